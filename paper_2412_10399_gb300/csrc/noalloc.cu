// Allocation-free particle-to-grid entry point (ckmpm_p2g_grids_static).
//
// Some callers cannot allocate device memory at the time they need a
// transfer: an application that hands the whole device to its own fixed
// memory arena and forbids further driver allocations, a real-time loop where
// cudaMalloc's implicit device synchronisation would stall other work, or a
// plug-in that must not change the host process's memory footprint after
// start-up.  This entry point serves them: it computes the same P2G grids as
// ckmpm_probe_grids + ckmpm_readback(GRID_M / GRID_P) on a context, but all
// of its working memory lives in one file-scope device array of fixed size,
// and it calls no cudaMalloc, cudaFree or allocating library routine.
//
// The array (kStaticBytes) is reserved on every GPU that loads the library,
// for the lifetime of the process; each GPU has its own copy.  Every call on
// a GPU shares that copy and it keeps the last call's contents (whatever must
// start at zero is cleared at the start of each call): two calls whose work
// overlaps on the same GPU, from different streams or host threads, race and
// corrupt each other's results.  The first call on a GPU looks up the array's
// device address (cudaGetSymbolAddress) with that GPU current; make that
// first call before capturing the stream into a CUDA graph.
//
// When the array's memory is taken: CUDA loads a library's device code
// lazily by default (CUDA_MODULE_LOADING=LAZY), and this file has no kernels
// of its own, so the module that holds the array is loaded on a GPU, and its
// 18 MiB reserved there, by the first cudaGetSymbolAddress, i.e. by the first
// call on that GPU (with CUDA_MODULE_LOADING=EAGER, when the library's
// context is created instead).  A caller whose own arena later claims the
// device memory should therefore make one small warm-up call per GPU at
// start-up, before the arena takes its share; a first call made after the
// memory is gone fails with CKMPM_ECUDA.  The call waits for its own work on
// its stream only: the error word is read back with an asynchronous copy on
// that stream followed by a synchronisation of that stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/ckmpm.h"
#include "common.cuh"
#include "launch.h"

namespace {

constexpr int64_t kStaticMaxN = 65536;    // particles per call
constexpr int kStaticMaxRes = 64;         // cells per axis
constexpr int kStaticMaxMats = 16;        // materials per scene
constexpr size_t kStaticBytes = 18u << 20;  // 18 MiB, enough for the limits above
constexpr int kMaxDevices = 64;

}  // namespace

// The scratch itself.  In host code this name is only a stand-in: its device
// address is obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_ckmpm_static_scratch[kStaticBytes];

namespace {

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (set up on the first
// call per device, with that device current).
cudaError_t scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_ckmpm_static_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// Bump carve-out of the scratch (256-byte aligned pieces).
struct Carve {
  char* base;
  size_t used = 0;
  bool ok = true;
  template <typename T>
  T* take(int64_t count) {
    size_t bytes = (sizeof(T) * (size_t)std::max<int64_t>(count, 1) + 255) & ~size_t(255);
    if (used + bytes > kStaticBytes) {
      ok = false;
      return nullptr;
    }
    T* p = (T*)(base + used);
    used += bytes;
    return p;
  }
};

}  // namespace

extern "C" CKMPM_API ckmpm_status ckmpm_p2g_grids_static(const ckmpm_scene* sc, int kernel, const float* B,
                                                        const float* F, float* grid_m, float* grid_p,
                                                        void* stream) {
  if (!sc || !sc->x || !grid_m || !grid_p) return CKMPM_EINVAL;
  if (kernel < 0 || kernel > 3) return CKMPM_EINVAL;  // APIC with the kernel gradient is not offered here
  const bool pic = (kernel & CKMPM_TRANSFER_PIC) != 0;
  if (pic && B) return CKMPM_EINVAL;  // the PIC transfer keeps no B
  kernel &= 1;
  if (!sc->is_device) return CKMPM_EINVAL;  // inputs must already be on the device
  if (sc->n < 1 || sc->n > kStaticMaxN) return CKMPM_EINVAL;
  if (sc->res < 4 || sc->res > kStaticMaxRes) return CKMPM_EINVAL;
  if (!(sc->dx > 0) || !(sc->dt > 0) || sc->ppc < 1 || !(sc->bc_cells >= 0)) return CKMPM_EINVAL;
  if (!std::isfinite(sc->dx) || !std::isfinite(sc->dt) || !std::isfinite(sc->bc_cells) ||
      !std::isfinite(sc->gravity[0]) || !std::isfinite(sc->gravity[1]) || !std::isfinite(sc->gravity[2]))
    return CKMPM_EINVAL;
  if (!sc->materials || sc->n_materials < 1 || sc->n_materials > kStaticMaxMats) return CKMPM_EINVAL;
  for (int i = 0; i < sc->n_materials; ++i) {
    const ckmpm_material& m = sc->materials[i];
    if (m.model == 1 && !(m.friction_deg >= 0 && m.friction_deg < 90)) return CKMPM_EINVAL;
    if (m.model < 0 || m.model > 2 || !(m.E >= 0) || !(m.nu > -1.0 && m.nu < 0.5) || !(m.rho > 0) ||
        (m.model == 2 && !(m.gamma > 0)) || !std::isfinite(m.E) || !std::isfinite(m.rho) ||
        !std::isfinite(m.friction_deg) || (m.model == 2 && !std::isfinite(m.gamma)))
      return CKMPM_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return CKMPM_ECUDA;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CKMPM_ECUDA;

  const int NG = kernel == 0 ? 2 : 1;
  const int64_t n = sc->n;
  const int64_t npb = (sc->res + 3) / 4, nb = npb + 1;
  const int64_t nkeys = npb * npb * npb, nvb = nb * nb * nb;
  const int64_t ntiles = (nkeys + ck::kScanTile - 1) / ck::kScanTile;

  Carve cv{(char*)base};
  ck::Pool P{};
  P.X = cv.take<float4>(n);
  P.VM0 = cv.take<float4>(n);
  P.VM1 = cv.take<float4>(n);
  P.VM2 = cv.take<float4>(n);
  P.F0 = cv.take<float4>(n);
  P.F1 = cv.take<float4>(n);
  P.F2 = cv.take<float>(n);
  P.ID = cv.take<uint32_t>(n);
  P.E = nullptr;
  ck::StepView v{};
  v.cur = P;
  v.nxt = P;  // not written: no G2P runs here
  v.key_cur = cv.take<uint32_t>(n);
  v.key_nxt = v.key_cur;
  v.cnt_cur = cv.take<uint32_t>(nkeys);
  v.cnt_nxt = cv.take<uint32_t>(nkeys);
  v.bnd_cur = cv.take<uint32_t>(2 * nkeys);
  v.bnd_nxt = cv.take<uint32_t>(2 * nkeys);
  v.offset = cv.take<uint32_t>(nkeys);
  v.cursor = cv.take<uint32_t>(nkeys);
  v.perm = cv.take<uint32_t>(n);
  v.pb_key = cv.take<uint32_t>(nkeys);
  v.pb_scene = cv.take<uint32_t>(nkeys);
  uint32_t* counters = cv.take<uint32_t>(8);
  v.n_pb = counters + 0;
  v.n_g = counters + 1;
  v.err = counters + 2;
  v.fp64_count = (unsigned long long*)(counters + 4);
  v.work = counters + 6;
  v.gflag = cv.take<uint32_t>(nvb);
  v.table = cv.take<uint32_t>(nvb);
  v.g_list = cv.take<uint32_t>(nvb);
  v.g_scene = cv.take<uint32_t>(nvb);
  v.pool_cap = (uint32_t)nvb;
  v.Gacc = cv.take<float4>(nvb * NG * ck::kBlockNodes);
  v.Gvel = v.Gacc;  // the grid update is not run
  ck::SceneDev* d_scene = cv.take<ck::SceneDev>(1);
  ck::MatDev* d_mats = cv.take<ck::MatDev>(kStaticMaxMats);
  uint32_t* scene_tab = cv.take<uint32_t>(2);
  ck::BinScratch bs{};
  bs.tile_cnt = cv.take<uint32_t>(ntiles + 1);
  bs.tile_ne = cv.take<uint32_t>(ntiles + 1);
  if (!cv.ok) return CKMPM_ENOMEM;  // cannot happen within the limits above
  v.scenes = d_scene;
  v.mats = d_mats;
  v.n_mats = kStaticMaxMats;
  v.n_keys = (uint32_t)nkeys;
  v.n_cur = (uint32_t)n;
  v.keep_gacc = 1;
  v.splits = 1;
  bs.scene_tab = scene_tab;
  bs.n_scene_tab = 1;

  // scene and material parameters (same definitions as a context's admission)
  ck::SceneDev h{};
  const double V0 = sc->dx * sc->dx * sc->dx / sc->ppc;
  h.dx = (float)sc->dx;
  h.inv_dx = (float)(1.0 / sc->dx);
  h.dt = (float)sc->dt;
  h.V0 = (float)V0;
  h.gx = (float)sc->gravity[0];
  h.gy = (float)sc->gravity[1];
  h.gz = (float)sc->gravity[2];
  h.bc = (float)sc->bc_cells;
  h.res = sc->res;
  h.npb = (int)npb;
  h.nb = (int)nb;
  h.key_base = 0;
  h.table_base = 0;
  h.j_tol = (float)sc->fp64_j_tol;
  h.cond_tol = (float)sc->fp64_cond_tol;
  h.gap_tol = (float)sc->fp64_gap_tol;
  h.alive = 1;
  ck::MatDev hm[kStaticMaxMats] = {};
  double mmax = 0.0;
  for (int i = 0; i < sc->n_materials; ++i) {
    const ckmpm_material& m = sc->materials[i];
    hm[i].model = m.model;
    hm[i].scene = 0;
    hm[i].mu = (float)(m.E / (2.0 * (1.0 + m.nu)));
    hm[i].lam = (float)(m.E * m.nu / ((1.0 + m.nu) * (1.0 - 2.0 * m.nu)));
    hm[i].mass = (float)(m.rho * V0);
    double s = std::sin(m.friction_deg * M_PI / 180.0);
    hm[i].alpha = (float)(std::sqrt(2.0 / 3.0) * 2.0 * s / (3.0 - s));
    hm[i].dpc = (float)((double)hm[i].alpha * (1.0 + m.nu) / (1.0 - 2.0 * m.nu));
    hm[i].gamma = (float)m.gamma;
    hm[i].E = (float)m.E;
    hm[i].nu = (float)m.nu;
    mmax = std::max(mmax, m.rho * V0);
  }
  h.mmax = (float)mmax;
  const uint32_t tab[2] = {0u, 0u};
  const int64_t nn = (int64_t)(sc->res + 1) * (sc->res + 1) * (sc->res + 1);

#define CK_S(expr)                                   \
  do {                                               \
    if ((expr) != cudaSuccess) return CKMPM_ECUDA;   \
  } while (0)
  CK_S(cudaMemcpyAsync(d_scene, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  CK_S(cudaMemcpyAsync(d_mats, hm, sizeof(ck::MatDev) * kStaticMaxMats, cudaMemcpyHostToDevice, st));
  CK_S(cudaMemcpyAsync(scene_tab, tab, sizeof(tab), cudaMemcpyHostToDevice, st));
  // everything a previous call may have left behind and the kernels expect zero
  CK_S(cudaMemsetAsync(v.cnt_cur, 0, sizeof(uint32_t) * nkeys, st));
  CK_S(cudaMemsetAsync(v.bnd_cur, 0, sizeof(uint32_t) * 2 * nkeys, st));
  CK_S(cudaMemsetAsync(counters, 0, sizeof(uint32_t) * 8, st));
  CK_S(cudaMemsetAsync(v.gflag, 0, sizeof(uint32_t) * nvb, st));
  CK_S(cudaMemsetAsync(v.Gacc, 0, sizeof(float4) * nvb * NG * ck::kBlockNodes, st));
  CK_S(cudaMemsetAsync(grid_m, 0, sizeof(float) * NG * nn, st));
  CK_S(cudaMemsetAsync(grid_p, 0, sizeof(float) * 3 * NG * nn, st));

  // particles: x, v, material; B = 0 and F = I, then the caller's F and B
  ck::launch_admit(kernel, st, P, v.key_cur, v.cnt_cur, v.bnd_cur, d_scene, d_mats, 0, 0u, (uint32_t)sc->n_materials,
                   0u, (uint32_t)n, sc->x, sc->v, sc->mat, nullptr, v.err);
  if (F || B) {
    if (F) ck::launch_write_particles(pic, st, P, d_scene, d_mats, 0, 0u, (uint32_t)n, CKMPM_FIELD_F, F);
    if (B) ck::launch_write_particles(pic, st, P, d_scene, d_mats, 0, 0u, (uint32_t)n, CKMPM_FIELD_B, B);
    // M changed: histogram and P2G bounds again
    CK_S(cudaMemsetAsync(v.cnt_cur, 0, sizeof(uint32_t) * nkeys, st));
    CK_S(cudaMemsetAsync(v.bnd_cur, 0, sizeof(uint32_t) * 2 * nkeys, st));
    ck::launch_rekey(kernel, st, P, v.key_cur, v.cnt_cur, v.bnd_cur, d_scene, d_mats, (uint32_t)n, v.err);
  }
  // binning and P2G, as in a context's step
  const int grid_ctas = sms * 4;
  ck::launch_bin(st, v, bs, ck::LB_SCAN_TILES, (uint32_t)nvb, grid_ctas);
  ck::launch_bin(st, v, bs, ck::LB_SCAN_TOP, (uint32_t)nvb, grid_ctas);
  ck::launch_bin(st, v, bs, ck::LB_SCAN_FINAL, (uint32_t)nvb, grid_ctas);
  ck::launch_bin(st, v, bs, ck::LB_SCATTER, (uint32_t)nvb, grid_ctas);
  ck::launch_bin(st, v, bs, ck::LB_GLIST, (uint32_t)nvb, grid_ctas);
  ck::LaunchCfg lc{st, sms * 8};
  lc.transfer = pic ? 1 : 0;
  ck::launch_transfer(kernel, lc, v, ck::LK_P2G);
  ck::launch_read_grid(kernel, st, v, 0, 0, grid_m);
  ck::launch_read_grid(kernel, st, v, 0, 1, grid_p);
  CK_S(cudaGetLastError());
  // the error word comes back on the caller's stream: waiting for that
  // stream alone leaves work on the device's other streams running
  uint32_t err = 0;
  CK_S(cudaMemcpyAsync(&err, v.err, sizeof(err), cudaMemcpyDeviceToHost, st));
  CK_S(cudaStreamSynchronize(st));
#undef CK_S
  if (err & CK_ERR_NONFINITE) return CKMPM_ENONFINITE;
  if (err & CK_ERR_DOMAIN) return CKMPM_EDOMAIN;
  if (err & (CK_ERR_POOL | CK_ERR_INTERNAL)) return CKMPM_EINVAL;
  return CKMPM_OK;
}
