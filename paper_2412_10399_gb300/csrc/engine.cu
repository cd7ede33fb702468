// Host runtime and C ABI of the CK-MPM library: contexts, scene admission,
// the per-step launch sequence, readback/upload and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ckmpm.h"
#include "common.cuh"
#include "launch.h"

namespace {

using ck::MatDev;
using ck::Pool;
using ck::SceneDev;

struct Range {
  int64_t start, len;
};

// First-fit allocator over an integer range.
struct RangeAlloc {
  std::vector<Range> free_;
  int64_t cap = 0, high = 0;
  void init(int64_t c) {
    cap = c;
    high = 0;
    free_.clear();
    if (c > 0) free_.push_back({0, c});
  }
  int64_t take(int64_t len) {
    for (size_t i = 0; i < free_.size(); ++i) {
      if (free_[i].len >= len) {
        int64_t s = free_[i].start;
        free_[i].start += len;
        free_[i].len -= len;
        if (free_[i].len == 0) free_.erase(free_.begin() + i);
        high = std::max(high, s + len);
        return s;
      }
    }
    return -1;
  }
  void give(int64_t s, int64_t len) {
    free_.push_back({s, len});
    std::sort(free_.begin(), free_.end(), [](const Range& a, const Range& b) { return a.start < b.start; });
    std::vector<Range> m;
    for (auto& r : free_) {
      if (!m.empty() && m.back().start + m.back().len == r.start)
        m.back().len += r.len;
      else
        m.push_back(r);
    }
    free_.swap(m);
  }
};

struct SceneHost {
  bool used = false, alive = false;
  int64_t n = 0;
  int64_t key_base = 0, nkeys = 0;
  int64_t table_base = 0, nvb = 0;
  int64_t mat_base = 0, nmat = 0;
  int res = 0;
};

struct Seg {
  int slot;
  int64_t start, n;
};

struct PendingFree {
  int slot;
};

}  // namespace

struct ckmpm_ctx {
  int kind = 0;      // 0 CK, 1 quadratic
  int transfer = 0;  // ckmpm_transfer
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  ckmpm_allocator alloc{};
  bool has_alloc = false;
  int device = 0, sm_count = 1;
  ck::LaunchCfg lc{};

  int64_t cap_n = 0, cap_keys = 0, cap_vblocks = 0, cap_pool = 0;
  int cap_scenes = 0, cap_mats = 0;
  bool per_E = false;

  Pool pool[2]{};
  int cur = 0;
  uint32_t* key[2]{};
  uint32_t* cnt[2]{};
  uint32_t* bnd[2]{};  // per key: P2G contribution bounds (2 floats as bits)
  uint32_t *offset = nullptr, *cursor = nullptr, *perm = nullptr, *pb_key = nullptr, *pb_scene = nullptr;
  uint32_t *counters = nullptr;  // [0] n_pb, [1] n_g, [2] err, [4..5] fp64 (64-bit), [6..7] work,
                                 // [8] n_g of the second table set, [9] leftover count
  // fused G2P2G steps: a second block-table set for the next step's grid,
  // which one maps the current grid velocities, and whether they are current
  bool fused = false;
  int splits_override = 0;  // CKMPM_SPLITS: work units per block (else chosen from the particle count)
  // steady-state steps replayed as CUDA graphs, one per parity of the
  // double-buffered state (particle buffer cur, plus table set tsel for
  // fused steps); dropped whenever the launch sequence or its arguments change
  bool graphs = false;
  cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t graph_steps = 0;  // steps launched as a graph
  int tsel = 0;
  bool grid_valid = false;
  uint32_t *table1 = nullptr, *g_list1 = nullptr, *g_scene1 = nullptr, *lo_list = nullptr;
  uint32_t* fp64_list = nullptr;  // particles of the float64 pass (capacity cap_n)
  uint32_t *gflag = nullptr, *table = nullptr, *g_list = nullptr, *g_scene = nullptr;
  uint32_t *tile_cnt = nullptr, *tile_ne = nullptr, *scene_tab = nullptr;
  float4 *Gacc = nullptr, *Gvel = nullptr;
  SceneDev* d_scenes = nullptr;
  MatDev* d_mats = nullptr;
  void* staging = nullptr;
  size_t staging_bytes = 0;
  // host readbacks: two device staging slots; the gather runs on the
  // context's stream, the device-to-host copy on copy_stream, so that the
  // copy of one step's field overlaps the next step
  struct RbSlot {
    void* buf = nullptr;
    size_t cap = 0;
    cudaEvent_t copied = nullptr;  // recorded on copy_stream after the slot's copies
    uint32_t* status = nullptr;    // pinned host word: the device status at the gather
    int64_t ticket = -1;
  };
  RbSlot rb[2];
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t rb_gathered = nullptr;
  int64_t rb_next = 0;

  std::vector<SceneHost> scenes;
  std::vector<SceneDev> h_scenes;
  std::vector<MatDev> h_mats;
  RangeAlloc keys_alloc, grid_alloc, mat_alloc;
  std::vector<int> pending_free;
  int64_t n_cur = 0;
  std::vector<Seg> layout;
  bool keys_dirty = false, grids_dirty = false;
  ckmpm_status sticky = CKMPM_OK;
  int64_t steps = 0;
  std::string msg;
  std::vector<std::pair<void*, size_t>> allocs;

  bool timing = false;
  struct EvPair {
    cudaEvent_t a, b;
    int which;
  };
  std::vector<EvPair> ev_used, ev_free;
  double ms_sum[8] = {0};
  int64_t ms_cnt[8] = {0};
  cudaEvent_t step_a = nullptr, step_b = nullptr;
  double ms_last_step = 0;
};

namespace {

ckmpm_status fail(ckmpm_ctx* c, ckmpm_status s, const std::string& m) {
  if (c) c->msg = m;
  return s;
}

ckmpm_status cuda_fail(ckmpm_ctx* c, cudaError_t e, const char* where) {
  return fail(c, CKMPM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK_TRY(expr, where)                                   \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where);  \
  } while (0)

void* dev_alloc(ckmpm_ctx* ctx, size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (ctx->has_alloc) {
    p = ctx->alloc.alloc(bytes, ctx->alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) ctx->allocs.push_back({p, bytes});
  return p;
}

void dev_free(ckmpm_ctx* ctx, void* p) {
  if (!p) return;
  for (size_t i = 0; i < ctx->allocs.size(); ++i) {
    if (ctx->allocs[i].first == p) {
      size_t b = ctx->allocs[i].second;
      ctx->allocs.erase(ctx->allocs.begin() + i);
      if (ctx->has_alloc)
        ctx->alloc.free(p, b, ctx->alloc.user);
      else
        cudaFree(p);
      return;
    }
  }
}

template <typename T>
bool alloc_n(ckmpm_ctx* ctx, T*& p, int64_t n) {
  p = (T*)dev_alloc(ctx, sizeof(T) * (size_t)std::max<int64_t>(n, 1));
  return p != nullptr;
}

bool alloc_pool(ckmpm_ctx* ctx, Pool& P, int64_t n) {
  P.E = nullptr;
  bool ok = alloc_n(ctx, P.X, n) && alloc_n(ctx, P.VM0, n) && alloc_n(ctx, P.VM1, n) && alloc_n(ctx, P.VM2, n) &&
            alloc_n(ctx, P.F0, n) && alloc_n(ctx, P.F1, n) && alloc_n(ctx, P.F2, n) && alloc_n(ctx, P.ID, n);
  if (ok && ctx->per_E) ok = alloc_n(ctx, P.E, n);
  P.T0 = P.T1 = nullptr;
  P.T2 = nullptr;
  if (ok && ctx->transfer == CKMPM_TRANSFER_APIC_GRAD)
    ok = alloc_n(ctx, P.T0, n) && alloc_n(ctx, P.T1, n) && alloc_n(ctx, P.T2, n);
  return ok;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

ck::StepView make_view(ckmpm_ctx* ctx) {
  ck::StepView v{};
  v.cur = ctx->pool[ctx->cur];
  v.nxt = ctx->pool[ctx->cur ^ 1];
  v.key_cur = ctx->key[ctx->cur];
  v.key_nxt = ctx->key[ctx->cur ^ 1];
  v.cnt_cur = ctx->cnt[ctx->cur];
  v.cnt_nxt = ctx->cnt[ctx->cur ^ 1];
  v.bnd_cur = ctx->bnd[ctx->cur];
  v.bnd_nxt = ctx->bnd[ctx->cur ^ 1];
  v.offset = ctx->offset;
  v.cursor = ctx->cursor;
  v.perm = ctx->perm;
  v.pb_key = ctx->pb_key;
  v.pb_scene = ctx->pb_scene;
  v.n_pb = ctx->counters + 0;
  v.n_g = ctx->counters + (ctx->tsel == 0 ? 1 : 8);
  v.err = ctx->counters + 2;
  v.fp64_count = (unsigned long long*)(ctx->counters + 4);
  v.fp64_list = ctx->fp64_list;
  v.work = ctx->counters + 6;
  v.gflag = ctx->gflag;
  v.table = ctx->tsel == 0 ? ctx->table : ctx->table1;
  v.pool_cap = (uint32_t)ctx->cap_pool;
  v.g_list = ctx->tsel == 0 ? ctx->g_list : ctx->g_list1;
  v.g_scene = ctx->tsel == 0 ? ctx->g_scene : ctx->g_scene1;
  v.Gacc = ctx->Gacc;
  v.Gvel = ctx->Gvel;
  v.scenes = ctx->d_scenes;
  v.mats = ctx->d_mats;
  v.n_mats = (uint32_t)ctx->cap_mats;
  v.n_keys = (uint32_t)std::max<int64_t>(ctx->keys_alloc.high, 1);
  v.n_cur = (uint32_t)ctx->n_cur;
  v.keep_gacc = 0;
  // a step with few particles splits each block over several work units, so
  // that the resident warps of the transfer kernels (about 20 per SM) get two
  // units of a few hundred particles each; large steps keep whole blocks
  {
    int64_t n_live = 0;
    for (auto& s : ctx->scenes) n_live += s.alive ? s.n : 0;
    const int64_t target = (int64_t)ctx->sm_count * 20 * 2 * 512;
    v.splits = (uint32_t)std::max<int64_t>(1, std::min<int64_t>(8, target / std::max<int64_t>(n_live, 1)));
    if (ctx->splits_override > 0) v.splits = (uint32_t)ctx->splits_override;
  }
  if (ctx->fused) {  // binning zeroes the leftover count every step
    v.lo_list = ctx->lo_list;
    v.lo_count = ctx->counters + 9;
  }
  return v;
}

ck::BinScratch make_bs(ckmpm_ctx* ctx, int n_tab) {
  ck::BinScratch bs{};
  bs.tile_cnt = ctx->tile_cnt;
  bs.tile_ne = ctx->tile_ne;
  bs.scene_tab = ctx->scene_tab;
  bs.n_scene_tab = n_tab;
  return bs;
}

// timing helpers
void tbeg(ckmpm_ctx* ctx, ckmpm_ctx::EvPair& ep, int which) {
  if (!ctx->timing) return;
  if (ctx->ev_free.empty()) {
    ckmpm_ctx::EvPair e{};
    cudaEventCreate(&e.a);
    cudaEventCreate(&e.b);
    ctx->ev_free.push_back(e);
  }
  ep = ctx->ev_free.back();
  ctx->ev_free.pop_back();
  ep.which = which;
  cudaEventRecord(ep.a, ctx->stream);
}
void tend(ckmpm_ctx* ctx, ckmpm_ctx::EvPair& ep) {
  if (!ctx->timing) return;
  cudaEventRecord(ep.b, ctx->stream);
  ctx->ev_used.push_back(ep);
}
void harvest_timing(ckmpm_ctx* ctx) {
  for (auto& e : ctx->ev_used) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
      ctx->ms_sum[e.which] += ms;
      ctx->ms_cnt[e.which] += 1;
    }
    ctx->ev_free.push_back(e);
  }
  ctx->ev_used.clear();
  cudaGetLastError();
}

int upload_scene_tab(ckmpm_ctx* ctx) {
  std::vector<uint32_t> tab;
  std::vector<std::pair<int64_t, int>> al;
  for (int s = 0; s < (int)ctx->scenes.size(); ++s)
    if (ctx->scenes[s].alive) al.push_back({ctx->scenes[s].key_base, s});
  std::sort(al.begin(), al.end());
  for (auto& a : al) {
    tab.push_back((uint32_t)a.first);
    tab.push_back((uint32_t)a.second);
  }
  if (tab.empty()) {
    tab.push_back(0);
    tab.push_back(0);
  }
  cudaMemcpyAsync(ctx->scene_tab, tab.data(), tab.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream);
  return (int)(tab.size() / 2);
}

int n_scene_tab(ckmpm_ctx* ctx) {
  int n = 0;
  for (auto& s : ctx->scenes) n += s.alive ? 1 : 0;
  return std::max(n, 1);
}

void process_pending(ckmpm_ctx* ctx) {
  for (int slot : ctx->pending_free) {
    SceneHost& s = ctx->scenes[slot];
    ctx->keys_alloc.give(s.key_base, s.nkeys);
    ctx->grid_alloc.give(s.table_base, s.nvb);
    ctx->mat_alloc.give(s.mat_base, s.nmat);
    s = SceneHost{};
  }
  ctx->pending_free.clear();
}

void rebuild_layout_sorted(ckmpm_ctx* ctx) {
  std::vector<std::pair<int64_t, int>> al;
  for (int s = 0; s < (int)ctx->scenes.size(); ++s)
    if (ctx->scenes[s].alive) al.push_back({ctx->scenes[s].key_base, s});
  std::sort(al.begin(), al.end());
  ctx->layout.clear();
  int64_t start = 0;
  for (auto& a : al) {
    ctx->layout.push_back({a.second, start, ctx->scenes[a.second].n});
    start += ctx->scenes[a.second].n;
  }
}

const Seg* find_seg(ckmpm_ctx* ctx, int slot) {
  for (auto& s : ctx->layout)
    if (s.slot == slot) return &s;
  return nullptr;
}

ckmpm_status apply_device_error(ckmpm_ctx* ctx, uint32_t e) {
  if (ctx->sticky == CKMPM_OK) {
    if (e & CK_ERR_NONFINITE) {
      ctx->sticky = CKMPM_ENONFINITE;
      ctx->msg = "a non-finite particle state was produced";
    } else if (e & CK_ERR_DOMAIN) {
      ctx->sticky = CKMPM_EDOMAIN;
      ctx->msg = "a particle left the valid interior [0.5 dx, (res-0.5) dx) and was clamped";
    } else if (e & CK_ERR_POOL) {
      ctx->sticky = CKMPM_ENOMEM;
      ctx->msg = "grid pool capacity exceeded: more active grid blocks than max_grid_blocks";
    } else if (e & CK_ERR_INTERNAL) {
      ctx->sticky = CKMPM_EINVAL;
      ctx->msg = "internal consistency check failed (particle outside its block)";
    } else if (e & CK_ERR_TIMEOUT) {
      ctx->sticky = CKMPM_ETIMEOUT;
      ctx->msg = "a bounded device wait gave up";
    }
  }
  return ctx->sticky;
}

ckmpm_status read_device_error(ckmpm_ctx* ctx) {
  uint32_t e = 0;
  cudaError_t ce = cudaMemcpy(&e, ctx->counters + 2, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (ce != cudaSuccess) return cuda_fail(ctx, ce, "reading the device status word");
  return apply_device_error(ctx, e);
}

bool ensure_staging(ckmpm_ctx* ctx, size_t bytes) {
  if (ctx->staging_bytes >= bytes) return true;
  if (ctx->staging) {
    cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, ctx->staging);
    ctx->staging = nullptr;
    ctx->staging_bytes = 0;
  }
  size_t b = std::max<size_t>(bytes, 1 << 20);
  ctx->staging = dev_alloc(ctx, b);
  if (!ctx->staging) return false;
  ctx->staging_bytes = b;
  return true;
}

// Whether any of the n bytes at p is >= k (1 <= k <= 255), eight bytes per
// step for k <= 128: with h = 127 - (k - 1), a byte b < 128 gets its top bit
// from b + h exactly when b >= k (b + h <= 254, so no carry leaves the byte),
// and a byte b >= 128 has it already, which OR-ing b keeps whatever carry the
// addition produced; a carry only ever leaves a byte whose top bit is set, so
// the word's answer is exact.
bool any_byte_at_least(const uint8_t* p, int64_t n, int k) {
  int64_t i = 0;
  if (k <= 128) {
    const uint64_t ones = 0x0101010101010101ull, tops = 0x8080808080808080ull;
    const uint64_t add = ones * (uint64_t)(128 - k);
    uint64_t acc = 0;
    for (; i + 8 <= n; i += 8) {
      uint64_t w;
      std::memcpy(&w, p + i, 8);
      acc |= ((w + add) | w) & tops;
    }
    if (acc) return true;
  }
  for (; i < n; ++i)
    if ((int)p[i] >= k) return true;
  return false;
}

ckmpm_status validate_scene(ckmpm_ctx* ctx, const ckmpm_scene* s) {
  if (!s) return fail(ctx, CKMPM_EINVAL, "scene is NULL");
  if (s->n < 1 || s->n > 0x7fffffffLL) return fail(ctx, CKMPM_EINVAL, "scene.n must be in [1, 2^31)");
  if (!s->x) return fail(ctx, CKMPM_EINVAL, "scene.x is NULL");
  if (s->res < 4 || s->res > 4096) return fail(ctx, CKMPM_EINVAL, "scene.res must be in [4, 4096]");
  if (!(s->dx > 0) || !(s->dt > 0) || !std::isfinite(s->dx) || !std::isfinite(s->dt))
    return fail(ctx, CKMPM_EINVAL, "scene.dx and scene.dt must be positive and finite");
  if (!std::isfinite(s->gravity[0]) || !std::isfinite(s->gravity[1]) || !std::isfinite(s->gravity[2]))
    return fail(ctx, CKMPM_EINVAL, "scene.gravity must be finite");
  if (!(s->fp64_j_tol >= 0) || !(s->fp64_cond_tol >= 0) || !(s->fp64_gap_tol >= 0) || !std::isfinite(s->fp64_j_tol) ||
      !std::isfinite(s->fp64_cond_tol) || !std::isfinite(s->fp64_gap_tol))
    return fail(ctx, CKMPM_EINVAL, "scene.fp64_*_tol must be finite and >= 0");
  if (s->ppc < 1) return fail(ctx, CKMPM_EINVAL, "scene.ppc must be >= 1");
  if (!s->materials || s->n_materials < 1 || s->n_materials > 255)
    return fail(ctx, CKMPM_EINVAL, "scene needs 1..255 materials");
  for (int i = 0; i < s->n_materials; ++i) {
    const ckmpm_material& m = s->materials[i];
    if (m.model < 0 || m.model > 2) return fail(ctx, CKMPM_EINVAL, "material.model must be 0, 1 or 2");
    if (m.model == 2 && !(m.gamma > 0)) return fail(ctx, CKMPM_EINVAL, "fluid material needs gamma > 0");
    if (m.model == 1 && !(m.friction_deg >= 0 && m.friction_deg < 90))
      return fail(ctx, CKMPM_EINVAL, "Drucker-Prager material needs a friction angle in [0, 90) degrees");
    if (!(m.E >= 0) || !(m.nu > -1.0 && m.nu < 0.5) || !(m.rho > 0) || !std::isfinite(m.E) || !std::isfinite(m.rho) ||
        !std::isfinite(m.friction_deg) || (m.model == 2 && !std::isfinite(m.gamma)))
      return fail(ctx, CKMPM_EINVAL, "material needs finite E >= 0, -1 < nu < 0.5, rho > 0");
  }
  if (!(s->bc_cells >= 0) || !std::isfinite(s->bc_cells))
    return fail(ctx, CKMPM_EINVAL, "scene.bc_cells must be finite and >= 0");
  // host material indices are checked here, before any device work; device
  // arrays are checked by the admission kernel (material 0 and EINVAL)
  if (s->mat && !s->is_device) {
    // a word-at-a-time test first; the offending index is searched for only
    // when there is one
    const uint8_t* mat = s->mat;
    const int64_t n = s->n;
    if (any_byte_at_least(mat, n, s->n_materials))
      for (int64_t i = 0; i < n; ++i)
        if ((int)mat[i] >= s->n_materials)
          return fail(ctx, CKMPM_EINVAL,
                      "scene.mat[" + std::to_string(i) + "] = " + std::to_string((int)mat[i]) +
                          " is not below n_materials");
  }
  return CKMPM_OK;
}

ckmpm_status init_ctx(ckmpm_ctx* ctx, const ckmpm_config* cfg) {
  if ((cfg->kernel & ~15) != 0 || (cfg->kernel & 6) == 6)
    return fail(ctx, CKMPM_EINVAL,
                "kernel must be 0 (CK) or 1 (quadratic), optionally | CKMPM_TRANSFER_PIC or CKMPM_TRANSFER_APIC_GRAD, "
                "and | CKMPM_STEP_G2P2G");
  ctx->kind = cfg->kernel & 1;
  ctx->transfer = cfg->kernel & 6;
  ctx->fused = (cfg->kernel & CKMPM_STEP_G2P2G) != 0;
  if (ctx->fused && ctx->transfer != CKMPM_TRANSFER_APIC_MLS)
    return fail(ctx, CKMPM_EINVAL, "the fused G2P2G step takes the APIC + MLS transfer only");
  if (cfg->max_particles < 1 || cfg->max_keys < 1 || cfg->max_grid_blocks < 1 || cfg->max_virtual_blocks < 1 ||
      cfg->max_scenes < 1 ||
      cfg->max_scenes > 1024 || cfg->max_materials < 1 || cfg->max_materials > 65535)
    return fail(ctx, CKMPM_EINVAL, "invalid capacities");
  if (cfg->max_particles > 0x7fffffffLL || cfg->max_keys > 0x7fffffffLL || cfg->max_grid_blocks > 0x7fffffffLL ||
      cfg->max_virtual_blocks > 0x7fffffffLL)
    return fail(ctx, CKMPM_EINVAL, "capacities must be below 2^31");
  if (cfg->allocator) {
    if (!cfg->allocator->alloc || !cfg->allocator->free) return fail(ctx, CKMPM_EINVAL, "allocator needs alloc and free");
    ctx->alloc = *cfg->allocator;
    ctx->has_alloc = true;
  }
  CK_TRY(cudaGetDevice(&ctx->device), "cudaGetDevice");
  CK_TRY(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device), "device attributes");
  int per_sm = 8;
  if (const char* e = getenv("CKMPM_CTAS_PER_SM")) per_sm = std::max(1, atoi(e));
  ctx->lc.persistent_ctas = ctx->sm_count * per_sm;
  ctx->lc.sm_count = ctx->sm_count;
  ctx->lc.g2p_minb = 5;
  ctx->lc.transfer = ctx->transfer == CKMPM_TRANSFER_PIC ? 1 : ctx->transfer == CKMPM_TRANSFER_APIC_GRAD ? 2 : 0;
  if (const char* e = getenv("CKMPM_G2P_MINB")) ctx->lc.g2p_minb = std::max(4, std::min(6, atoi(e)));
  // two copies of the P2G accumulators are the faster choice for the
  // quadratic twin (27-node stencils collide more); the compact kernel keeps
  // one copy and issues its components in the lane-rotated order.  Both
  // round contributions by a fused multiply-add in blocks of >= 256 particles.
  ctx->lc.p2g_rep = ctx->kind == 1 ? 2 : 1;
  ctx->lc.p2g_rot = ctx->kind == 1 ? 0 : 1;
  ctx->lc.p2g_fma = 1;
  if (const char* e = getenv("CKMPM_P2G_REP")) ctx->lc.p2g_rep = atoi(e) == 2 ? 2 : 1;
  if (const char* e = getenv("CKMPM_P2G_ROT")) ctx->lc.p2g_rot = atoi(e) != 0;
  if (const char* e = getenv("CKMPM_P2G_FMA")) ctx->lc.p2g_fma = atoi(e) != 0;
  if (const char* e = getenv("CKMPM_SPLITS")) ctx->splits_override = std::max(1, std::min(8, atoi(e)));
  // steady steps run as CUDA graphs (CKMPM_GRAPHS=0 turns them off); the
  // legacy stream cannot be captured, so a context on it launches directly
  ctx->graphs = true;
  if (const char* e = getenv("CKMPM_GRAPHS")) ctx->graphs = atoi(e) != 0;
  if (cfg->stream) {
    ctx->stream = (cudaStream_t)cfg->stream;
  } else {
    CK_TRY(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking), "cudaStreamCreate");
    ctx->own_stream = true;
  }
  ctx->lc.stream = ctx->stream;
  if (!ctx->stream) ctx->graphs = false;
  ctx->cap_n = cfg->max_particles;
  ctx->cap_keys = cfg->max_keys;
  ctx->cap_pool = cfg->max_grid_blocks;
  ctx->cap_vblocks = cfg->max_virtual_blocks;
  ctx->cap_scenes = cfg->max_scenes;
  ctx->cap_mats = cfg->max_materials;
  ctx->per_E = cfg->per_particle_E != 0;
  const int NG = ctx->kind == 0 ? 2 : 1;
  bool ok = alloc_pool(ctx, ctx->pool[0], ctx->cap_n) && alloc_pool(ctx, ctx->pool[1], ctx->cap_n) &&
            alloc_n(ctx, ctx->key[0], ctx->cap_n) && alloc_n(ctx, ctx->key[1], ctx->cap_n) &&
            alloc_n(ctx, ctx->perm, ctx->cap_n) && alloc_n(ctx, ctx->fp64_list, ctx->cap_n) &&
            alloc_n(ctx, ctx->cnt[0], ctx->cap_keys) &&
            alloc_n(ctx, ctx->cnt[1], ctx->cap_keys) && alloc_n(ctx, ctx->bnd[0], 2 * ctx->cap_keys) &&
            alloc_n(ctx, ctx->bnd[1], 2 * ctx->cap_keys) && alloc_n(ctx, ctx->offset, ctx->cap_keys) &&
            alloc_n(ctx, ctx->cursor, ctx->cap_keys) && alloc_n(ctx, ctx->pb_key, ctx->cap_keys) &&
            alloc_n(ctx, ctx->pb_scene, ctx->cap_keys) && alloc_n(ctx, ctx->counters, 12) &&
            alloc_n(ctx, ctx->gflag, ctx->cap_vblocks) && alloc_n(ctx, ctx->table, ctx->cap_vblocks) &&
            alloc_n(ctx, ctx->g_list, ctx->cap_pool) && alloc_n(ctx, ctx->g_scene, ctx->cap_pool) &&
            alloc_n(ctx, ctx->tile_cnt, ceil_div(ctx->cap_keys, ck::kScanTile) + 1) &&
            alloc_n(ctx, ctx->tile_ne, ceil_div(ctx->cap_keys, ck::kScanTile) + 1) &&
            alloc_n(ctx, ctx->scene_tab, 2 * (int64_t)ctx->cap_scenes + 2) &&
            alloc_n(ctx, ctx->Gacc, ctx->cap_pool * NG * ck::kBlockNodes) &&
            alloc_n(ctx, ctx->Gvel, ctx->cap_pool * NG * ck::kBlockNodes) &&
            alloc_n(ctx, ctx->d_scenes, ctx->cap_scenes) && alloc_n(ctx, ctx->d_mats, ctx->cap_mats);
  if (ok && ctx->fused)
    ok = alloc_n(ctx, ctx->table1, ctx->cap_vblocks) && alloc_n(ctx, ctx->g_list1, ctx->cap_pool) &&
         alloc_n(ctx, ctx->g_scene1, ctx->cap_pool) && alloc_n(ctx, ctx->lo_list, ctx->cap_n);
  if (!ok) return fail(ctx, CKMPM_ENOMEM, "device memory allocation failed");
  if (ctx->fused) CK_TRY(cudaMemsetAsync(ctx->table1, 0xff, sizeof(uint32_t) * ctx->cap_vblocks, ctx->stream), "memset");
  CK_TRY(cudaMemsetAsync(ctx->cnt[0], 0, sizeof(uint32_t) * ctx->cap_keys, ctx->stream), "memset");
  CK_TRY(cudaMemsetAsync(ctx->cnt[1], 0, sizeof(uint32_t) * ctx->cap_keys, ctx->stream), "memset");
  CK_TRY(cudaMemsetAsync(ctx->bnd[0], 0, sizeof(uint32_t) * 2 * ctx->cap_keys, ctx->stream), "memset");
  CK_TRY(cudaMemsetAsync(ctx->bnd[1], 0, sizeof(uint32_t) * 2 * ctx->cap_keys, ctx->stream), "memset");
  CK_TRY(cudaMemsetAsync(ctx->counters, 0, sizeof(uint32_t) * 12, ctx->stream), "memset");
  CK_TRY(cudaMemsetAsync(ctx->gflag, 0, sizeof(uint32_t) * ctx->cap_vblocks, ctx->stream), "memset");
  CK_TRY(cudaMemsetAsync(ctx->table, 0xff, sizeof(uint32_t) * ctx->cap_vblocks, ctx->stream), "memset");
  CK_TRY(cudaMemsetAsync(ctx->Gacc, 0, sizeof(float4) * ctx->cap_pool * NG * ck::kBlockNodes, ctx->stream), "memset");
  CK_TRY(cudaMemsetAsync(ctx->Gvel, 0, sizeof(float4) * ctx->cap_pool * NG * ck::kBlockNodes, ctx->stream), "memset");
  ctx->scenes.assign(ctx->cap_scenes, SceneHost{});
  ctx->h_scenes.assign(ctx->cap_scenes, SceneDev{});
  ctx->h_mats.assign(ctx->cap_mats, MatDev{});
  ctx->keys_alloc.init(ctx->cap_keys);
  ctx->grid_alloc.init(ctx->cap_vblocks);
  ctx->mat_alloc.init(ctx->cap_mats);
  CK_TRY(cudaEventCreate(&ctx->step_a), "event");
  CK_TRY(cudaEventCreate(&ctx->step_b), "event");
  CK_TRY(cudaGetLastError(), "init");
  return CKMPM_OK;
}

void scene_dims(int res, int64_t& npb, int64_t& nb) {
  npb = ceil_div(res, 4);
  nb = npb + 1;
}

bool capturing(ckmpm_ctx* ctx) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(ctx->stream, &st);
  return st != cudaStreamCaptureStatusNone;
}

void drop_graphs(ckmpm_ctx* ctx) {
  for (auto& g : ctx->gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

// Run a step's launch sequence as the CUDA graph of state parity `key`,
// capturing it on first use; false when the step must be issued directly
// instead (capture is not possible on this stream -- the legacy stream, or
// one the caller is capturing itself -- or it failed; graphs are then off
// for the context and nothing of the sequence has run).
template <typename Issue>
bool graph_step(ckmpm_ctx* ctx, int key, Issue&& issue) {
  if (!ctx->graphs) return false;
  cudaGraphExec_t& ex = ctx->gexec[key];
  if (!ex) {
    if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      ctx->graphs = false;
      return false;
    }
    issue();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (e != cudaSuccess || !g || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      ex = nullptr;
      ctx->graphs = false;
      return false;
    }
    cudaGraphDestroy(g);
  }
  if (cudaGraphLaunch(ex, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    drop_graphs(ctx);
    ctx->graphs = false;
    return false;
  }
  ctx->graph_steps++;
  return true;
}

ckmpm_status run_step_fused(ckmpm_ctx* ctx);

ckmpm_status run_step(ckmpm_ctx* ctx, bool probe) {
  if (ctx->fused && !probe) return run_step_fused(ctx);
  if (ctx->fused) ctx->grid_valid = false;  // a probe reuses the grid arrays
  ck::StepView v = make_view(ctx);
  ckmpm_ctx::EvPair ep{};
  const bool steady = !probe && !ctx->timing && !ctx->grids_dirty && !ctx->keys_dirty;
  if (probe) drop_graphs(ctx);  // the probe refills the block table the graphs were captured with
  if (ctx->grids_dirty) {
    ck::launch_transfer(ctx->kind, ctx->lc, v, ck::LK_CLEAR);
    ctx->grids_dirty = false;
  }
  if (ctx->keys_dirty) {
    CK_TRY(cudaMemsetAsync(ctx->cnt[ctx->cur], 0, sizeof(uint32_t) * v.n_keys, ctx->stream), "memset");
    CK_TRY(cudaMemsetAsync(ctx->bnd[ctx->cur], 0, sizeof(uint32_t) * 2 * v.n_keys, ctx->stream), "memset");
    if (ctx->n_cur > 0)
      ck::launch_rekey(ctx->kind, ctx->stream, ctx->pool[ctx->cur], ctx->key[ctx->cur], ctx->cnt[ctx->cur],
                       ctx->bnd[ctx->cur],
                       ctx->d_scenes, ctx->d_mats, (uint32_t)ctx->n_cur, v.err);
    ctx->keys_dirty = false;
  }
  int64_t n_live = 0;
  for (auto& s : ctx->scenes) n_live += s.alive ? s.n : 0;
  if (n_live == 0) {
    if (!probe) {
      ctx->n_cur = 0;
      ctx->layout.clear();
      ctx->steps++;
      process_pending(ctx);
    }
    CK_TRY(cudaGetLastError(), "step launch");
    return CKMPM_OK;
  }
  ck::BinScratch bs = make_bs(ctx, n_scene_tab(ctx));
  const uint32_t ngb = (uint32_t)std::max<int64_t>(ctx->grid_alloc.high, 1);
  const int grid_ctas = ctx->sm_count * 4;
  // fused contexts keep each table set's assigned entries listed, so that a
  // set is cleared before it is filled again (a probe fills set tsel)
  if (ctx->fused) ck::launch_table_reset(ctx->stream, v.table, v.g_list, v.n_g, v.pool_cap, grid_ctas);
  if (ctx->timing && !probe) cudaEventRecord(ctx->step_a, ctx->stream);
  v.keep_gacc = probe ? 1u : 0u;
  auto issue = [&]() {
  tbeg(ctx, ep, 0);
  ck::launch_bin(ctx->stream, v, bs, ck::LB_SCAN_TILES, ngb, grid_ctas);
  ck::launch_bin(ctx->stream, v, bs, ck::LB_SCAN_TOP, ngb, grid_ctas);
  ck::launch_bin(ctx->stream, v, bs, ck::LB_SCAN_FINAL, ngb, grid_ctas);
  tend(ctx, ep);
  tbeg(ctx, ep, 1);
  ck::launch_bin(ctx->stream, v, bs, ck::LB_SCATTER, ngb, grid_ctas);
  tend(ctx, ep);
  tbeg(ctx, ep, 5);
  ck::launch_bin(ctx->stream, v, bs, ck::LB_GLIST, ngb, grid_ctas);
  tend(ctx, ep);
  tbeg(ctx, ep, 2);
  ck::launch_transfer(ctx->kind, ctx->lc, v, ck::LK_P2G);
  tend(ctx, ep);
  tbeg(ctx, ep, 3);
  ck::launch_transfer(ctx->kind, ctx->lc, v, ck::LK_UPDATE);
  tend(ctx, ep);
  if (probe) return;
  tbeg(ctx, ep, 4);
  ck::launch_transfer(ctx->kind, ctx->lc, v, ck::LK_G2P);
  tend(ctx, ep);
  tbeg(ctx, ep, 6);
  ck::launch_transfer(ctx->kind, ctx->lc, v, ck::LK_G2P_FP64);
  tend(ctx, ep);
  };
  if (!(steady && !ctx->fused && graph_step(ctx, ctx->cur, issue))) issue();
  if (probe) {
    ctx->grids_dirty = true;
    CK_TRY(cudaGetLastError(), "probe launch");
    return CKMPM_OK;
  }
  if (ctx->timing) cudaEventRecord(ctx->step_b, ctx->stream);
  CK_TRY(cudaGetLastError(), "step launch");
  ctx->cur ^= 1;
  // a step that drops released particles changes the pool's count, which the
  // graphs were captured with
  if (ctx->n_cur != n_live) drop_graphs(ctx);
  ctx->n_cur = n_live;
  rebuild_layout_sorted(ctx);
  ctx->steps++;
  process_pending(ctx);
  return CKMPM_OK;
}

// One fused step (CKMPM_STEP_G2P2G).  The grid of the current state (Gvel
// through block-table set tsel) comes from the previous fused step, or from
// a prologue that runs the split path's binning, P2G and grid update when
// the state changed outside a step (admission, release, upload, probe).
// Then: the other table set is cleared of its last use and filled from this
// step's particle blocks (2x2x2 grid blocks each); the fused kernel runs G2P
// and scatters the particles that stayed in their block into that grid; the
// float64 pass; the leftover P2G (claiming any further grid blocks); the grid
// update of the new grid; and the sets swap.
ckmpm_status run_step_fused(ckmpm_ctx* ctx) {
  const bool was_clean = !ctx->grids_dirty && !ctx->keys_dirty && ctx->grid_valid && !ctx->timing;
  if (ctx->grids_dirty) {
    ck::launch_transfer(ctx->kind, ctx->lc, make_view(ctx), ck::LK_CLEAR);
    ctx->grids_dirty = false;
    ctx->grid_valid = false;
  }
  if (ctx->keys_dirty) {
    ck::StepView v = make_view(ctx);
    CK_TRY(cudaMemsetAsync(ctx->cnt[ctx->cur], 0, sizeof(uint32_t) * v.n_keys, ctx->stream), "memset");
    CK_TRY(cudaMemsetAsync(ctx->bnd[ctx->cur], 0, sizeof(uint32_t) * 2 * v.n_keys, ctx->stream), "memset");
    if (ctx->n_cur > 0)
      ck::launch_rekey(ctx->kind, ctx->stream, ctx->pool[ctx->cur], ctx->key[ctx->cur], ctx->cnt[ctx->cur],
                       ctx->bnd[ctx->cur], ctx->d_scenes, ctx->d_mats, (uint32_t)ctx->n_cur, v.err);
    ctx->keys_dirty = false;
    ctx->grid_valid = false;
  }
  int64_t n_live = 0;
  for (auto& s : ctx->scenes) n_live += s.alive ? s.n : 0;
  if (n_live == 0) {
    ctx->n_cur = 0;
    ctx->layout.clear();
    ctx->steps++;
    process_pending(ctx);
    ctx->grid_valid = false;
    CK_TRY(cudaGetLastError(), "step launch");
    return CKMPM_OK;
  }
  ck::BinScratch bs = make_bs(ctx, n_scene_tab(ctx));
  const uint32_t ngb = (uint32_t)std::max<int64_t>(ctx->grid_alloc.high, 1);
  const int grid_ctas = ctx->sm_count * 4;
  const int cs = ctx->tsel, ns = cs ^ 1;
  // views over table set cs (this step's grid) and ns (the next step's)
  ck::StepView vc = make_view(ctx);
  ctx->tsel = ns;
  ck::StepView vn = make_view(ctx);
  ctx->tsel = cs;
  ckmpm_ctx::EvPair ep{};
  if (ctx->timing) cudaEventRecord(ctx->step_a, ctx->stream);
  // the fused kernel gathers through set cs and scatters through set ns
  ck::StepView vf = vc;
  vf.table_nxt = vn.table;
  vf.g_list_nxt = vn.g_list;
  vf.g_scene_nxt = vn.g_scene;
  vf.n_g_nxt = vn.n_g;
  auto issue_fused = [&]() {
    tbeg(ctx, ep, 7);
    ck::launch_transfer(ctx->kind, ctx->lc, vf, ck::LK_G2P2G);
    tend(ctx, ep);
    tbeg(ctx, ep, 6);
    ck::launch_transfer(ctx->kind, ctx->lc, vf, ck::LK_G2P_FP64);
    tend(ctx, ep);
    tbeg(ctx, ep, 2);
    ck::launch_transfer(ctx->kind, ctx->lc, vf, ck::LK_LEFTOVER);
    tend(ctx, ep);
    tbeg(ctx, ep, 3);
    ck::launch_transfer(ctx->kind, ctx->lc, vn, ck::LK_UPDATE);
    tend(ctx, ep);
  };
  // the steady step: the next table set cleared and filled from this step's
  // blocks, then the fused kernel, the float64 pass, the leftover P2G and the
  // grid update
  auto issue_steady = [&]() {
    ck::launch_table_reset(ctx->stream, vn.table, vn.g_list, vn.n_g, vn.pool_cap, grid_ctas);
    tbeg(ctx, ep, 0);
    ck::launch_bin(ctx->stream, vn, bs, ck::LB_SCAN_TILES, ngb, grid_ctas);
    ck::launch_bin(ctx->stream, vn, bs, ck::LB_SCAN_TOP, ngb, grid_ctas);
    ck::launch_bin(ctx->stream, vn, bs, ck::LB_SCAN_FINAL, ngb, grid_ctas);
    tend(ctx, ep);
    tbeg(ctx, ep, 1);
    ck::launch_bin(ctx->stream, vn, bs, ck::LB_SCATTER, ngb, grid_ctas);
    tend(ctx, ep);
    tbeg(ctx, ep, 5);
    ck::launch_bin(ctx->stream, vn, bs, ck::LB_GLIST, ngb, grid_ctas);
    tend(ctx, ep);
    issue_fused();
  };
  if (ctx->grid_valid) {
    if (!(was_clean && graph_step(ctx, ctx->cur + 2 * ctx->tsel, issue_steady))) issue_steady();
  } else {
    // every table set is cleared of the entries its last fill assigned (its
    // list records them, slots claimed by the leftover P2G included) before
    // it is filled again
    ck::launch_table_reset(ctx->stream, vn.table, vn.g_list, vn.n_g, vn.pool_cap, grid_ctas);
    // prologue: binning, P2G and grid update of the current state into set cs
    ck::launch_table_reset(ctx->stream, vc.table, vc.g_list, vc.n_g, vc.pool_cap, grid_ctas);
    ck::launch_bin(ctx->stream, vc, bs, ck::LB_SCAN_TILES, ngb, grid_ctas);
    ck::launch_bin(ctx->stream, vc, bs, ck::LB_SCAN_TOP, ngb, grid_ctas);
    ck::launch_bin(ctx->stream, vc, bs, ck::LB_SCAN_FINAL, ngb, grid_ctas);
    ck::launch_bin(ctx->stream, vc, bs, ck::LB_SCATTER, ngb, grid_ctas);
    ck::launch_bin(ctx->stream, vc, bs, ck::LB_GLIST, ngb, grid_ctas);
    ck::launch_transfer(ctx->kind, ctx->lc, vc, ck::LK_P2G);
    ck::launch_transfer(ctx->kind, ctx->lc, vc, ck::LK_UPDATE);
    // the same particle blocks flag the next step's grid blocks
    CK_TRY(cudaMemsetAsync(vn.n_g, 0, sizeof(uint32_t), ctx->stream), "memset");
    ck::launch_bin(ctx->stream, vn, bs, ck::LB_SCAN_FINAL, ngb, grid_ctas);
    ck::launch_bin(ctx->stream, vn, bs, ck::LB_GLIST, ngb, grid_ctas);
    issue_fused();
    ctx->grid_valid = true;
  }
  if (ctx->timing) cudaEventRecord(ctx->step_b, ctx->stream);
  CK_TRY(cudaGetLastError(), "step launch");
  ctx->cur ^= 1;
  ctx->tsel = ns;
  if (ctx->n_cur != n_live) drop_graphs(ctx);
  ctx->n_cur = n_live;
  rebuild_layout_sorted(ctx);
  ctx->steps++;
  process_pending(ctx);
  return CKMPM_OK;
}

ckmpm_status admit_impl(ckmpm_ctx* ctx, const ckmpm_scene* sc, int* scene_id) {
  ckmpm_status st = validate_scene(ctx, sc);
  if (st != CKMPM_OK) return st;
  if (capturing(ctx)) return fail(ctx, CKMPM_EBUSY, "admission is not allowed during stream capture");
  int64_t npb, nb;
  scene_dims(sc->res, npb, nb);
  const int64_t nkeys = npb * npb * npb, nvb = nb * nb * nb;
  if (ctx->n_cur + sc->n > ctx->cap_n) return fail(ctx, CKMPM_ENOMEM, "particle capacity exceeded");
  int slot = -1;
  for (int s = 0; s < ctx->cap_scenes; ++s)
    if (!ctx->scenes[s].used) {
      slot = s;
      break;
    }
  if (slot < 0) return fail(ctx, CKMPM_ENOMEM, "no free scene slot");
  int64_t kb = ctx->keys_alloc.take(nkeys);
  if (kb < 0) return fail(ctx, CKMPM_ENOMEM, "key-space capacity exceeded");
  int64_t gb = ctx->grid_alloc.take(nvb);
  if (gb < 0) {
    ctx->keys_alloc.give(kb, nkeys);
    return fail(ctx, CKMPM_ENOMEM, "virtual grid-block capacity exceeded");
  }
  int64_t mb = ctx->mat_alloc.take(sc->n_materials);
  if (mb < 0) {
    ctx->keys_alloc.give(kb, nkeys);
    ctx->grid_alloc.give(gb, nvb);
    return fail(ctx, CKMPM_ENOMEM, "material-table capacity exceeded");
  }
  size_t bx = sizeof(float) * 3 * sc->n;
  size_t need = sc->is_device ? 0 : (2 * bx + (size_t)sc->n + 64);
  if (need && !ensure_staging(ctx, need)) {
    ctx->keys_alloc.give(kb, nkeys);
    ctx->grid_alloc.give(gb, nvb);
    ctx->mat_alloc.give(mb, sc->n_materials);
    return fail(ctx, CKMPM_ENOMEM, "staging allocation failed");
  }
  // per-particle E defaults to the material's E; its temporary is taken
  // before the scene is recorded, so that a failure leaves nothing behind
  float* dE = nullptr;
  if (ctx->per_E) {
    std::vector<float> Ehost((size_t)sc->n);
    std::vector<uint8_t> mh;
    auto give_back = [&]() {
      ctx->keys_alloc.give(kb, nkeys);
      ctx->grid_alloc.give(gb, nvb);
      ctx->mat_alloc.give(mb, sc->n_materials);
    };
    if (sc->mat) {
      mh.resize((size_t)sc->n);
      cudaError_t ce = cudaSuccess;
      if (sc->is_device)
        ce = cudaMemcpy(mh.data(), sc->mat, (size_t)sc->n, cudaMemcpyDeviceToHost);
      else
        std::memcpy(mh.data(), sc->mat, (size_t)sc->n);
      if (ce != cudaSuccess) {
        give_back();
        return cuda_fail(ctx, ce, "read mat");
      }
    }
    // the material table is indexed on the host here, so every index is
    // checked before it is used (the kernels check it again on the device)
    for (int64_t i = 0; i < sc->n; ++i) {
      const int mi = sc->mat ? (int)mh[i] : 0;
      if (mi >= sc->n_materials) {
        give_back();
        return fail(ctx, CKMPM_EINVAL,
                    "scene.mat[" + std::to_string(i) + "] = " + std::to_string(mi) + " is not below n_materials");
      }
      Ehost[i] = (float)sc->materials[mi].E;
    }
    dE = (float*)dev_alloc(ctx, sizeof(float) * (size_t)sc->n);
    if (!dE) {
      give_back();
      return fail(ctx, CKMPM_ENOMEM, "allocation failed");
    }
    CK_TRY(cudaMemcpyAsync(dE, Ehost.data(), sizeof(float) * sc->n, cudaMemcpyHostToDevice, ctx->stream), "upload E");
  }
  SceneHost& h = ctx->scenes[slot];
  h.used = true;
  h.alive = true;
  h.n = sc->n;
  h.key_base = kb;
  h.nkeys = nkeys;
  h.table_base = gb;
  h.nvb = nvb;
  h.mat_base = mb;
  h.nmat = sc->n_materials;
  h.res = sc->res;
  SceneDev& d = ctx->h_scenes[slot];
  d.dx = (float)sc->dx;
  d.inv_dx = (float)(1.0 / sc->dx);
  d.dt = (float)sc->dt;
  d.V0 = (float)(sc->dx * sc->dx * sc->dx / sc->ppc);
  d.gx = (float)sc->gravity[0];
  d.gy = (float)sc->gravity[1];
  d.gz = (float)sc->gravity[2];
  d.bc = (float)sc->bc_cells;
  d.res = sc->res;
  d.npb = (int)npb;
  d.nb = (int)nb;
  d.key_base = (uint32_t)kb;
  d.table_base = gb;
  d.j_tol = (float)sc->fp64_j_tol;
  d.cond_tol = (float)sc->fp64_cond_tol;
  d.gap_tol = (float)sc->fp64_gap_tol;
  d.alive = 1;
  const double V0 = sc->dx * sc->dx * sc->dx / sc->ppc;
  double mmax = 0.0;
  for (int i = 0; i < sc->n_materials; ++i) mmax = std::max(mmax, sc->materials[i].rho * V0);
  d.mmax = (float)mmax;
  for (int i = 0; i < sc->n_materials; ++i) {
    const ckmpm_material& m = sc->materials[i];
    MatDev& md = ctx->h_mats[mb + i];
    md.model = m.model;
    md.scene = slot;
    md.mu = (float)(m.E / (2.0 * (1.0 + m.nu)));
    md.lam = (float)(m.E * m.nu / ((1.0 + m.nu) * (1.0 - 2.0 * m.nu)));
    md.mass = (float)(m.rho * V0);
    double s = std::sin(m.friction_deg * M_PI / 180.0);
    md.alpha = (float)(std::sqrt(2.0 / 3.0) * 2.0 * s / (3.0 - s));
    md.dpc = (float)((double)md.alpha * (1.0 + m.nu) / (1.0 - 2.0 * m.nu));
    md.gamma = (float)m.gamma;
    md.E = (float)m.E;
    md.nu = (float)m.nu;
  }
  CK_TRY(cudaMemcpyAsync(ctx->d_scenes + slot, &d, sizeof(SceneDev), cudaMemcpyHostToDevice, ctx->stream), "upload scene");
  CK_TRY(cudaMemcpyAsync(ctx->d_mats + mb, &ctx->h_mats[mb], sizeof(MatDev) * sc->n_materials, cudaMemcpyHostToDevice,
                         ctx->stream),
         "upload materials");
  upload_scene_tab(ctx);
  const float* dx_ = sc->x;
  const float* dv_ = sc->v;
  const uint8_t* dm_ = sc->mat;
  if (!sc->is_device) {
    char* stg = (char*)ctx->staging;
    CK_TRY(cudaMemcpyAsync(stg, sc->x, bx, cudaMemcpyHostToDevice, ctx->stream), "upload x");
    dx_ = (const float*)stg;
    if (sc->v) {
      CK_TRY(cudaMemcpyAsync(stg + bx, sc->v, bx, cudaMemcpyHostToDevice, ctx->stream), "upload v");
      dv_ = (const float*)(stg + bx);
    }
    if (sc->mat) {
      CK_TRY(cudaMemcpyAsync(stg + 2 * bx, sc->mat, (size_t)sc->n, cudaMemcpyHostToDevice, ctx->stream), "upload mat");
      dm_ = (const uint8_t*)(stg + 2 * bx);
    }
  }
  ck::launch_admit(ctx->kind, ctx->stream, ctx->pool[ctx->cur], ctx->key[ctx->cur], ctx->cnt[ctx->cur],
                   ctx->bnd[ctx->cur], ctx->d_scenes, ctx->d_mats, slot, (uint32_t)mb, (uint32_t)sc->n_materials, (uint32_t)ctx->n_cur, (uint32_t)sc->n, dx_, dv_, dm_, dE,
                   ctx->counters + 2);
  CK_TRY(cudaGetLastError(), "admit launch");
  if (dE) {
    CK_TRY(cudaStreamSynchronize(ctx->stream), "sync");
    dev_free(ctx, dE);
  }
  ctx->layout.push_back({slot, ctx->n_cur, sc->n});
  ctx->grid_valid = false;
  drop_graphs(ctx);  // particle count, key space and scene table changed
  ctx->n_cur += sc->n;
  if (scene_id) *scene_id = slot;
  return CKMPM_OK;
}

int64_t field_floats(int field) {
  switch (field) {
    case CKMPM_FIELD_X:
    case CKMPM_FIELD_V:
      return 3;
    case CKMPM_FIELD_B:
    case CKMPM_FIELD_C:
    case CKMPM_FIELD_F:
      return 9;
    case CKMPM_FIELD_E:
      return 1;
    default:
      return 0;
  }
}

}  // namespace

// ============================================================== C ABI

extern "C" {

const char* ckmpm_version(void) { return "ckmpm 0.1 (sm_103a)"; }

ckmpm_status ckmpm_create_server(const ckmpm_config* cfg, ckmpm_ctx** out) {
  if (!out) return CKMPM_EINVAL;
  *out = nullptr;
  if (!cfg) return CKMPM_EINVAL;
  ckmpm_ctx* ctx = new (std::nothrow) ckmpm_ctx();
  if (!ctx) return CKMPM_ENOMEM;
  ckmpm_status st = init_ctx(ctx, cfg);
  if (st != CKMPM_OK) {
    ckmpm_destroy(ctx);
    return st;
  }
  *out = ctx;
  return CKMPM_OK;
}

ckmpm_status ckmpm_create(const ckmpm_scene* scene, int kernel, void* stream, ckmpm_ctx** out) {
  if (!out) return CKMPM_EINVAL;
  *out = nullptr;
  ckmpm_status st = validate_scene(nullptr, scene);
  if (st != CKMPM_OK) return st;
  int64_t npb, nb;
  scene_dims(scene->res, npb, nb);
  ckmpm_config cfg{};
  cfg.kernel = kernel;
  cfg.max_particles = scene->n;
  cfg.max_keys = npb * npb * npb;
  cfg.max_virtual_blocks = nb * nb * nb;
  // pool for the active blocks: a compact scene at 8 particles per cell
  // touches about n/512 blocks per grid; n/64 leaves 8x headroom for spreading
  cfg.max_grid_blocks = std::min<int64_t>(nb * nb * nb, scene->n / 64 + 4096);
  cfg.max_scenes = 1;
  cfg.max_materials = scene->n_materials;
  cfg.per_particle_E = 0;
  cfg.stream = stream;
  ckmpm_ctx* ctx = nullptr;
  st = ckmpm_create_server(&cfg, &ctx);
  if (st != CKMPM_OK) return st;
  int sid = -1;
  st = admit_impl(ctx, scene, &sid);
  if (st != CKMPM_OK) {
    ckmpm_destroy(ctx);
    return st;
  }
  *out = ctx;
  return CKMPM_OK;
}

ckmpm_status ckmpm_admit(ckmpm_ctx* ctx, const ckmpm_scene* scene, int* scene_id) {
  if (!ctx) return CKMPM_EINVAL;
  return admit_impl(ctx, scene, scene_id);
}

ckmpm_status ckmpm_release(ckmpm_ctx* ctx, int scene_id) {
  if (!ctx) return CKMPM_EINVAL;
  if (scene_id < 0 || scene_id >= ctx->cap_scenes || !ctx->scenes[scene_id].alive)
    return fail(ctx, CKMPM_ENOTFOUND, "unknown scene id");
  if (capturing(ctx)) return fail(ctx, CKMPM_EBUSY, "release is not allowed during stream capture");
  SceneHost& h = ctx->scenes[scene_id];
  // retire its particles now (dead keys, cleared histogram range) so that its
  // slot, key range, block table and materials can be reused at once; the
  // particles themselves leave the pool at the next step
  for (size_t i = 0; i < ctx->layout.size(); ++i) {
    if (ctx->layout[i].slot == scene_id) {
      ck::launch_mark_dead(ctx->stream, ctx->key[ctx->cur], (uint32_t)ctx->layout[i].start,
                           (uint32_t)ctx->layout[i].n);
      ctx->layout.erase(ctx->layout.begin() + i);
      break;
    }
  }
  CK_TRY(cudaMemsetAsync(ctx->cnt[ctx->cur] + h.key_base, 0, sizeof(uint32_t) * h.nkeys, ctx->stream), "memset");
  CK_TRY(cudaMemsetAsync(ctx->bnd[ctx->cur] + 2 * h.key_base, 0, sizeof(uint32_t) * 2 * h.nkeys, ctx->stream),
         "memset");
  h.alive = false;
  ctx->grid_valid = false;
  drop_graphs(ctx);
  ctx->h_scenes[scene_id].alive = 0;
  CK_TRY(cudaMemcpyAsync(ctx->d_scenes + scene_id, &ctx->h_scenes[scene_id], sizeof(SceneDev), cudaMemcpyHostToDevice,
                         ctx->stream),
         "upload scene");
  upload_scene_tab(ctx);
  ctx->pending_free.push_back(scene_id);
  process_pending(ctx);
  CK_TRY(cudaGetLastError(), "release");
  return CKMPM_OK;
}

ckmpm_status ckmpm_step(ckmpm_ctx* ctx, int n) {
  if (!ctx) return CKMPM_EINVAL;
  if (n < 0) return fail(ctx, CKMPM_EINVAL, "n must be >= 0");
  if (ctx->sticky != CKMPM_OK) return ctx->sticky;
  for (int i = 0; i < n; ++i) {
    ckmpm_status st = run_step(ctx, false);
    if (st != CKMPM_OK) return st;
  }
  return CKMPM_OK;
}

ckmpm_status ckmpm_probe_grids(ckmpm_ctx* ctx) {
  if (!ctx) return CKMPM_EINVAL;
  if (ctx->sticky != CKMPM_OK) return ctx->sticky;
  return run_step(ctx, true);
}

ckmpm_status ckmpm_sync(ckmpm_ctx* ctx) {
  if (!ctx) return CKMPM_EINVAL;
  CK_TRY(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  return read_device_error(ctx);
}

int64_t ckmpm_scene_particles(const ckmpm_ctx* ctx, int scene_id) {
  if (!ctx || scene_id < 0 || scene_id >= ctx->cap_scenes || !ctx->scenes[scene_id].alive) return -1;
  return ctx->scenes[scene_id].n;
}

}  // extern "C"

namespace {

// Checks a readback request; on success *want is the field's size in bytes
// and *which the grid field to gather (the velocity/mass of the next step's
// grid after a fused step).
ckmpm_status readback_check(ckmpm_ctx* ctx, int scene_id, int field, const void* dst, size_t bytes, size_t* want,
                            int* which) {
  if (!ctx) return CKMPM_EINVAL;
  if (scene_id < 0 || scene_id >= ctx->cap_scenes || !ctx->scenes[scene_id].alive)
    return fail(ctx, CKMPM_ENOTFOUND, "unknown scene id");
  if (!dst) return fail(ctx, CKMPM_EINVAL, "dst is NULL");
  if (capturing(ctx)) return fail(ctx, CKMPM_EBUSY, "readback is not allowed during stream capture");
  const SceneHost& h = ctx->scenes[scene_id];
  const int NG = ctx->kind == 0 ? 2 : 1;
  *want = 0;
  if (field >= CKMPM_FIELD_GRID_M && field <= CKMPM_FIELD_GRID_V) {
    int64_t n = h.res + 1;
    *want = sizeof(float) * (size_t)(NG * n * n * n) * (field == CKMPM_FIELD_GRID_M ? 1 : 3);
  } else {
    int64_t f = field_floats(field);
    if (f == 0) return fail(ctx, CKMPM_EINVAL, "unknown field");
    if (field == CKMPM_FIELD_E && !ctx->per_E) return fail(ctx, CKMPM_EINVAL, "context has no per-particle E");
    *want = sizeof(float) * (size_t)(f * h.n);
  }
  if (bytes != *want) return fail(ctx, CKMPM_EINVAL, "readback size mismatch: expected " + std::to_string(*want));
  // a fused step leaves the next step's grid as velocities and masses only
  // (its grid update consumed the momenta): mass and velocity come from
  // there until a probe replaces them
  *which = field - CKMPM_FIELD_GRID_M;
  if (field >= CKMPM_FIELD_GRID_M && ctx->fused && ctx->grid_valid) {
    if (field == CKMPM_FIELD_GRID_P)
      return fail(ctx, CKMPM_EINVAL, "after a fused step the grid momentum is consumed; probe the grids for it");
    *which = field == CKMPM_FIELD_GRID_M ? 3 : 4;
  }
  return CKMPM_OK;
}

// Enqueues the gather of one field into the device buffer out (want bytes)
// on the context's stream.
ckmpm_status readback_gather(ckmpm_ctx* ctx, int scene_id, int field, int which, size_t want, float* out) {
  if (field >= CKMPM_FIELD_GRID_M) {
    CK_TRY(cudaMemsetAsync(out, 0, want, ctx->stream), "memset");
    ck::launch_read_grid(ctx->kind, ctx->stream, make_view(ctx), scene_id, which, out);
  } else {
    const Seg* sg = find_seg(ctx, scene_id);
    if (!sg) return fail(ctx, CKMPM_EINVAL, "scene has no particles in the pool");
    ck::launch_read_particles(ctx->kind, ctx->transfer == CKMPM_TRANSFER_PIC, ctx->stream, ctx->pool[ctx->cur],
                              ctx->d_scenes, ctx->d_mats, scene_id, (uint32_t)sg->start, (uint32_t)sg->n, field, out);
  }
  CK_TRY(cudaGetLastError(), "readback gather");
  return CKMPM_OK;
}

// The readback slot of a ticket; waits for the slot's last copies first when
// its buffer has to grow.
ckmpm_status readback_slot(ckmpm_ctx* ctx, size_t want, ckmpm_ctx::RbSlot** out) {
  if (!ctx->copy_stream) {
    CK_TRY(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking), "copy stream");
    CK_TRY(cudaEventCreateWithFlags(&ctx->rb_gathered, cudaEventDisableTiming), "readback event");
    for (auto& sl : ctx->rb) {
      CK_TRY(cudaEventCreateWithFlags(&sl.copied, cudaEventDisableTiming), "readback event");
      CK_TRY(cudaHostAlloc((void**)&sl.status, sizeof(uint32_t), cudaHostAllocDefault), "readback status word");
      *sl.status = 0;
    }
  }
  ckmpm_ctx::RbSlot& sl = ctx->rb[ctx->rb_next & 1];
  if (sl.cap < want) {
    if (sl.buf) {
      CK_TRY(cudaEventSynchronize(sl.copied), "readback slot");
      dev_free(ctx, sl.buf);
      sl.buf = nullptr;
      sl.cap = 0;
    }
    sl.buf = dev_alloc(ctx, want);
    if (!sl.buf) return fail(ctx, CKMPM_ENOMEM, "readback staging allocation failed");
    sl.cap = want;
  } else if (sl.ticket >= 0) {
    // the gather must not overwrite the slot while its previous copy runs
    CK_TRY(cudaStreamWaitEvent(ctx->stream, sl.copied, 0), "readback slot");
  }
  *out = &sl;
  return CKMPM_OK;
}

}  // namespace

extern "C" {

ckmpm_status ckmpm_readback_async(ckmpm_ctx* ctx, int scene_id, int field, void* dst, size_t bytes,
                                  int64_t* ticket) {
  if (ticket) *ticket = -1;
  if (!ctx) return CKMPM_EINVAL;
  if (!ticket) return fail(ctx, CKMPM_EINVAL, "ticket is NULL");
  size_t want = 0;
  int which = 0;
  ckmpm_status s = readback_check(ctx, scene_id, field, dst, bytes, &want, &which);
  if (s != CKMPM_OK) return s;
  ckmpm_ctx::RbSlot* sl = nullptr;
  if ((s = readback_slot(ctx, want, &sl)) != CKMPM_OK) return s;
  if ((s = readback_gather(ctx, scene_id, field, which, want, (float*)sl->buf)) != CKMPM_OK) return s;
  CK_TRY(cudaEventRecord(ctx->rb_gathered, ctx->stream), "readback event");
  CK_TRY(cudaStreamWaitEvent(ctx->copy_stream, ctx->rb_gathered, 0), "readback event");
  CK_TRY(cudaMemcpyAsync(dst, sl->buf, want, cudaMemcpyDeviceToHost, ctx->copy_stream), "readback copy");
  CK_TRY(cudaMemcpyAsync(sl->status, ctx->counters + 2, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->copy_stream),
         "readback copy");
  CK_TRY(cudaEventRecord(sl->copied, ctx->copy_stream), "readback event");
  sl->ticket = ctx->rb_next;
  *ticket = ctx->rb_next++;
  return CKMPM_OK;
}

ckmpm_status ckmpm_readback_wait(ckmpm_ctx* ctx, int64_t ticket) {
  if (!ctx) return CKMPM_EINVAL;
  if (ticket < 0 || ticket >= ctx->rb_next) return fail(ctx, CKMPM_EINVAL, "unknown readback ticket");
  // a slot's copies run in ticket order behind its previous ones, so the
  // slot's latest copy completing implies every older ticket of the slot
  ckmpm_ctx::RbSlot& sl = ctx->rb[ticket & 1];
  CK_TRY(cudaEventSynchronize(sl.copied), "readback wait");
  return apply_device_error(ctx, *sl.status);
}

ckmpm_status ckmpm_readback(ckmpm_ctx* ctx, int scene_id, int field, void* dst, size_t bytes, int dst_is_device) {
  if (!ctx) return CKMPM_EINVAL;
  if (!dst_is_device) {
    int64_t t = -1;
    ckmpm_status s = ckmpm_readback_async(ctx, scene_id, field, dst, bytes, &t);
    if (s != CKMPM_OK) return s;
    return ckmpm_readback_wait(ctx, t);
  }
  size_t want = 0;
  int which = 0;
  ckmpm_status s = readback_check(ctx, scene_id, field, dst, bytes, &want, &which);
  if (s != CKMPM_OK) return s;
  if ((s = readback_gather(ctx, scene_id, field, which, want, (float*)dst)) != CKMPM_OK) return s;
  CK_TRY(cudaStreamSynchronize(ctx->stream), "readback");
  return read_device_error(ctx);
}

ckmpm_status ckmpm_upload(ckmpm_ctx* ctx, int scene_id, int field, const void* src, size_t bytes, int src_is_device) {
  if (!ctx) return CKMPM_EINVAL;
  if (scene_id < 0 || scene_id >= ctx->cap_scenes || !ctx->scenes[scene_id].alive)
    return fail(ctx, CKMPM_ENOTFOUND, "unknown scene id");
  if (!src) return fail(ctx, CKMPM_EINVAL, "src is NULL");
  if (capturing(ctx)) return fail(ctx, CKMPM_EBUSY, "upload is not allowed during stream capture");
  if (!(field == CKMPM_FIELD_X || field == CKMPM_FIELD_V || field == CKMPM_FIELD_B || field == CKMPM_FIELD_F ||
        field == CKMPM_FIELD_E))
    return fail(ctx, CKMPM_EINVAL, "field cannot be uploaded");
  if (field == CKMPM_FIELD_E && !ctx->per_E) return fail(ctx, CKMPM_EINVAL, "context has no per-particle E");
  if (field == CKMPM_FIELD_B && ctx->transfer == CKMPM_TRANSFER_PIC) return fail(ctx, CKMPM_EINVAL, "the PIC transfer keeps no B");
  const SceneHost& h = ctx->scenes[scene_id];
  size_t want = sizeof(float) * (size_t)(field_floats(field) * h.n);
  if (bytes != want) return fail(ctx, CKMPM_EINVAL, "upload size mismatch: expected " + std::to_string(want));
  const Seg* sg = find_seg(ctx, scene_id);
  if (!sg) return fail(ctx, CKMPM_EINVAL, "scene has no particles in the pool");
  const float* in = (const float*)src;
  void* tmp = nullptr;
  if (!src_is_device) {
    tmp = dev_alloc(ctx, want);
    if (!tmp) return fail(ctx, CKMPM_ENOMEM, "temporary allocation failed");
    CK_TRY(cudaMemcpyAsync(tmp, src, want, cudaMemcpyHostToDevice, ctx->stream), "upload copy");
    in = (const float*)tmp;
  }
  ck::launch_write_particles(ctx->transfer == CKMPM_TRANSFER_PIC, ctx->stream, ctx->pool[ctx->cur], ctx->d_scenes, ctx->d_mats, scene_id, (uint32_t)sg->start,
                             (uint32_t)sg->n, field, in);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (tmp) dev_free(ctx, tmp);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "upload");
  // keys (positions) or P2G bounds (velocity, M through B, F or E) changed:
  // the next step re-bins the pool first
  ctx->keys_dirty = true;
  drop_graphs(ctx);
  return read_device_error(ctx);
}

ckmpm_status ckmpm_get_stats(ckmpm_ctx* ctx, ckmpm_stats* out) {
  if (!ctx || !out) return CKMPM_EINVAL;
  CK_TRY(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  uint32_t c[12];
  CK_TRY(cudaMemcpy(c, ctx->counters, sizeof(c), cudaMemcpyDeviceToHost), "read counters");
  std::memset(out, 0, sizeof(*out));
  out->n_particles = ctx->n_cur;
  out->n_particle_blocks = c[0];
  out->n_grid_blocks = c[ctx->tsel == 0 ? 1 : 8];
  out->leftover_particles = ctx->fused ? c[9] : 0;
  out->graph_steps = ctx->graph_steps;
  out->steps = ctx->steps;
  unsigned long long f64 = 0;
  std::memcpy(&f64, &c[4], sizeof(f64));
  out->fp64_particles = (int64_t)f64;
  harvest_timing(ctx);
  if (ctx->timing) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->step_a, ctx->step_b) == cudaSuccess) ctx->ms_last_step = ms;
    cudaGetLastError();
  }
  out->ms_last_step = ctx->ms_last_step;
  for (int i = 0; i < 8; ++i) {
    out->ms_kernel[i] = ctx->ms_cnt[i] ? ctx->ms_sum[i] / ctx->ms_cnt[i] : 0.0;
    out->launches_kernel[i] = ctx->ms_cnt[i];
  }
  out->launches_per_step = ctx->fused ? 11 : 9;
  return CKMPM_OK;
}

ckmpm_status ckmpm_set_timing(ckmpm_ctx* ctx, int on) {
  if (!ctx) return CKMPM_EINVAL;
  ctx->timing = on != 0;
  return CKMPM_OK;
}

ckmpm_status ckmpm_reset_timing(ckmpm_ctx* ctx) {
  if (!ctx) return CKMPM_EINVAL;
  CK_TRY(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  harvest_timing(ctx);
  for (int i = 0; i < 8; ++i) {
    ctx->ms_sum[i] = 0;
    ctx->ms_cnt[i] = 0;
  }
  return CKMPM_OK;
}

ckmpm_status ckmpm_destroy(ckmpm_ctx* ctx) {
  if (!ctx) return CKMPM_OK;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  drop_graphs(ctx);
  harvest_timing(ctx);
  for (auto& e : ctx->ev_free) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  if (ctx->step_a) cudaEventDestroy(ctx->step_a);
  if (ctx->step_b) cudaEventDestroy(ctx->step_b);
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    for (auto& sl : ctx->rb) {
      if (sl.copied) cudaEventDestroy(sl.copied);
      if (sl.status) cudaFreeHost(sl.status);
    }
    if (ctx->rb_gathered) cudaEventDestroy(ctx->rb_gathered);
    cudaStreamDestroy(ctx->copy_stream);
  }
  while (!ctx->allocs.empty()) dev_free(ctx, ctx->allocs.back().first);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  cudaGetLastError();
  delete ctx;
  return CKMPM_OK;
}

const char* ckmpm_last_error(const ckmpm_ctx* ctx) {
  if (!ctx) return "no context";
  return ctx->msg.empty() ? "no error" : ctx->msg.c_str();
}

}  // extern "C"
