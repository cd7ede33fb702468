// Device-side data layout and helpers shared by the CK-MPM kernels.
//
// Particle pool (structure of arrays, double-buffered, 16-byte vectors):
//   X   float4 (x, y, z, material index as bits)
//   VM0 float4 (vx, vy, vz, M00)   VM1 (M01, M02, M10, M11)   VM2 (M12, M20, M21, M22)
//   F0  float4 (F00, F01, F02, F10)  F1 (F11, F12, F20, F21)  F2 float F22
//   ID  uint32 scene-local particle index
// M = m B - dt V0 tau(F) is the per-particle matrix that P2G multiplies by
// D(x)^-1: it carries both the APIC affine momentum (Sec. 4.4) and the MLS
// stress force (Sec. 4.3.2 with reading R4).  Storing M instead of B lets P2G
// run without an SVD; B is recovered exactly as (M + dt V0 tau(F)) / m.
//
// Sparse grid: each scene's domain is a virtual array of 4x4x4-node blocks;
// a block table maps the blocks touched this step to slots of a compact pool
// (slot = position in the active-block list, reassigned every step).  Per
// pool slot and grid 64 float4:
//   Gacc  (m, p_x, p_y, p_z) accumulated by P2G, zeroed by the grid update
//   Gvel  (v~_x, v~_y, v~_z, m) written by the grid update, gathered by G2P
// CK uses two grids per block (0: G-, 1: G+), quadratic one.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define CK_ERR_DOMAIN 1u
#define CK_ERR_NONFINITE 2u
#define CK_ERR_INTERNAL 4u
#define CK_ERR_TIMEOUT 8u
#define CK_ERR_POOL 16u
#define CK_NO_SLOT 0xFFFFFFFFu

#define CK_DEAD_KEY 0xFFFFFFFFu

namespace ck {

constexpr int kBlock = 4;        // nodes / cells per block edge
constexpr int kBlockNodes = 64;  // nodes per block and grid

struct SceneDev {
  float dx, inv_dx, dt, V0;
  float gx, gy, gz;
  float bc;           // sticky wall thickness in cells
  int res;            // cells per axis
  int npb;            // particle blocks per axis = ceil(res/4)
  int nb;             // grid blocks per axis = npb + 1
  uint32_t key_base;  // first particle-block key of this scene
  long long table_base;  // first entry of this scene's block table
  float j_tol, cond_tol, gap_tol;  // float64 SVD criteria
  float mmax;         // largest particle mass of the scene's materials
  int alive;
};

struct MatDev {
  int model;      // 0 fixed-corotated, 1 Drucker-Prager, 2 J-based fluid
  int scene;      // owning scene slot
  float mu, lam;  // Lame parameters
  float mass;     // rho * V0
  float alpha;    // Drucker-Prager cone coefficient
  float dpc;      // Drucker-Prager: (3 lam + 2 mu) / (2 mu) alpha = alpha (1 + nu) / (1 - 2 nu), any E
  float E, nu;    // for per-particle E; the fluid's equation-of-state constant B is E
  float gamma;    // fluid equation-of-state exponent
};

// Pointers to one buffer of the particle pool.
struct Pool {
  float4* X;
  float4* VM0;
  float4* VM1;
  float4* VM2;
  float4* F0;
  float4* F1;
  float* F2;
  uint32_t* ID;
  float* E;  // optional per-particle Young's modulus (may be null)
  // APIC with the kernel gradient only (else null): T = -dt V0 tau, row-major
  // in T0 (T00, T01, T02, T10), T1 (T11, T12, T20, T21), T2 T22; VM then
  // holds m B without the stress
  float4* T0;
  float4* T1;
  float* T2;
};

// Everything the per-step kernels read; passed by value.
struct StepView {
  Pool cur, nxt;
  uint32_t* key_cur;    // keys of cur (input of the sort)
  uint32_t* key_nxt;    // keys written by G2P for nxt
  uint32_t* cnt_cur;    // histogram of key_cur over the key space
  uint32_t* cnt_nxt;    // histogram written by G2P (all zero before it: G2P clears cnt_cur after use)
  uint32_t* bnd_cur;    // per key: P2G contribution bounds (mass, momentum) of cur, float
                        // bits; P2G clears an active block's pair after use
  uint32_t* bnd_nxt;    // the same for nxt, written by G2P (all zero before it)
  uint32_t* offset;     // exclusive scan of cnt_cur
  uint32_t* cursor;     // scatter cursors
  uint32_t* perm;       // sorted slot -> index into cur
  uint32_t* pb_key;     // non-empty particle blocks: key
  uint32_t* pb_scene;   // and owning scene
  uint32_t* n_pb;       // number of non-empty particle blocks
  uint32_t* gflag;      // per virtual grid block: scene+1 if touched this step
  uint32_t* table;      // per virtual grid block: pool slot (valid if touched this step)
  uint32_t* g_list;     // pool slot -> virtual grid block
  uint32_t* g_scene;    // pool slot -> owning scene
  uint32_t* n_g;        // number of active grid blocks (may exceed pool_cap on overflow)
  uint32_t pool_cap;    // pool capacity in blocks
  float4* Gacc;
  float4* Gvel;
  const SceneDev* scenes;
  const MatDev* mats;
  uint32_t* err;
  unsigned long long* fp64_count;  // particles listed for the float64 pass this step
  uint32_t* fp64_list;  // their slots in nxt (capacity: the pool)
  uint32_t* work;       // [0] next P2G block, [1] next G2P block (dynamic scheduling)
  uint32_t n_keys;      // size of the key space
  uint32_t n_cur;       // particles in cur (including dead ones)
  uint32_t keep_gacc;   // probe: the grid update leaves Gacc, P2G keeps bnd_cur
  uint32_t splits;      // work units per particle block of the transfer kernels (>= 1)
  uint32_t n_mats;      // entries of the material table
  // fused G2P2G step only (else null): the block table of the next step's
  // grid (the gather reads Gvel through `table`, the scatter adds to Gacc
  // through these), and the list of particles the fused kernel leaves to the
  // leftover P2G (changed block, float64 pass, non-finite)
  uint32_t* table_nxt;
  uint32_t* g_list_nxt;
  uint32_t* g_scene_nxt;
  uint32_t* n_g_nxt;
  uint32_t* lo_list;
  uint32_t* lo_count;
};

__device__ __forceinline__ void flag_error(uint32_t* err, uint32_t bit) { atomicOr(err, bit); }

// Work unit u of the transfer kernels: particle block u / splits, part
// u % splits of its particles, in whole chunks of `align` particles (a step
// with few blocks splits each over several units so that every resident
// warp gets work).  Returns false when that part is empty.
__device__ __forceinline__ bool unit_range(const StepView& v, uint32_t u, uint32_t align, uint32_t& bi,
                                           uint32_t& lo, uint32_t& hi) {
  const uint32_t S = v.splits;
  bi = u / S;
  const uint32_t part = u - bi * S;
  const uint32_t cnt = v.cnt_cur[v.pb_key[bi]];
  const uint32_t per = ((cnt + S - 1) / S + align - 1) / align * align;
  lo = part * per;
  hi = min(cnt, lo + per);
  return lo < hi;
}

// Cell decomposition shared by every kernel that maps a position to nodes.
// u0 = x/dx.  CK: t = u0 + 1/4, b+ = floor(t), f+ = t - b+ (exact when dx is a
// power of two), b- = b+ or b+ - 1 with f- = f+ -+ 1/2 (Sec. 4.2 offsets).
// The particle block is floor(b-/4) for CK (G- blocks are the reference
// blocks, Sec. 5.1) and floor(base/4) for the quadratic stencil.
template <int KIND>
struct Cell;

template <>
struct Cell<0> {
  int bp, bm;   // base node on G+ and G-
  float fp, fm; // fractions in [0,1)
  __device__ __forceinline__ void set(float u0) {
    float t = u0 + 0.25f;
    float fb = floorf(t);
    bp = (int)fb;
    fp = t - fb;
    if (fp >= 0.5f) {
      bm = bp;
      fm = fp - 0.5f;
    } else {
      bm = bp - 1;
      fm = fp + 0.5f;
    }
  }
  __device__ __forceinline__ int block() const { return bm >> 2; }
};

template <>
struct Cell<1> {
  int b;
  float f;  // in [0.5, 1.5)
  __device__ __forceinline__ void set(float u0) {
    float t = u0 - 0.5f;
    float fb = floorf(t);
    b = (int)fb;
    f = u0 - fb;
  }
  __device__ __forceinline__ int block() const { return b >> 2; }
};

// Valid interior for both stencils: 0.5 <= x/dx < res - 0.5.
__device__ __forceinline__ bool in_domain(float u, int res) {
  return u >= 0.5f && u < (float)res - 0.5f;
}

template <int KIND>
__device__ __forceinline__ uint32_t particle_key(const SceneDev& s, float ux, float uy, float uz) {
  Cell<KIND> cx, cy, cz;
  cx.set(ux);
  cy.set(uy);
  cz.set(uz);
  int bx = cx.block(), by = cy.block(), bz = cz.block();
  return s.key_base + (uint32_t)((bz * s.npb + by) * s.npb + bx);
}

__device__ __forceinline__ uint32_t warp_aggregated_inc(uint32_t* counters, uint32_t key) {
  // lanes with equal keys add once
  unsigned mask = __activemask();
  unsigned peers = __match_any_sync(mask, key);
  int leader = __ffs(peers) - 1;
  int lane = threadIdx.x & 31;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&counters[key], (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

// Histogram increment and P2G contribution bounds of particles binned under
// `key` (lanes with equal keys add once).  The bounds are non-negative floats
// kept as bit patterns (whose unsigned order is the float order); each warp
// contributes the largest bound over all its active lanes, which may only
// overestimate a block's bound.
__device__ __forceinline__ void warp_aggregated_bin(uint32_t* cnt, uint32_t* bnd, uint32_t key, float bmass,
                                                    float bmom) {
  const unsigned mask = __activemask();
  const uint32_t bm = __reduce_max_sync(mask, __float_as_uint(bmass));
  const uint32_t bp = __reduce_max_sync(mask, __float_as_uint(bmom));
  const unsigned peers = __match_any_sync(mask, key);
  if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) {
    atomicAdd(&cnt[key], (uint32_t)__popc(peers));
    atomicMax(&bnd[2 * key], bm);
    atomicMax(&bnd[2 * key + 1], bp);
  }
}

__device__ __forceinline__ bool finite4(float4 a) {
  return isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(a.w);
}

}  // namespace ck
