// Per-step particle binning by particle block (counting sort on block keys).
//
// The histogram of the keys is produced by the previous G2P (or by admission
// / re-keying).  One step then runs:
//   scan_tiles  per 4096-key tile: particle count and non-empty key count
//   scan_top    one CTA: exclusive scan over tiles; resets per-step counters
//   scan_final  per non-empty key: offset and scatter cursor; non-empty keys
//               become the particle-block list (in key order, so the list is
//               deterministic) and flag the 2x2x2 grid blocks they touch
// (G2P clears each histogram entry it has used, so the buffer it fills next
// step starts at zero without a pass over the whole key space.)
//   scatter     perm[cursor[key]++] = particle (warp-aggregated atomics)
//   glist       flagged grid blocks -> active grid-block list; flags cleared
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "launch.h"

namespace ck {

constexpr int kScanThreads = 256;
constexpr int kPerThread = kScanTile / kScanThreads;  // 16

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(StepView v, BinScratch bs) {
  const uint32_t base = blockIdx.x * kScanTile;
  uint32_t c = 0, ne = 0;
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) {
    uint32_t k = base + q * kScanThreads + threadIdx.x;
    if (k < v.n_keys) {
      uint32_t x = v.cnt_cur[k];
      c += x;
      ne += x ? 1u : 0u;
    }
  }
  __shared__ uint32_t sc[kScanThreads / 32], sn[kScanThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_down_sync(0xffffffffu, c, o);
    ne += __shfl_down_sync(0xffffffffu, ne, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sc[threadIdx.x >> 5] = c;
    sn[threadIdx.x >> 5] = ne;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tc = 0, tn = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
      tc += sc[w];
      tn += sn[w];
    }
    bs.tile_cnt[blockIdx.x] = tc;
    bs.tile_ne[blockIdx.x] = tn;
  }
}

// Exclusive scan of (tile_cnt, tile_ne) in place by one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_top(StepView v, BinScratch bs, uint32_t ntiles) {
  __shared__ uint32_t wc[32], wn[32];
  __shared__ uint32_t carry_c, carry_n;
  if (threadIdx.x == 0) {
    carry_c = 0;
    carry_n = 0;
    *v.n_g = 0;
    *v.fp64_count = 0ull;
    v.work[0] = 0u;
    v.work[1] = 0u;
    if (v.lo_count) *v.lo_count = 0u;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t b0 = 0; b0 < ntiles; b0 += 1024) {
    uint32_t i = b0 + threadIdx.x;
    uint32_t c = i < ntiles ? bs.tile_cnt[i] : 0u;
    uint32_t n = i < ntiles ? bs.tile_ne[i] : 0u;
    uint32_t ic = c, in = n;  // inclusive within warp
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t yc = __shfl_up_sync(0xffffffffu, ic, o);
      uint32_t yn = __shfl_up_sync(0xffffffffu, in, o);
      if (lane >= o) {
        ic += yc;
        in += yn;
      }
    }
    if (lane == 31) {
      wc[warp] = ic;
      wn[warp] = in;
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t xc = wc[lane], xn = wn[lane];
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t yc = __shfl_up_sync(0xffffffffu, xc, o);
        uint32_t yn = __shfl_up_sync(0xffffffffu, xn, o);
        if (lane >= o) {
          xc += yc;
          xn += yn;
        }
      }
      wc[lane] = xc;
      wn[lane] = xn;
    }
    __syncthreads();
    uint32_t pc = (warp ? wc[warp - 1] : 0u) + ic - c + carry_c;
    uint32_t pn = (warp ? wn[warp - 1] : 0u) + in - n + carry_n;
    if (i < ntiles) {
      bs.tile_cnt[i] = pc;
      bs.tile_ne[i] = pn;
    }
    __syncthreads();
    if (threadIdx.x == 1023) {
      carry_c = pc + c;
      carry_n = pn + n;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *v.n_pb = carry_n;
}

__device__ __forceinline__ int scene_of_key(const BinScratch& bs, uint32_t key) {
  int lo = 0, hi = bs.n_scene_tab - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (bs.scene_tab[2 * mid] <= key)
      lo = mid;
    else
      hi = mid - 1;
  }
  return (int)bs.scene_tab[2 * lo + 1];
}

__global__ void __launch_bounds__(kScanThreads) k_scan_final(StepView v, BinScratch bs) {
  const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kPerThread;
  uint32_t c[kPerThread];
  uint32_t tc = 0, tn = 0;
  if (base + kPerThread <= v.n_keys) {  // 16 consecutive counts as four 16-byte loads
    const uint4* p4 = reinterpret_cast<const uint4*>(v.cnt_cur + base);
#pragma unroll
    for (int q = 0; q < kPerThread / 4; ++q) {
      const uint4 x = p4[q];
      c[4 * q] = x.x;
      c[4 * q + 1] = x.y;
      c[4 * q + 2] = x.z;
      c[4 * q + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) c[q] = base + q < v.n_keys ? v.cnt_cur[base + q] : 0u;
  }
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) {
    tc += c[q];
    tn += c[q] ? 1u : 0u;
  }
  // block-wide exclusive scan of (tc, tn)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t ic = tc, in = tn;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t yc = __shfl_up_sync(0xffffffffu, ic, o);
    uint32_t yn = __shfl_up_sync(0xffffffffu, in, o);
    if (lane >= o) {
      ic += yc;
      in += yn;
    }
  }
  __shared__ uint32_t wc[kScanThreads / 32], wn[kScanThreads / 32];
  if (lane == 31) {
    wc[warp] = ic;
    wn[warp] = in;
  }
  __syncthreads();
  uint32_t pc = bs.tile_cnt[blockIdx.x], pn = bs.tile_ne[blockIdx.x];
  for (int w = 0; w < warp; ++w) {
    pc += wc[w];
    pn += wn[w];
  }
  pc += ic - tc;
  pn += in - tn;
  // the owning scene of the thread's keys, looked up once and kept in
  // registers while the keys stay inside its key range (the stores below
  // could alias the scene table, so reading it per key reloads it each time)
  int sl = -1, npb = 1, nb = 1;
  uint32_t klo = 1u;
  uint64_t khi = 0u;
  long long tbase = 0;
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) {
    uint32_t k = base + q;
    if (k >= v.n_keys) break;
    if (c[q]) {
      v.offset[k] = pc;
      v.cursor[k] = pc;
      if (!(k >= klo && (uint64_t)k < khi)) {
        sl = scene_of_key(bs, k);
        const SceneDev& s = v.scenes[sl];
        klo = s.key_base;
        npb = s.npb;
        nb = s.nb;
        tbase = s.table_base;
        khi = (uint64_t)klo + (uint64_t)npb * (uint64_t)npb * (uint64_t)npb;
      }
      v.pb_key[pn] = k;
      v.pb_scene[pn] = (uint32_t)sl;
      int lb = (int)(k - klo);
      int bx = lb % npb, by = (lb / npb) % npb, bz = lb / (npb * npb);
      for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
          for (int dx = 0; dx < 2; ++dx)
            v.gflag[tbase + ((long long)(bz + dz) * nb + (by + dy)) * nb + (bx + dx)] = (uint32_t)sl + 1u;
      pn += 1;
    }
    pc += c[q];
  }
}

// Each warp handles kScatterUnroll groups of 32 particles per pass and issues
// the cursor atomics of all of them before it waits for the first result: the
// pass is one atomic round trip instead of kScatterUnroll.
constexpr int kScatterUnroll = 8;

__global__ void __launch_bounds__(256) k_scatter(StepView v) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t stride = gridDim.x * blockDim.x * kScatterUnroll;
  // the loop runs on the warp's first index, so every lane of a warp takes
  // the same iterations (the full-mask warp intrinsics below need that)
  for (uint32_t w0 = blockIdx.x * blockDim.x * kScatterUnroll + (threadIdx.x - lane) * kScatterUnroll;
       w0 < v.n_cur; w0 += stride) {
    const uint32_t j0 = w0 + lane;
    uint32_t key[kScatterUnroll], peers[kScatterUnroll], base[kScatterUnroll];
#pragma unroll
    for (int u = 0; u < kScatterUnroll; ++u) {
      const uint32_t j = j0 + 32u * u;
      key[u] = j < v.n_cur ? v.key_cur[j] : CK_DEAD_KEY;
    }
#pragma unroll
    for (int u = 0; u < kScatterUnroll; ++u) {
      peers[u] = __match_any_sync(0xffffffffu, key[u]);
      base[u] = 0u;
      if (key[u] != CK_DEAD_KEY && (int)lane == __ffs(peers[u]) - 1)
        base[u] = atomicAdd(&v.cursor[key[u]], (uint32_t)__popc(peers[u]));
    }
#pragma unroll
    for (int u = 0; u < kScatterUnroll; ++u) {
      const uint32_t b = __shfl_sync(0xffffffffu, base[u], __ffs(peers[u]) - 1);
      if (key[u] != CK_DEAD_KEY) v.perm[b + __popc(peers[u] & ((1u << lane) - 1u))] = j0 + 32u * u;
    }
  }
}

// Flagged virtual blocks get pool slots in list order; the block table maps
// each of them to its slot.  Entries of untouched blocks are stale and never
// read (P2G/G2P only look up the blocks their own particle block flagged).
// A warp reads 32 x 4 flags with one 16-byte load per lane; a warp scan of
// the lanes' flag counts and one atomic per warp give every flagged block its
// slot.  The tail (fewer than four flags) and an unaligned array are read one
// flag at a time.
__device__ __forceinline__ void glist_assign(const StepView& v, uint32_t g, uint32_t f, uint32_t idx) {
  if (idx < v.pool_cap) {
    v.g_list[idx] = g;
    v.g_scene[idx] = f - 1u;
    v.table[g] = idx;
  } else {
    v.table[g] = CK_NO_SLOT;
    flag_error(v.err, CK_ERR_POOL);
  }
  v.gflag[g] = 0u;
}

__global__ void k_glist(StepView v, uint32_t n_vblocks) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n4 = (reinterpret_cast<uintptr_t>(v.gflag) & 15u) ? 0u : n_vblocks / 4u;
  const uint4* f4 = reinterpret_cast<const uint4*>(v.gflag);
  const uint32_t wstride = gridDim.x * blockDim.x;
  // every lane of a warp runs the same iterations (full-mask intrinsics)
  for (uint32_t q0 = blockIdx.x * blockDim.x + (threadIdx.x - lane); q0 < n4; q0 += wstride) {
    const uint32_t q = q0 + lane;
    const uint4 f = q < n4 ? f4[q] : make_uint4(0u, 0u, 0u, 0u);
    const uint32_t nf = (f.x != 0u) + (f.y != 0u) + (f.z != 0u) + (f.w != 0u);
    if (__ballot_sync(0xffffffffu, nf != 0u) == 0u) continue;
    uint32_t inc = nf;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if ((int)lane >= o) inc += y;
    }
    uint32_t start = 0u;
    if (lane == 31u) start = atomicAdd(v.n_g, inc);
    start = __shfl_sync(0xffffffffu, start, 31);
    uint32_t idx = start + inc - nf;
    if (f.x) glist_assign(v, 4u * q, f.x, idx++);
    if (f.y) glist_assign(v, 4u * q + 1u, f.y, idx++);
    if (f.z) glist_assign(v, 4u * q + 2u, f.z, idx++);
    if (f.w) glist_assign(v, 4u * q + 3u, f.w, idx++);
  }
  for (uint32_t g = 4u * n4 + blockIdx.x * blockDim.x + threadIdx.x; g < n_vblocks; g += wstride) {
    const uint32_t f = v.gflag[g];
    if (f) glist_assign(v, g, f, atomicAdd(v.n_g, 1u));
  }
}

// Fused step: before a block table is filled again, the entries its last
// use assigned (the first *n_g entries of its list, slots claimed by the
// leftover P2G included) go back to CK_NO_SLOT, so that every entry not
// assigned in this step reads as unassigned.
__global__ void k_table_reset(uint32_t* table, const uint32_t* g_list, const uint32_t* n_g, uint32_t pool_cap) {
  const uint32_t n = min(*n_g, pool_cap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    table[g_list[i]] = CK_NO_SLOT;
}

void launch_table_reset(cudaStream_t st, uint32_t* table, const uint32_t* g_list, const uint32_t* n_g,
                        uint32_t pool_cap, int grid_ctas) {
  k_table_reset<<<grid_ctas, 256, 0, st>>>(table, g_list, n_g, pool_cap);
}

// Retire particles [start, start + n) of the current pool (a released scene):
// they get the dead key and leave the pool at the next step.
__global__ void k_mark_dead(uint32_t* key, uint32_t start, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    key[start + i] = CK_DEAD_KEY;
}

void launch_mark_dead(cudaStream_t st, uint32_t* key, uint32_t start, uint32_t n) {
  int blocks = (int)((n + 255) / 256);
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  k_mark_dead<<<blocks, 256, 0, st>>>(key, start, n);
}

void launch_bin(cudaStream_t st, const StepView& v, const BinScratch& bs, int which, uint32_t n_gblocks,
                int grid_ctas) {
  uint32_t ntiles = (v.n_keys + kScanTile - 1) / kScanTile;
  if (ntiles == 0) ntiles = 1;
  switch (which) {
    case LB_SCAN_TILES: k_scan_tiles<<<ntiles, kScanThreads, 0, st>>>(v, bs); break;
    case LB_SCAN_TOP: k_scan_top<<<1, 1024, 0, st>>>(v, bs, ntiles); break;
    case LB_SCAN_FINAL: k_scan_final<<<ntiles, kScanThreads, 0, st>>>(v, bs); break;
    case LB_SCATTER: k_scatter<<<grid_ctas, 256, 0, st>>>(v); break;
    case LB_GLIST: k_glist<<<grid_ctas, 256, 0, st>>>(v, n_gblocks); break;
  }
}

}  // namespace ck
