// P2G, grid update and fused G2P + constitutive kernels of the CK-MPM step,
// for the compact kernel on the dual grid (KIND 0) and the quadratic
// B-spline comparison path (KIND 1).
//
// One CTA works on one particle block (4x4x4 cells of the reference grid G-,
// Sec. 5.1) at a time and loops over the block list (persistent grid-stride
// launch over all resident scenes).  The nodes that the block's particles can
// touch are staged in shared memory:
//   CK:  G- nodes [4P, 4P+4]^3 (125) and G+ nodes [4P, 4P+5]^3 (216) = 341
//   quadratic: nodes [4P, 4P+5]^3 = 216
// P2G accumulates there with shared-memory atomics and flushes each touched
// node once with a 16-byte global atomic; G2P gathers from the staged copy.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "launch.h"
#include "svd3.cuh"

namespace ck {

constexpr float kInv2Pi = 0.15915494309189535f;

// Asynchronous global -> shared copies: a CTA issues the gathers of a whole
// chunk of particles before it waits for any.  The 16-byte copies stream
// through L2 only (.cg), so that the particle stream does not evict the small
// tables every particle reads through L1 (materials, scenes, block lists).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Material tables of up to this many entries are staged in shared memory by
// the transfer kernels (one copy per CTA).
constexpr int kSmemMats = 8;

// sin(2 pi f) for f in [0, 1): reduce to t = f - rint(f) in [-1/2, 1/2], fold
// |t| > 1/4 with sin(2 pi t) = sin(2 pi (sign(t)/2 - t)) (both steps exact in
// float), then the Taylor series of sin x at x = 2 pi t, |x| <= pi/2, through
// x^11: coefficients (-1)^k (2 pi)^(2k+1) / (2k+1)!, truncation error below
// (pi/2)^13 / 13! = 1.5e-8, about 1.6e-7 after float rounding.
__device__ __forceinline__ float sin_2pi(float f) {
  float t = f - rintf(f);
  const float h = copysignf(0.5f, t) - t;
  t = fabsf(t) > 0.25f ? h : t;
  const float t2 = t * t;
  float p = -15.094642576822984f;
  p = fmaf(p, t2, 42.058693944897634f);
  p = fmaf(p, t2, -76.70585975306136f);
  p = fmaf(p, t2, 81.60524927607504f);
  p = fmaf(p, t2, -41.341702240399755f);
  p = fmaf(p, t2, 6.283185307179586f);
  return t * p;
}

// cos(2 pi f) for f in [0, 1): the reduction of sin_2pi, where the fold
// t -> sign(t)/2 - t flips the cosine's sign, then the Taylor series of cos x
// at x = 2 pi t, |x| <= pi/2, through x^12: coefficients
// (-1)^k (2 pi)^(2k) / (2k)!, truncation error below (pi/2)^14 / 14! = 6.4e-9.
__device__ __forceinline__ float cos_2pi(float f) {
  float t = f - rintf(f);
  const float h = copysignf(0.5f, t) - t;
  const bool fold = fabsf(t) > 0.25f;
  t = fold ? h : t;
  const float t2 = t * t;
  float p = 7.903536371318465f;
  p = fmaf(p, t2, -26.426256783374388f);
  p = fmaf(p, t2, 60.24464137187664f);
  p = fmaf(p, t2, -85.45681720669371f);
  p = fmaf(p, t2, 64.93939402266828f);
  p = fmaf(p, t2, -19.739208802178716f);
  p = fmaf(p, t2, 1.0f);
  return fold ? -p : p;
}

// 1/x for a normal float x: the hardware approximation refined by one
// Newton-Raphson step e = 1 - x y, y <- y + y e (the classical iteration for
// the reciprocal; the error after one step is about the square of the
// approximation's, below one ulp).  No special-case branches: callers pass
// values bounded away from 0 and infinity.
__device__ __forceinline__ float rcp_nr(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  const float e = fmaf(-x, y, 1.0f);
  return fmaf(y, e, y);
}

template <int KIND>
struct Geo;
template <>
struct Geo<0> {
  static constexpr int NG = 2;
  static constexpr int E0 = 5, E1 = 6;
  static constexpr int N0 = 125;
  static constexpr int NS = 341;
  static constexpr float half = 0.5f;
};
template <>
struct Geo<1> {
  static constexpr int NG = 1;
  static constexpr int E0 = 6, E1 = 6;
  static constexpr int N0 = 216;
  static constexpr int NS = 216;
  static constexpr float half = 1.0f;
};

// staged index -> (slot, local node coordinates)
template <int KIND>
__device__ __forceinline__ void staged_coords(int j, int& slot, int& lx, int& ly, int& lz) {
  constexpr int E0 = Geo<KIND>::E0;
  if (j < Geo<KIND>::N0) {
    slot = 0;
    lx = j % E0;
    ly = (j / E0) % E0;
    lz = j / (E0 * E0);
  } else {
    j -= Geo<KIND>::N0;
    slot = 1;
    lx = j % 6;
    ly = (j / 6) % 6;
    lz = j / 36;
  }
}

// Pool index of a staged node (grid g, local coordinates relative to the
// particle block's origin 4P) from the pool slots of the 2x2x2 grid blocks
// the particle block touches; -1 if that block has no slot (pool overflow).
template <int KIND>
__device__ __forceinline__ long long pool_index(const uint32_t* bslot, int g, int lx, int ly, int lz) {
  uint32_t sl = bslot[((lz >> 2) * 2 + (ly >> 2)) * 2 + (lx >> 2)];
  if (sl == CK_NO_SLOT) return -1;
  int l = ((lz & 3) * 4 + (ly & 3)) * 4 + (lx & 3);
  return ((long long)sl * Geo<KIND>::NG + g) * kBlockNodes + l;
}

// Slots of the 2x2x2 grid blocks touched by particle block (bx, by, bz).
__device__ __forceinline__ void load_block_slots(const StepView& v, const SceneDev& s, int ox, int oy, int oz,
                                                 uint32_t* bslot) {
  if (threadIdx.x < 8) {
    int t = threadIdx.x;
    int bx = (ox >> 2) + (t & 1), by = (oy >> 2) + ((t >> 1) & 1), bz = (oz >> 2) + (t >> 2);
    bslot[t] = v.table[s.table_base + ((long long)bz * s.nb + by) * s.nb + bx];
  }
}

// ------------------------------------------------------------------ stencils

// Weights, node offsets (x_i - x_p in cells) and D^-1 (cells^-2) of one
// particle.  CK: K1 weights on both grids from one sine per axis
// (sin 2 pi f- = -sin 2 pi f+), D = Lambda + s s^T with the closed form
// Lambda_a = (m2(f+) + m2(f-))/2 - s_a^2, s_a = sin(2 pi f+_a)/(2 pi),
// inverted by Sherman-Morrison.  Quadratic: B-spline weights, D^-1 = 4 I.
template <int KIND>
struct Sten;

template <>
struct Sten<0> {
  int r[2][3];        // base node of each slot relative to the block origin
  float w[2][3][2];   // per slot, axis, node
  float d[2][3][2];
  float li[3], y[3], den;  // D^-1 = diag(li) - den y y^T (cells^-2)
  float k[2][3][2];        // PIC transfer: K1'(d) per slot, axis, node (set_grad)
  __device__ __forceinline__ bool set(float ux, float uy, float uz, int ox, int oy, int oz) {
    float u[3] = {ux, uy, uz};
    int o[3] = {ox, oy, oz};
    float s[3], lam[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Cell<0> c;
      c.set(u[a]);
      r[0][a] = c.bm - o[a];
      r[1][a] = c.bp - o[a];
      ok = ok && (unsigned)r[0][a] <= 3u;  // then the G+ base, r[0][a] or r[0][a] + 1, is in [0, 4]
      float sg = sin_2pi(c.fp) * kInv2Pi;
      w[1][a][0] = 1.0f - c.fp + sg;
      w[1][a][1] = c.fp - sg;
      d[1][a][0] = -c.fp;
      d[1][a][1] = 1.0f - c.fp;
      w[0][a][0] = 1.0f - c.fm - sg;
      w[0][a][1] = c.fm + sg;
      d[0][a][0] = -c.fm;
      d[0][a][1] = 1.0f - c.fm;
      float m2p = c.fp * (1.0f - c.fp) - sg * (1.0f - 2.0f * c.fp);
      float m2m = c.fm * (1.0f - c.fm) + sg * (1.0f - 2.0f * c.fm);
      lam[a] = 0.5f * (m2p + m2m) - sg * sg;
      s[a] = sg;
    }
    // Lambda_a in [0.0826, 0.1586] and 1 + s^T Lambda^-1 s in [1, 1.3]
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      li[a] = rcp_nr(lam[a]);
      y[a] = li[a] * s[a];
    }
    den = rcp_nr(1.0f + s[0] * y[0] + s[1] * y[1] + s[2] * y[2]);
    return ok;
  }
  // K1'(x) = sgn(x) (cos(2 pi |x|) - 1) at the node offsets d = -f, 1 - f:
  // with c = cos(2 pi f+), 1 - c and c - 1 on G+; cos(2 pi f-) = -c, so
  // 1 + c and -1 - c on G-.  Each pair sums to 0 (the weights sum to 1).
  __device__ __forceinline__ void set_grad() {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float c = cos_2pi(-d[1][a][0]);
      k[1][a][0] = 1.0f - c;
      k[1][a][1] = c - 1.0f;
      k[0][a][0] = 1.0f + c;
      k[0][a][1] = -1.0f - c;
    }
  }
};

template <>
struct Sten<1> {
  int r[3];
  float w[3][3];
  float d[3][3];
  float k[3][3];  // PIC transfer: N'(d) per axis, node (set_grad)
  __device__ __forceinline__ bool set(float ux, float uy, float uz, int ox, int oy, int oz) {
    float u[3] = {ux, uy, uz};
    int o[3] = {ox, oy, oz};
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Cell<1> c;
      c.set(u[a]);
      r[a] = c.b - o[a];
      ok = ok && (unsigned)r[a] <= 3u;
      float f = c.f;
      w[a][0] = 0.5f * (1.5f - f) * (1.5f - f);
      w[a][1] = 0.75f - (f - 1.0f) * (f - 1.0f);
      w[a][2] = 0.5f * (f - 0.5f) * (f - 0.5f);
      d[a][0] = -f;
      d[a][1] = 1.0f - f;
      d[a][2] = 2.0f - f;
    }
    return ok;
  }
  // N'(x) of the quadratic B-spline at d = -f, 1 - f, 2 - f (f in [1/2, 3/2)):
  // 3/2 - f, 2 (f - 1), 1/2 - f.
  __device__ __forceinline__ void set_grad() {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float f = -d[a][0];
      k[a][0] = 1.5f - f;
      k[a][1] = 2.0f * (f - 1.0f);
      k[a][2] = 0.5f - f;
    }
  }
};

// Visit every (node, weight, offset) of a stencil: fn(staged_index, w, dx, dy, dz).
template <typename Fn>
__device__ __forceinline__ void for_nodes(const Sten<0>& st, Fn&& fn) {
#pragma unroll
  for (int slot = 0; slot < 2; ++slot) {
    const int E = slot == 0 ? 5 : 6;
    const int base = slot == 0 ? 0 : 125;
#pragma unroll
    for (int sz = 0; sz < 2; ++sz)
#pragma unroll
      for (int sy = 0; sy < 2; ++sy) {
        float wyz = st.w[slot][1][sy] * st.w[slot][2][sz];
        int row = base + ((st.r[slot][2] + sz) * E + (st.r[slot][1] + sy)) * E + st.r[slot][0];
#pragma unroll
        for (int sx = 0; sx < 2; ++sx)
          fn(row + sx, st.w[slot][0][sx] * wyz, st.d[slot][0][sx], st.d[slot][1][sy], st.d[slot][2][sz]);
      }
  }
}

template <typename Fn>
__device__ __forceinline__ void for_nodes(const Sten<1>& st, Fn&& fn) {
#pragma unroll
  for (int sz = 0; sz < 3; ++sz)
#pragma unroll
    for (int sy = 0; sy < 3; ++sy) {
      float wyz = st.w[1][sy] * st.w[2][sz];
      int row = ((st.r[2] + sz) * 6 + (st.r[1] + sy)) * 6 + st.r[0];
#pragma unroll
      for (int sx = 0; sx < 3; ++sx) fn(row + sx, st.w[0][sx] * wyz, st.d[0][sx], st.d[1][sy], st.d[2][sz]);
    }
}

// Kernel-gradient transfers: visit every (node, weight, kernel-derivative
// products, offsets) of a stencil, fn(staged_index, w, gx, gy, gz, dx, dy, dz)
// with w = Kx Ky Kz and g = (K'x Ky Kz, Kx K'y Kz, Kx Ky K'z), so that
// grad w = -g / dx (the gradient with respect to the particle position), and
// d the node offset in cells.  Needs set_grad().
template <typename Fn>
__device__ __forceinline__ void for_nodes_grad(const Sten<0>& st, Fn&& fn) {
#pragma unroll
  for (int slot = 0; slot < 2; ++slot) {
    const int E = slot == 0 ? 5 : 6;
    const int base = slot == 0 ? 0 : 125;
#pragma unroll
    for (int sz = 0; sz < 2; ++sz)
#pragma unroll
      for (int sy = 0; sy < 2; ++sy) {
        const float wyz = st.w[slot][1][sy] * st.w[slot][2][sz];
        const float kyz = st.k[slot][1][sy] * st.w[slot][2][sz];
        const float ykz = st.w[slot][1][sy] * st.k[slot][2][sz];
        const int row = base + ((st.r[slot][2] + sz) * E + (st.r[slot][1] + sy)) * E + st.r[slot][0];
#pragma unroll
        for (int sx = 0; sx < 2; ++sx) {
          const float wx = st.w[slot][0][sx];
          fn(row + sx, wx * wyz, st.k[slot][0][sx] * wyz, wx * kyz, wx * ykz, st.d[slot][0][sx], st.d[slot][1][sy],
             st.d[slot][2][sz]);
        }
      }
  }
}

template <typename Fn>
__device__ __forceinline__ void for_nodes_grad(const Sten<1>& st, Fn&& fn) {
#pragma unroll
  for (int sz = 0; sz < 3; ++sz)
#pragma unroll
    for (int sy = 0; sy < 3; ++sy) {
      const float wyz = st.w[1][sy] * st.w[2][sz];
      const float kyz = st.k[1][sy] * st.w[2][sz];
      const float ykz = st.w[1][sy] * st.k[2][sz];
      const int row = ((st.r[2] + sz) * 6 + (st.r[1] + sy)) * 6 + st.r[0];
#pragma unroll
      for (int sx = 0; sx < 3; ++sx) {
        const float wx = st.w[0][sx];
        fn(row + sx, wx * wyz, st.k[0][sx] * wyz, wx * kyz, wx * ykz, st.d[0][sx], st.d[1][sy], st.d[2][sz]);
      }
    }
}

// G2P gather as a tensor-product contraction (a node's weight is the product
// of per-axis weights): over one grid's N^3 stencil, S = sum w v~ and the
// first moments M_a = sum w v~ s_a (s_a in 0..N-1: the node's offset in the
// stencil along axis a), reducing x, then y, then z.  With x_i - x_p =
// (s - f) dx per axis, sum w v~ (x_i - x_p)_a / dx = M_a - f_a S.  sv holds
// the staged nodes with row pitch E; base is the stencil's first node.
template <int N, int E>
__device__ __forceinline__ void gather_moments(const float4* sv, int base, const float* wx, const float* wy,
                                               const float* wz, float* S, float* Mx, float* My, float* Mz) {
#pragma unroll
  for (int sz = 0; sz < N; ++sz) {
    float Ps[3], Px[3], Py[3];
#pragma unroll
    for (int sy = 0; sy < N; ++sy) {
      float Rs[3], Rx[3];
      const int row = base + (sz * E + sy) * E;
#pragma unroll
      for (int sx = N - 1; sx >= 0; --sx) {
        const float4 a = sv[row + sx];
        const float t[3] = {wx[sx] * a.x, wx[sx] * a.y, wx[sx] * a.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (sx == N - 1) {
            Rs[c] = t[c];
            Rx[c] = (float)sx * t[c];
          } else {
            Rs[c] += t[c];
            if (sx > 0) Rx[c] = fmaf((float)sx, t[c], Rx[c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float u = wy[sy] * Rs[c];
        if (sy == 0) {
          Ps[c] = u;
          Px[c] = wy[sy] * Rx[c];
        } else {
          Ps[c] += u;
          Px[c] = fmaf(wy[sy], Rx[c], Px[c]);
          Py[c] = sy == 1 ? u : fmaf((float)sy, u, Py[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float u = wz[sz] * Ps[c];
      if (sz == 0) {
        S[c] = u;
        Mx[c] = wz[sz] * Px[c];
        My[c] = wz[sz] * Py[c];
      } else {
        S[c] += u;
        Mx[c] = fmaf(wz[sz], Px[c], Mx[c]);
        My[c] = fmaf(wz[sz], Py[c], My[c]);
        Mz[c] = sz == 1 ? u : fmaf((float)sz, u, Mz[c]);
      }
    }
  }
}

// v = h sum w v~ and Bh = h sum w v~ (x_i - x_p)^T / dx (row c, column a) over
// the particle's stencil; h = 1/2 averages the two CK grids.  Every sum is
// linear in the z weights, so h is applied to those (four products) instead
// of to the twelve results; scaling by a power of two is exact, so the
// results are the same bits.
__device__ __forceinline__ void g2p_gather(const Sten<0>& st, const float4* sv, float* vel, float* Bh) {
  float S[2][3], M[2][3][3];
  const float hz0[2] = {0.5f * st.w[0][2][0], 0.5f * st.w[0][2][1]};
  const float hz1[2] = {0.5f * st.w[1][2][0], 0.5f * st.w[1][2][1]};
  gather_moments<2, 5>(sv, (st.r[0][2] * 5 + st.r[0][1]) * 5 + st.r[0][0], st.w[0][0], st.w[0][1], hz0, S[0],
                       M[0][0], M[0][1], M[0][2]);
  gather_moments<2, 6>(sv, 125 + (st.r[1][2] * 6 + st.r[1][1]) * 6 + st.r[1][0], st.w[1][0], st.w[1][1], hz1,
                       S[1], M[1][0], M[1][1], M[1][2]);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    vel[c] = S[0][c] + S[1][c];
#pragma unroll
    for (int a = 0; a < 3; ++a)  // f_a = -d[g][a][0]
      Bh[c * 3 + a] = fmaf(st.d[0][a][0], S[0][c], M[0][a][c]) + fmaf(st.d[1][a][0], S[1][c], M[1][a][c]);
  }
}

__device__ __forceinline__ void g2p_gather(const Sten<1>& st, const float4* sv, float* vel, float* Bh) {
  float S[3], M[3][3];
  gather_moments<3, 6>(sv, (st.r[2] * 6 + st.r[1]) * 6 + st.r[0], st.w[0], st.w[1], st.w[2], S, M[0], M[1], M[2]);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    vel[c] = S[c];
#pragma unroll
    for (int a = 0; a < 3; ++a) Bh[c * 3 + a] = fmaf(st.d[a][0], S[c], M[a][c]);
  }
}

// PIC transfer: S = sum w v~ and the derivative sums G_a = sum g_a v~ over one
// grid's N^3 stencil (g as in for_nodes_grad), by the same x, y, z reduction
// as gather_moments with the kernel derivative in place of the offset.
template <int N, int E>
__device__ __forceinline__ void gather_grad(const float4* sv, int base, const float* wx, const float* wy,
                                            const float* wz, const float* kx, const float* ky, const float* kz,
                                            float* S, float* Gx, float* Gy, float* Gz) {
#pragma unroll
  for (int sz = 0; sz < N; ++sz) {
    float Ps[3], Px[3], Py[3];
#pragma unroll
    for (int sy = 0; sy < N; ++sy) {
      float Rs[3], Rx[3];
      const int row = base + (sz * E + sy) * E;
#pragma unroll
      for (int sx = 0; sx < N; ++sx) {
        const float4 a = sv[row + sx];
        const float t[3] = {a.x, a.y, a.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Rs[c] = sx == 0 ? wx[sx] * t[c] : fmaf(wx[sx], t[c], Rs[c]);
          Rx[c] = sx == 0 ? kx[sx] * t[c] : fmaf(kx[sx], t[c], Rx[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Ps[c] = sy == 0 ? wy[sy] * Rs[c] : fmaf(wy[sy], Rs[c], Ps[c]);
        Px[c] = sy == 0 ? wy[sy] * Rx[c] : fmaf(wy[sy], Rx[c], Px[c]);
        Py[c] = sy == 0 ? ky[sy] * Rs[c] : fmaf(ky[sy], Rs[c], Py[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      S[c] = sz == 0 ? wz[sz] * Ps[c] : fmaf(wz[sz], Ps[c], S[c]);
      Gx[c] = sz == 0 ? wz[sz] * Px[c] : fmaf(wz[sz], Px[c], Gx[c]);
      Gy[c] = sz == 0 ? wz[sz] * Py[c] : fmaf(wz[sz], Py[c], Gy[c]);
      Gz[c] = sz == 0 ? kz[sz] * Ps[c] : fmaf(kz[sz], Ps[c], Gz[c]);
    }
  }
}

// PIC transfer: v = h sum w v~ and Gr = h sum v~ g^T (row c, column a), so
// that grad v = -Gr / dx; h = 1/2 averages the two CK grids.  Needs set_grad().
__device__ __forceinline__ void g2p_gather_grad(const Sten<0>& st, const float4* sv, float* vel, float* Gr) {
  float S[2][3], D[2][3][3];
  gather_grad<2, 5>(sv, (st.r[0][2] * 5 + st.r[0][1]) * 5 + st.r[0][0], st.w[0][0], st.w[0][1], st.w[0][2],
                    st.k[0][0], st.k[0][1], st.k[0][2], S[0], D[0][0], D[0][1], D[0][2]);
  gather_grad<2, 6>(sv, 125 + (st.r[1][2] * 6 + st.r[1][1]) * 6 + st.r[1][0], st.w[1][0], st.w[1][1], st.w[1][2],
                    st.k[1][0], st.k[1][1], st.k[1][2], S[1], D[1][0], D[1][1], D[1][2]);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    vel[c] = 0.5f * (S[0][c] + S[1][c]);
#pragma unroll
    for (int a = 0; a < 3; ++a) Gr[c * 3 + a] = 0.5f * (D[0][a][c] + D[1][a][c]);
  }
}

__device__ __forceinline__ void g2p_gather_grad(const Sten<1>& st, const float4* sv, float* vel, float* Gr) {
  float S[3], D[3][3];
  gather_grad<3, 6>(sv, (st.r[2] * 6 + st.r[1]) * 6 + st.r[0], st.w[0], st.w[1], st.w[2], st.k[0], st.k[1],
                    st.k[2], S, D[0], D[1], D[2]);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    vel[c] = S[c];
#pragma unroll
    for (int a = 0; a < 3; ++a) Gr[c * 3 + a] = D[a][c];
  }
}

// R = scale Q D^-1 for a row-major 3x3 Q.  CK: D^-1 = diag(li) - den y y^T,
// so each row costs one dot product with y and three fused updates instead of
// a full 3x3 product; quadratic: D^-1 = 4 I.
__device__ __forceinline__ void mul_dinv(const Sten<0>& st, const float* Q, float scale, float* R) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float t = (Q[r * 3] * st.y[0] + Q[r * 3 + 1] * st.y[1] + Q[r * 3 + 2] * st.y[2]) * st.den;
#pragma unroll
    for (int q = 0; q < 3; ++q) R[r * 3 + q] = scale * (Q[r * 3 + q] * st.li[q] - t * st.y[q]);
  }
}
__device__ __forceinline__ void mul_dinv(const Sten<1>&, const float* Q, float scale, float* R) {
#pragma unroll
  for (int q = 0; q < 9; ++q) R[q] = (4.0f * scale) * Q[q];
}

__device__ __forceinline__ void decode_block(const SceneDev& s, uint32_t key, int& ox, int& oy, int& oz) {
  int lb = (int)(key - s.key_base);
  int bx = lb % s.npb;
  int by = (lb / s.npb) % s.npb;
  int bz = lb / (s.npb * s.npb);
  ox = bx * 4;
  oy = by * 4;
  oz = bz * 4;
}

// ------------------------------------------------------------------------ P2G

// Shared-memory accumulation is in 32-bit fixed point: integer shared
// atomics run about 4x faster than float ones on this part (measured), and
// integer sums do not depend on the order of the atomics.  A first pass over
// the block's particles bounds every contribution each can make (p2g_bound,
// from the largest weight, weight times offset and row sum of D^-1 of the
// stencil), so with cnt particles no node sum can exceed cnt times the
// block's largest bound, and the scale maps that to 2^30 (no overflow).
// Rounding costs at most half a unit per contribution, cnt * bound * 2^-31.

// P2G runs one warp per CTA and streams a block's particles through shared
// memory in chunks of kP2GStage (cp.async gathers through the binned order,
// all in flight together); lanes take a chunk's particles C = kP2GStage / 32
// apart (C odd), so each quarter-warp's 16-byte reads fall on distinct bank
// groups and neighbouring lanes come from different cells.
constexpr int kP2GWarp = 32;
constexpr int kP2GStage = 96;  // 3 * 32

struct P2GPart {
  float4 X, a, b, c;
};

// Per-stencil bounds of one P2G contribution w (m v + A^ d) (d: node offset
// in cells); wmax and the product wd * dinv keep a margin of at least 0.3%
// over the exact maxima for float rounding:
//   wmax  largest node weight: CK 1 (K1(0)); quadratic 0.75^3;
//   wd    largest |w d_a|: max over one axis of |d| K(|d|) times the largest
//         weight of the other two: CK 0.27751 (at |d| = 0.394) x 1;
//         quadratic 0.25 (at |d| = 1/2) x 0.75^2 = 0.140625;
//   dinv  largest row abs-sum of D^-1 in cells^-2: CK 14.04 (over a 121^3
//         grid of fractions), quadratic 4 (D^-1 = 4 I).
template <int KIND>
struct P2GBound;
template <>
struct P2GBound<0> {
  static constexpr float wmax = 1.003f;
  static constexpr float wd = 0.2785f;
  static constexpr float dinv = 14.5f;
};
template <>
struct P2GBound<1> {
  static constexpr float wmax = 0.4232f;
  static constexpr float wd = 0.1411f;
  static constexpr float dinv = 4.0f;
};

// Bound of |w (m v + A^ d)|_inf over every node a particle touches:
// wmax m |v|_inf + wd * dinv * max_row sum_k |M_rk| / dx, since
// |w (A^ d)_r| <= sum_k |A^_rk| |w d_k| and the rows of A^ = M D^-1 / dx sum
// to at most sum_j |M_rj| * dinv / dx.
// The PIC transfer's contribution w m v + M grad w (M = -dt V0 tau) has the
// same bound with wd * dinv replaced by the largest |g_a| of for_nodes_grad:
// CK 2 (|K1'| <= 2, at |x| = 1/2, times weights <= 1), quadratic 0.5625
// (|N'| <= 1 times 0.75^2); both are below wd * dinv (4.04 and 0.5644), so
// one bound serves every transfer.  APIC with the kernel gradient keeps m B
// and T = -dt V0 tau apart and passes |m B| + |T| (elementwise) as M.
// The particle's two bounds (mass, momentum) go into its block's entry of
// the per-key bound table when it is binned (G2P for the next step, admission
// and re-keying otherwise), so P2G reads a block's bounds without a pass over
// its particles.
template <int KIND>
__device__ __forceinline__ void p2g_bounds(float inv_dx, float mass, float vx, float vy, float vz, const float* M,
                                           float& bmass, float& bmom) {
  const float r0 = fabsf(M[0]) + fabsf(M[1]) + fabsf(M[2]);
  const float r1 = fabsf(M[3]) + fabsf(M[4]) + fabsf(M[5]);
  const float r2 = fabsf(M[6]) + fabsf(M[7]) + fabsf(M[8]);
  const float rm = fmaxf(r0, fmaxf(r1, r2));
  bmass = P2GBound<KIND>::wmax * mass;
  bmom = bmass * fmaxf(fabsf(vx), fmaxf(fabsf(vy), fabsf(vz))) +
         P2GBound<KIND>::wd * P2GBound<KIND>::dinv * rm * inv_dx;
}

// FMA: a block of at least kP2GFmaCount particles has every scaled
// contribution within 2^30 / count <= 2^22 in magnitude, where one fused
// multiply-add with 1.5 * 2^23 rounds w * (...) to the nearest integer in the
// low mantissa bits (the sum lies in [2^23, 2^24), whose spacing is 1): the
// integer is the float's bits minus those of 1.5 * 2^23.  That takes the
// conversion off the XU pipe; smaller blocks convert with __float2int_rn.
constexpr uint32_t kP2GFmaCount = 256;

template <bool FMA>
__device__ __forceinline__ int p2g_fixed(float w, float val) {
  if constexpr (FMA)
    return __float_as_int(fmaf(w, val, 12582912.0f)) - 0x4B400000;
  else
    return __float2int_rn(w * val);
}

template <int KIND, bool FMA = false>
__device__ __forceinline__ void p2g_scatter(const SceneDev& s, const MatDev* mats, uint32_t* err, const P2GPart& q,
                                            int ox, int oy, int oz, float Sm, float Sp, int (*sm)[Geo<KIND>::NS]) {
  Sten<KIND> st;
  if (!st.set(q.X.x * s.inv_dx, q.X.y * s.inv_dx, q.X.z * s.inv_dx, ox, oy, oz)) {
    flag_error(err, CK_ERR_INTERNAL);
    return;
  }
  const float M[9] = {q.a.w, q.b.x, q.b.y, q.b.z, q.b.w, q.c.x, q.c.y, q.c.z, q.c.w};
  // A^ = M D^-1 / dx so that A (x_i - x_p) = A^ (offset in cells), pre-scaled
  float A[9];
  mul_dinv(st, M, s.inv_dx * Sp, A);
  const float mass = mats[__float_as_uint(q.X.w)].mass;
  const float ms = mass * Sm;
  const float px = mass * q.a.x * Sp, py = mass * q.a.y * Sp, pz = mass * q.a.z * Sp;
  for_nodes(st, [&](int j, float w, float dx, float dy, float dz) {
    atomicAdd(&sm[0][j], p2g_fixed<FMA>(w, ms));
    atomicAdd(&sm[1][j], p2g_fixed<FMA>(w, px + A[0] * dx + A[1] * dy + A[2] * dz));
    atomicAdd(&sm[2][j], p2g_fixed<FMA>(w, py + A[3] * dx + A[4] * dy + A[5] * dz));
    atomicAdd(&sm[3][j], p2g_fixed<FMA>(w, pz + A[6] * dx + A[7] * dy + A[8] * dz));
  });
}

// The same sums with the four components issued in a lane-rotated order.
// A shared atomic instruction costs about the largest number of its lanes
// that fall in one bank, and lanes on one address count like lanes on
// distinct addresses of that bank: about three lanes of an instruction share
// a cell and so every node of the stencil.  Here the instruction of slot c
// (c = 0..3) adds component (c + rot) & 3, rot = (3 lane) & 3, so
// neighbouring lanes of one cell write different planes (plane stride
// kP2GRotPlane, 24 banks apart).  Every component is written as
// w (R0 + R1 dx + R2 dy + R3 dz) with the rows R of the mass (m, 0, 0, 0) and
// of the momenta (p_c, row c of A^); the lane's rows are permuted once per
// particle by two selects each, so no register array is indexed at run
// time.  pl[c] is the plane that instruction slot c writes.
template <int KIND>
struct P2GRotPlane {
  static constexpr int value = ((Geo<KIND>::NS + 7) / 32) * 32 + 24;  // >= NS, = 24 mod 32
};

template <int KIND, bool FMA = false>
__device__ __forceinline__ void p2g_scatter_rot(const SceneDev& s, const MatDev* mats, uint32_t* err,
                                                const P2GPart& q, int ox, int oy, int oz, float Sm, float Sp,
                                                int* const* pl, uint32_t rot) {
  Sten<KIND> st;
  if (!st.set(q.X.x * s.inv_dx, q.X.y * s.inv_dx, q.X.z * s.inv_dx, ox, oy, oz)) {
    flag_error(err, CK_ERR_INTERNAL);
    return;
  }
  const float M[9] = {q.a.w, q.b.x, q.b.y, q.b.z, q.b.w, q.c.x, q.c.y, q.c.z, q.c.w};
  float A[9];
  mul_dinv(st, M, s.inv_dx * Sp, A);
  const float mass = mats[__float_as_uint(q.X.w)].mass;
  const float R[4][4] = {{mass * Sm, 0.f, 0.f, 0.f},
                         {mass * q.a.x * Sp, A[0], A[1], A[2]},
                         {mass * q.a.y * Sp, A[3], A[4], A[5]},
                         {mass * q.a.z * Sp, A[6], A[7], A[8]}};
  const bool r1 = (rot & 1u) != 0u, r2 = (rot & 2u) != 0u;
  float T[4][4], Q[4][4];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e) T[c][e] = r1 ? R[(c + 1) & 3][e] : R[c][e];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e) Q[c][e] = r2 ? T[(c + 2) & 3][e] : T[c][e];
  if constexpr (KIND == 0) {
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int E = g == 0 ? 5 : 6;
      const int jb = (g == 0 ? 0 : 125) + (st.r[g][2] * E + st.r[g][1]) * E + st.r[g][0];
      int* const b0 = pl[0] + jb;
      int* const b1 = pl[1] + jb;
      int* const b2 = pl[2] + jb;
      int* const b3 = pl[3] + jb;
#pragma unroll
      for (int sz = 0; sz < 2; ++sz)
#pragma unroll
        for (int sy = 0; sy < 2; ++sy) {
          const float wyz = st.w[g][1][sy] * st.w[g][2][sz];
          const float dy = st.d[g][1][sy], dz = st.d[g][2][sz];
          float e[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) e[c] = fmaf(Q[c][3], dz, fmaf(Q[c][2], dy, Q[c][0]));
#pragma unroll
          for (int sx = 0; sx < 2; ++sx) {
            const int o = (sz * E + sy) * E + sx;
            const float w = st.w[g][0][sx] * wyz;
            const float dx = st.d[g][0][sx];
            atomicAdd(b0 + o, p2g_fixed<FMA>(w, fmaf(Q[0][1], dx, e[0])));
            atomicAdd(b1 + o, p2g_fixed<FMA>(w, fmaf(Q[1][1], dx, e[1])));
            atomicAdd(b2 + o, p2g_fixed<FMA>(w, fmaf(Q[2][1], dx, e[2])));
            atomicAdd(b3 + o, p2g_fixed<FMA>(w, fmaf(Q[3][1], dx, e[3])));
          }
        }
    }
  } else {
    const int jb = (st.r[2] * 6 + st.r[1]) * 6 + st.r[0];
    int* const b0 = pl[0] + jb;
    int* const b1 = pl[1] + jb;
    int* const b2 = pl[2] + jb;
    int* const b3 = pl[3] + jb;
#pragma unroll
    for (int sz = 0; sz < 3; ++sz)
#pragma unroll
      for (int sy = 0; sy < 3; ++sy) {
        const float wyz = st.w[1][sy] * st.w[2][sz];
        const float dy = st.d[1][sy], dz = st.d[2][sz];
        float e[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) e[c] = fmaf(Q[c][3], dz, fmaf(Q[c][2], dy, Q[c][0]));
#pragma unroll
        for (int sx = 0; sx < 3; ++sx) {
          const int o = (sz * 6 + sy) * 6 + sx;
          const float w = st.w[0][sx] * wyz;
          const float dx = st.d[0][sx];
          atomicAdd(b0 + o, p2g_fixed<FMA>(w, fmaf(Q[0][1], dx, e[0])));
          atomicAdd(b1 + o, p2g_fixed<FMA>(w, fmaf(Q[1][1], dx, e[1])));
          atomicAdd(b2 + o, p2g_fixed<FMA>(w, fmaf(Q[2][1], dx, e[2])));
          atomicAdd(b3 + o, p2g_fixed<FMA>(w, fmaf(Q[3][1], dx, e[3])));
        }
      }
  }
}

// PIC transfer (Sec. 4.3 with the kernel gradient): the state holds
// M = -dt V0 tau (B = 0), and a node receives w m v + M grad w with
// grad w = -g / dx, i.e. w m v + A g with A = -M / dx, pre-scaled.
template <int KIND>
__device__ __forceinline__ void p2g_scatter_pic(const SceneDev& s, const MatDev* mats, uint32_t* err,
                                                const P2GPart& q, int ox, int oy, int oz, float Sm, float Sp,
                                                int (*sm)[Geo<KIND>::NS]) {
  Sten<KIND> st;
  if (!st.set(q.X.x * s.inv_dx, q.X.y * s.inv_dx, q.X.z * s.inv_dx, ox, oy, oz)) {
    flag_error(err, CK_ERR_INTERNAL);
    return;
  }
  st.set_grad();
  const float M[9] = {q.a.w, q.b.x, q.b.y, q.b.z, q.b.w, q.c.x, q.c.y, q.c.z, q.c.w};
  const float sc = -s.inv_dx * Sp;
  float A[9];
#pragma unroll
  for (int r = 0; r < 9; ++r) A[r] = sc * M[r];
  const float mass = mats[__float_as_uint(q.X.w)].mass;
  const float ms = mass * Sm;
  const float px = mass * q.a.x * Sp, py = mass * q.a.y * Sp, pz = mass * q.a.z * Sp;
  for_nodes_grad(st, [&](int j, float w, float gx, float gy, float gz, float, float, float) {
    atomicAdd(&sm[0][j], __float2int_rn(w * ms));
    atomicAdd(&sm[1][j], __float2int_rn(fmaf(w, px, A[0] * gx + A[1] * gy + A[2] * gz)));
    atomicAdd(&sm[2][j], __float2int_rn(fmaf(w, py, A[3] * gx + A[4] * gy + A[5] * gz)));
    atomicAdd(&sm[3][j], __float2int_rn(fmaf(w, pz, A[6] * gx + A[7] * gy + A[8] * gz)));
  });
}

// APIC with the kernel gradient: M = m B (state), T = -dt V0 tau (separate
// arrays); a node receives w (m v + A d) + G g with A = m B D^-1 / dx (the
// APIC momentum) and G = -T / dx (the force), both pre-scaled.
template <int KIND>
__device__ __forceinline__ void p2g_scatter_grad(const SceneDev& s, const MatDev* mats, uint32_t* err,
                                                 const P2GPart& q, const float* T, int ox, int oy, int oz, float Sm,
                                                 float Sp, int (*sm)[Geo<KIND>::NS]) {
  Sten<KIND> st;
  if (!st.set(q.X.x * s.inv_dx, q.X.y * s.inv_dx, q.X.z * s.inv_dx, ox, oy, oz)) {
    flag_error(err, CK_ERR_INTERNAL);
    return;
  }
  st.set_grad();
  const float M[9] = {q.a.w, q.b.x, q.b.y, q.b.z, q.b.w, q.c.x, q.c.y, q.c.z, q.c.w};
  float A[9], G[9];
  mul_dinv(st, M, s.inv_dx * Sp, A);
  const float sc = -s.inv_dx * Sp;
#pragma unroll
  for (int r = 0; r < 9; ++r) G[r] = sc * T[r];
  const float mass = mats[__float_as_uint(q.X.w)].mass;
  const float ms = mass * Sm;
  const float px = mass * q.a.x * Sp, py = mass * q.a.y * Sp, pz = mass * q.a.z * Sp;
  for_nodes_grad(st, [&](int j, float w, float gx, float gy, float gz, float dx, float dy, float dz) {
    atomicAdd(&sm[0][j], __float2int_rn(w * ms));
    atomicAdd(&sm[1][j], __float2int_rn(fmaf(w, px + A[0] * dx + A[1] * dy + A[2] * dz,
                                             G[0] * gx + G[1] * gy + G[2] * gz)));
    atomicAdd(&sm[2][j], __float2int_rn(fmaf(w, py + A[3] * dx + A[4] * dy + A[5] * dz,
                                             G[3] * gx + G[4] * gy + G[5] * gz)));
    atomicAdd(&sm[3][j], __float2int_rn(fmaf(w, pz + A[6] * dx + A[7] * dy + A[8] * dz,
                                             G[6] * gx + G[7] * gy + G[8] * gz)));
  });
}

// Replicated accumulators: with REP = 2 the staged sums exist twice and a
// lane adds into copy (lane & 1).  Lanes of one cell are neighbours (they
// take particles C apart in binned order), and k lanes on one shared address
// cost about k cycles, so splitting neighbours over two copies halves those
// collisions; the copies start 16 banks apart, so the same node in both
// copies is on different banks.  The copies are summed at the flush.
template <int KIND, int REP>
struct P2GRep {
  static constexpr int NS = Geo<KIND>::NS;
  static constexpr int stride = REP == 1 ? 4 * NS : ((4 * NS + 15) / 32) * 32 + 16;  // ints per copy
};

// TR: transfer, 0 APIC + MLS, 1 PIC, 2 APIC with the kernel gradient.
// ROT (APIC + MLS, one copy): components issued in the lane-rotated order of
// p2g_scatter_rot, planes kP2GRotPlane apart.  FMA (APIC + MLS): blocks of
// at least kP2GFmaCount particles round their contributions by p2g_fixed's
// fused multiply-add instead of a conversion.
template <int KIND, int TR, int REP, int ROT = 0, int FMA = 0>
__global__ void __launch_bounds__(kP2GWarp) k_p2g(StepView v) {
  constexpr int NS = Geo<KIND>::NS;
  static_assert(ROT == 0 || (REP == 1 && TR == 0), "the rotated order takes one copy and APIC + MLS");
  static_assert(FMA == 0 || TR == 0, "fused-multiply-add rounding is built for APIC + MLS");
  constexpr int PL = ROT ? P2GRotPlane<KIND>::value : NS;  // plane stride of the components
  constexpr int RS = ROT ? 4 * PL : P2GRep<KIND, REP>::stride;
  constexpr uint32_t CAP = kP2GStage, C = kP2GStage / 32;
  static_assert(C % 2 == 1, "lane stride must be odd");
  static_assert(RS % 4 == 0, "copies must keep 16-byte alignment");
  __shared__ __align__(16) int small[REP * RS];
  int(*sm)[NS] = reinterpret_cast<int(*)[NS]>(small + (REP == 1 ? 0 : (int)(threadIdx.x & 1u) * RS));
  const uint32_t rot = (threadIdx.x * 3u) & 3u;
  int* const pl[4] = {small + ((0u + rot) & 3u) * PL, small + ((1u + rot) & 3u) * PL,
                      small + ((2u + rot) & 3u) * PL, small + ((3u + rot) & 3u) * PL};
  __shared__ float4 sX[CAP], sA[CAP], sB[CAP], sC[CAP];
  constexpr uint32_t TCAP = TR == 2 ? CAP : 1;  // the stress term T (kernel-gradient APIC only)
  __shared__ float4 sT0[TCAP], sT1[TCAP];
  __shared__ float sT2[TCAP];
  __shared__ uint32_t bslot[8];
  const uint32_t nunits = *v.n_pb * v.splits;
  const uint32_t lane = threadIdx.x;
  for (;;) {
    // dynamic scheduling: one work unit (a block or a part of one) at a time
    uint32_t u = 0;
    if (lane == 0) u = atomicAdd(&v.work[0], 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= nunits) break;
    uint32_t bi, lo, hi;
    if (!unit_range(v, u, CAP, bi, lo, hi)) continue;
    const uint32_t key = v.pb_key[bi];
    const SceneDev s = v.scenes[v.pb_scene[bi]];
    const uint32_t start = v.offset[key];
    const uint32_t cnt = v.cnt_cur[key];
    // the block's largest contribution bounds, recorded when its particles
    // were binned
    const float bmass = __uint_as_float(v.bnd_cur[2 * key]);
    const float bmom = __uint_as_float(v.bnd_cur[2 * key + 1]);
    int ox, oy, oz;
    decode_block(s, key, ox, oy, oz);
    load_block_slots(v, s, ox, oy, oz, bslot);
    for (int j = lane; j < REP * RS / 4; j += kP2GWarp) reinterpret_cast<int4*>(small)[j] = make_int4(0, 0, 0, 0);
    // the scale covers the block's whole count, so any part of it is bounded
    const float fcnt = (float)cnt;
    const float Sm = bmass > 0.f ? 1073741824.0f / (fcnt * bmass) : 1.0f;
    const float Sp = bmom > 0.f ? 1073741824.0f / (fcnt * bmom) : 1.0f;
    for (uint32_t c0 = lo; c0 < hi; c0 += CAP) {
      const uint32_t m = min(hi - c0, CAP);
#pragma unroll
      for (uint32_t r = 0; r < C; ++r) {
        const uint32_t i = lane + r * kP2GWarp;
        if (i < m) {
          const uint32_t p = v.perm[start + c0 + i];
          cp_async16(&sX[i], &v.cur.X[p]);
          cp_async16(&sA[i], &v.cur.VM0[p]);
          cp_async16(&sB[i], &v.cur.VM1[p]);
          cp_async16(&sC[i], &v.cur.VM2[p]);
          if constexpr (TR == 2) {
            cp_async16(&sT0[i], &v.cur.T0[p]);
            cp_async16(&sT1[i], &v.cur.T1[p]);
            cp_async4(&sT2[i], &v.cur.T2[p]);
          }
        }
      }
      cp_async_wait_all();
      __syncwarp();
#pragma unroll 1
      for (uint32_t r = 0; r < C; ++r) {
        const uint32_t i = lane * C + r;
        if (i < m) {
          const P2GPart q{sX[i], sA[i], sB[i], sC[i]};
          if constexpr (TR == 1) {
            p2g_scatter_pic<KIND>(s, v.mats, v.err, q, ox, oy, oz, Sm, Sp, sm);
          } else if constexpr (TR == 2) {
            const float4 t0 = sT0[i], t1 = sT1[i];
            const float T[9] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w, sT2[i]};
            p2g_scatter_grad<KIND>(s, v.mats, v.err, q, T, ox, oy, oz, Sm, Sp, sm);
          } else if constexpr (ROT != 0) {
            if (FMA && cnt >= kP2GFmaCount)
              p2g_scatter_rot<KIND, true>(s, v.mats, v.err, q, ox, oy, oz, Sm, Sp, pl, rot);
            else
              p2g_scatter_rot<KIND, false>(s, v.mats, v.err, q, ox, oy, oz, Sm, Sp, pl, rot);
          } else {
            if (FMA && cnt >= kP2GFmaCount)
              p2g_scatter<KIND, true>(s, v.mats, v.err, q, ox, oy, oz, Sm, Sp, sm);
            else
              p2g_scatter<KIND, false>(s, v.mats, v.err, q, ox, oy, oz, Sm, Sp, sm);
          }
        }
      }
      __syncwarp();  // the next chunk overwrites the staged copies
    }
    const float iSm = 1.0f / Sm, iSp = 1.0f / Sp;
    for (int j = lane; j < NS; j += kP2GWarp) {
      // the copies' sums: each copy's sum is bounded like the whole, and
      // their total too, so adding them as integers cannot overflow
      int q[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        q[c] = small[c * PL + j];
        if (REP == 2) q[c] += small[RS + c * NS + j];
      }
      if (q[0] != 0) {
        int g, lx, ly, lz;
        staged_coords<KIND>(j, g, lx, ly, lz);
        long long gi = pool_index<KIND>(bslot, g, lx, ly, lz);
        if (gi >= 0)
          atomicAdd(&v.Gacc[gi], make_float4((float)q[0] * iSm, (float)q[1] * iSp, (float)q[2] * iSp,
                                             (float)q[3] * iSp));
      }
    }
    // (the block's bounds are cleared after G2P, by the float64 pass: other
    // units of this block may still be reading them)
    __syncwarp();  // the next unit clears the accumulators
  }
}

// ---------------------------------------------------------------- grid update

// Sec. 4.3.3 per grid: v~ = (m v + dt f)/m + dt g on nodes with m > 0, zero
// elsewhere; sticky walls zero v~ where a node coordinate (in cells, node i of
// G- at i + 1/4, of G+ at i - 1/4, quadratic at i) is < bc or > res - bc.
template <int KIND>
__global__ void __launch_bounds__(128) k_grid_update(StepView v) {
  constexpr int NG = Geo<KIND>::NG;
  // blocks per iteration: their dependent loads (list entry, scene, sums)
  // overlap (four measured slower: registers)
  constexpr int PB = 2;
  const uint32_t ng = min(*v.n_g, v.pool_cap);
  for (uint32_t g0 = blockIdx.x * PB; g0 < ng; g0 += gridDim.x * PB) {
    uint32_t gb[PB];
    SceneDev sd[PB];
#pragma unroll
    for (int k = 0; k < PB; ++k) {
      const uint32_t gi = min(g0 + k, ng - 1);  // a missing second block repeats the first's reads
      gb[k] = v.g_list[gi];
      sd[k] = v.scenes[v.g_scene[gi]];
    }
    for (int t = threadIdx.x; t < NG * kBlockNodes; t += blockDim.x) {
      const int grid = t / kBlockNodes, l = t % kBlockNodes;
      float4 acc[PB];
#pragma unroll
      for (int k = 0; k < PB; ++k)
        acc[k] = g0 + k < ng ? v.Gacc[((long long)(g0 + k) * NG + grid) * kBlockNodes + l] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < PB; ++k) {
        if (g0 + k >= ng) break;
        const SceneDev& s = sd[k];
        const long long lb = (long long)gb[k] - s.table_base;
        const int gx = (int)(lb % s.nb), gy = (int)((lb / s.nb) % s.nb), gz = (int)(lb / ((long long)s.nb * s.nb));
        const int ix = gx * 4 + (l & 3), iy = gy * 4 + ((l >> 2) & 3), iz = gz * 4 + (l >> 4);
        const float off = KIND == 0 ? (grid == 0 ? 0.25f : -0.25f) : 0.0f;
        const long long idx = ((long long)(g0 + k) * NG + grid) * kBlockNodes + l;
        float4 o = make_float4(0.f, 0.f, 0.f, acc[k].x);
        if (acc[k].x > 0.f) {
          o.x = acc[k].y / acc[k].x + s.dt * s.gx;
          o.y = acc[k].z / acc[k].x + s.dt * s.gy;
          o.z = acc[k].w / acc[k].x + s.dt * s.gz;
        }
        const float px = ix + off, py = iy + off, pz = iz + off;
        const float hi = (float)s.res - s.bc;
        const bool wall = px < s.bc || py < s.bc || pz < s.bc || px > hi || py > hi || pz > hi;
        if (wall) o.x = o.y = o.z = 0.f;
        v.Gvel[idx] = o;
        if (!v.keep_gacc) v.Gacc[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
}

// ------------------------------------------------------ G2P + constitutive

__device__ __forceinline__ float min3(float a, float b, float c) { return fminf(a, fminf(b, c)); }

// G2P runs one warp per CTA: a particle block's ~400-500 particles leave a
// partly idle last round on 32 lanes instead of on 128, and the staging
// waits are warp-level, so a lane that finishes early never holds up three
// other warps at a block barrier.  MINB counts 4-warp equivalents per SM.
// The fused G2P2G kernel stages g2p_stage(MINB) particles per chunk (64 at
// 5 or more, so that shared memory admits the extra warps).
constexpr int kG2PWarp = 32;
__host__ __device__ constexpr int g2p_stage(int minb) { return minb >= 5 ? 64 : 128; }  // particles per chunk

// Result of one particle's G2P: its next key and P2G contribution bounds,
// whether its constitutive update was deferred to the float64 pass, and
// whether its new state is finite.
struct G2POut {
  uint32_t nk;
  float bmass, bmom;
  bool use64, fin;
};

// G2P of one particle (slot t of the current binned order): gather v and B
// (or the kernel-gradient sums) from the staged grid velocities sv, F update,
// constitutive update (or listing for the float64 pass), advection, next key
// and bounds; stores the new state at slot t of nxt.  Returns false (and
// flags CK_ERR_INTERNAL) for a particle outside its block.
template <int KIND, int TR>
__device__ __forceinline__ bool g2p_particle(const StepView& v, const SceneDev& s, int ox, int oy, int oz,
                                             const float4* sv, uint32_t t, const float4 X, const float4 f0,
                                             const float4 f1, const float f2, const uint32_t id, const float Eraw,
                                             G2POut& out, const MatDev* smat = nullptr) {
  out.use64 = false;
  const uint32_t mi = __float_as_uint(X.w);
  // the material table from shared memory when the kernel staged it there
  const MatDev mt = smat ? smat[mi] : v.mats[mi];
  float mu = mt.mu, lam = mt.lam;
  float Ep = 0.f;
  if (v.cur.E) {
    Ep = Eraw;
    mu = Ep / (2.0f * (1.0f + mt.nu));
    lam = Ep * mt.nu / ((1.0f + mt.nu) * (1.0f - 2.0f * mt.nu));
  }
  Sten<KIND> st;
  if (!st.set(X.x * s.inv_dx, X.y * s.inv_dx, X.z * s.inv_dx, ox, oy, oz)) {
    flag_error(v.err, CK_ERR_INTERNAL);
    return false;
  }
  float vel[3], Bh[9], G[9];
  if constexpr (TR == 1) {
    // grad v = -Gr / dx (Gr in Bh); F' = (I + dt grad v) F
    st.set_grad();
    g2p_gather_grad(st, sv, vel, Bh);
    const float sc = -s.dt * s.inv_dx;
#pragma unroll
    for (int q = 0; q < 9; ++q) G[q] = sc * Bh[q];
  } else if constexpr (TR == 2) {
    // B from the APIC moments, grad v = -Gr / dx from the derivative sums
    g2p_gather(st, sv, vel, Bh);
    st.set_grad();
    float vg[3];
    g2p_gather_grad(st, sv, vg, G);
    const float sc = -s.dt * s.inv_dx;
#pragma unroll
    for (int q = 0; q < 9; ++q) G[q] *= sc;
  } else {
    // C = B D^-1 = Bh D^-1 / dx ; F' = (I + dt C) F
    g2p_gather(st, sv, vel, Bh);
    mul_dinv(st, Bh, s.dt * s.inv_dx, G);
  }
  const float vx = vel[0], vy = vel[1], vz = vel[2];
  G[0] += 1.0f;
  G[4] += 1.0f;
  G[8] += 1.0f;
  const float Fo[9] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w, f2};
  float F[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q)
      F[r * 3 + q] = G[r * 3 + 0] * Fo[0 * 3 + q] + G[r * 3 + 1] * Fo[1 * 3 + q] + G[r * 3 + 2] * Fo[2 * 3 + q];
  // constitutive update in float32 from the left stretch; degenerate or
  // inverted F is deferred to the float64 pass (precision extension):
  // this kernel stores F' and M = m B' (no stress) and lists the particle
  float tau[9];
  // Drucker-Prager at small stretch: matrix log/exp series, no eigen-
  // decomposition (such F is far from every float64 criterion)
  float Xs[6];
  const float xr = mt.model == 1 ? left_strain(F, Xs) : 1.f;
  const bool small_dp = mt.model == 1 && s.gap_tol <= 0.f && s.j_tol < 0.9f && s.cond_tol < 0.9f &&
                        xr <= (1.f / 48.f);
  const int sdeg = dp_lane_degree(xr);
  if (mt.model == 2) {
    // J-based fluid: volume ratio only, stress from J (no decomposition)
    fluid_update<float>(F, mt.E, mt.gamma, tau);
  } else if (small_dp) {
    dp_small_strain(F, Xs, sdeg, mu, lam, mt.dpc, tau);
  } else {
    // b = F F^T = U diag(sigma^2) U^T
    float bq[9], U[9], e[3], sg[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = r; q < 3; ++q) {
        const float d = F[r * 3] * F[q * 3] + F[r * 3 + 1] * F[q * 3 + 1] + F[r * 3 + 2] * F[q * 3 + 2];
        bq[r * 3 + q] = d;
        bq[q * 3 + r] = d;
      }
    sym_eig3<float>(bq, U, e);
    sg[0] = sqrtf(fmaxf(e[0], 0.f));
    sg[1] = sqrtf(fmaxf(e[1], 0.f));
    sg[2] = sqrtf(fmaxf(e[2], 0.f));
    const float J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                    F[2] * (F[3] * F[7] - F[4] * F[6]);
    const float smax = fmaxf(sg[0], fmaxf(sg[1], sg[2]));
    const float smin = min3(sg[0], sg[1], sg[2]);
    const float gap = min3(fabsf(sg[0] - sg[1]), fabsf(sg[0] - sg[2]), fabsf(sg[1] - sg[2]));
    const bool use64 = !(J > 0.f) || (fabsf(J) < s.j_tol) || (smin < s.cond_tol * smax) ||
                       (gap < s.gap_tol * smax);
    out.use64 = use64;
    if (use64) {
      const unsigned long long slot = atomicAdd(v.fp64_count, 1ull);
      v.fp64_list[slot] = t;
#pragma unroll
      for (int q = 0; q < 9; ++q) tau[q] = 0.f;
    } else {
      constitutive_left<float>(mt.model, F, mu, lam, mt.alpha, tau, U, e, sg);
    }
  }
  // M' = m B' - dt V0 tau, B' = dx Bh (APIC) or 0 (PIC); the kernel-
  // gradient APIC keeps M' = m B' and T' = -dt V0 tau apart
  const float mdx = mt.mass * s.dx, dtv = s.dt * s.V0;
  float Mn[9];
#pragma unroll
  for (int q = 0; q < 9; ++q)
    Mn[q] = TR == 1 ? -dtv * tau[q] : TR == 2 ? mdx * Bh[q] : mdx * Bh[q] - dtv * tau[q];
  float4 Xn = make_float4(X.x + s.dt * vx, X.y + s.dt * vy, X.z + s.dt * vz, X.w);
  // next key; particles leaving the interior are clamped and flagged
  float ux = Xn.x * s.inv_dx, uy = Xn.y * s.inv_dx, uz = Xn.z * s.inv_dx;
  // x was finite, so x + dt v is finite when v is.  x * 0 is 0 for a finite
  // x and NaN for an infinite or NaN one, so one sum of such products tests
  // every value at one fused multiply-add each
  float z = fmaf(vx, 0.f, fmaf(vy, 0.f, vz * 0.f));
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    z = fmaf(F[q], 0.f, fmaf(Mn[q], 0.f, z));
    if constexpr (TR == 2) z = fmaf(tau[q], 0.f, z);
  }
  const bool fin = z == 0.f;
  if (!fin) flag_error(v.err, CK_ERR_NONFINITE);
  out.fin = fin;
  if (!(in_domain(ux, s.res) && in_domain(uy, s.res) && in_domain(uz, s.res))) {
    flag_error(v.err, CK_ERR_DOMAIN);
    const float lo = 0.5f, hi = (float)s.res - 0.5f - 1e-3f;
    ux = fminf(fmaxf(isfinite(ux) ? ux : lo, lo), hi);
    uy = fminf(fmaxf(isfinite(uy) ? uy : lo, lo), hi);
    uz = fminf(fmaxf(isfinite(uz) ? uz : lo, lo), hi);
    Xn.x = ux * s.dx;
    Xn.y = uy * s.dx;
    Xn.z = uz * s.dx;
    ux = Xn.x * s.inv_dx;
    uy = Xn.y * s.inv_dx;
    uz = Xn.z * s.inv_dx;
  }
  const uint32_t nk = particle_key<KIND>(s, ux, uy, uz);
  v.nxt.X[t] = Xn;
  v.nxt.VM0[t] = make_float4(vx, vy, vz, Mn[0]);
  v.nxt.VM1[t] = make_float4(Mn[1], Mn[2], Mn[3], Mn[4]);
  v.nxt.VM2[t] = make_float4(Mn[5], Mn[6], Mn[7], Mn[8]);
  v.nxt.F0[t] = make_float4(F[0], F[1], F[2], F[3]);
  v.nxt.F1[t] = make_float4(F[4], F[5], F[6], F[7]);
  v.nxt.F2[t] = F[8];
  v.nxt.ID[t] = id;
  if (v.nxt.E) v.nxt.E[t] = Ep;
  v.key_nxt[t] = nk;
  out.nk = nk;
  float& bmass = out.bmass;
  float& bmom = out.bmom;
  if constexpr (TR == 2) {
    float Tn[9], Mb[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      Tn[q] = -dtv * tau[q];
      Mb[q] = fabsf(Mn[q]) + fabsf(Tn[q]);
    }
    v.nxt.T0[t] = make_float4(Tn[0], Tn[1], Tn[2], Tn[3]);
    v.nxt.T1[t] = make_float4(Tn[4], Tn[5], Tn[6], Tn[7]);
    v.nxt.T2[t] = Tn[8];
    p2g_bounds<KIND>(s.inv_dx, mt.mass, vx, vy, vz, Mb, bmass, bmom);
  } else {
    p2g_bounds<KIND>(s.inv_dx, mt.mass, vx, vy, vz, Mn, bmass, bmom);
  }
  return true;
}

// G2P with the next chunk's particle state in flight.  Chunks of 32
// particles (one per lane; each lane stages and reads only its own
// particle's slot) alternate between two staging buffers: while chunk k is
// computed, chunk k+1 is being gathered with cp.async.  The binned-order
// indices (perm) that address those gathers travel by cp.async into shared
// memory too, three chunks ahead, so inside a block no load result is waited
// on and no index is held in a register across a chunk's computation (held
// there, one was spilled to local memory at this register budget, and its
// spill store waited for the load).

// TR: transfer, 0 APIC + MLS, 1 PIC, 2 APIC with the kernel gradient.
template <int KIND, int MINB, int TR>
__global__ void __launch_bounds__(kG2PWarp, 4 * MINB) k_g2p(StepView v) {
  constexpr int NS = Geo<KIND>::NS;
  constexpr int CH = 32;
  constexpr int NB = 2;       // staging buffers (four measured slower: registers)
  constexpr int D = NB - 1;   // chunks in flight ahead of the computed one
  constexpr int PS = 2 * NB;  // slots of binned-order indices (D + 2 live at a time)
  static_assert((NB & (NB - 1)) == 0, "NB must be a power of two");
  __shared__ float4 sv[NS];
  __shared__ float4 sX[NB][CH], sF0[NB][CH], sF1[NB][CH];
  __shared__ float sF2[NB][CH], sE[NB][CH];
  __shared__ uint32_t sID[NB][CH];
  __shared__ uint32_t sP[PS][CH];
  __shared__ uint32_t bslot[8];
  __shared__ MatDev smat[kSmemMats];
  const uint32_t lane = threadIdx.x;
  const bool mat_smem = v.n_mats <= (uint32_t)kSmemMats;
  if (mat_smem) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(v.mats);
    uint32_t* dst = reinterpret_cast<uint32_t*>(smat);
    const uint32_t words = v.n_mats * (uint32_t)(sizeof(MatDev) / 4);
    for (uint32_t w = lane; w < words; w += CH) dst[w] = src[w];
  }
  __syncwarp();
  const uint32_t nunits = *v.n_pb * v.splits;
  for (;;) {
    uint32_t u = 0;
    if (lane == 0) u = atomicAdd(&v.work[1], 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= nunits) break;
    uint32_t bi, lo, hi;
    if (!unit_range(v, u, CH, bi, lo, hi)) continue;
    const uint32_t key = v.pb_key[bi];
    const SceneDev s = v.scenes[v.pb_scene[bi]];
    const uint32_t start = v.offset[key];
    int ox, oy, oz;
    decode_block(s, key, ox, oy, oz);
    load_block_slots(v, s, ox, oy, oz, bslot);
    const uint32_t nch = (hi - lo + CH - 1) / CH;
    // Each lane stages and reads only its own slot of every buffer, so the
    // index and particle buffers need no cross-lane ordering; sv does.
    // Binned-order indices of chunks 0 .. 2D: loaded together; chunks
    // 0 .. D-1 are staged at once, D .. 2D parked in sP.  The index of chunk
    // c >= 2D + 1 is fetched by cp.async in the group of chunk c - D - 1,
    // which has landed before chunk c is staged.
    uint32_t pp[2 * D + 1];
#pragma unroll
    for (int j = 0; j <= 2 * D; ++j) {
      const uint32_t i = lo + (uint32_t)j * CH + lane;
      pp[j] = i < hi ? v.perm[start + i] : 0u;
    }
#pragma unroll
    for (int j = D; j <= 2 * D; ++j) sP[j % PS][lane] = pp[j];
    __syncwarp();  // bslot
    for (int j = lane; j < NS; j += CH) {
      int g, lx, ly, lz;
      staged_coords<KIND>(j, g, lx, ly, lz);
      const long long gi = pool_index<KIND>(bslot, g, lx, ly, lz);
      if (gi >= 0)
        cp_async16(&sv[j], &v.Gvel[gi]);
      else
        sv[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    auto stage = [&](uint32_t c, uint32_t p) {
      const uint32_t b = c & (NB - 1);
      if (lo + c * CH + lane < hi) {
        cp_async16(&sX[b][lane], &v.cur.X[p]);
        cp_async16(&sF0[b][lane], &v.cur.F0[p]);
        cp_async16(&sF1[b][lane], &v.cur.F1[p]);
        cp_async4(&sF2[b][lane], &v.cur.F2[p]);
        cp_async4(&sID[b][lane], &v.cur.ID[p]);
        if (v.cur.E) cp_async4(&sE[b][lane], &v.cur.E[p]);
      }
    };
    // chunks 0 .. D-1 (the grid velocities go with chunk 0's group)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      if ((uint32_t)j < nch) stage((uint32_t)j, pp[j]);
      cp_async_commit();
    }
    for (uint32_t k = 0; k < nch; ++k) {
      const uint32_t kn = k + D;
      if (kn < nch) stage(kn, sP[kn % PS][lane]);
      const uint32_t kp = k + 2 * D + 1;
      if (kp < nch) {
        const uint32_t i = lo + kp * CH + lane;
        if (i < hi) cp_async4(&sP[kp % PS][lane], &v.perm[start + i]);
      }
      cp_async_commit();
      cp_async_wait<D>();  // the D newest groups may still be in flight: chunk k has landed
      __syncwarp();
      const uint32_t b = k & (NB - 1);
      const uint32_t i = lo + k * CH + lane;
      if (i < hi) {
        G2POut o;
        if (g2p_particle<KIND, TR>(v, s, ox, oy, oz, sv, start + i, sX[b][lane], sF0[b][lane], sF1[b][lane],
                                   sF2[b][lane], sID[b][lane], v.cur.E ? sE[b][lane] : 0.f, o,
                                   mat_smem ? smat : nullptr))
          warp_aggregated_bin(v.cnt_nxt, v.bnd_nxt, o.nk, o.bmass, o.bmom);
      }
      __syncwarp();  // chunk k + NB is staged into this buffer next
    }
  }
}

// ------------------------------------------------------------ fused G2P2G
//
// The paper's G2P2G (Sec. 5.1, after Wang 2020) gathers step n and scatters
// step n + 1 in one kernel.  Here one CTA (one warp) takes a particle block
// of step n and
//   1. runs G2P on every particle of the block exactly as k_g2p does
//      (new state, next key, histogram and bounds for the next binning);
//   2. scatters the particles that stay in the block (same key, float32
//      constitutive update, finite) into the block's staged nodes with the
//      fixed-point shared atomics of k_p2g, and flushes them into the next
//      step's grid through its block table.
// The fixed-point scale needs the bound of the block's new contributions
// before the first atomic, so the scatter is a second pass that reads the
// new state the first pass just wrote (contiguous, from L2), instead of a
// stash in shared memory that would cost occupancy.  Particles that moved to
// another block, took the float64 pass or became non-finite go to a list
// that k_p2g_leftover scatters after the float64 pass.
// The staged grid velocities of pass 1 and the accumulators of pass 2 share
// one shared-memory arena.
constexpr int kFuseMaxCnt = 4096;  // block particle count up to which stays are tracked (larger: all leftover)

template <int KIND, int MINB>
struct FuseSmem {
  static constexpr int NS = Geo<KIND>::NS;
  static constexpr int CAP = g2p_stage(MINB);
  struct Ph1 {
    float4 sv[NS];
    float4 sX[CAP], sF0[CAP], sF1[CAP];
    float sF2[CAP], sE[CAP];
    uint32_t sID[CAP];
  };
  struct Ph2 {
    int sm[4][NS];
    float4 sX[kP2GStage], sA[kP2GStage], sB[kP2GStage], sC[kP2GStage];
  };
  static constexpr size_t bytes = sizeof(Ph1) > sizeof(Ph2) ? sizeof(Ph1) : sizeof(Ph2);
};

// Append value to a global list when pred holds (one atomic per warp).
__device__ __forceinline__ void warp_append(uint32_t* count, uint32_t* list, uint32_t value, bool pred) {
  const unsigned am = __activemask();
  const unsigned m = __ballot_sync(am, pred);
  if (!m) return;
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(m));
  base = __shfl_sync(am, base, leader);
  if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = value;
}

template <int KIND, int MINB>
__global__ void __launch_bounds__(kG2PWarp, 4 * MINB) k_g2p2g(StepView v) {
  using SM = FuseSmem<KIND, MINB>;
  constexpr int NS = SM::NS;
  constexpr int CAP = SM::CAP;
  constexpr uint32_t PCAP = kP2GStage, PC = kP2GStage / 32;
  static_assert(CAP % 32 == 0, "the stay mask takes one ballot per 32 particles");
  __shared__ __align__(16) unsigned char arena[SM::bytes];
  __shared__ uint32_t stay[kFuseMaxCnt / 32];
  __shared__ uint32_t bslot[8];
  auto& p1 = *reinterpret_cast<typename SM::Ph1*>(arena);
  auto& p2 = *reinterpret_cast<typename SM::Ph2*>(arena);
  const uint32_t nunits = *v.n_pb * v.splits;
  const uint32_t lane = threadIdx.x;
  for (;;) {
    uint32_t u = 0;
    if (lane == 0) u = atomicAdd(&v.work[1], 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= nunits) break;
    uint32_t bi, lo, hi;
    if (!unit_range(v, u, CAP, bi, lo, hi)) continue;
    const uint32_t key = v.pb_key[bi];
    const SceneDev s = v.scenes[v.pb_scene[bi]];
    const uint32_t start = v.offset[key];
    const bool track = hi - lo <= (uint32_t)kFuseMaxCnt;
    int ox, oy, oz;
    decode_block(s, key, ox, oy, oz);
    load_block_slots(v, s, ox, oy, oz, bslot);  // this step's grid (gather)
    __syncwarp();
    // ---- pass 1: G2P of the block
    float bm_max = 0.f, bp_max = 0.f;
    uint32_t nstay = 0;
    for (uint32_t c0 = lo; c0 < hi; c0 += CAP) {
      const uint32_t m = min(hi - c0, (uint32_t)CAP);
#pragma unroll 4
      for (uint32_t i = lane; i < m; i += 32) {
        const uint32_t p = v.perm[start + c0 + i];
        cp_async16(&p1.sX[i], &v.cur.X[p]);
        cp_async16(&p1.sF0[i], &v.cur.F0[p]);
        cp_async16(&p1.sF1[i], &v.cur.F1[p]);
        cp_async4(&p1.sF2[i], &v.cur.F2[p]);
        cp_async4(&p1.sID[i], &v.cur.ID[p]);
        if (v.cur.E) cp_async4(&p1.sE[i], &v.cur.E[p]);
      }
      if (c0 == lo) {
        for (int j = lane; j < NS; j += 32) {
          int g, lx, ly, lz;
          staged_coords<KIND>(j, g, lx, ly, lz);
          long long gi = pool_index<KIND>(bslot, g, lx, ly, lz);
          if (gi >= 0)
            cp_async16(&p1.sv[j], &v.Gvel[gi]);
          else
            p1.sv[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      cp_async_wait_all();
      __syncwarp();
      for (uint32_t i = lane; i < m; i += 32) {
        const uint32_t t = start + c0 + i;
        G2POut o;
        const bool ok = g2p_particle<KIND, 0>(v, s, ox, oy, oz, p1.sv, t, p1.sX[i], p1.sF0[i], p1.sF1[i],
                                              p1.sF2[i], p1.sID[i], v.cur.E ? p1.sE[i] : 0.f, o);
        if (ok) warp_aggregated_bin(v.cnt_nxt, v.bnd_nxt, o.nk, o.bmass, o.bmom);
        const bool st = ok && track && o.nk == key && !o.use64 && o.fin;
        if (st) {
          bm_max = fmaxf(bm_max, o.bmass);
          bp_max = fmaxf(bp_max, o.bmom);
          nstay += 1;
        }
        warp_append(v.lo_count, v.lo_list, t, ok && !st);
        const unsigned am = __activemask();
        const unsigned w = __ballot_sync(am, st);
        if (track && (int)lane == __ffs(am) - 1) stay[(c0 - lo + i - lane) >> 5] = w;
      }
      __syncwarp();  // the next chunk overwrites the staged copies
    }
    // ---- pass 2: P2G of the particles that stayed, into the next grid
    bm_max = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(bm_max)));
    bp_max = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(bp_max)));
    nstay = __reduce_add_sync(0xffffffffu, nstay);
    if (nstay > 0) {
      if (lane < 8) {  // the next step's grid blocks (scatter)
        const int bx = (ox >> 2) + (lane & 1), by = (oy >> 2) + ((lane >> 1) & 1), bz = (oz >> 2) + (lane >> 2);
        bslot[lane] = v.table_nxt[s.table_base + ((long long)bz * s.nb + by) * s.nb + bx];
      }
      for (int j = lane; j < NS; j += 32) reinterpret_cast<int4*>(&p2.sm[0][0])[j] = make_int4(0, 0, 0, 0);
      const float fst = (float)nstay;
      const float Sm = bm_max > 0.f ? 1073741824.0f / (fst * bm_max) : 1.0f;
      const float Sp = bp_max > 0.f ? 1073741824.0f / (fst * bp_max) : 1.0f;
      for (uint32_t c0 = lo; c0 < hi; c0 += PCAP) {
        const uint32_t m = min(hi - c0, PCAP);
#pragma unroll
        for (uint32_t r = 0; r < PC; ++r) {
          const uint32_t i = lane + r * 32;
          if (i < m) {
            const uint32_t t = start + c0 + i;
            cp_async16(&p2.sX[i], &v.nxt.X[t]);
            cp_async16(&p2.sA[i], &v.nxt.VM0[t]);
            cp_async16(&p2.sB[i], &v.nxt.VM1[t]);
            cp_async16(&p2.sC[i], &v.nxt.VM2[t]);
          }
        }
        cp_async_wait_all();
        __syncwarp();
#pragma unroll 1
        for (uint32_t r = 0; r < PC; ++r) {
          const uint32_t i = lane * PC + r;
          const uint32_t q = c0 - lo + i;
          if (i < m && ((stay[q >> 5] >> (q & 31)) & 1u)) {
            const P2GPart part{p2.sX[i], p2.sA[i], p2.sB[i], p2.sC[i]};
            p2g_scatter<KIND>(s, v.mats, v.err, part, ox, oy, oz, Sm, Sp, p2.sm);
          }
        }
        __syncwarp();
      }
      const float iSm = 1.0f / Sm, iSp = 1.0f / Sp;
      for (int j = lane; j < NS; j += 32) {
        const int mi = p2.sm[0][j];
        if (mi != 0) {
          int g, lx, ly, lz;
          staged_coords<KIND>(j, g, lx, ly, lz);
          const long long gi = pool_index<KIND>(bslot, g, lx, ly, lz);
          if (gi >= 0)
            atomicAdd(&v.Gacc[gi], make_float4((float)mi * iSm, (float)p2.sm[1][j] * iSp,
                                               (float)p2.sm[2][j] * iSp, (float)p2.sm[3][j] * iSp));
          else
            flag_error(v.err, CK_ERR_POOL);
        }
      }
    }
    __syncwarp();  // the next unit reuses the arena and the slots
  }
}

// Pool slot of virtual grid block g in the next step's table; a block no
// fused scatter touched is claimed here: a slot is taken from the counter
// and offered to the table with one compare-and-swap; when another thread
// got there first its slot is used and this one stays empty (its
// accumulators are zero, so the grid update leaves it at rest).  No thread
// waits on another.
__device__ __forceinline__ uint32_t claim_slot(const StepView& v, long long g, uint32_t scene) {
  const uint32_t cur = v.table_nxt[g];
  if (cur != CK_NO_SLOT) return cur;
  const uint32_t ns = atomicAdd(v.n_g_nxt, 1u);
  if (ns >= v.pool_cap) {
    flag_error(v.err, CK_ERR_POOL);
    return CK_NO_SLOT;
  }
  v.g_list_nxt[ns] = (uint32_t)g;
  v.g_scene_nxt[ns] = scene;
  const uint32_t old = atomicCAS(&v.table_nxt[g], CK_NO_SLOT, ns);
  return old == CK_NO_SLOT ? ns : old;
}

// P2G of the particles the fused kernel left over (new state in nxt, after
// the float64 pass): one particle per thread, contributions in float added
// with one 16-byte global atomic per node (APIC + MLS; quadratic or CK).
template <int KIND>
__global__ void __launch_bounds__(128) k_p2g_leftover(StepView v) {
  constexpr int NG = Geo<KIND>::NG;
  const uint32_t n = min(*v.lo_count, v.n_cur);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t t = v.lo_list[i];
    const float4 X = v.nxt.X[t];
    const MatDev mt = v.mats[__float_as_uint(X.w)];
    const SceneDev s = v.scenes[mt.scene];
    const float ux = X.x * s.inv_dx, uy = X.y * s.inv_dx, uz = X.z * s.inv_dx;
    Cell<KIND> cx, cy, cz;
    cx.set(ux);
    cy.set(uy);
    cz.set(uz);
    const int ox = cx.block() * 4, oy = cy.block() * 4, oz = cz.block() * 4;
    Sten<KIND> st;
    if (!st.set(ux, uy, uz, ox, oy, oz)) {
      flag_error(v.err, CK_ERR_INTERNAL);
      continue;
    }
    float M[9];
    const float4 a = v.nxt.VM0[t], b = v.nxt.VM1[t], c = v.nxt.VM2[t];
    M[0] = a.w; M[1] = b.x; M[2] = b.y; M[3] = b.z; M[4] = b.w; M[5] = c.x; M[6] = c.y; M[7] = c.z; M[8] = c.w;
    float A[9];
    mul_dinv(st, M, s.inv_dx, A);
    const float mass = mt.mass;
    const float px = mass * a.x, py = mass * a.y, pz = mass * a.z;
    for_nodes(st, [&](int j, float w, float dx, float dy, float dz) {
      int g, lx, ly, lz;
      staged_coords<KIND>(j, g, lx, ly, lz);
      const int ix = ox + lx, iy = oy + ly, iz = oz + lz;
      const long long gb = s.table_base + ((long long)(iz >> 2) * s.nb + (iy >> 2)) * s.nb + (ix >> 2);
      const uint32_t sl = claim_slot(v, gb, mt.scene);
      if (sl == CK_NO_SLOT) return;
      const int l = ((iz & 3) * 4 + (iy & 3)) * 4 + (ix & 3);
      atomicAdd(&v.Gacc[((long long)sl * NG + g) * kBlockNodes + l],
                make_float4(w * mass, w * (px + A[0] * dx + A[1] * dy + A[2] * dz),
                            w * (py + A[3] * dx + A[4] * dy + A[5] * dz), w * (pz + A[6] * dx + A[7] * dy + A[8] * dz)));
    });
  }
}

// Float64 pass of the precision extension: the particles G2P listed (F
// degenerate, inverted or flagged by the scene's criteria) get the full
// rotation-variant SVD and constitutive update in float64.  G2P stored the
// advanced F' and M = m B'; this pass stores the projected F, subtracts
// dt V0 tau from M (with the kernel-gradient APIC: stores T = -dt V0 tau) and
// raises the particle's block bounds to cover the new M.
// Grid-stride over the list; an empty list returns at once.
template <int KIND>
__global__ void __launch_bounds__(128) k_g2p_fp64(StepView v) {
  // every transfer kernel of the step is done with the histogram entries and
  // P2G bounds of this step's blocks: clear them, so that this buffer is all
  // zero when G2P fills it for the step after next
  const uint32_t npb = *v.n_pb;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < npb; i += gridDim.x * blockDim.x) {
    const uint32_t key = v.pb_key[i];
    v.cnt_cur[key] = 0u;
    v.bnd_cur[2 * key] = 0u;
    v.bnd_cur[2 * key + 1] = 0u;
  }
  const uint32_t n = (uint32_t)min(*v.fp64_count, (unsigned long long)v.n_cur);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t t = v.fp64_list[i];
    const float4 X = v.nxt.X[t];
    const MatDev mt = v.mats[__float_as_uint(X.w)];
    const SceneDev s = v.scenes[mt.scene];
    double mu = mt.mu, lam = mt.lam;
    if (v.nxt.E) {
      const double E = v.nxt.E[t], nu = mt.nu;
      mu = E / (2.0 * (1.0 + nu));
      lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    }
    const float4 f0 = v.nxt.F0[t], f1 = v.nxt.F1[t];
    double F[9] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w, v.nxt.F2[t]};
    double tau[9], sg[3];
    constitutive<double>(mt.model, F, mu, lam, (double)mt.alpha, tau, sg);
    const double dtv = (double)s.dt * (double)s.V0;
    float4 a = v.nxt.VM0[t], b = v.nxt.VM1[t], c = v.nxt.VM2[t];
    float Tn[9];
    const bool sep = v.nxt.T0 != nullptr;  // stress term kept apart from m B
#pragma unroll
    for (int q = 0; q < 9; ++q) Tn[q] = (float)(-dtv * tau[q]);
    if (sep) {
      v.nxt.T0[t] = make_float4(Tn[0], Tn[1], Tn[2], Tn[3]);
      v.nxt.T1[t] = make_float4(Tn[4], Tn[5], Tn[6], Tn[7]);
      v.nxt.T2[t] = Tn[8];
    } else {
      a.w = (float)(a.w - dtv * tau[0]);
      b = make_float4((float)(b.x - dtv * tau[1]), (float)(b.y - dtv * tau[2]), (float)(b.z - dtv * tau[3]),
                      (float)(b.w - dtv * tau[4]));
      c = make_float4((float)(c.x - dtv * tau[5]), (float)(c.y - dtv * tau[6]), (float)(c.z - dtv * tau[7]),
                      (float)(c.w - dtv * tau[8]));
    }
    float Ff[9];
    bool fin = isfinite(a.w) && isfinite(b.x) && isfinite(b.y) && isfinite(b.z) && isfinite(b.w) &&
               isfinite(c.x) && isfinite(c.y) && isfinite(c.z) && isfinite(c.w);
#pragma unroll
    for (int q = 0; q < 9; ++q) fin = fin && isfinite(Tn[q]);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      Ff[q] = (float)F[q];
      fin = fin && isfinite(Ff[q]);
    }
    if (!fin) flag_error(v.err, CK_ERR_NONFINITE);
    v.nxt.VM0[t] = a;
    v.nxt.VM1[t] = b;
    v.nxt.VM2[t] = c;
    v.nxt.F0[t] = make_float4(Ff[0], Ff[1], Ff[2], Ff[3]);
    v.nxt.F1[t] = make_float4(Ff[4], Ff[5], Ff[6], Ff[7]);
    v.nxt.F2[t] = Ff[8];
    float Mn[9] = {a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
    if (sep) {
#pragma unroll
      for (int q = 0; q < 9; ++q) Mn[q] = fabsf(Mn[q]) + fabsf(Tn[q]);
    }
    float bmass, bmom;
    p2g_bounds<KIND>(s.inv_dx, mt.mass, a.x, a.y, a.z, Mn, bmass, bmom);
    const uint32_t nk = v.key_nxt[t];
    atomicMax(&v.bnd_nxt[2 * nk], __float_as_uint(bmass));
    atomicMax(&v.bnd_nxt[2 * nk + 1], __float_as_uint(bmom));
  }
}

// Zero the accumulators of the blocks listed by the last probe.
template <int KIND>
__global__ void k_clear_gacc(StepView v) {
  constexpr int NG = Geo<KIND>::NG;
  const uint32_t ng = min(*v.n_g, v.pool_cap);
  for (uint32_t gi = blockIdx.x; gi < ng; gi += gridDim.x) {
    for (int t = threadIdx.x; t < NG * kBlockNodes; t += blockDim.x)
      v.Gacc[((long long)gi * NG + (t / kBlockNodes)) * kBlockNodes + (t % kBlockNodes)] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// ------------------------------------------------------- readback / upload

// Kirchhoff stress of a stored F (no plasticity), any material.
__device__ __forceinline__ void stress_of(const MatDev& mt, const float* F, float mu, float lam, float* tau) {
  if (mt.model == 2)
    fluid_tau_of_J<float>(det3(F), mt.E, mt.gamma, tau);
  else
    stress_only<float>(mt.model, F, mu, lam, tau);
}

__device__ __forceinline__ void load_F(const Pool& P, uint32_t t, float* F) {
  float4 a = P.F0[t], b = P.F1[t];
  F[0] = a.x; F[1] = a.y; F[2] = a.z; F[3] = a.w;
  F[4] = b.x; F[5] = b.y; F[6] = b.z; F[7] = b.w;
  F[8] = P.F2[t];
}

__device__ __forceinline__ void load_M(const Pool& P, uint32_t t, float* M) {
  float4 a = P.VM0[t], b = P.VM1[t], c = P.VM2[t];
  M[0] = a.w; M[1] = b.x; M[2] = b.y; M[3] = b.z;
  M[4] = b.w; M[5] = c.x; M[6] = c.y; M[7] = c.z; M[8] = c.w;
}

__device__ __forceinline__ void store_M(Pool& P, uint32_t t, const float* M) {
  float4 a = P.VM0[t];
  a.w = M[0];
  P.VM0[t] = a;
  P.VM1[t] = make_float4(M[1], M[2], M[3], M[4]);
  P.VM2[t] = make_float4(M[5], M[6], M[7], M[8]);
}

__device__ __forceinline__ void lame_of(const MatDev& mt, const Pool& P, uint32_t t, float& mu, float& lam) {
  mu = mt.mu;
  lam = mt.lam;
  if (P.E) {
    float E = P.E[t];
    mu = E / (2.0f * (1.0f + mt.nu));
    lam = E * mt.nu / ((1.0f + mt.nu) * (1.0f - 2.0f * mt.nu));
  }
}

// B = (M + dt V0 tau(F)) / m; with the stress term kept apart, B = M / m
__device__ __forceinline__ void recover_B(const Pool& P, const SceneDev& s, const MatDev& mt, uint32_t t, float* B) {
  float F[9], M[9], tau[9];
  load_M(P, t, M);
  if (P.T0) {
    const float im = 1.0f / mt.mass;
#pragma unroll
    for (int q = 0; q < 9; ++q) B[q] = M[q] * im;
    return;
  }
  load_F(P, t, F);
  float mu, lam;
  lame_of(mt, P, t, mu, lam);
  stress_of(mt, F, mu, lam, tau);
  float dtv = s.dt * s.V0, im = 1.0f / mt.mass;
#pragma unroll
  for (int q = 0; q < 9; ++q) B[q] = (M[q] + dtv * tau[q]) * im;
}

// pic: the PIC transfer keeps B = 0, so B and C read as 0.
template <int KIND>
__global__ void k_read_particles(Pool P, const SceneDev* scenes, const MatDev* mats, int scene, uint32_t start,
                                 uint32_t n, int field, int pic, float* out) {
  const SceneDev s = scenes[scene];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t t = start + i;
    uint32_t id = P.ID[t];
    float4 X = P.X[t];
    const MatDev mt = mats[__float_as_uint(X.w)];
    if (field == 0) {
      out[3 * id] = X.x; out[3 * id + 1] = X.y; out[3 * id + 2] = X.z;
    } else if (field == 1) {
      float4 a = P.VM0[t];
      out[3 * id] = a.x; out[3 * id + 1] = a.y; out[3 * id + 2] = a.z;
    } else if (field == 4) {
      float F[9];
      load_F(P, t, F);
      for (int q = 0; q < 9; ++q) out[9 * id + q] = F[q];
    } else if (field == 5) {
      out[id] = P.E ? P.E[t] : 0.f;
    } else if (pic) {
      for (int q = 0; q < 9; ++q) out[9 * id + q] = 0.f;
    } else {
      float B[9];
      recover_B(P, s, mt, t, B);
      if (field == 2) {
        for (int q = 0; q < 9; ++q) out[9 * id + q] = B[q];
      } else {  // C = B D^-1 = B Di / dx^2
        Sten<KIND> st;
        float ux = X.x * s.inv_dx, uy = X.y * s.inv_dx, uz = X.z * s.inv_dx;
        Cell<KIND> cx, cy, cz;
        cx.set(ux); cy.set(uy); cz.set(uz);
        st.set(ux, uy, uz, cx.block() * 4, cy.block() * 4, cz.block() * 4);
        float C[9];
        mul_dinv(st, B, s.inv_dx * s.inv_dx, C);
        for (int q = 0; q < 9; ++q) out[9 * id + q] = C[q];
      }
    }
  }
}

// Overwrite one field from original-order input; keeps M = m B - dt V0 tau(F)
// (pic: B = 0, the host refuses uploads of B).
__global__ void k_write_particles(Pool P, const SceneDev* scenes, const MatDev* mats, int scene, uint32_t start,
                                  uint32_t n, int field, int pic, const float* in) {
  const SceneDev s = scenes[scene];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t t = start + i;
    uint32_t id = P.ID[t];
    float4 X = P.X[t];
    const MatDev mt = mats[__float_as_uint(X.w)];
    float dtv = s.dt * s.V0;
    if (field == 0) {
      P.X[t] = make_float4(in[3 * id], in[3 * id + 1], in[3 * id + 2], X.w);
    } else if (field == 1) {
      float4 a = P.VM0[t];
      P.VM0[t] = make_float4(in[3 * id], in[3 * id + 1], in[3 * id + 2], a.w);
    } else if (field == 2) {
      float F[9], tau[9], M[9], mu, lam;
      load_F(P, t, F);
      lame_of(mt, P, t, mu, lam);
      stress_of(mt, F, mu, lam, tau);
      for (int q = 0; q < 9; ++q) M[q] = mt.mass * in[9 * id + q] - (P.T0 ? 0.f : dtv * tau[q]);
      store_M(P, t, M);
    } else if (field == 4 || field == 5) {
      float B[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (!pic) recover_B(P, s, mt, t, B);
      if (field == 4) {
        P.F0[t] = make_float4(in[9 * id], in[9 * id + 1], in[9 * id + 2], in[9 * id + 3]);
        P.F1[t] = make_float4(in[9 * id + 4], in[9 * id + 5], in[9 * id + 6], in[9 * id + 7]);
        P.F2[t] = in[9 * id + 8];
      } else if (P.E) {
        P.E[t] = in[id];
      }
      float F[9], tau[9], M[9], mu, lam;
      load_F(P, t, F);
      lame_of(mt, P, t, mu, lam);
      stress_of(mt, F, mu, lam, tau);
      if (P.T0) {  // m B stays; the stress term follows the new F (or E)
        P.T0[t] = make_float4(-dtv * tau[0], -dtv * tau[1], -dtv * tau[2], -dtv * tau[3]);
        P.T1[t] = make_float4(-dtv * tau[4], -dtv * tau[5], -dtv * tau[6], -dtv * tau[7]);
        P.T2[t] = -dtv * tau[8];
      } else {
        for (int q = 0; q < 9; ++q) M[q] = mt.mass * B[q] - dtv * tau[q];
        store_M(P, t, M);
      }
    }
  }
}

// Dense grid fields of one scene: out[grid][iz][iy][ix] (x fastest) over
// 0..res per axis, written from the active blocks of the last step (the
// caller zeroes out first); which: 0 mass, 1 momentum (3), 2 velocity (3)
// from a probe's accumulators; 3 mass, 4 velocity (3) from the grid a fused
// step left (velocity and mass after its update), nodes with mass only, so
// that a slot the leftover P2G claimed in vain (empty) writes nothing.
template <int KIND>
__global__ void k_read_grid(const float4* Gacc, const float4* Gvel, const uint32_t* g_list, const uint32_t* g_scene,
                            const uint32_t* n_g, uint32_t pool_cap, const SceneDev* scenes, int scene, int which,
                            float* out) {
  constexpr int NG = Geo<KIND>::NG;
  const SceneDev s = scenes[scene];
  const int n = s.res + 1;
  const long long nnode = (long long)n * n * n;
  const uint32_t ng = min(*n_g, pool_cap);
  for (uint32_t gi = blockIdx.x; gi < ng; gi += gridDim.x) {
    if ((int)g_scene[gi] != scene) continue;
    long long lb = (long long)g_list[gi] - s.table_base;
    int gx = (int)(lb % s.nb), gy = (int)((lb / s.nb) % s.nb), gz = (int)(lb / ((long long)s.nb * s.nb));
    for (int t = threadIdx.x; t < NG * kBlockNodes; t += blockDim.x) {
      int grid = t / kBlockNodes, l = t % kBlockNodes;
      int ix = gx * 4 + (l & 3), iy = gy * 4 + ((l >> 2) & 3), iz = gz * 4 + (l >> 4);
      if (ix >= n || iy >= n || iz >= n) continue;
      long long q = grid * nnode + ((long long)iz * n + iy) * n + ix;
      long long idx = ((long long)gi * NG + grid) * kBlockNodes + l;
      if (which >= 3) {
        const float4 g = Gvel[idx];
        if (g.w > 0.f) {
          if (which == 3) {
            out[q] = g.w;
          } else {
            out[3 * q] = g.x; out[3 * q + 1] = g.y; out[3 * q + 2] = g.z;
          }
        }
        continue;
      }
      float4 a = Gacc[idx];
      if (which == 0) {
        out[q] = a.x;
      } else if (which == 1) {
        out[3 * q] = a.y; out[3 * q + 1] = a.z; out[3 * q + 2] = a.w;
      } else {
        float4 g = Gvel[idx];
        bool has = a.x > 0.f;
        out[3 * q] = has ? g.x : 0.f;
        out[3 * q + 1] = has ? g.y : 0.f;
        out[3 * q + 2] = has ? g.z : 0.f;
      }
    }
  }
}

// Append a new scene's particles: X (x, mat_base + mat), v, M = 0 (B = 0 and
// tau(I) = 0), F = I, ID = index; plus keys and the histogram.
template <int KIND>
__global__ void k_admit(Pool P, uint32_t* key, uint32_t* cnt, uint32_t* bnd, const SceneDev* scenes,
                        const MatDev* mats, int scene, uint32_t mat_base, uint32_t nmat, uint32_t start, uint32_t n,
                        const float* x, const float* vel, const uint8_t* mat, const float* E, uint32_t* err) {
  const SceneDev s = scenes[scene];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t t = start + i;
    float px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2];
    float ux = px * s.inv_dx, uy = py * s.inv_dx, uz = pz * s.inv_dx;
    if (!(in_domain(ux, s.res) && in_domain(uy, s.res) && in_domain(uz, s.res))) {
      flag_error(err, CK_ERR_DOMAIN);
      const float lo = 0.5f, hi = (float)s.res - 0.5f - 1e-3f;
      ux = fminf(fmaxf(isfinite(ux) ? ux : lo, lo), hi);
      uy = fminf(fmaxf(isfinite(uy) ? uy : lo, lo), hi);
      uz = fminf(fmaxf(isfinite(uz) ? uz : lo, lo), hi);
      px = ux * s.dx; py = uy * s.dx; pz = uz * s.dx;
      ux = px * s.inv_dx; uy = py * s.inv_dx; uz = pz * s.inv_dx;
    }
    uint32_t mloc = mat ? (uint32_t)mat[i] : 0u;
    if (mloc >= nmat) {  // unknown material index: use material 0 and report
      flag_error(err, CK_ERR_INTERNAL);
      mloc = 0;
    }
    uint32_t m = mat_base + mloc;
    P.X[t] = make_float4(px, py, pz, __uint_as_float(m));
    float vx = vel ? vel[3 * i] : 0.f, vy = vel ? vel[3 * i + 1] : 0.f, vz = vel ? vel[3 * i + 2] : 0.f;
    P.VM0[t] = make_float4(vx, vy, vz, 0.f);
    P.VM1[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    P.VM2[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    P.F0[t] = make_float4(1.f, 0.f, 0.f, 0.f);
    P.F1[t] = make_float4(1.f, 0.f, 0.f, 0.f);
    P.F2[t] = 1.f;
    P.ID[t] = i;
    if (P.E) P.E[t] = E ? E[i] : 0.f;
    if (P.T0) {  // tau(I) = 0 for every model
      P.T0[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      P.T1[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      P.T2[t] = 0.f;
    }
    uint32_t k = particle_key<KIND>(s, ux, uy, uz);
    key[t] = k;
    const float M0[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float bmass, bmom;
    p2g_bounds<KIND>(s.inv_dx, mats[m].mass, vx, vy, vz, M0, bmass, bmom);
    warp_aggregated_bin(cnt, bnd, k, bmass, bmom);
  }
}

// Recompute keys and the histogram of the whole current pool (after an
// upload of positions); particles already retired by a release keep the dead
// key and leave the pool at the next step.
template <int KIND>
__global__ void k_rekey(Pool P, uint32_t* key, uint32_t* cnt, uint32_t* bnd, const SceneDev* scenes,
                        const MatDev* mats, uint32_t n, uint32_t* err) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    if (key[t] == CK_DEAD_KEY) continue;  // retired by a release; its slot may already be reused
    float4 X = P.X[t];
    const MatDev mt = mats[__float_as_uint(X.w)];
    const SceneDev s = scenes[mt.scene];
    if (!s.alive) {
      key[t] = CK_DEAD_KEY;
      continue;
    }
    float ux = X.x * s.inv_dx, uy = X.y * s.inv_dx, uz = X.z * s.inv_dx;
    if (!(in_domain(ux, s.res) && in_domain(uy, s.res) && in_domain(uz, s.res))) {
      flag_error(err, CK_ERR_DOMAIN);
      const float lo = 0.5f, hi = (float)s.res - 0.5f - 1e-3f;
      ux = fminf(fmaxf(isfinite(ux) ? ux : lo, lo), hi);
      uy = fminf(fmaxf(isfinite(uy) ? uy : lo, lo), hi);
      uz = fminf(fmaxf(isfinite(uz) ? uz : lo, lo), hi);
      X.x = ux * s.dx; X.y = uy * s.dx; X.z = uz * s.dx;
      P.X[t] = X;
      ux = X.x * s.inv_dx; uy = X.y * s.inv_dx; uz = X.z * s.inv_dx;
    }
    uint32_t k = particle_key<KIND>(s, ux, uy, uz);
    key[t] = k;
    const float4 a = P.VM0[t], b = P.VM1[t], c = P.VM2[t];
    float M[9] = {a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
    if (P.T0) {
      const float4 t0 = P.T0[t], t1 = P.T1[t];
      const float T[9] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w, P.T2[t]};
      for (int q = 0; q < 9; ++q) M[q] = fabsf(M[q]) + fabsf(T[q]);
    }
    float bmass, bmom;
    p2g_bounds<KIND>(s.inv_dx, mt.mass, a.x, a.y, a.z, M, bmass, bmom);
    warp_aggregated_bin(cnt, bnd, k, bmass, bmom);
  }
}

// ------------------------------------------------------------ host launchers

// P2G of the APIC + MLS transfer: accumulator copies, component order and
// rounding as the launch configuration asks.
template <int KIND>
static void launch_p2g_apic(const LaunchCfg& lc, StepView v) {
  const int g = lc.sm_count * 32;
  if (lc.p2g_rep == 2) {
    if (lc.p2g_fma)
      k_p2g<KIND, 0, 2, 0, 1><<<g, kP2GWarp, 0, lc.stream>>>(v);
    else
      k_p2g<KIND, 0, 2, 0, 0><<<g, kP2GWarp, 0, lc.stream>>>(v);
  } else if (lc.p2g_rot) {
    if (lc.p2g_fma)
      k_p2g<KIND, 0, 1, 1, 1><<<g, kP2GWarp, 0, lc.stream>>>(v);
    else
      k_p2g<KIND, 0, 1, 1, 0><<<g, kP2GWarp, 0, lc.stream>>>(v);
  } else {
    if (lc.p2g_fma)
      k_p2g<KIND, 0, 1, 0, 1><<<g, kP2GWarp, 0, lc.stream>>>(v);
    else
      k_p2g<KIND, 0, 1, 0, 0><<<g, kP2GWarp, 0, lc.stream>>>(v);
  }
}

template <int KIND>
static void launch_all(const LaunchCfg& lc, StepView v, int which) {
  switch (which) {
    case LK_P2G:
      if (lc.transfer == 1)
        k_p2g<KIND, 1, 1><<<lc.sm_count * 32, kP2GWarp, 0, lc.stream>>>(v);
      else if (lc.transfer == 2)
        k_p2g<KIND, 2, 1><<<lc.sm_count * 32, kP2GWarp, 0, lc.stream>>>(v);
      else
        launch_p2g_apic<KIND>(lc, v);
      break;
    // a wide grid: each CTA's block loop is short, so the dependent loads of
    // one block (list entry, scene, accumulators) overlap across CTAs
    case LK_UPDATE: k_grid_update<KIND><<<lc.sm_count * 64, 128, 0, lc.stream>>>(v); break;
    case LK_G2P:
      // register budget of G2P: 20 warps/SM (96 registers) by default, the
      // faster for both kernels on the large-impact scene; 16 (119-124
      // registers) or 24 (80) on request.  One resident wave.  The kernel-
      // gradient transfers run one budget each: PIC the APIC default (16
      // warps/SM for the quadratic twin); the kernel-gradient APIC (two
      // gathers) 16 warps/SM for CK and 12 (168 registers, no spills) for
      // the quadratic twin.
      if (lc.transfer == 1)
        k_g2p<KIND, KIND == 0 ? 5 : 4, 1><<<lc.sm_count * (KIND == 0 ? 20 : 16), kG2PWarp, 0, lc.stream>>>(v);
      else if (lc.transfer == 2)
        k_g2p<KIND, KIND == 0 ? 4 : 3, 2><<<lc.sm_count * (KIND == 0 ? 16 : 12), kG2PWarp, 0, lc.stream>>>(v);
      else if (lc.g2p_minb >= 6)
        k_g2p<KIND, 6, 0><<<lc.sm_count * 24, kG2PWarp, 0, lc.stream>>>(v);
      else if (lc.g2p_minb == 5)
        k_g2p<KIND, 5, 0><<<lc.sm_count * 20, kG2PWarp, 0, lc.stream>>>(v);
      else
        k_g2p<KIND, 4, 0><<<lc.sm_count * 16, kG2PWarp, 0, lc.stream>>>(v);
      break;
    case LK_G2P_FP64: k_g2p_fp64<KIND><<<lc.sm_count * 4, 128, 0, lc.stream>>>(v); break;
    // fused step (APIC + MLS): one resident wave at the G2P register budget
    case LK_G2P2G:
      if constexpr (KIND == 0)
        k_g2p2g<KIND, 5><<<lc.sm_count * 20, kG2PWarp, 0, lc.stream>>>(v);
      else
        k_g2p2g<KIND, 4><<<lc.sm_count * 16, kG2PWarp, 0, lc.stream>>>(v);
      break;
    case LK_LEFTOVER: k_p2g_leftover<KIND><<<lc.sm_count * 4, 128, 0, lc.stream>>>(v); break;
    case LK_CLEAR: k_clear_gacc<KIND><<<lc.persistent_ctas, 128, 0, lc.stream>>>(v); break;
  }
}

void launch_transfer(int kind, const LaunchCfg& lc, const StepView& v, int which) {
  if (kind == 0)
    launch_all<0>(lc, v, which);
  else
    launch_all<1>(lc, v, which);
}

void launch_read_particles(int kind, bool pic, cudaStream_t st, Pool P, const SceneDev* scenes, const MatDev* mats,
                           int scene, uint32_t start, uint32_t n, int field, float* out) {
  int blocks = (int)((n + 255) / 256);
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  if (kind == 0)
    k_read_particles<0><<<blocks, 256, 0, st>>>(P, scenes, mats, scene, start, n, field, pic ? 1 : 0, out);
  else
    k_read_particles<1><<<blocks, 256, 0, st>>>(P, scenes, mats, scene, start, n, field, pic ? 1 : 0, out);
}

void launch_write_particles(bool pic, cudaStream_t st, Pool P, const SceneDev* scenes, const MatDev* mats, int scene,
                            uint32_t start, uint32_t n, int field, const float* in) {
  int blocks = (int)((n + 255) / 256);
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  k_write_particles<<<blocks, 256, 0, st>>>(P, scenes, mats, scene, start, n, field, pic ? 1 : 0, in);
}

void launch_read_grid(int kind, cudaStream_t st, const StepView& v, int scene, int which, float* out) {
  if (kind == 0)
    k_read_grid<0><<<1024, 128, 0, st>>>(v.Gacc, v.Gvel, v.g_list, v.g_scene, v.n_g, v.pool_cap, v.scenes, scene,
                                          which, out);
  else
    k_read_grid<1><<<1024, 128, 0, st>>>(v.Gacc, v.Gvel, v.g_list, v.g_scene, v.n_g, v.pool_cap, v.scenes, scene,
                                          which, out);
}

void launch_admit(int kind, cudaStream_t st, Pool P, uint32_t* key, uint32_t* cnt, uint32_t* bnd,
                  const SceneDev* scenes, const MatDev* mats, int scene, uint32_t mat_base, uint32_t nmat,
                  uint32_t start, uint32_t n, const float* x, const float* v, const uint8_t* mat, const float* E,
                  uint32_t* err) {
  int blocks = (int)((n + 255) / 256);
  if (blocks < 1) blocks = 1;
  if (blocks > 8192) blocks = 8192;
  if (kind == 0)
    k_admit<0><<<blocks, 256, 0, st>>>(P, key, cnt, bnd, scenes, mats, scene, mat_base, nmat, start, n, x, v, mat, E,
                                        err);
  else
    k_admit<1><<<blocks, 256, 0, st>>>(P, key, cnt, bnd, scenes, mats, scene, mat_base, nmat, start, n, x, v, mat, E,
                                        err);
}

void launch_rekey(int kind, cudaStream_t st, Pool P, uint32_t* key, uint32_t* cnt, uint32_t* bnd,
                  const SceneDev* scenes, const MatDev* mats, uint32_t n, uint32_t* err) {
  int blocks = (int)((n + 255) / 256);
  if (blocks < 1) blocks = 1;
  if (blocks > 8192) blocks = 8192;
  if (kind == 0)
    k_rekey<0><<<blocks, 256, 0, st>>>(P, key, cnt, bnd, scenes, mats, n, err);
  else
    k_rekey<1><<<blocks, 256, 0, st>>>(P, key, cnt, bnd, scenes, mats, n, err);
}

}  // namespace ck
