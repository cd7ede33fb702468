// Differentiable CK-MPM step: forward and hand-written adjoint kernels.
//
// One step of the compact-kernel MPM on the dual grid (Sec. 4.3-4.5) with the
// fixed-corotated model, written as a pure function of the particle state
// (x, v, B, F) and a per-particle Young's modulus E, with particles kept in
// the caller's order and a dense grid of (res+1)^3 nodes per grid:
//   P2G   m_i = sum w m,  P_i = sum w (m v + A d),  A = (m B - dt V0 tau(F)) D^-1
//   grid  v~_i = mask (P_i / m_i + dt g)   (m_i > 0; sticky walls)
//   G2P   v' = 1/2 sum w v~,  B' = 1/2 sum w v~ (x_i - x_p)^T,
//         F' = (I + dt B' D^-1) F,  x' = x + dt v'
// (readings R4-R8 of the forward engine).  The adjoint of a step runs the
// reverse of these three stages: G2P^T scatters the velocity adjoint to the
// grid, the grid stage maps it to momentum and mass adjoints, and P2G^T
// gathers them back to the particles; weights, offsets and D depend on x and
// are differentiated in closed form (K1 is C^2, so dK1 is continuous).  The
// stress adjoint goes through the polar decomposition F = R S with
// dR = R Omega, Omega S + S Omega = R^T dF - dF^T R, whose (sigma_i + sigma_j)
// denominators stay well conditioned when singular values coincide.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "../../include/ckmpm.h"
#include "svd3.cuh"

namespace ckd {

using ck::svd3;

struct DP {
  float dx, inv_dx, dt, V0, mass, nu, gx, gy, gz, bc;
  int res, nn, n;
};

constexpr float kInv2Pi = 0.15915494309189535f;
constexpr float kTwoPi = 6.283185307179586f;

// Per-particle stencil on both grids with derivatives with respect to x.
struct DS {
  int base[2][3];      // base node per grid (0: G-, 1: G+) and axis
  float W[2][3][2];    // 1-D weights
  float dW[2][3][2];   // d W / d x (per unit length)
  float d[2][3][2];    // x_i - x_p in cells
  float Di[9];         // D^-1 (cells^-2)
  float sg[3], dsg[3]; // sigma = sin(2 pi f+)/(2 pi) and d sigma / dx
  float dLam[3];       // d Lambda / dx
  __device__ void set(const DP& p, float x0, float x1, float x2) {
    float xs[3] = {x0, x1, x2};
    float lam[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float u = xs[a] * p.inv_dx;
      float t = u + 0.25f;
      float fb = floorf(t);
      int bp = (int)fb;
      float fp = t - fb, fm;
      int bm;
      if (fp >= 0.5f) {
        bm = bp;
        fm = fp - 0.5f;
      } else {
        bm = bp - 1;
        fm = fp + 0.5f;
      }
      float s2, c2;
      sincospif(2.0f * fp, &s2, &c2);
      float s = s2 * kInv2Pi;
      base[0][a] = bm;
      base[1][a] = bp;
      W[1][a][0] = 1.0f - fp + s;
      W[1][a][1] = fp - s;
      W[0][a][0] = 1.0f - fm - s;
      W[0][a][1] = fm + s;
      dW[1][a][0] = (-1.0f + c2) * p.inv_dx;
      dW[1][a][1] = (1.0f - c2) * p.inv_dx;
      dW[0][a][0] = (-1.0f - c2) * p.inv_dx;
      dW[0][a][1] = (1.0f + c2) * p.inv_dx;
      d[1][a][0] = -fp;
      d[1][a][1] = 1.0f - fp;
      d[0][a][0] = -fm;
      d[0][a][1] = 1.0f - fm;
      float m2p = fp * (1.0f - fp) - s * (1.0f - 2.0f * fp);
      float m2m = fm * (1.0f - fm) + s * (1.0f - 2.0f * fm);
      lam[a] = 0.5f * (m2p + m2m) - s * s;
      float dm2p = (1.0f - 2.0f * fp) * (1.0f - c2) + 2.0f * s;
      float dm2m = (1.0f - 2.0f * fm) * (1.0f + c2) - 2.0f * s;
      dLam[a] = (0.5f * (dm2p + dm2m) - 2.0f * s * c2) * p.inv_dx;
      sg[a] = s;
      dsg[a] = c2 * p.inv_dx;
    }
    float li[3] = {1.0f / lam[0], 1.0f / lam[1], 1.0f / lam[2]};
    float y[3] = {li[0] * sg[0], li[1] * sg[1], li[2] * sg[2]};
    float den = 1.0f / (1.0f + sg[0] * y[0] + sg[1] * y[1] + sg[2] * y[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Di[i * 3 + j] = (i == j ? li[i] : 0.0f) - y[i] * y[j] * den;
  }
  // x_bar contribution of an adjoint Dib on D^-1 (cells^-2)
  __device__ void dinv_to_x(const float* Dib, float* xb) const {
    // D_bar = -Di^T Dib Di^T  (Di symmetric)
    float T[9], Db[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) T[i * 3 + j] = Di[i * 3 + 0] * Dib[0 * 3 + j] + Di[i * 3 + 1] * Dib[1 * 3 + j] + Di[i * 3 + 2] * Dib[2 * 3 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Db[i * 3 + j] = -(T[i * 3 + 0] * Di[0 * 3 + j] + T[i * 3 + 1] * Di[1 * 3 + j] + T[i * 3 + 2] * Di[2 * 3 + j]);
    // D_ab = Lam_a delta_ab + sg_a sg_b
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float sym = 0.f;
#pragma unroll
      for (int b = 0; b < 3; ++b) sym += (Db[c * 3 + b] + Db[b * 3 + c]) * sg[b];
      xb[c] += Db[c * 4] * dLam[c] + dsg[c] * sym;
    }
  }
};

__device__ __forceinline__ long long node_index(const DP& p, int g, int ix, int iy, int iz) {
  return (((long long)g * p.nn + iz) * p.nn + iy) * p.nn + ix;
}

__device__ __forceinline__ bool nodes_in_range(const DP& p, const DS& s) {
  bool ok = true;
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int a = 0; a < 3; ++a) ok = ok && s.base[g][a] >= 0 && s.base[g][a] + 1 <= p.res;
  return ok;
}

__device__ __forceinline__ void load9(const float* a, long long i, float* o) {
#pragma unroll
  for (int q = 0; q < 9; ++q) o[q] = a[9 * i + q];
}

__device__ __forceinline__ void mat3(const float* A, const float* B, float* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[i * 3 + j] = A[i * 3] * B[j] + A[i * 3 + 1] * B[3 + j] + A[i * 3 + 2] * B[6 + j];
}
__device__ __forceinline__ void mat3_bt(const float* A, const float* B, float* C) {  // A B^T
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[i * 3 + j] = A[i * 3] * B[j * 3] + A[i * 3 + 1] * B[j * 3 + 1] + A[i * 3 + 2] * B[j * 3 + 2];
}
__device__ __forceinline__ void mat3_at(const float* A, const float* B, float* C) {  // A^T B
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[i * 3 + j] = A[i] * B[j] + A[3 + i] * B[3 + j] + A[6 + i] * B[6 + j];
}

__device__ __forceinline__ void lame(const DP& p, float E, float& mu, float& lam) {
  mu = E / (2.0f * (1.0f + p.nu));
  lam = E * p.nu / ((1.0f + p.nu) * (1.0f - 2.0f * p.nu));
}

// tau = 2 mu (F - R) F^T + lam J (J - 1) I
__device__ __forceinline__ void fc_stress(const float* F, float mu, float lam, float* tau, float* U, float* sig, float* V) {
  svd3<float>(F, U, sig, V);
  ck::fc_tau<float>(F, U, sig, V, mu, lam, tau);
}

// Adjoint of tau(F; E) for the fixed-corotated model: F_bar += d tau/dF ^T : tb,
// E_bar += <tb, tau> / E (tau is proportional to E at fixed F).
__device__ void fc_stress_vjp(const float* F, float E, float mu, float lam, const float* tb, float* Fb, float& Eb) {
  float U[9], V[9], sig[3], tau[9];
  fc_stress(F, mu, lam, tau, U, sig, V);
  float R[9];
  mat3_bt(U, V, R);
  float J = sig[0] * sig[1] * sig[2];
  float G[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) G[q] = F[q] - R[q];
  // 2 mu (tb F + tb^T G)
  float t1[9], t2[9];
  mat3(tb, F, t1);
  mat3_at(tb, G, t2);
#pragma unroll
  for (int q = 0; q < 9; ++q) Fb[q] += 2.0f * mu * (t1[q] + t2[q]);
  // lam (2J - 1) tr(tb) cof(F)
  float tr = tb[0] + tb[4] + tb[8];
  float cof[9] = {F[4] * F[8] - F[5] * F[7], F[5] * F[6] - F[3] * F[8], F[3] * F[7] - F[4] * F[6],
                  F[2] * F[7] - F[1] * F[8], F[0] * F[8] - F[2] * F[6], F[1] * F[6] - F[0] * F[7],
                  F[1] * F[5] - F[2] * F[4], F[2] * F[3] - F[0] * F[5], F[0] * F[4] - F[1] * F[3]};
  float kv = lam * (2.0f * J - 1.0f) * tr;
#pragma unroll
  for (int q = 0; q < 9; ++q) Fb[q] += kv * cof[q];
  // R_bar = -2 mu tb F ; F_bar += 2 U Z V^T, Z_ij = skew(U^T R_bar V)_ij / (sig_i + sig_j)
  float Rb[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) Rb[q] = -2.0f * mu * t1[q];
  float T[9], A[9];
  mat3_at(U, Rb, T);
  mat3(T, V, A);
  float Z[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float den = sig[i] + sig[j];
      den = fabsf(den) < 1e-6f ? (den < 0.f ? -1e-6f : 1e-6f) : den;
      Z[i * 3 + j] = (i == j) ? 0.0f : 0.5f * (A[i * 3 + j] - A[j * 3 + i]) / den;
    }
  float UZ[9], UZV[9];
  mat3(U, Z, UZ);
  mat3_bt(UZ, V, UZV);
#pragma unroll
  for (int q = 0; q < 9; ++q) Fb[q] += 2.0f * UZV[q];
  float dot = 0.f;
#pragma unroll
  for (int q = 0; q < 9; ++q) dot += tb[q] * tau[q];
  Eb += E > 0.f ? dot / E : 0.0f;
}

// --------------------------------------------------------------- forward

__global__ void k_fwd_p2g(DP p, const float* x, const float* v, const float* B, const float* F, const float* E,
                          float* gm, float* gp, uint32_t* err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gridDim.x * blockDim.x) {
    DS s;
    s.set(p, x[3 * i], x[3 * i + 1], x[3 * i + 2]);
    if (!nodes_in_range(p, s)) {
      atomicOr(err, 1u);
      continue;
    }
    float Fi[9], Bi[9], tau[9], U[9], V[9], sig[3], mu, lam;
    load9(F, i, Fi);
    load9(B, i, Bi);
    lame(p, E[i], mu, lam);
    fc_stress(Fi, mu, lam, tau, U, sig, V);
    float M[9], A[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) M[q] = p.mass * Bi[q] - p.dt * p.V0 * tau[q];
    mat3(M, s.Di, A);
#pragma unroll
    for (int q = 0; q < 9; ++q) A[q] *= p.inv_dx;
    const float mv0 = p.mass * v[3 * i], mv1 = p.mass * v[3 * i + 1], mv2 = p.mass * v[3 * i + 2];
    for (int g = 0; g < 2; ++g)
      for (int sz = 0; sz < 2; ++sz)
        for (int sy = 0; sy < 2; ++sy)
          for (int sx = 0; sx < 2; ++sx) {
            float w = s.W[g][0][sx] * s.W[g][1][sy] * s.W[g][2][sz];
            float d0 = s.d[g][0][sx], d1 = s.d[g][1][sy], d2 = s.d[g][2][sz];
            long long ni = node_index(p, g, s.base[g][0] + sx, s.base[g][1] + sy, s.base[g][2] + sz);
            atomicAdd(&gm[ni], w * p.mass);
            atomicAdd(&gp[3 * ni], w * (mv0 + A[0] * d0 + A[1] * d1 + A[2] * d2));
            atomicAdd(&gp[3 * ni + 1], w * (mv1 + A[3] * d0 + A[4] * d1 + A[5] * d2));
            atomicAdd(&gp[3 * ni + 2], w * (mv2 + A[6] * d0 + A[7] * d1 + A[8] * d2));
          }
  }
}

__device__ __forceinline__ bool wall(const DP& p, int g, long long r) {
  int ix = (int)(r % p.nn), iy = (int)((r / p.nn) % p.nn), iz = (int)(r / ((long long)p.nn * p.nn));
  float off = g == 0 ? 0.25f : -0.25f;
  float hi = (float)p.res - p.bc;
  float a = ix + off, b = iy + off, c = iz + off;
  return a < p.bc || b < p.bc || c < p.bc || a > hi || b > hi || c > hi;
}

__global__ void k_fwd_grid(DP p, const float* gm, const float* gp, float* gv) {
  const long long per = (long long)p.nn * p.nn * p.nn;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 2 * per; q += (long long)gridDim.x * blockDim.x) {
    float m = gm[q];
    float o0 = 0.f, o1 = 0.f, o2 = 0.f;
    if (m > 0.f && !wall(p, (int)(q / per), q % per)) {
      o0 = gp[3 * q] / m + p.dt * p.gx;
      o1 = gp[3 * q + 1] / m + p.dt * p.gy;
      o2 = gp[3 * q + 2] / m + p.dt * p.gz;
    }
    gv[3 * q] = o0;
    gv[3 * q + 1] = o1;
    gv[3 * q + 2] = o2;
  }
}

__global__ void k_fwd_g2p(DP p, const float* x, const float* F, const float* gv, float* x1, float* v1, float* B1,
                          float* F1, uint32_t* err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gridDim.x * blockDim.x) {
    DS s;
    s.set(p, x[3 * i], x[3 * i + 1], x[3 * i + 2]);
    if (!nodes_in_range(p, s)) {  // reported by ckmpm_diff_sync; the particle is left in place
      atomicOr(err, 1u);
      for (int q = 0; q < 9; ++q) {
        if (q < 3) {
          x1[3 * i + q] = x[3 * i + q];
          v1[3 * i + q] = 0.f;
        }
        B1[9 * i + q] = 0.f;
        F1[9 * i + q] = F[9 * i + q];
      }
      continue;
    }
    float vv[3] = {0.f, 0.f, 0.f}, Bh[9] = {0.f};
    for (int g = 0; g < 2; ++g)
      for (int sz = 0; sz < 2; ++sz)
        for (int sy = 0; sy < 2; ++sy)
          for (int sx = 0; sx < 2; ++sx) {
            float w = 0.5f * s.W[g][0][sx] * s.W[g][1][sy] * s.W[g][2][sz];
            float dd[3] = {s.d[g][0][sx], s.d[g][1][sy], s.d[g][2][sz]};
            long long ni = node_index(p, g, s.base[g][0] + sx, s.base[g][1] + sy, s.base[g][2] + sz);
            float g3[3] = {gv[3 * ni], gv[3 * ni + 1], gv[3 * ni + 2]};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              vv[a] += w * g3[a];
#pragma unroll
              for (int b = 0; b < 3; ++b) Bh[a * 3 + b] += w * g3[a] * dd[b];
            }
          }
    float Fi[9], C[9], Fn[9];
    load9(F, i, Fi);
    mat3(Bh, s.Di, C);
#pragma unroll
    for (int q = 0; q < 9; ++q) C[q] = (q % 4 == 0 ? 1.0f : 0.0f) + p.dt * p.inv_dx * C[q];
    mat3(C, Fi, Fn);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      x1[3 * i + a] = x[3 * i + a] + p.dt * vv[a];
      v1[3 * i + a] = vv[a];
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      B1[9 * i + q] = p.dx * Bh[q];
      F1[9 * i + q] = Fn[q];
    }
  }
}

// --------------------------------------------------------------- adjoint

// x_bar contribution of per-node (w_bar, d_bar) for node (g, sx, sy, sz)
__device__ __forceinline__ void node_to_x(const DS& s, int g, int sx, int sy, int sz, float wb, const float* db,
                                          const DP& p, float* xb) {
  float w0 = s.W[g][0][sx], w1 = s.W[g][1][sy], w2 = s.W[g][2][sz];
  xb[0] += wb * s.dW[g][0][sx] * w1 * w2 - db[0] * p.inv_dx;
  xb[1] += wb * w0 * s.dW[g][1][sy] * w2 - db[1] * p.inv_dx;
  xb[2] += wb * w0 * w1 * s.dW[g][2][sz] - db[2] * p.inv_dx;
}

// G2P^T: given the step's output adjoints, write x_bar and F_bar (partial) of
// the step inputs and scatter the grid-velocity adjoint gvb.
__global__ void k_bwd_g2p(DP p, const float* x, const float* F, const float* gv, const float* gx1, const float* gv1,
                          const float* gB1, const float* gF1, float* gx, float* gF, float* gvb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gridDim.x * blockDim.x) {
    DS s;
    s.set(p, x[3 * i], x[3 * i + 1], x[3 * i + 2]);
    if (!nodes_in_range(p, s)) {
      for (int q = 0; q < 9; ++q) {
        if (q < 3) gx[3 * i + q] = 0.f;
        gF[9 * i + q] = 0.f;
      }
      continue;
    }
    // recompute the forward gather
    float vv[3] = {0.f, 0.f, 0.f}, Bh[9] = {0.f};
    for (int g = 0; g < 2; ++g)
      for (int sz = 0; sz < 2; ++sz)
        for (int sy = 0; sy < 2; ++sy)
          for (int sx = 0; sx < 2; ++sx) {
            float w = 0.5f * s.W[g][0][sx] * s.W[g][1][sy] * s.W[g][2][sz];
            float dd[3] = {s.d[g][0][sx], s.d[g][1][sy], s.d[g][2][sz]};
            long long ni = node_index(p, g, s.base[g][0] + sx, s.base[g][1] + sy, s.base[g][2] + sz);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              float ga = gv[3 * ni + a];
              vv[a] += w * ga;
#pragma unroll
              for (int b = 0; b < 3; ++b) Bh[a * 3 + b] += w * ga * dd[b];
            }
          }
    float Fi[9], Fb1[9], Bb1[9];
    load9(F, i, Fi);
    load9(gF1, i, Fb1);
    load9(gB1, i, Bb1);
    float xb[3] = {gx1[3 * i], gx1[3 * i + 1], gx1[3 * i + 2]};
    float vb[3] = {gv1[3 * i] + p.dt * xb[0], gv1[3 * i + 1] + p.dt * xb[1], gv1[3 * i + 2] + p.dt * xb[2]};
    // F' = G F, G = I + k Bh Di, k = dt/dx
    const float k = p.dt * p.inv_dx;
    float C[9], G[9];
    mat3(Bh, s.Di, C);
#pragma unroll
    for (int q = 0; q < 9; ++q) G[q] = (q % 4 == 0 ? 1.0f : 0.0f) + k * C[q];
    float Fbo[9];
    mat3_at(G, Fb1, Fbo);  // G^T F'_bar
#pragma unroll
    for (int q = 0; q < 9; ++q) gF[9 * i + q] = Fbo[q];
    float Gb[9];
    mat3_bt(Fb1, Fi, Gb);  // F'_bar F^T
    // C = Bh Di: Bh_bar = k Gb Di^T, Di_bar = k Bh^T Gb ; plus B' = dx Bh
    float Bhb[9], Dib[9];
    mat3_bt(Gb, s.Di, Bhb);
#pragma unroll
    for (int q = 0; q < 9; ++q) Bhb[q] = k * Bhb[q] + p.dx * Bb1[q];
    mat3_at(Bh, Gb, Dib);
#pragma unroll
    for (int q = 0; q < 9; ++q) Dib[q] *= k;
    // gather adjoints: v = 1/2 sum w v~, Bh = 1/2 sum w v~ d^T
    for (int g = 0; g < 2; ++g)
      for (int sz = 0; sz < 2; ++sz)
        for (int sy = 0; sy < 2; ++sy)
          for (int sx = 0; sx < 2; ++sx) {
            float w = 0.5f * s.W[g][0][sx] * s.W[g][1][sy] * s.W[g][2][sz];
            float dd[3] = {s.d[g][0][sx], s.d[g][1][sy], s.d[g][2][sz]};
            long long ni = node_index(p, g, s.base[g][0] + sx, s.base[g][1] + sy, s.base[g][2] + sz);
            float q3[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) q3[a] = vb[a] + Bhb[a * 3] * dd[0] + Bhb[a * 3 + 1] * dd[1] + Bhb[a * 3 + 2] * dd[2];
            float g3[3] = {gv[3 * ni], gv[3 * ni + 1], gv[3 * ni + 2]};
            atomicAdd(&gvb[3 * ni], w * q3[0]);
            atomicAdd(&gvb[3 * ni + 1], w * q3[1]);
            atomicAdd(&gvb[3 * ni + 2], w * q3[2]);
            float wb = 0.5f * (g3[0] * q3[0] + g3[1] * q3[1] + g3[2] * q3[2]);
            float db[3];
#pragma unroll
            for (int b = 0; b < 3; ++b) db[b] = w * (Bhb[b] * g3[0] + Bhb[3 + b] * g3[1] + Bhb[6 + b] * g3[2]);
            node_to_x(s, g, sx, sy, sz, wb, db, p, xb);
          }
    s.dinv_to_x(Dib, xb);
    gx[3 * i] = xb[0];
    gx[3 * i + 1] = xb[1];
    gx[3 * i + 2] = xb[2];
  }
}

// grid^T: v~ = (P/m + dt g) on nodes with mass off the walls
__global__ void k_bwd_grid(DP p, const float* gm, const float* gp, const float* gvb, float* gpb, float* gmb) {
  const long long per = (long long)p.nn * p.nn * p.nn;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 2 * per; q += (long long)gridDim.x * blockDim.x) {
    float m = gm[q];
    float b0 = 0.f, b1 = 0.f, b2 = 0.f, bm = 0.f;
    if (m > 0.f && !wall(p, (int)(q / per), q % per)) {
      float im = 1.0f / m;
      b0 = gvb[3 * q] * im;
      b1 = gvb[3 * q + 1] * im;
      b2 = gvb[3 * q + 2] * im;
      bm = -(b0 * gp[3 * q] + b1 * gp[3 * q + 1] + b2 * gp[3 * q + 2]) * im;
    }
    gpb[3 * q] = b0;
    gpb[3 * q + 1] = b1;
    gpb[3 * q + 2] = b2;
    gmb[q] = bm;
  }
}

// P2G^T: gather the grid adjoints back to the particles.
__global__ void k_bwd_p2g(DP p, const float* x, const float* v, const float* B, const float* F, const float* E,
                          const float* gpb, const float* gmb, float* gx, float* gv, float* gB, float* gF, float* gE) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gridDim.x * blockDim.x) {
    DS s;
    s.set(p, x[3 * i], x[3 * i + 1], x[3 * i + 2]);
    if (!nodes_in_range(p, s)) {
      for (int q = 0; q < 9; ++q) {
        if (q < 3) gv[3 * i + q] = 0.f;
        gB[9 * i + q] = 0.f;
      }
      continue;
    }
    float Fi[9], Bi[9], tau[9], U[9], V[9], sig[3], mu, lam;
    load9(F, i, Fi);
    load9(B, i, Bi);
    const float Ei = E[i];
    lame(p, Ei, mu, lam);
    fc_stress(Fi, mu, lam, tau, U, sig, V);
    float M[9], A[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) M[q] = p.mass * Bi[q] - p.dt * p.V0 * tau[q];
    mat3(M, s.Di, A);
#pragma unroll
    for (int q = 0; q < 9; ++q) A[q] *= p.inv_dx;
    const float mv[3] = {p.mass * v[3 * i], p.mass * v[3 * i + 1], p.mass * v[3 * i + 2]};
    float xb[3] = {0.f, 0.f, 0.f}, vb[3] = {0.f, 0.f, 0.f}, Ab[9] = {0.f};
    for (int g = 0; g < 2; ++g)
      for (int sz = 0; sz < 2; ++sz)
        for (int sy = 0; sy < 2; ++sy)
          for (int sx = 0; sx < 2; ++sx) {
            float w = s.W[g][0][sx] * s.W[g][1][sy] * s.W[g][2][sz];
            float dd[3] = {s.d[g][0][sx], s.d[g][1][sy], s.d[g][2][sz]};
            long long ni = node_index(p, g, s.base[g][0] + sx, s.base[g][1] + sy, s.base[g][2] + sz);
            float pb[3] = {gpb[3 * ni], gpb[3 * ni + 1], gpb[3 * ni + 2]};
            float mb = gmb[ni];
            float c3[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) c3[a] = mv[a] + A[a * 3] * dd[0] + A[a * 3 + 1] * dd[1] + A[a * 3 + 2] * dd[2];
            float wb = p.mass * mb + pb[0] * c3[0] + pb[1] * c3[1] + pb[2] * c3[2];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              vb[a] += w * p.mass * pb[a];
#pragma unroll
              for (int b = 0; b < 3; ++b) Ab[a * 3 + b] += w * pb[a] * dd[b];
            }
            float db[3];
#pragma unroll
            for (int b = 0; b < 3; ++b) db[b] = w * (A[b] * pb[0] + A[3 + b] * pb[1] + A[6 + b] * pb[2]);
            node_to_x(s, g, sx, sy, sz, wb, db, p, xb);
          }
    // A = M Di / dx: M_bar = Ab Di^T / dx ; Di_bar = M^T Ab / dx
    float Mb[9], Dib[9];
    mat3_bt(Ab, s.Di, Mb);
    mat3_at(M, Ab, Dib);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      Mb[q] *= p.inv_dx;
      Dib[q] *= p.inv_dx;
    }
    s.dinv_to_x(Dib, xb);
    // M = m B - dt V0 tau
    float tb[9], Fb[9] = {0.f}, Eb = 0.f;
#pragma unroll
    for (int q = 0; q < 9; ++q) tb[q] = -p.dt * p.V0 * Mb[q];
    fc_stress_vjp(Fi, Ei, mu, lam, tb, Fb, Eb);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      gx[3 * i + a] += xb[a];
      gv[3 * i + a] = vb[a];
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      gB[9 * i + q] = p.mass * Mb[q];
      gF[9 * i + q] += Fb[q];
    }
    gE[i] += Eb;
  }
}

}  // namespace ckd

struct ckmpm_diff {
  ckd::DP p{};
  cudaStream_t stream = nullptr;
  float *gm = nullptr, *gp = nullptr, *gv = nullptr, *gvb = nullptr, *gpb = nullptr, *gmb = nullptr;
  uint32_t* err = nullptr;
  int blocks = 1024;
};

extern "C" {

ckmpm_status ckmpm_diff_create(const ckmpm_scene* sc, void* stream, ckmpm_diff** out) {
  if (!out) return CKMPM_EINVAL;
  *out = nullptr;
  if (!sc || sc->n < 1 || sc->res < 4 || sc->res > 1024 || !(sc->dx > 0) || !(sc->dt > 0) || sc->ppc < 1 ||
      !sc->materials || sc->n_materials < 1 || sc->materials[0].model != CKMPM_FIXED_COROTATED ||
      !(sc->materials[0].rho > 0) || !(sc->materials[0].nu > -1.0 && sc->materials[0].nu < 0.5))
    return CKMPM_EINVAL;
  ckmpm_diff* d = new (std::nothrow) ckmpm_diff();
  if (!d) return CKMPM_ENOMEM;
  ckd::DP& p = d->p;
  p.dx = (float)sc->dx;
  p.inv_dx = (float)(1.0 / sc->dx);
  p.dt = (float)sc->dt;
  p.V0 = (float)(sc->dx * sc->dx * sc->dx / sc->ppc);
  p.mass = (float)(sc->materials[0].rho * sc->dx * sc->dx * sc->dx / sc->ppc);
  p.nu = (float)sc->materials[0].nu;
  p.gx = (float)sc->gravity[0];
  p.gy = (float)sc->gravity[1];
  p.gz = (float)sc->gravity[2];
  p.bc = (float)sc->bc_cells;
  p.res = sc->res;
  p.nn = sc->res + 1;
  p.n = (int)sc->n;
  d->stream = (cudaStream_t)stream;
  size_t nodes = 2ull * p.nn * p.nn * p.nn;
  bool ok = cudaMalloc(&d->gm, nodes * 4) == cudaSuccess && cudaMalloc(&d->gp, nodes * 12) == cudaSuccess &&
            cudaMalloc(&d->gv, nodes * 12) == cudaSuccess && cudaMalloc(&d->gvb, nodes * 12) == cudaSuccess &&
            cudaMalloc(&d->gpb, nodes * 12) == cudaSuccess && cudaMalloc(&d->gmb, nodes * 4) == cudaSuccess &&
            cudaMalloc(&d->err, 4) == cudaSuccess;
  if (!ok || cudaMemset(d->err, 0, 4) != cudaSuccess) {
    cudaGetLastError();
    ckmpm_diff_destroy(d);
    return CKMPM_ENOMEM;
  }
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  d->blocks = sms * 8;
  *out = d;
  return CKMPM_OK;
}

static ckmpm_status diff_forward_grid(ckmpm_diff* d, const float* x, const float* v, const float* B, const float* F,
                                      const float* E) {
  const ckd::DP& p = d->p;
  size_t nodes = 2ull * p.nn * p.nn * p.nn;
  if (cudaMemsetAsync(d->gm, 0, nodes * 4, d->stream) != cudaSuccess ||
      cudaMemsetAsync(d->gp, 0, nodes * 12, d->stream) != cudaSuccess)
    return CKMPM_ECUDA;
  ckd::k_fwd_p2g<<<d->blocks, 128, 0, d->stream>>>(p, x, v, B, F, E, d->gm, d->gp, d->err);
  ckd::k_fwd_grid<<<d->blocks, 256, 0, d->stream>>>(p, d->gm, d->gp, d->gv);
  return cudaGetLastError() == cudaSuccess ? CKMPM_OK : CKMPM_ECUDA;
}

ckmpm_status ckmpm_diff_step(ckmpm_diff* d, const float* x, const float* v, const float* B, const float* F,
                             const float* E, float* x1, float* v1, float* B1, float* F1) {
  if (!d || !x || !v || !B || !F || !E || !x1 || !v1 || !B1 || !F1) return CKMPM_EINVAL;
  ckmpm_status st = diff_forward_grid(d, x, v, B, F, E);
  if (st != CKMPM_OK) return st;
  ckd::k_fwd_g2p<<<d->blocks, 128, 0, d->stream>>>(d->p, x, F, d->gv, x1, v1, B1, F1, d->err);
  return cudaGetLastError() == cudaSuccess ? CKMPM_OK : CKMPM_ECUDA;
}

ckmpm_status ckmpm_diff_step_backward(ckmpm_diff* d, const float* x, const float* v, const float* B, const float* F,
                                      const float* E, const float* gx1, const float* gv1, const float* gB1,
                                      const float* gF1, float* gx, float* gv, float* gB, float* gF, float* gE) {
  if (!d || !x || !v || !B || !F || !E || !gx1 || !gv1 || !gB1 || !gF1 || !gx || !gv || !gB || !gF || !gE)
    return CKMPM_EINVAL;
  ckmpm_status st = diff_forward_grid(d, x, v, B, F, E);
  if (st != CKMPM_OK) return st;
  const ckd::DP& p = d->p;
  size_t nodes = 2ull * p.nn * p.nn * p.nn;
  if (cudaMemsetAsync(d->gvb, 0, nodes * 12, d->stream) != cudaSuccess) return CKMPM_ECUDA;
  ckd::k_bwd_g2p<<<d->blocks, 128, 0, d->stream>>>(p, x, F, d->gv, gx1, gv1, gB1, gF1, gx, gF, d->gvb);
  ckd::k_bwd_grid<<<d->blocks, 256, 0, d->stream>>>(p, d->gm, d->gp, d->gvb, d->gpb, d->gmb);
  ckd::k_bwd_p2g<<<d->blocks, 128, 0, d->stream>>>(p, x, v, B, F, E, d->gpb, d->gmb, gx, gv, gB, gF, gE);
  return cudaGetLastError() == cudaSuccess ? CKMPM_OK : CKMPM_ECUDA;
}

ckmpm_status ckmpm_diff_sync(ckmpm_diff* d) {
  if (!d) return CKMPM_EINVAL;
  if (cudaStreamSynchronize(d->stream) != cudaSuccess) return CKMPM_ECUDA;
  uint32_t e = 0;
  if (cudaMemcpy(&e, d->err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return CKMPM_ECUDA;
  return e ? CKMPM_EDOMAIN : CKMPM_OK;
}

ckmpm_status ckmpm_diff_destroy(ckmpm_diff* d) {
  if (!d) return CKMPM_OK;
  if (d->stream) cudaStreamSynchronize(d->stream);
  cudaFree(d->gm);
  cudaFree(d->gp);
  cudaFree(d->gv);
  cudaFree(d->gvb);
  cudaFree(d->gpb);
  cudaFree(d->gmb);
  cudaFree(d->err);
  cudaGetLastError();
  delete d;
  return CKMPM_OK;
}

}  // extern "C"
