// 3x3 singular value decomposition and the constitutive models, templated on
// the floating-point type so the same code runs in float32 and float64.
//
// SVD method: one-sided Jacobi in the spirit of McAdams, Selle, Tamstorf,
// Teran and Sifakis, "Computing the Singular Value Decomposition of 3x3
// matrices with minimal branching and elementary floating point operations"
// (UW-Madison TR1690, 2011): a symmetric cyclic Jacobi eigen-sweep on F^T F
// gives V, then a Givens QR of F V gives U and the singular values.  Each
// Jacobi rotation is exact (it zeroes its off-diagonal), with its angle taken
// from the half-angle identities cos^2(phi) = (1 + cos 2phi)/2,
// sin(phi) = sin(2phi) / (2 cos phi), so that it needs two reciprocal square
// roots and no division; the angle is kept in [-pi/4, pi/4].
// The result is rotation-variant: det U = det V = +1, sigma_0 >= sigma_1 >= 0
// and sigma_2 carries the sign of det F.
#pragma once
#include <cuda_runtime.h>

namespace ck {

template <typename T>
struct Num;
template <>
struct Num<float> {
  __device__ static __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  // reciprocal square root refined by one Newton step y <- y (3 - x y^2) / 2
  __device__ static __forceinline__ float rsqrt_(float x) {
    float y = rsqrtf(x);
    return y * (1.5f - 0.5f * x * y * y);
  }
  __device__ static __forceinline__ float abs_(float x) { return fabsf(x); }
  __device__ static __forceinline__ float log_(float x) { return logf(x); }
  __device__ static __forceinline__ float exp_(float x) { return expf(x); }
  __device__ static __forceinline__ float pow_(float x, float y) { return powf(x, y); }
  __device__ static __forceinline__ float cbrt_(float x) { return cbrtf(x); }
  static constexpr int sweeps = 4;
  static constexpr float eps = 5.9604645e-8f;  // 2^-24
};
template <>
struct Num<double> {
  __device__ static __forceinline__ double sqrt_(double x) { return sqrt(x); }
  __device__ static __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
  __device__ static __forceinline__ double abs_(double x) { return fabs(x); }
  __device__ static __forceinline__ double log_(double x) { return log(x); }
  __device__ static __forceinline__ double exp_(double x) { return exp(x); }
  __device__ static __forceinline__ double pow_(double x, double y) { return pow(x, y); }
  __device__ static __forceinline__ double cbrt_(double x) { return cbrt(x); }
  static constexpr int sweeps = 6;
  static constexpr double eps = 1.1102230246251565e-16;  // 2^-53
};

// Row-major 3x3 helpers.
#define CK_M(a, i, j) (a)[(i)*3 + (j)]

// Jacobi rotation zeroing S[p][q].  An off-diagonal below half an ulp of the
// diagonal is dropped without rotating: rotating it away (a 45 degree turn
// when S[p][p] ~ S[q][q], e.g. F ~ I) changes nothing exact but rounds the
// rotation's c and s and puts an ulp of noise into the singular values.
template <typename T>
__device__ __forceinline__ void jacobi_rotate(T* S, T* V, int p, int q, int r) {
  const T apq = CK_M(S, p, q), spp = CK_M(S, p, p), sqq = CK_M(S, q, q);
  if (Num<T>::abs_(apq) <= Num<T>::eps * (Num<T>::abs_(spp) + Num<T>::abs_(sqq))) {
    CK_M(S, p, q) = T(0);
    CK_M(S, q, p) = T(0);
    return;
  }
  // S' = J^T S J, J = [[c, s], [-s, c]] in the (p, q) plane; S'_pq = 0 needs
  // cos(2phi) S_pq + sin(2phi) (S_pp - S_qq) / 2 = 0.
  const T x = spp - sqq, y = T(2) * apq;
  const T ir = Num<T>::rsqrt_(x * x + y * y);
  const T c2 = Num<T>::abs_(x) * ir;            // cos 2phi >= 0
  const T s2 = (x >= T(0) ? -y : y) * ir;      // sin 2phi
  const T h = T(0.5) + T(0.5) * c2;            // cos^2 phi in [1/2, 1]
  const T rh = Num<T>::rsqrt_(h);
  const T c = h * rh;
  const T s = T(0.5) * s2 * rh;
  const T cc = c * c, ss = s * s, cs2 = T(2) * c * s;
  const T srp = CK_M(S, r, p), srq = CK_M(S, r, q);
  const T nrp = c * srp - s * srq;
  const T nrq = s * srp + c * srq;
  CK_M(S, p, p) = cc * spp - cs2 * apq + ss * sqq;
  CK_M(S, q, q) = ss * spp + cs2 * apq + cc * sqq;
  CK_M(S, p, q) = T(0);
  CK_M(S, q, p) = T(0);
  CK_M(S, r, p) = nrp;
  CK_M(S, p, r) = nrp;
  CK_M(S, r, q) = nrq;
  CK_M(S, q, r) = nrq;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T vp = CK_M(V, i, p), vq = CK_M(V, i, q);
    CK_M(V, i, p) = c * vp - s * vq;
    CK_M(V, i, q) = s * vp + c * vq;
  }
}

template <typename T>
__device__ __forceinline__ void swap_cols_neg(T* V, T* e, int a, int b) {
  // swap eigenpairs a and b; negate one column so det V stays +1
  T t = e[a];
  e[a] = e[b];
  e[b] = t;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T va = CK_M(V, i, a);
    CK_M(V, i, a) = CK_M(V, i, b);
    CK_M(V, i, b) = -va;
  }
}

template <typename T>
__device__ __forceinline__ void givens_rows(T* Bm, T* U, int p, int q) {
  // zero Bm[q][p] by rotating rows p and q (Bm[p][p] ends >= 0); U <- U G^T
  const T a = CK_M(Bm, p, p), b = CK_M(Bm, q, p);
  T c, s;
  if (b == T(0)) {
    c = a >= T(0) ? T(1) : T(-1);
    s = T(0);
  } else {
    const T ir = Num<T>::rsqrt_(a * a + b * b);
    c = a * ir;
    s = b * ir;
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    T bp = CK_M(Bm, p, j), bq = CK_M(Bm, q, j);
    CK_M(Bm, p, j) = c * bp + s * bq;
    CK_M(Bm, q, j) = -s * bp + c * bq;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T up = CK_M(U, i, p), uq = CK_M(U, i, q);
    CK_M(U, i, p) = c * up + s * uq;
    CK_M(U, i, q) = -s * up + c * uq;
  }
}

// F = U diag(sig) V^T, rotation-variant.
template <typename T>
__device__ __forceinline__ void svd3(const T* F, T* U, T* sig, T* V) {
  T S[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      CK_M(S, i, j) = CK_M(F, 0, i) * CK_M(F, 0, j) + CK_M(F, 1, i) * CK_M(F, 1, j) + CK_M(F, 2, i) * CK_M(F, 2, j);
#pragma unroll
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? T(1) : T(0);
  // cyclic sweeps until every off-diagonal is below half an ulp of its
  // diagonal pair (Jacobi converges quadratically; F near a rotation times a
  // small stretch needs about two sweeps), at most Num<T>::sweeps
#pragma unroll 1
  for (int sw = 0; sw < Num<T>::sweeps; ++sw) {
    jacobi_rotate(S, V, 0, 1, 2);
    jacobi_rotate(S, V, 0, 2, 1);
    jacobi_rotate(S, V, 1, 2, 0);
    const T e = Num<T>::eps;
    if (Num<T>::abs_(CK_M(S, 0, 1)) <= e * (Num<T>::abs_(CK_M(S, 0, 0)) + Num<T>::abs_(CK_M(S, 1, 1))) &&
        Num<T>::abs_(CK_M(S, 0, 2)) <= e * (Num<T>::abs_(CK_M(S, 0, 0)) + Num<T>::abs_(CK_M(S, 2, 2))) &&
        Num<T>::abs_(CK_M(S, 1, 2)) <= e * (Num<T>::abs_(CK_M(S, 1, 1)) + Num<T>::abs_(CK_M(S, 2, 2))))
      break;
  }
  T e[3] = {CK_M(S, 0, 0), CK_M(S, 1, 1), CK_M(S, 2, 2)};
  if (e[0] < e[1]) swap_cols_neg(V, e, 0, 1);
  if (e[0] < e[2]) swap_cols_neg(V, e, 0, 2);
  if (e[1] < e[2]) swap_cols_neg(V, e, 1, 2);
  T Bm[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      CK_M(Bm, i, j) = CK_M(F, i, 0) * CK_M(V, 0, j) + CK_M(F, i, 1) * CK_M(V, 1, j) + CK_M(F, i, 2) * CK_M(V, 2, j);
#pragma unroll
  for (int i = 0; i < 9; ++i) U[i] = (i % 4 == 0) ? T(1) : T(0);
  givens_rows(Bm, U, 0, 1);
  givens_rows(Bm, U, 0, 2);
  givens_rows(Bm, U, 1, 2);
  sig[0] = CK_M(Bm, 0, 0);
  sig[1] = CK_M(Bm, 1, 1);
  sig[2] = CK_M(Bm, 2, 2);
}

// Symmetric eigen-decomposition S = Q diag(e) Q^T by the same cyclic Jacobi
// sweeps (no sorting); S is overwritten.
template <typename T>
__device__ __forceinline__ void sym_eig3(T* S, T* Q, T* e) {
#pragma unroll
  for (int i = 0; i < 9; ++i) Q[i] = (i % 4 == 0) ? T(1) : T(0);
#pragma unroll 1
  for (int sw = 0; sw < Num<T>::sweeps; ++sw) {
    jacobi_rotate(S, Q, 0, 1, 2);
    jacobi_rotate(S, Q, 0, 2, 1);
    jacobi_rotate(S, Q, 1, 2, 0);
    const T ep = Num<T>::eps;
    if (Num<T>::abs_(CK_M(S, 0, 1)) <= ep * (Num<T>::abs_(CK_M(S, 0, 0)) + Num<T>::abs_(CK_M(S, 1, 1))) &&
        Num<T>::abs_(CK_M(S, 0, 2)) <= ep * (Num<T>::abs_(CK_M(S, 0, 0)) + Num<T>::abs_(CK_M(S, 2, 2))) &&
        Num<T>::abs_(CK_M(S, 1, 2)) <= ep * (Num<T>::abs_(CK_M(S, 1, 1)) + Num<T>::abs_(CK_M(S, 2, 2))))
      break;
  }
  e[0] = CK_M(S, 0, 0);
  e[1] = CK_M(S, 1, 1);
  e[2] = CK_M(S, 2, 2);
}

// ---------------------------------------------------------------- materials

constexpr float kSigmaFloor = 1e-6f;

// Fixed-corotated Kirchhoff stress tau = 2 mu (F - R) F^T + lam J (J - 1) I,
// R = U V^T (stomakhin2012, cited in Sec. 6.1).
template <typename T>
__device__ __forceinline__ void fc_tau(const T* F, const T* U, const T* sig, const T* V, T mu, T lam, T* tau) {
  T R[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      CK_M(R, i, j) = CK_M(U, i, 0) * CK_M(V, j, 0) + CK_M(U, i, 1) * CK_M(V, j, 1) + CK_M(U, i, 2) * CK_M(V, j, 2);
  T J = sig[0] * sig[1] * sig[2];
  T D[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) D[i] = F[i] - R[i];
  T vol = lam * J * (J - T(1));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      CK_M(tau, i, j) = T(2) * mu * (CK_M(D, i, 0) * CK_M(F, j, 0) + CK_M(D, i, 1) * CK_M(F, j, 1) + CK_M(D, i, 2) * CK_M(F, j, 2)) +
                        (i == j ? vol : T(0));
}

// Hencky Kirchhoff stress U diag(2 mu eps + lam tr eps) U^T, eps = ln sigma.
template <typename T>
__device__ __forceinline__ void hencky_tau(const T* U, const T* sig, T mu, T lam, T* tau) {
  T e0 = Num<T>::log_(sig[0] > T(kSigmaFloor) ? sig[0] : T(kSigmaFloor));
  T e1 = Num<T>::log_(sig[1] > T(kSigmaFloor) ? sig[1] : T(kSigmaFloor));
  T e2 = Num<T>::log_(sig[2] > T(kSigmaFloor) ? sig[2] : T(kSigmaFloor));
  T tr = e0 + e1 + e2;
  T d0 = T(2) * mu * e0 + lam * tr, d1 = T(2) * mu * e1 + lam * tr, d2 = T(2) * mu * e2 + lam * tr;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      CK_M(tau, i, j) = CK_M(U, i, 0) * d0 * CK_M(U, j, 0) + CK_M(U, i, 1) * d1 * CK_M(U, j, 1) + CK_M(U, i, 2) * d2 * CK_M(U, j, 2);
}

// Drucker-Prager projection of the singular values (klar2016): returns true
// when sigma changed.  Tension (tr eps >= 0) goes to the tip; otherwise the
// state moves only when dgamma > 0, which with tr eps < 0 implies
// |eps^| > 0, so a purely volumetric compression (eps^ = 0) stays inside.
template <typename T>
__device__ __forceinline__ bool dp_project(T* sig, T mu, T lam, T alpha) {
  T e0 = Num<T>::log_(sig[0] > T(kSigmaFloor) ? sig[0] : T(kSigmaFloor));
  T e1 = Num<T>::log_(sig[1] > T(kSigmaFloor) ? sig[1] : T(kSigmaFloor));
  T e2 = Num<T>::log_(sig[2] > T(kSigmaFloor) ? sig[2] : T(kSigmaFloor));
  T tr = e0 + e1 + e2;
  T h0 = e0 - tr / T(3), h1 = e1 - tr / T(3), h2 = e2 - tr / T(3);
  T nrm = Num<T>::sqrt_(h0 * h0 + h1 * h1 + h2 * h2);
  if (tr >= T(0)) {
    sig[0] = sig[1] = sig[2] = T(1);
    return true;
  }
  T dg = nrm + (T(3) * lam + T(2) * mu) / (T(2) * mu) * tr * alpha;
  if (!(dg > T(0) && nrm > T(0))) return false;  // inside the cone (nrm > 0 follows for alpha >= 0)
  T k = dg / nrm;
  sig[0] = Num<T>::exp_(e0 - k * h0);
  sig[1] = Num<T>::exp_(e1 - k * h1);
  sig[2] = Num<T>::exp_(e2 - k * h2);
  return true;
}

// U diag(sig) V^T
template <typename T>
__device__ __forceinline__ void usvt(const T* U, const T* sig, const T* V, T* F) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      CK_M(F, i, j) = CK_M(U, i, 0) * sig[0] * CK_M(V, j, 0) + CK_M(U, i, 1) * sig[1] * CK_M(V, j, 1) +
                      CK_M(U, i, 2) * sig[2] * CK_M(V, j, 2);
}

// Constitutive update on F (already advanced by (I + dt C)): plasticity for
// Drucker-Prager, then the Kirchhoff stress of the resulting F.
template <typename T>
__device__ __forceinline__ void constitutive(int model, T* F, T mu, T lam, T alpha, T* tau, T* sig_out) {
  T U[9], V[9], sig[3];
  svd3<T>(F, U, sig, V);
  if (model == 1) {
    if (dp_project<T>(sig, mu, lam, alpha)) usvt<T>(U, sig, V, F);
    hencky_tau<T>(U, sig, mu, lam, tau);
  } else {
    fc_tau<T>(F, U, sig, V, mu, lam, tau);
  }
  sig_out[0] = sig[0];
  sig_out[1] = sig[1];
  sig_out[2] = sig[2];
}

// Constitutive update from the left stretch: b = F F^T = U diag(e) U^T,
// e = sigma^2, gives U and sigma without V (F = U Sigma V^T, det F > 0).
// Drucker-Prager works on the log strains eps = ln(e) / 2 directly: the
// return map gives eps_new, then F <- U diag(exp(eps_new - eps)) U^T F
// (= U Sigma_new V^T) and the Hencky stress U diag(2 mu eps_new + lam tr
// eps_new) U^T, with no log of the projected sigma and no division.
// Fixed-corotated: R = U diag(1 / sigma) U^T F (= U V^T) and 2 mu (F - R) F^T
// + lam J (J - 1) I.  Used in float32 for well-conditioned F with det F > 0.
template <typename T>
__device__ __forceinline__ void constitutive_left(int model, T* F, T mu, T lam, T alpha, T* tau, const T* U,
                                                  const T* e, const T* sig) {
  if (model == 1) {
    const T fl = T(kSigmaFloor) * T(kSigmaFloor);
    T ep[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) ep[a] = T(0.5) * Num<T>::log_(e[a] > fl ? e[a] : fl);
    const T tr = ep[0] + ep[1] + ep[2];
    const T h0 = ep[0] - tr / T(3), h1 = ep[1] - tr / T(3), h2 = ep[2] - tr / T(3);
    const T nrm = Num<T>::sqrt_(h0 * h0 + h1 * h1 + h2 * h2);
    T en[3] = {ep[0], ep[1], ep[2]};
    bool moved = false;
    if (tr >= T(0)) {  // tension: the tip
      en[0] = en[1] = en[2] = T(0);
      moved = true;
    } else {
      const T dg = nrm + (T(3) * lam + T(2) * mu) / (T(2) * mu) * tr * alpha;
      if (dg > T(0) && nrm > T(0)) {
        const T k = dg / nrm;
        en[0] = ep[0] - k * h0;
        en[1] = ep[1] - k * h1;
        en[2] = ep[2] - k * h2;
        moved = true;
      }
    }
    if (moved) {
      const T k[3] = {Num<T>::exp_(en[0] - ep[0]), Num<T>::exp_(en[1] - ep[1]), Num<T>::exp_(en[2] - ep[2])};
      T W[9], Fn[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          CK_M(W, i, j) = CK_M(U, i, 0) * k[0] * CK_M(U, j, 0) + CK_M(U, i, 1) * k[1] * CK_M(U, j, 1) +
                          CK_M(U, i, 2) * k[2] * CK_M(U, j, 2);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          CK_M(Fn, i, j) = CK_M(W, i, 0) * CK_M(F, 0, j) + CK_M(W, i, 1) * CK_M(F, 1, j) + CK_M(W, i, 2) * CK_M(F, 2, j);
#pragma unroll
      for (int q = 0; q < 9; ++q) F[q] = Fn[q];
    }
    const T trn = en[0] + en[1] + en[2];
    const T d0 = T(2) * mu * en[0] + lam * trn, d1 = T(2) * mu * en[1] + lam * trn, d2 = T(2) * mu * en[2] + lam * trn;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        CK_M(tau, i, j) = CK_M(U, i, 0) * d0 * CK_M(U, j, 0) + CK_M(U, i, 1) * d1 * CK_M(U, j, 1) +
                          CK_M(U, i, 2) * d2 * CK_M(U, j, 2);
  } else {
    T k[3] = {T(1) / sig[0], T(1) / sig[1], T(1) / sig[2]};
    T W[9], R[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        CK_M(W, i, j) = CK_M(U, i, 0) * k[0] * CK_M(U, j, 0) + CK_M(U, i, 1) * k[1] * CK_M(U, j, 1) +
                        CK_M(U, i, 2) * k[2] * CK_M(U, j, 2);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        CK_M(R, i, j) = CK_M(W, i, 0) * CK_M(F, 0, j) + CK_M(W, i, 1) * CK_M(F, 1, j) + CK_M(W, i, 2) * CK_M(F, 2, j);
    const T J = sig[0] * sig[1] * sig[2];
    T D[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) D[i] = F[i] - R[i];
    const T vol = lam * J * (J - T(1));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        CK_M(tau, i, j) = T(2) * mu * (CK_M(D, i, 0) * CK_M(F, j, 0) + CK_M(D, i, 1) * CK_M(F, j, 1) + CK_M(D, i, 2) * CK_M(F, j, 2)) +
                          (i == j ? vol : T(0));
  }
}

// ------------------------------------------- Drucker-Prager for small stretches
//
// Symmetric 3x3 matrices as (00, 11, 22, 01, 02, 12).  sym_mul forms A B for
// commuting symmetric A and B (polynomials in one matrix), which is symmetric.
__device__ __forceinline__ void sym_mul(const float* a, const float* b, float* c) {
  c[0] = a[0] * b[0] + a[3] * b[3] + a[4] * b[4];
  c[1] = a[3] * b[3] + a[1] * b[1] + a[5] * b[5];
  c[2] = a[4] * b[4] + a[5] * b[5] + a[2] * b[2];
  c[3] = a[0] * b[3] + a[3] * b[1] + a[4] * b[5];
  c[4] = a[0] * b[4] + a[3] * b[5] + a[4] * b[2];
  c[5] = a[3] * b[4] + a[1] * b[5] + a[5] * b[2];
}

// X = F F^T - I from D = F - I as D + D^T + D D^T (no cancellation against the
// identity), and its largest row abs-sum.
__device__ __forceinline__ float left_strain(const float* F, float* X) {
  const float d[9] = {F[0] - 1.f, F[1], F[2], F[3], F[4] - 1.f, F[5], F[6], F[7], F[8] - 1.f};
  X[0] = 2.f * d[0] + (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  X[1] = 2.f * d[4] + (d[3] * d[3] + d[4] * d[4] + d[5] * d[5]);
  X[2] = 2.f * d[8] + (d[6] * d[6] + d[7] * d[7] + d[8] * d[8]);
  X[3] = d[1] + d[3] + (d[0] * d[3] + d[1] * d[4] + d[2] * d[5]);
  X[4] = d[2] + d[6] + (d[0] * d[6] + d[1] * d[7] + d[2] * d[8]);
  X[5] = d[5] + d[7] + (d[3] * d[6] + d[4] * d[7] + d[5] * d[8]);
  const float r0 = fabsf(X[0]) + fabsf(X[3]) + fabsf(X[4]);
  const float r1 = fabsf(X[3]) + fabsf(X[1]) + fabsf(X[5]);
  const float r2 = fabsf(X[4]) + fabsf(X[5]) + fabsf(X[2]);
  return fmaxf(r0, fmaxf(r1, r2));
}

// The Drucker-Prager update of Sec. 3.2 step 4 (klar2016 return map, Hencky
// elasticity) without an eigen-decomposition, for F F^T = I + X with the
// largest row abs-sum xr of X at most 1/48 (every stretch within about 1% of 1).
// The log strain is a matrix function of the left stretch V = (F F^T)^(1/2):
// L = log V = log(I + X) / 2 has the eigenvectors U of F F^T and eigenvalues
// eps_i = ln sigma_i, so tr eps = tr L and |eps^| = |dev L|_F.  The return map
// moves eps along eps^ (or to 0 at the tip), which is L_new = L - k dev L (or
// 0); then F_new = U diag(exp(eps_new - eps)) U^T F = exp(L_new - L) F and the
// Hencky stress is 2 mu L_new + lam tr(L_new) I.  log(I + X) and exp(Y) are
// their series through the d-th power in Horner form (products of commuting
// symmetric matrices), with d chosen from xr (the spectral radius of X is at
// most xr; L's is about xr/2, so that of Y, -L or a part of dev L, is below
// xr): the log's truncation is below
// xr^(d+1) / ((d+1)(1-xr)), i.e. below 4e-8 xr, for d = 2 up to xr = 3.4e-4,
// d = 3 up to 5.4e-3 and d = 4 up to 1/48; the exponential's is smaller at the
// same d.  One degree serves the warp (its largest), so neighbouring particles
// do not diverge; the degree-4 case is the one this update always used.
__device__ __forceinline__ int dp_lane_degree(float xr) { return xr <= 3.4e-4f ? 2 : xr <= 5.4e-3f ? 3 : 4; }

// lane_deg: dp_lane_degree of the particle's xr
__device__ __forceinline__ void dp_small_strain(float* F, const float* X, int lane_deg, float mu, float lam,
                                                float dpc, float* tau) {
  const int deg = __reduce_max_sync(__activemask(), lane_deg);
  float Z[6], W[6];
  // log(I + X) = X Q(X), Q = I - X/2 + X^2/3 - X^3/4 through degree deg:
  // Z = I/(deg-1) - X/deg, then Z = I/k - X Z for k = deg-2 .. 1
  const float za = deg == 4 ? 1.f / 3.f : deg == 3 ? 0.5f : 1.f;
  const float zb = deg == 4 ? 0.25f : deg == 3 ? 1.f / 3.f : 0.5f;
#pragma unroll
  for (int q = 0; q < 6; ++q) Z[q] = -zb * X[q] + (q < 3 ? za : 0.f);
  if (deg == 4) {
    sym_mul(X, Z, W);
#pragma unroll
    for (int q = 0; q < 6; ++q) Z[q] = -W[q] + (q < 3 ? 0.5f : 0.f);
  }
  if (deg >= 3) {
    sym_mul(X, Z, W);
#pragma unroll
    for (int q = 0; q < 6; ++q) Z[q] = -W[q] + (q < 3 ? 1.f : 0.f);
  }
  float L[6];
  sym_mul(X, Z, L);
#pragma unroll
  for (int q = 0; q < 6; ++q) L[q] *= 0.5f;
  const float tr = L[0] + L[1] + L[2];
  const float h[6] = {L[0] - tr * (1.f / 3.f), L[1] - tr * (1.f / 3.f), L[2] - tr * (1.f / 3.f), L[3], L[4], L[5]};
  const float nrm = sqrtf(h[0] * h[0] + h[1] * h[1] + h[2] * h[2] + 2.f * (h[3] * h[3] + h[4] * h[4] + h[5] * h[5]));
  float Ln[6] = {L[0], L[1], L[2], L[3], L[4], L[5]};
  float Y[6];
  bool moved = false;
  if (tr >= 0.f) {  // tension: the tip
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      Ln[q] = 0.f;
      Y[q] = -L[q];
    }
    moved = true;
  } else {
    const float dg = nrm + dpc * tr;
    if (dg > 0.f && nrm > 0.f) {
      const float k = dg / nrm;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        Y[q] = -k * h[q];
        Ln[q] = L[q] + Y[q];
      }
      moved = true;
    }
  }
  if (moved) {
    // exp(Y) = I + Y P(Y), P = I + Y/2 + Y^2/6 + Y^3/24 through degree deg:
    // Z = I/(deg-1)! + Y/deg!, then Z = I/k! + Y Z for k = deg-2 .. 1
    const float ea = deg == 4 ? 1.f / 6.f : deg == 3 ? 0.5f : 1.f;
    const float eb = deg == 4 ? 1.f / 24.f : deg == 3 ? 1.f / 6.f : 0.5f;
#pragma unroll
    for (int q = 0; q < 6; ++q) Z[q] = Y[q] * eb + (q < 3 ? ea : 0.f);
    if (deg == 4) {
      sym_mul(Y, Z, W);
#pragma unroll
      for (int q = 0; q < 6; ++q) Z[q] = W[q] + (q < 3 ? 0.5f : 0.f);
    }
    if (deg >= 3) {
      sym_mul(Y, Z, W);
#pragma unroll
      for (int q = 0; q < 6; ++q) Z[q] = W[q] + (q < 3 ? 1.f : 0.f);
    }
    float Ex[6];
    sym_mul(Y, Z, Ex);
    Ex[0] += 1.f;
    Ex[1] += 1.f;
    Ex[2] += 1.f;
    const float Em[9] = {Ex[0], Ex[3], Ex[4], Ex[3], Ex[1], Ex[5], Ex[4], Ex[5], Ex[2]};
    float Fn[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        CK_M(Fn, i, j) = CK_M(Em, i, 0) * CK_M(F, 0, j) + CK_M(Em, i, 1) * CK_M(F, 1, j) + CK_M(Em, i, 2) * CK_M(F, 2, j);
#pragma unroll
    for (int q = 0; q < 9; ++q) F[q] = Fn[q];
  }
  const float trn = Ln[0] + Ln[1] + Ln[2];
  const float m2 = 2.f * mu, vol = lam * trn;
  tau[0] = m2 * Ln[0] + vol;
  tau[4] = m2 * Ln[1] + vol;
  tau[8] = m2 * Ln[2] + vol;
  tau[1] = tau[3] = m2 * Ln[3];
  tau[2] = tau[6] = m2 * Ln[4];
  tau[5] = tau[7] = m2 * Ln[5];
}

// J-based fluid (the equation of state of the dam-break scenes): J = det F,
// pressure p = B (J^-gamma - 1), Kirchhoff stress tau = -J p I.
template <typename T>
__device__ __forceinline__ T det3(const T* F) {
  return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) + F[2] * (F[3] * F[7] - F[4] * F[6]);
}
template <typename T>
__device__ __forceinline__ void fluid_tau_of_J(T J, T Bk, T gamma, T* tau) {
  const T s = -J * Bk * (Num<T>::pow_(J, -gamma) - T(1));
#pragma unroll
  for (int q = 0; q < 9; ++q) tau[q] = (q % 4 == 0) ? s : T(0);
}
// The fluid's update after F' = (I + dt C) F: it keeps only the volume ratio,
// F <- J^(1/3) I, and its stress depends on J alone.
template <typename T>
__device__ __forceinline__ void fluid_update(T* F, T Bk, T gamma, T* tau) {
  const T J = det3(F);
  const T c = Num<T>::cbrt_(J);
#pragma unroll
  for (int q = 0; q < 9; ++q) F[q] = (q % 4 == 0) ? c : T(0);
  fluid_tau_of_J(J, Bk, gamma, tau);
}

// Kirchhoff stress of a given F without plasticity (used by readback/upload).
template <typename T>
__device__ __forceinline__ void stress_only(int model, const T* F, T mu, T lam, T* tau) {
  T U[9], V[9], sig[3];
  svd3<T>(F, U, sig, V);
  if (model == 1)
    hencky_tau<T>(U, sig, mu, lam, tau);
  else
    fc_tau<T>(F, U, sig, V, mu, lam, tau);
}

}  // namespace ck
