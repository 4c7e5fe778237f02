// Device helpers shared by the upper-level band factorisations (one CTA in
// coarse_solve.cu, a cluster of CTAs in coarse_factor_cluster.cu).
#pragma once
#include "hms_internal.cuh"

namespace hms {
namespace coarse {

constexpr int NB = 16;  // block of columns / rows (the serial diagonal work per block grows as NB^3)

template <typename T>
struct Tau;
template <>
struct Tau<float> {
  static constexpr float v = 1e-6f;
};
template <>
struct Tau<double> {
  static constexpr double v = 1e-14;
};
// 1/sqrt(x): the hardware approximation in FP32 (the factor only needs to be a
// good preconditioner: FP64 refinement restores the accuracy), exact in FP64
__device__ inline float trsqrt(float x) { return rsqrtf(x); }
__device__ inline double trsqrt(double x) { return 1.0 / sqrt(x); }

// Column C of the register-resident Cholesky of an NB x NB diagonal block
// (lane = row; lanes >= NB hold zero rows).  A dropped column becomes a unit column with a zero row.
template <typename T, int C>
__device__ __forceinline__ void diag_steps(T (&a)[NB], unsigned dmask, int lane, unsigned& dropped_out,
                                           T (&rdiag)[NB]) {
  if constexpr (C < NB) {
    const T piv = __shfl_sync(0xffffffffu, a[C], C);
    const bool drop = ((dmask >> C) & 1u) != 0 || !(piv > Tau<T>::v);
    const T inv = drop ? T(1) : trsqrt(piv);
    const T d = drop ? T(1) : piv * inv;
    rdiag[C] = inv;  // 1 / L_CC
    const bool mine = lane == C;
    const T acl = a[C];
    a[C] = mine ? d : (lane > C ? (drop ? T(0) : acl * inv) : acl);
    if (drop) {  // warp-uniform and rare: the dropped row becomes zero
#pragma unroll
      for (int j = 0; j < C; ++j) a[j] = mine ? T(0) : a[j];
    }
    const T lc = a[C];
    // entries above the diagonal (lane < j) are never read: update them too
#pragma unroll
    for (int j = C + 1; j < NB; ++j) {
      const T ljc = __shfl_sync(0xffffffffu, lc, j);
      a[j] = fma(-lc, ljc, a[j]);
    }
    if (drop) dropped_out |= (1u << C);
    diag_steps<T, C + 1>(a, dmask, lane, dropped_out, rdiag);
  }
}

// four consecutive elements from 16-byte-aligned shared memory
__device__ inline void ld4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}
__device__ inline void ld4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}
__device__ inline void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ inline void st4(double* p, double a, double b, double c, double d) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
  *reinterpret_cast<double2*>(p + 2) = make_double2(c, d);
}

// The window holds band rows [k0, k0 + W) in circular row slots; row i keeps
// its entry of column j at position j mod lda.  lda >= bw + 4 is a multiple
// of 4 with lda / 4 odd, so the four entries (i, j..j+3), j = 0 mod 4, are one
// aligned 16-byte word, and such words of consecutive rows fall in different
// bank groups; positions outside the row's band [i - bw, i] are never read.
__host__ __device__ inline int window_lda(int bw) {
  int m = (bw + 4 + 3) / 4;
  if ((m & 1) == 0) ++m;
  return 4 * m;
}
// Warp 0: factor the diagonal block starting at row k (nbk rows) held in a[],
// write L to Ls, X = L^-1 to Xs and dinv, and the drop decisions.
template <typename T>
__device__ __forceinline__ void factor_diag_block(T (&a)[NB], int k, int nbk, int lane, int* sdrop, T* Ls, T* Xs,
                                                  T* __restrict__ dinv, unsigned* dropblk) {
  const unsigned dmask = __ballot_sync(0xffffffffu, lane >= nbk || sdrop[k + lane] != 0);
  unsigned dout = 0;
  T rdiag[NB];
  diag_steps<T, 0>(a, dmask, lane, dout, rdiag);
  if (lane < NB) {
#pragma unroll
    for (int j = 0; j < NB; ++j) Ls[lane * (NB + 1) + j] = (j <= lane) ? a[j] : T(0);
  }
  if (lane == 0) *dropblk = dout;
  __syncwarp();
  if (lane < nbk) sdrop[k + lane] = (dout >> lane) & 1u;
  // X = L^-1, lane c computes column c column-oriented: once x_q is known it
  // is subtracted from every later row, so the dependent chain is NB steps long
  T x[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) x[r] = (r == lane) ? T(1) : T(0);
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const T xq = (q >= lane) ? x[q] * rdiag[q] : T(0);
    x[q] = xq;
#pragma unroll
    for (int r = q + 1; r < NB; ++r) x[r] = fma(-Ls[r * (NB + 1) + q], xq, x[r]);
  }
  if (lane < NB) {
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      Xs[r * (NB + 1) + lane] = x[r];
      dinv[(size_t)(k / NB) * NB * NB + r * NB + lane] = x[r];
    }
  }
  __syncwarp();
}

}  // namespace coarse
}  // namespace hms
