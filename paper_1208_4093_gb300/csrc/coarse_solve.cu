// K4: the upper-level ("master") solve of Eq. 8.
//
// K_aa is symmetric positive (semi)definite and banded when its unknowns are
// ordered set by set (9 per set) over the row-major set grid: set I couples to
// its eight neighbours, the farthest at I + Mx + 1, so the half-bandwidth is
// bw = 9 (Mx + 2) - 1.  With D = diag(K_aa) the Jacobi-scaled matrix
// A = D^-1/2 K_aa D^-1/2 has a unit diagonal and a condition number of a few
// thousand on these lattices, so it is factored in FP32 and the solution is
// refined in FP64:
//   x = 0, res = b = D^-1/2 P;  repeat: x += A32^-1 res, res = b - A x (FP64)
// reaching the FP64 solution after a few solves.  A mode is dropped (a = 0)
// when its diagonal is <= 1e-300 or its FP32 pivot is <= 1e-6, in the fixed
// order of the unknowns.
//
//   k_coarse_factor  one CTA: right-looking band Cholesky in 32-column blocks;
//                    the active window (bw + 32 rows of the band) lives in
//                    shared memory as circular row-band storage; the diagonal
//                    block is factored in registers by one warp, inverted, and
//                    the panel and rank-32 trailing update follow.  Writes L in
//                    column-band and row-band layouts and the inverted 32 x 32
//                    diagonal blocks.
//   k_coarse_solve   one CTA: block forward / back substitution (32 rows per
//                    step, products with the inverted diagonal blocks); adds
//                    the FP32 correction to the FP64 solution; the last solve
//                    also writes a = D^-1/2 x.
//   k_coarse_residual many CTAs, FP64: res = b - A x over the band.
#include "hms_internal.cuh"

namespace hms {
namespace {

constexpr int NB = 32;          // block of columns
constexpr int FT = 1024;        // threads of the factor / solve CTA
constexpr float TAU32 = 1e-6f;  // FP32 pivot drop threshold (unit-diagonal matrix)

__device__ inline float warp_sum_f(float v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}
__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

struct FactorSmem {
  int W, ldw, pstr;
  size_t aw_off, pc_off, ls_off, xs_off, total_floats;
};
__host__ __device__ inline FactorSmem factor_layout(int bw) {
  FactorSmem L;
  L.W = bw + NB;
  L.ldw = bw + 1;
  L.pstr = ((bw + 3) / 4) * 4 + 4;
  L.aw_off = 0;
  L.pc_off = L.aw_off + (size_t)L.W * L.ldw;
  L.pc_off = (L.pc_off + 3) / 4 * 4;
  L.ls_off = L.pc_off + (size_t)NB * L.pstr;
  L.xs_off = L.ls_off + NB * (NB + 1);
  L.total_floats = L.xs_off + NB * (NB + 1);
  return L;
}

// fband: scaled FP32 band in column layout [c][k] = A[c+k][c]; overwritten by L.
// lrow: L in row layout [i][k] = L[i][i-k].  dinv: inverted diagonal blocks,
// block K at dinv[K*NB*NB], row-major X[r][c].
__global__ void __launch_bounds__(FT) k_coarse_factor(int n, int bw, float* __restrict__ fband,
                                                      float* __restrict__ lrow, float* __restrict__ dinv,
                                                      int* __restrict__ dropped, const IterCtl* ctl) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  extern __shared__ float fs[];
  const FactorSmem LY = factor_layout(bw);
  const int W = LY.W, ldw = LY.ldw, pstr = LY.pstr;
  float* Aw = fs + LY.aw_off;
  float* Pc = fs + LY.pc_off;
  float* Ls = fs + LY.ls_off;
  float* Xs = fs + LY.xs_off;
  __shared__ int dropblk[NB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // initial window: rows [0, min(n, W))
  {
    const int rows = n < W ? n : W;
    for (int q = tid; q < rows * ldw; q += FT) {
      const int i = q / ldw, kk = q % ldw;
      const int j = i - kk;
      Aw[(i % W) * ldw + kk] = (j >= 0) ? fband[(size_t)j * ldw + kk] : 0.0f;
    }
  }
  __syncthreads();

  for (int k0 = 0; k0 < n; k0 += NB) {
    const int k1 = min(k0 + NB, n), nbk = k1 - k0;
    const int rend = min(n, k1 + bw), np = rend - k1;
    // (1) diagonal block in registers of warp 0 (lane = row)
    if (warp == 0) {
      float a[NB];
      const int row = k0 + lane;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int col = k0 + j;
        a[j] = (lane < nbk && j <= lane && row - col <= bw) ? Aw[(row % W) * ldw + (row - col)] : 0.0f;
      }
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        const float piv = __shfl_sync(0xffffffffu, a[c], c);
        bool drop = (c >= nbk);
        if (!drop) drop = dropped[k0 + c] != 0 || !(piv > TAU32);
        const float d = drop ? 1.0f : sqrtf(piv);
        const float inv = 1.0f / d;
        if (lane == c) {
          a[c] = d;
          if (drop) {
#pragma unroll
            for (int j = 0; j < c; ++j) a[j] = 0.0f;
          }
        }
        if (lane > c) a[c] = drop ? 0.0f : a[c] * inv;
#pragma unroll
        for (int j = c + 1; j < NB; ++j) {
          const float ljc = __shfl_sync(0xffffffffu, a[c], j);
          if (lane >= j) a[j] = fmaf(-a[c], ljc, a[j]);
        }
        if (lane == 0) dropblk[c] = drop ? 1 : 0;
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) Ls[lane * (NB + 1) + j] = (j <= lane) ? a[j] : 0.0f;
      __syncwarp();
      if (lane < nbk) dropped[k0 + lane] = dropblk[lane];
      // X = Ls^-1, lane c computes column c
      float x[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        float acc = (r == lane) ? 1.0f : 0.0f;
#pragma unroll
        for (int kq = 0; kq < r; ++kq) acc = fmaf(-Ls[r * (NB + 1) + kq], x[kq], acc);
        x[r] = (r >= lane) ? acc / Ls[r * (NB + 1) + r] : 0.0f;
      }
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        Xs[r * (NB + 1) + lane] = x[r];
        dinv[(size_t)(k0 / NB) * NB * NB + r * NB + lane] = x[r];
      }
    }
    __syncthreads();
    // (2) panel: P[i][c] = sum_{c' <= c} A[i][k0+c'] X[c][c'],  i in [k1, rend)
    for (int q = tid; q < np * NB; q += FT) {
      const int il = q / NB, c = q % NB;
      const int i = k1 + il;
      float acc = 0.0f;
      if (c < nbk && !dropblk[c]) {
        const float* arow = Aw + (i % W) * ldw;
        for (int cp = 0; cp <= c; ++cp) {
          const int kk = i - (k0 + cp);
          if (kk <= bw) acc = fmaf(arow[kk], Xs[c * (NB + 1) + cp], acc);
        }
      }
      Pc[c * pstr + il] = acc;
    }
    __syncthreads();
    // (3) finished columns [k0, k1) of L to global, both layouts
    for (int q = tid; q < nbk * ldw; q += FT) {
      const int cl = q / ldw, kk = q % ldw;
      const int c = k0 + cl, i = c + kk;
      float v = 0.0f;
      if (i < n) {
        if (i < k1) v = Ls[(i - k0) * (NB + 1) + cl];
        else if (i < rend) v = Pc[cl * pstr + (i - k1)];
      }
      fband[(size_t)c * ldw + kk] = v;
      if (i < n) lrow[(size_t)i * ldw + kk] = v;
    }
    // (4) trailing update A[i][j] -= sum_c P[i][c] P[j][c], k1 <= j <= i < rend, 4 x 4 tiles
    {
      const int T = (np + 3) / 4;
      const int npairs = T * (T + 1) / 2;
      for (int q = tid; q < npairs; q += FT) {
        int ti = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
        while (ti * (ti + 1) / 2 > q) --ti;
        while ((ti + 1) * (ti + 2) / 2 <= q) ++ti;
        const int tj = q - ti * (ti + 1) / 2;
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
        for (int c = 0; c < nbk; ++c) {
          const float4 pi = *reinterpret_cast<const float4*>(Pc + c * pstr + 4 * ti);
          const float4 pj = *reinterpret_cast<const float4*>(Pc + c * pstr + 4 * tj);
          const float ri[4] = {pi.x, pi.y, pi.z, pi.w}, rj[4] = {pj.x, pj.y, pj.z, pj.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(ri[u], rj[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int i = k1 + 4 * ti + u, j = k1 + 4 * tj + v;
            if (i < rend && j <= i) Aw[(i % W) * ldw + (i - j)] -= acc[u][v];
          }
      }
    }
    __syncthreads();
    // (5) slide the window: rows [k0 + W, k1 + W) enter
    {
      const int r0 = k0 + W, r1 = min(k1 + W, n);
      for (int q = tid; q < (r1 > r0 ? r1 - r0 : 0) * ldw; q += FT) {
        const int i = r0 + q / ldw, kk = q % ldw;
        const int j = i - kk;
        Aw[(i % W) * ldw + kk] = fband[(size_t)j * ldw + kk];
      }
    }
    __syncthreads();
  }
}

// One FP32 solve with the factor, added to the FP64 solution x.
__global__ void __launch_bounds__(FT) k_coarse_solve(int n, int bw, const float* __restrict__ lcol,
                                                     const float* __restrict__ lrow,
                                                     const float* __restrict__ dinv,
                                                     const int* __restrict__ dropped,
                                                     const double* __restrict__ res, double* __restrict__ x,
                                                     const double* __restrict__ scale, double* __restrict__ a_out,
                                                     const IterCtl* ctl) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  extern __shared__ float ss[];
  float* y = ss;            // n
  __shared__ float ts[NB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ldw = bw + 1;
  for (int i = tid; i < n; i += FT) y[i] = dropped[i] ? 0.0f : (float)res[i];
  __syncthreads();
  const int nblk = (n + NB - 1) / NB;
  // forward: L y = z
  for (int K = 0; K < nblk; ++K) {
    const int r0 = K * NB, r1 = min(r0 + NB, n);
    const int r = r0 + warp;
    if (r < r1) {
      float acc = 0.0f;
      const float* lr = lrow + (size_t)r * ldw;
      for (int kk = r - r0 + 1 + lane; kk <= bw && kk <= r; kk += 32) acc = fmaf(lr[kk], y[r - kk], acc);
      acc = warp_sum_f(acc);
      if (lane == 0) ts[warp] = y[r] - acc;
    } else if (lane == 0) {
      ts[warp] = 0.0f;
    }
    __syncthreads();
    if (warp == 0) {
      const float* X = dinv + (size_t)K * NB * NB;
      float acc = 0.0f;
#pragma unroll 8
      for (int c = 0; c <= lane; ++c) acc = fmaf(X[lane * NB + c], ts[c], acc);
      if (r0 + lane < r1) y[r0 + lane] = dropped[r0 + lane] ? 0.0f : acc;
    }
    __syncthreads();
  }
  // backward: L^T x = y
  for (int K = nblk - 1; K >= 0; --K) {
    const int r0 = K * NB, r1 = min(r0 + NB, n);
    const int r = r0 + warp;
    if (r < r1) {
      float acc = 0.0f;
      const float* lc = lcol + (size_t)r * ldw;
      for (int kk = r1 - r + lane; kk <= bw && r + kk < n; kk += 32) acc = fmaf(lc[kk], y[r + kk], acc);
      acc = warp_sum_f(acc);
      if (lane == 0) ts[warp] = y[r] - acc;
    } else if (lane == 0) {
      ts[warp] = 0.0f;
    }
    __syncthreads();
    if (warp == 0) {
      const float* X = dinv + (size_t)K * NB * NB;
      float acc = 0.0f;
#pragma unroll 8
      for (int c = lane; c < NB; ++c) acc = fmaf(X[c * NB + lane], ts[c], acc);
      if (r0 + lane < r1) y[r0 + lane] = dropped[r0 + lane] ? 0.0f : acc;
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += FT) {
    const double xi = dropped[i] ? 0.0 : x[i] + (double)y[i];
    x[i] = xi;
    if (a_out) a_out[i] = scale[i] * xi;
  }
}

// res = b - A x in FP64 (A symmetric band: column layout sband, row layout sbandR).
__global__ void k_coarse_residual(int n, int bw, const double* __restrict__ sband,
                                  const double* __restrict__ sbandR, const double* __restrict__ b,
                                  const double* __restrict__ x, const int* __restrict__ dropped,
                                  double* __restrict__ res, const IterCtl* ctl) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const int ldw = bw + 1;
  double acc = 0.0;
  const double* up = sband + (size_t)row * ldw;
  const double* lo = sbandR + (size_t)row * ldw;
  for (int kk = lane; kk <= bw; kk += 32) {
    if (row + kk < n) acc = fma(up[kk], x[row + kk], acc);
    if (kk >= 1 && row - kk >= 0) acc = fma(lo[kk], x[row - kk], acc);
  }
  acc = warp_sum_d(acc);
  if (lane == 0) res[row] = dropped[row] ? 0.0 : b[row] - acc;
}

}  // namespace

cudaError_t configure_coarse_solve(int max_smem) {
  cudaError_t e = set_max_dynamic_smem(k_coarse_factor, max_smem);
  if (e != cudaSuccess) return e;
  return set_max_dynamic_smem(k_coarse_solve, max_smem);
}

size_t coarse_factor_smem_bytes(int bw) { return factor_layout(bw).total_floats * sizeof(float); }
int coarse_dinv_size(int n) { return ((n + NB - 1) / NB) * NB * NB; }

cudaError_t launch_coarse_factor(cudaStream_t s, int n, int bw, float* fband, float* dinv, int* dropped,
                                 const IterCtl* ctl, int* /*err*/) {
  const size_t smem = coarse_factor_smem_bytes(bw);
  float* lrow = fband + (size_t)n * (bw + 1);
  k_coarse_factor<<<1, FT, smem, s>>>(n, bw, fband, lrow, dinv, dropped, ctl);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve(cudaStream_t s, int n, int bw, const float* fband, const float* dinv,
                                const int* dropped, const double* res, double* x, const double* scale,
                                double* a_out, const IterCtl* ctl) {
  const size_t smem = (size_t)n * sizeof(float);
  const float* lrow = fband + (size_t)n * (bw + 1);
  k_coarse_solve<<<1, FT, smem, s>>>(n, bw, fband, lrow, dinv, dropped, res, x, scale, a_out, ctl);
  return cudaGetLastError();
}

cudaError_t launch_coarse_residual(cudaStream_t s, int n, int bw, const double* sband, const double* b,
                                   const double* x, const int* dropped, double* res, const IterCtl* ctl) {
  const double* sbandR = sband + (size_t)n * (bw + 1);
  const int threads = 256;
  const int blocks = (int)(((size_t)n * 32 + threads - 1) / threads);
  k_coarse_residual<<<blocks, threads, 0, s>>>(n, bw, sband, sbandR, b, x, dropped, res, ctl);
  return cudaGetLastError();
}

}  // namespace hms
