// K4: the upper-level ("master") solve of Eq. 8.
//
// K_aa is symmetric positive (semi)definite and banded when its unknowns are
// ordered set by set (9 per set) over the row-major set grid: set I couples to
// its eight neighbours, the farthest at I + Mx + 1, so the half-bandwidth is
// bw = 9 (Mx + 2) - 1.  With D = diag(K_aa) the Jacobi-scaled matrix
// A = D^-1/2 K_aa D^-1/2 has a unit diagonal and, on these lattices, a
// condition number of a few thousand, so it is factored in T = float and the
// solution is refined in FP64:
//   x = 0, res = b = D^-1/2 P;  repeat: x += A_T^-1 res, res = b - A x (FP64)
// (T = double for ill-conditioned systems of degenerate set shapes).  Modes
// already marked as dropped (zero or dependent, decided in FP64) are unit rows;
// a pivot at or below Tau<T> drops its mode too.
//
//   k_coarse_factor  one CTA of 512 threads: right-looking band Cholesky in
//                    16-column blocks over a window of bw + 16 band rows held in
//                    shared memory (circular row-band storage).  Look-ahead:
//                    while warps 1-15 apply block K's rank-16 update to the
//                    rest of the window, write block K's columns of L and load
//                    the next band rows, warp 0 updates, factors (registers)
//                    and inverts the diagonal block K+1.
//   k_coarse_solve   one CTA of 512 threads: block forward / back substitution,
//                    16 rows per step (one warp per row), products with the
//                    inverted diagonal blocks; the rows of L each step needs
//                    are staged by bulk copies several steps ahead.  Adds the
//                    correction to the FP64 solution and writes a = D^-1/2 x.
//   k_coarse_residual many CTAs, FP64: res = b - A x over the band.
#include "hms_internal.cuh"
#include "ptx.cuh"

namespace hms {
namespace {

constexpr int NB = 16;     // block of columns / rows (the serial diagonal work per block grows as NB^3)
constexpr int FTF = 512;   // threads of the factor CTA
constexpr int FTS = 32 * NB;  // threads of the solve CTA (one warp per row of a block)

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
template <typename T>
struct Stages;
template <>
struct Stages<float> {
  static constexpr int v = 4;
};
template <>
struct Stages<double> {
  static constexpr int v = 2;
};

__device__ inline float wsum(float v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}
__device__ inline double wsum(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}
// 1/sqrt(x): the hardware approximation in FP32 (the factor only needs to be a
// good preconditioner: FP64 refinement restores the accuracy), exact in FP64
__device__ inline float trsqrt(float x) { return rsqrtf(x); }
__device__ inline double trsqrt(double x) { return 1.0 / sqrt(x); }

// Column C of the register-resident Cholesky of an NB x NB diagonal block
// (lane = row; lanes >= NB hold zero rows).  A dropped column becomes a unit column with a zero row.
template <typename T, int C>
__device__ __forceinline__ void diag_steps(T (&a)[NB], unsigned dmask, int lane, unsigned& dropped_out) {
  if constexpr (C < NB) {
    const T piv = __shfl_sync(0xffffffffu, a[C], C);
    const bool drop = ((dmask >> C) & 1u) != 0 || !(piv > Tau<T>::v);
    const T inv = drop ? T(1) : trsqrt(piv);
    const T d = drop ? T(1) : piv * inv;
    const bool mine = lane == C;
    const T acl = a[C];
    a[C] = mine ? d : (lane > C ? (drop ? T(0) : acl * inv) : acl);
#pragma unroll
    for (int j = 0; j < C; ++j) a[j] = (mine && drop) ? T(0) : a[j];
    const T lc = a[C];
#pragma unroll
    for (int j = C + 1; j < NB; ++j) {
      const T ljc = __shfl_sync(0xffffffffu, lc, j);
      a[j] = (lane >= j) ? fma(-lc, ljc, a[j]) : a[j];
    }
    if (drop) dropped_out |= (1u << C);
    diag_steps<T, C + 1>(a, dmask, lane, dropped_out);
  }
}

template <typename T>
struct FactorLayout {
  int W, ldw, pstr;
  size_t aw, pc, ls, xs, total;
};
template <typename T>
__host__ __device__ inline FactorLayout<T> factor_layout(int bw) {
  FactorLayout<T> L;
  // rows [k0, k0 + W) cover block K's band rows and the next diagonal block
  L.W = (bw > NB ? bw : NB) + NB;
  L.ldw = bw + 1;
  L.pstr = ((bw + 3) / 4) * 4 + 4;
  L.aw = 0;
  L.pc = ((size_t)L.W * L.ldw + 3) / 4 * 4;
  L.ls = L.pc + (size_t)NB * L.pstr;  // 2 buffers of NB x (NB+1)
  L.xs = L.ls + 2 * NB * (NB + 1);    // 2 buffers of NB x (NB+1)
  L.total = L.xs + 2 * NB * (NB + 1);
  return L;
}

// Warp 0: factor the diagonal block starting at row k (nbk rows) held in a[],
// write L to Ls, X = L^-1 to Xs and dinv, and the drop decisions.
template <typename T>
__device__ __forceinline__ void factor_diag_block(T (&a)[NB], int k, int nbk, int lane, int* __restrict__ dropped,
                                                  T* Ls, T* Xs, T* __restrict__ dinv, unsigned* dropblk) {
  const unsigned dmask = __ballot_sync(0xffffffffu, lane >= nbk || dropped[k + lane] != 0);
  unsigned dout = 0;
  diag_steps<T, 0>(a, dmask, lane, dout);
  if (lane < NB) {
#pragma unroll
    for (int j = 0; j < NB; ++j) Ls[lane * (NB + 1) + j] = (j <= lane) ? a[j] : T(0);
  }
  if (lane == 0) *dropblk = dout;
  __syncwarp();
  if (lane < nbk) dropped[k + lane] = (dout >> lane) & 1u;
  // X = L^-1, lane c computes column c column-oriented: once x_q is known it
  // is subtracted from every later row, so the dependent chain is NB steps long
  T x[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) x[r] = (r == lane) ? T(1) : T(0);
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const T xq = (q >= lane) ? x[q] / Ls[q * (NB + 1) + q] : T(0);
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

// lrow: input = scaled band in row layout [i][kk] = A[i][i-kk]; output = L in
// row layout.  lcol: output = L in column layout [c][kk] = L[c+kk][c].
template <typename T>
__global__ void __launch_bounds__(FTF, 1) k_coarse_factor(int n, int bw, T* __restrict__ lrow, T* __restrict__ lcol,
                                                          T* __restrict__ dinv, int* __restrict__ dropped,
                                                          const IterCtl* ctl) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  extern __shared__ __align__(16) unsigned char fsraw[];
  T* fs = reinterpret_cast<T*>(fsraw);
  const FactorLayout<T> LY = factor_layout<T>(bw);
  const int W = LY.W, ldw = LY.ldw, pstr = LY.pstr;
  T* Aw = fs + LY.aw;
  T* Pc = fs + LY.pc;
  __shared__ unsigned dropblk[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nblk = (n + NB - 1) / NB;

  // window rows [0, min(n, W))
  for (int q = tid; q < min(n, W) * ldw; q += FTF) {
    const int i = q / ldw, kk = q - (q / ldw) * ldw;
    Aw[(size_t)(i % W) * ldw + kk] = (kk <= i) ? lrow[(size_t)i * ldw + kk] : T(0);
  }
  __syncthreads();
  // diagonal block 0
  if (warp == 0) {
    T a[NB];
    const int nbk = min(NB, n);
#pragma unroll
    for (int j = 0; j < NB; ++j)
      a[j] = (lane < nbk && j <= lane && lane - j <= bw) ? Aw[(size_t)lane * ldw + (lane - j)] : T(0);
    factor_diag_block<T>(a, 0, nbk, lane, dropped, fs + LY.ls, fs + LY.xs, dinv, &dropblk[0]);
  }
  __syncthreads();

  for (int K = 0; K < nblk; ++K) {
    const int cur = K & 1, nxt = cur ^ 1;
    const int k0 = K * NB, k1 = min(k0 + NB, n), nbk = k1 - k0;
    const int rend = min(n, k1 + bw), np = rend - k1;
    const T* Ls = fs + LY.ls + cur * NB * (NB + 1);
    const T* Xs = fs + LY.xs + cur * NB * (NB + 1);
    const unsigned dblk = dropblk[cur];
    // (a) panel P[i][c] = sum_{c' <= c} A[i][k0 + c'] X[c][c'], i in [k1, rend); 4 x 4 tiles
    {
      const int nrq = (np + 3) / 4;
      for (int q = tid; q < nrq * (NB / 4); q += FTF) {
        const int rq = q / (NB / 4), cq = q - rq * (NB / 4);
        int rowoff[4];
        int il[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          il[u] = 4 * rq + u;
          const int i = k1 + (il[u] < np ? il[u] : np - 1);
          rowoff[u] = (i % W) * ldw + (i - k0);
        }
        T acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
        const int cmax = min(4 * cq + 3, nbk - 1);
        for (int cp = 0; cp <= cmax; ++cp) {
          T av[4], xv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int kk = k1 + il[u] - k0 - cp;  // i - (k0 + cp)
            av[u] = (il[u] < np && kk <= bw) ? Aw[rowoff[u] - cp] : T(0);
          }
#pragma unroll
          for (int v = 0; v < 4; ++v) xv[v] = Xs[(4 * cq + v) * (NB + 1) + cp];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], xv[v], acc[u][v]);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int c = 4 * cq + v;
          const bool keep = c < nbk && !((dblk >> c) & 1u);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (il[u] < np) Pc[c * pstr + il[u]] = keep ? acc[u][v] : T(0);
        }
      }
    }
    __syncthreads();
    // (a2) rank-NB update of the next diagonal block, by all threads
    const int nbk2 = (K + 1 < nblk) ? min(NB, n - k1) : 0;
    for (int q = tid; q < NB * NB; q += FTF) {
      const int l = q / NB, j = q - l * NB;
      if (l < nbk2 && j <= l && l < np && l - j <= bw) {
        T v = T(0);
        for (int c = 0; c < nbk; ++c) v = fma(Pc[c * pstr + l], Pc[c * pstr + j], v);
        Aw[(size_t)((k1 + l) % W) * ldw + (l - j)] -= v;
      }
    }
    __syncthreads();
    if (warp == 0) {
      // (b0) look-ahead: factor the diagonal block K+1
      if (K + 1 < nblk) {
        T a[NB];
        const size_t rbase = (size_t)((k1 + lane) % W) * ldw;
#pragma unroll
        for (int j = 0; j < NB; ++j)
          a[j] = (lane < nbk2 && j <= lane && lane - j <= bw) ? Aw[rbase + (lane - j)] : T(0);
        factor_diag_block<T>(a, k1, nbk2, lane, dropped, fs + LY.ls + nxt * NB * (NB + 1),
                             fs + LY.xs + nxt * NB * (NB + 1), dinv, &dropblk[nxt]);
      }
    } else {
      const int t2 = tid - 32, nt2 = FTF - 32;
      // (b1) trailing update of the window except the next diagonal block
      {
        const int T4 = (np + 3) / 4;
        const int first = (NB / 4) * (NB / 4 + 1) / 2;  // tile pairs inside rows [k1, k1 + NB)
        const int npairs = T4 * (T4 + 1) / 2;
        for (int q = first + t2; q < npairs; q += nt2) {
          int ti = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
          while (ti * (ti + 1) / 2 > q) --ti;
          while ((ti + 1) * (ti + 2) / 2 <= q) ++ti;
          const int tj = q - ti * (ti + 1) / 2;
          if (ti < NB / 4) continue;
          T acc[4][4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
          for (int c = 0; c < nbk; ++c) {
            const T* pc = Pc + c * pstr;
            T ri[4], rj[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              ri[u] = pc[4 * ti + u];
              rj[u] = pc[4 * tj + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) acc[u][v] = fma(ri[u], rj[v], acc[u][v]);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = k1 + 4 * ti + u;
            if (i >= rend) continue;
            const size_t rb = (size_t)(i % W) * ldw;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const int j = k1 + 4 * tj + v;
              if (j <= i) Aw[rb + (i - j)] -= acc[u][v];
            }
          }
        }
      }
      // (b2) columns [k0, k1) of L to global, both layouts
      for (int q = t2; q < nbk * ldw; q += nt2) {
        const int cl = q / ldw, kk = q - (q / ldw) * ldw;
        const int c = k0 + cl, i = c + kk;
        T v = T(0);
        if (i < n) {
          if (i < k1) v = Ls[(i - k0) * (NB + 1) + cl];
          else if (i < rend) v = Pc[cl * pstr + (i - k1)];
        }
        lcol[(size_t)c * ldw + kk] = v;
        if (i < n) lrow[(size_t)i * ldw + kk] = v;
      }
      // (b3) band rows [k0 + W, k1 + W) enter the window (slots of rows [k0, k1))
      const int r0 = k0 + W, r1 = min(k1 + W, n);
      for (int q = t2; q < (r1 > r0 ? r1 - r0 : 0) * ldw; q += nt2) {
        const int i = r0 + q / ldw, kk = q - (q / ldw) * ldw;
        Aw[(size_t)(i % W) * ldw + kk] = (kk <= i) ? lrow[(size_t)i * ldw + kk] : T(0);
      }
    }
    __syncthreads();
  }
}

// One solve with the factor, added to the FP64 solution x; writes a = s x.
template <typename T>
__host__ __device__ inline int solve_stage_elems(int bw) {
  return ((NB * (bw + 1) + 3) / 4) * 4 + NB * NB;
}

template <typename T>
__global__ void __launch_bounds__(FTS) k_coarse_solve(int n, int bw, const T* __restrict__ lcol,
                                                      const T* __restrict__ lrow, const T* __restrict__ dinv,
                                                      const int* __restrict__ dropped, const double* __restrict__ res,
                                                      double* __restrict__ x, const double* __restrict__ scale,
                                                      double* __restrict__ a_out, const IterCtl* ctl, int* err) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  constexpr int S = Stages<T>::v;
  extern __shared__ __align__(16) unsigned char ssraw[];
  T* ss = reinterpret_cast<T*>(ssraw);
  __shared__ uint64_t bars[S];
  __shared__ T ts[NB];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ldw = bw + 1;
  const int nblk = (n + NB - 1) / NB;
  const int nops = 2 * nblk;
  const int stage = solve_stage_elems<T>(bw);
  const int ybase = (n + 3) / 4 * 4;
  T* y = ss;
  const int dinv_off = stage - NB * NB;

  auto issue = [&](int o) {
    const bool fwd = o < nblk;
    const int K = fwd ? o : nops - 1 - o;
    const int rows = min(NB, n - K * NB);
    const uint32_t rb = (uint32_t)((((size_t)rows * ldw * sizeof(T)) + 15) / 16 * 16);
    const uint32_t db = NB * NB * sizeof(T);
    uint64_t* bar = &bars[o % S];
    T* dst = ss + ybase + (size_t)(o % S) * stage;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, rb + db);
    bulk_g2s(dst, (fwd ? lrow : lcol) + (size_t)K * NB * ldw, rb, bar);
    bulk_g2s(dst + dinv_off, dinv + (size_t)K * NB * NB, db, bar);
  };
  if (tid == 0) {
    abort_flag = 0;
    for (int k = 0; k < S; ++k) mbar_init(&bars[k], 1);
    fence_mbar_init();
  }
  for (int i = tid; i < n; i += FTS) y[i] = dropped[i] ? T(0) : (T)res[i];
  __syncthreads();
  if (tid == 0)
    for (int o = 0; o < S - 1 && o < nops; ++o) issue(o);
  for (int o = 0; o < nops; ++o) {
    const bool fwd = o < nblk;
    const int K = fwd ? o : nops - 1 - o;
    const int r0 = K * NB, r1 = min(r0 + NB, n);
    if (!mbar_wait_bounded(&bars[o % S], (uint32_t)((o / S) & 1))) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    if (tid == 32 && o + S - 1 < nops) issue(o + S - 1);
    const T* Lb = ss + ybase + (size_t)(o % S) * stage;
    const T* X = Lb + dinv_off;
    const int r = r0 + warp;
    T acc = T(0);
    if (r < r1) {
      const T* lr = Lb + (size_t)warp * ldw;
      if (fwd) {
        for (int kk = r - r0 + 1 + lane; kk <= bw && kk <= r; kk += 32) acc = fma(lr[kk], y[r - kk], acc);
      } else {
        for (int kk = r1 - r + lane; kk <= bw && r + kk < n; kk += 32) acc = fma(lr[kk], y[r + kk], acc);
      }
      acc = wsum(acc);
    }
    if (lane == 0) ts[warp] = (r < r1) ? y[r] - acc : T(0);
    __syncthreads();
    // y (or x) of this block: row w = warp, lanes over the block's columns
    if (r < r1) {
      T v = T(0);
      if (lane < NB) {
        const int w = warp, c = lane;
        v = fwd ? (c <= w ? X[w * NB + c] * ts[c] : T(0)) : (c >= w ? X[c * NB + w] * ts[c] : T(0));
      }
#pragma unroll
      for (int m = NB / 2; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
      if (lane == 0) y[r] = dropped[r] ? T(0) : v;
    }
    __syncthreads();
  }
  if (abort_flag) {
    if (tid == 0) {
      for (int b2 = 0; b2 < S; ++b2) mbar_wait_bounded(&bars[b2], 0u), mbar_wait_bounded(&bars[b2], 1u);
      if (err) atomicOr(err, (int)DEVERR_TIMEOUT);
    }
    return;
  }
  for (int i = tid; i < n; i += FTS) {
    const double xi = dropped[i] ? 0.0 : x[i] + (double)y[i];
    x[i] = xi;
    a_out[i] = scale[i] * xi;
  }
}

__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
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
  cudaError_t e;
  if ((e = set_max_dynamic_smem(k_coarse_factor<float>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_coarse_factor<double>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_coarse_solve<float>, max_smem)) != cudaSuccess) return e;
  return set_max_dynamic_smem(k_coarse_solve<double>, max_smem);
}

size_t coarse_factor_smem_bytes(int bw, bool fp64) {
  return fp64 ? factor_layout<double>(bw).total * sizeof(double) : factor_layout<float>(bw).total * sizeof(float);
}
size_t coarse_solve_smem_bytes(int n, int bw, bool fp64) {
  if (fp64)
    return (((size_t)n + 3) / 4 * 4 + (size_t)Stages<double>::v * solve_stage_elems<double>(bw)) * sizeof(double);
  return (((size_t)n + 3) / 4 * 4 + (size_t)Stages<float>::v * solve_stage_elems<float>(bw)) * sizeof(float);
}
int coarse_dinv_size(int n) { return ((n + NB - 1) / NB) * NB * NB; }

cudaError_t launch_coarse_factor(cudaStream_t s, int n, int bw, bool fp64, void* lrow, void* lcol, void* dinv,
                                 int* dropped, const IterCtl* ctl) {
  const size_t smem = coarse_factor_smem_bytes(bw, fp64);
  if (fp64)
    k_coarse_factor<double><<<1, FTF, smem, s>>>(n, bw, (double*)lrow, (double*)lcol, (double*)dinv, dropped, ctl);
  else
    k_coarse_factor<float><<<1, FTF, smem, s>>>(n, bw, (float*)lrow, (float*)lcol, (float*)dinv, dropped, ctl);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve(cudaStream_t s, int n, int bw, bool fp64, const void* lcol, const void* lrow,
                                const void* dinv, const int* dropped, const double* res, double* x,
                                const double* scale, double* a_out, const IterCtl* ctl, int* err) {
  const size_t smem = coarse_solve_smem_bytes(n, bw, fp64);
  if (fp64)
    k_coarse_solve<double><<<1, FTS, smem, s>>>(n, bw, (const double*)lcol, (const double*)lrow,
                                                (const double*)dinv, dropped, res, x, scale, a_out, ctl, err);
  else
    k_coarse_solve<float><<<1, FTS, smem, s>>>(n, bw, (const float*)lcol, (const float*)lrow, (const float*)dinv,
                                               dropped, res, x, scale, a_out, ctl, err);
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
