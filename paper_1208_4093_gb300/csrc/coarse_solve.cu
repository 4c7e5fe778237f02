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
//                    while 12 warps apply block K's rank-16 update to the rest
//                    of the window and load the next band rows, and warps 4,
//                    8, 12 write block K's columns of L, warp 0 factors
//                    (registers) and inverts the diagonal block K+1.
//   k_coarse_solve   one CTA of 512 threads: right-looking block forward / back
//                    substitution, 16 rows per step: the inverted diagonal
//                    block, then the block's contribution to the next bw rows;
//                    the columns (rows) of L each step needs are staged by bulk
//                    copies several steps ahead.  Adds the correction to the
//                    FP64 solution and writes a = D^-1/2 x.
//   k_coarse_blockinv / k_coarse_solve_big  (FP32 factor, when it fits in
//                    shared memory): the inverses of the 64 x 64 diagonal
//                    blocks of L are formed once per factor (one CTA per
//                    block), and each solve then takes n/64 block steps of a
//                    dense 64 x 64 product and a one-thread-per-row update.
//   k_coarse_residual many CTAs, FP64: res = b - A x over the band.
#include <cooperative_groups.h>

#include "coarse_common.cuh"
#include "hms_internal.cuh"
#include "ptx.cuh"

namespace hms {
namespace {

using namespace coarse;
namespace cg = cooperative_groups;
constexpr int FTF = 512;   // threads of the factor CTA
constexpr int FTS = 32 * NB;  // threads of the solve CTA (one warp per row of a block)

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

template <typename T>
struct FactorLayout {
  int W, ldw, lda, pstr;
  size_t aw, pc, ls, xs, total;
};
template <typename T>
__host__ __device__ inline FactorLayout<T> factor_layout(int bw) {
  FactorLayout<T> L;
  // rows [k0, k0 + W) cover block K's band rows and the next diagonal block
  L.W = (bw > NB ? bw : NB) + NB;
  L.ldw = bw + 1;
  L.lda = window_lda(bw);
  L.pstr = ((bw + 3) / 4) * 4 + 4;
  L.aw = 0;
  L.pc = ((size_t)L.W * L.lda + 3) / 4 * 4;
  L.ls = L.pc + (size_t)NB * L.pstr;  // 2 buffers of NB x (NB+1)
  L.xs = L.ls + 2 * NB * (NB + 1);    // 2 buffers of NB x (NB+1)
  L.total = L.xs + 2 * NB * (NB + 1);
  return L;
}
// extra shared memory of the factor after the T-typed part: the drop flags
// (int per unknown) and the trailing update's 4 x 4 tile pairs (ti, tj)
__host__ __device__ inline int factor_tile_pairs(int bw) {
  const int t4 = (bw + 3) / 4;
  return t4 * (t4 + 1) / 2;
}

// lrow: input = scaled band in row layout [i][kk] = A[i][i-kk]; output = L in
// row layout if write_lrow (the 16-row substitution reads it).  lcol: output
// = L in column layout [c][kk] = L[c+kk][c].
//
// Only the first npiv rows are pivots (npiv = n: the whole factor; else a
// multiple of 4).  Columns [0, npiv) of L are written with all their band
// rows, and rows [npiv, n) end with the Schur complement of the pivots,
// A - L L^T.  If schur is set, the part of it the pivots changed is written
// out as a dense s x s lower triangle: schur[i s + j] = (A - S)[npiv + i][npiv
// + j] for j <= i < min(bw, s), else 0.
template <typename T>
__device__ __forceinline__ void factor_run(int n, int npiv, int bw, T* __restrict__ lrow, T* __restrict__ lcol,
                                           T* __restrict__ dinv, int* __restrict__ dropped, int write_lrow,
                                           T* __restrict__ schur, int s) {
  extern __shared__ __align__(16) unsigned char fsraw[];
  T* fs = reinterpret_cast<T*>(fsraw);
  const FactorLayout<T> LY = factor_layout<T>(bw);
  const int W = LY.W, ldw = LY.ldw, lda = LY.lda, pstr = LY.pstr;
  T* Aw = fs + LY.aw;
  T* Pc = fs + LY.pc;
  int* sdrop = reinterpret_cast<int*>(fs + LY.total);
  unsigned short* tpair = reinterpret_cast<unsigned short*>(sdrop + n);
  __shared__ unsigned dropblk[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nblk = (npiv + NB - 1) / NB;
  const int npairs_max = factor_tile_pairs(bw);
  // lrow and dropped may have been written earlier in the same kernel (the
  // two-sided factor's second part): coherent loads (__ldcg), never the
  // read-only path
  for (int i = tid; i < n; i += FTF) sdrop[i] = __ldcg(dropped + i);
  for (int q = tid; q < npairs_max; q += FTF) {
    int ti = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
    while (ti * (ti + 1) / 2 > q) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= q) ++ti;
    tpair[2 * q] = (unsigned short)ti;
    tpair[2 * q + 1] = (unsigned short)(q - ti * (ti + 1) / 2);
  }

  // window rows [0, min(n, W))
  for (int q = tid; q < min(n, W) * ldw; q += FTF) {
    const int i = q / ldw, kk = q - (q / ldw) * ldw;
    if (kk <= i) Aw[(size_t)(i % W) * lda + (i - kk) % lda] = __ldcg(lrow + (size_t)i * ldw + kk);
  }
  __syncthreads();
  // diagonal block 0
  if (warp == 0) {
    T a[NB];
    const int nbk = min(NB, npiv);
#pragma unroll
    for (int j = 0; j < NB; ++j)
      a[j] = (lane < nbk && j <= lane && lane - j <= bw) ? Aw[(size_t)lane * lda + j] : T(0);
    factor_diag_block<T>(a, 0, nbk, lane, sdrop, fs + LY.ls, fs + LY.xs, dinv, &dropblk[0]);
  }
  __syncthreads();

  for (int K = 0; K < nblk; ++K) {
    const int cur = K & 1, nxt = cur ^ 1;
    const int k0 = K * NB, k1 = min(k0 + NB, npiv), nbk = k1 - k0;
    const int rend = min(n, k1 + bw), np = rend - k1;
    const T* Ls = fs + LY.ls + cur * NB * (NB + 1);
    const T* Xs = fs + LY.xs + cur * NB * (NB + 1);
    const unsigned dblk = dropblk[cur];
    const int slot_k1 = k1 % W;  // window slot of row k1; row k1 + d sits at slot_k1 + d (mod W)
    auto slot = [&](int i) { const int v = slot_k1 + (i - k1); return v >= W ? v - W : v; };
    // (a) panel P[i][c] = sum_{c' <= c} A[i][k0 + c'] X[c][c'], i in [k1, rend);
    // tiles of 4 rows (interleaved by nrq, so that neighbouring threads read
    // neighbouring rows) x 4 columns
    const int ck0 = k0 % lda;  // position of column k0 in a window row
    {
      const int nrq = (np + 3) / 4;
      for (int q = tid; q < nrq * (NB / 4); q += FTF) {
        const int rq = q / (NB / 4), cq = q - rq * (NB / 4);
        int rowoff[4];
        int il[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          il[u] = rq + u * nrq;
          const int i = k1 + (il[u] < np ? il[u] : np - 1);
          rowoff[u] = slot(i) * lda;
        }
        T acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
        // X is zero above its diagonal: run all NB columns (unrolled by 8:
        // fully unrolled, the kernel's 128 registers spill)
#pragma unroll 8
        for (int cp = 0; cp < NB; ++cp) {
          T av[4], xv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            // kk = i - (k0 + cp) < 0 only in a short last block followed by
            // rows that are no pivots (npiv < n): column k0 + cp is then right
            // of row i's band, a window position never loaded, and X's zero
            // there must not meet it (0 * NaN)
            const int kk = k1 + il[u] - k0 - cp;  // i - (k0 + cp)
            const int pos = ck0 + cp;
            av[u] = (il[u] < np && kk >= 0 && kk <= bw) ? Aw[rowoff[u] + (pos >= lda ? pos - lda : pos)] : T(0);
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
    // (a2) rank-NB update of the next diagonal block, by all threads (its
    // rows past npiv are not pivots but are updated all the same)
    const int nbu = min(NB, n - k1);
    const int nbk2 = (K + 1 < nblk) ? min(NB, npiv - k1) : 0;
    for (int q = tid; q < NB * NB; q += FTF) {
      const int l = q / NB, j = q - l * NB;
      if (l < nbu && j <= l && l < np && l - j <= bw) {
        T v = T(0);
        for (int c = 0; c < nbk; ++c) v = fma(Pc[c * pstr + l], Pc[c * pstr + j], v);
        Aw[(size_t)slot(k1 + l) * lda + (k1 + j) % lda] -= v;
      }
    }
    __syncthreads();
    if (warp == 0) {
      // (b0) look-ahead: factor the diagonal block K+1
      if (K + 1 < nblk) {
        T a[NB];
        const size_t rbase = (size_t)slot(min(k1 + lane, n - 1)) * lda;
        const int ck1 = k1 % lda;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          const int pos = ck1 + j;
          a[j] = (lane < nbk2 && j <= lane && lane - j <= bw) ? Aw[rbase + (pos >= lda ? pos - lda : pos)] : T(0);
        }
        factor_diag_block<T>(a, k1, nbk2, lane, sdrop, fs + LY.ls + nxt * NB * (NB + 1),
                             fs + LY.xs + nxt * NB * (NB + 1), dinv, &dropblk[nxt]);
      }
    } else if ((warp & 3) == 0) {
      // warps 4, 8, 12 share warp 0's scheduler, so they take only light
      // work that does not wait on the update: band rows [k0 + W, k1 + W)
      // enter the window in the slots of rows [k0, k1), which nothing reads
      // in this phase
      const int er0 = k0 + W, er1 = min(k1 + W, n);
      for (int i = er0 + (warp >> 2) - 1; i < er1; i += FTF / 128 - 1) {
        const T* src = lrow + (size_t)i * ldw;
        T* dst = Aw + (size_t)(i % W) * lda;
        const int ci = i % lda;  // position of column i; column i - kk wraps at most once (kk < ldw <= lda)
        T v[7];  // ldw <= 224: all loads first, then the stores
#pragma unroll
        for (int u = 0; u < 7; ++u) {
          const int kk = lane + 32 * u;
          v[u] = (kk < ldw && kk <= i) ? __ldcg(src + kk) : T(0);
        }
#pragma unroll
        for (int u = 0; u < 7; ++u) {
          const int kk = lane + 32 * u;
          const int pos = ci - kk;
          if (kk < ldw && kk <= i) dst[pos < 0 ? pos + lda : pos] = v[u];
        }
      }
    } else {
      // the other 12 warps: trailing update, then block K's columns of L
      const int wi = warp - 1 - (warp >> 2), nwi = FTF / 32 - FTF / 128;
      const int t2 = wi * 32 + lane, nt2 = nwi * 32;
      // (b1) trailing update of the window except the next diagonal block
      {
        const int T4 = (np + 3) / 4;
        const int first = (NB / 4) * (NB / 4 + 1) / 2;  // tile pairs inside rows [k1, k1 + NB)
        const int npairs = T4 * (T4 + 1) / 2;
        for (int q = first + t2; q < npairs; q += nt2) {
          const int ti = tpair[2 * q], tj = tpair[2 * q + 1];
          T acc[4][4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
          // columns of Pc past nbk are zero (a short last block): always NB
#pragma unroll
          for (int c = 0; c < NB; ++c) {
            const T* pc = Pc + c * pstr;
            T ri[4], rj[4];
            ld4(pc + 4 * ti, ri);
            ld4(pc + 4 * tj, rj);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) acc[u][v] = fma(ri[u], rj[v], acc[u][v]);
          }
          // (i, k1 + 4 tj .. + 3) is one aligned 16-byte word of row i; in a
          // diagonal tile the entries right of the diagonal land on unused
          // positions of the row
          const int pj = (k1 + 4 * tj) % lda;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = k1 + 4 * ti + u;
            if (i >= rend) continue;
            T* w4 = Aw + (size_t)slot(i) * lda + pj;
            T old[4];
            ld4(w4, old);
            st4(w4, old[0] - acc[u][0], old[1] - acc[u][1], old[2] - acc[u][2], old[3] - acc[u][3]);
          }
        }
      }
      // (b2) columns [k0, k1) of L to global (and the row layout if asked)
      for (int cl = wi; cl < nbk; cl += nwi) {
        const int c = k0 + cl;
        T v[7];  // ldw <= 224: all loads first, then the stores
#pragma unroll
        for (int u = 0; u < 7; ++u) {
          const int kk = lane + 32 * u, i = c + kk;
          v[u] = T(0);
          if (kk < ldw && i < n) {
            if (i < k1) v[u] = Ls[(i - k0) * (NB + 1) + cl];
            else if (i < rend) v[u] = Pc[cl * pstr + (i - k1)];
          }
        }
#pragma unroll
        for (int u = 0; u < 7; ++u) {
          const int kk = lane + 32 * u, i = c + kk;
          if (kk < ldw) {
            lcol[(size_t)c * ldw + kk] = v[u];
            if (write_lrow && i < n) lrow[(size_t)i * ldw + kk] = v[u];
          }
        }
      }
    }
    __syncthreads();
  }
  if (schur) {
    // rows [npiv, npiv + bw) are still in the window: slot i mod W
    for (int q = tid; q < s * s; q += FTF) {
      const int i = q / s, j = q - (q / s) * s;
      const int gi = npiv + i, gj = npiv + j;
      T v = T(0);
      if (j <= i && i < bw && gi < n)
        v = __ldcg(lrow + (size_t)gi * ldw + (gi - gj)) - Aw[(size_t)(gi % W) * lda + gj % lda];
      schur[q] = v;
    }
  }
  for (int i = tid; i < n; i += FTF) dropped[i] = sdrop[i];
}

template <typename T>
__global__ void __launch_bounds__(FTF, 1) k_coarse_factor(int n, int bw, T* __restrict__ lrow, T* __restrict__ lcol,
                                                          T* __restrict__ dinv, int* __restrict__ dropped,
                                                          int write_lrow, const IterCtl* ctl) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  factor_run<T>(n, n, bw, lrow, lcol, dinv, dropped, write_lrow, nullptr, 0);
}

// One solve with the factor, added to the FP64 solution x; writes a = s x.
// Right-looking substitution: step K applies the inverted diagonal block to
// block K's right-hand side (final by then), then subtracts block K's
// contribution from the next bw rows (forward: columns of L, backward: rows of
// L), so the chain from one block to the next is two short phases.
template <typename T>
__host__ __device__ inline int solve_stage_elems(int bw) {
  return ((NB * (bw + 1) + 3) / 4) * 4 + NB * NB;
}

// cstat[0]: bits of max |b| (set by the first solve), cstat[1]: bits of the
// last residual's max |res| (k_coarse_residual), cstat[2]: 1 once refinement
// has converged (max |res| <= 1e-14 max |b|); later solves then return at once;
// cstat[3]: updates whose last allowed solve still ran (refinement not
// converged before it), counted over a whole hms_solve.
template <typename T>
__global__ void __launch_bounds__(FTS) k_coarse_solve(int n, int bw, const T* __restrict__ lcol,
                                                      const T* __restrict__ lrow, const T* __restrict__ dinv,
                                                      const int* __restrict__ dropped, const double* __restrict__ res,
                                                      double* __restrict__ x, const double* __restrict__ scale,
                                                      double* __restrict__ a_out, unsigned long long* cstat, int first,
                                                      const IterCtl* ctl, int* err) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  // first: bit 0 = the solve of b, bit 1 = the last solve the update allows
  const bool last = (first & 2) != 0;
  first &= 1;
  __shared__ int skip;
  if (threadIdx.x == 0) {
    if (first) {
      skip = 0;
    } else {
      const double bmax = __longlong_as_double((long long)cstat[0]);
      const double rmax = __longlong_as_double((long long)cstat[1]);
      skip = (cstat[2] != 0ull) || !(rmax > 1e-14 * bmax);
      if (skip) cstat[2] = 1ull;
      else if (last) atomicAdd(&cstat[3], 1ull);  // refinement used every solve it may
    }
  }
  __syncthreads();
  if (skip) return;
  constexpr int S = Stages<T>::v;
  extern __shared__ __align__(16) unsigned char ssraw[];
  T* ss = reinterpret_cast<T*>(ssraw);
  __shared__ uint64_t bars[S];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ldw = bw + 1;
  const int nblk = (n + NB - 1) / NB;
  const int nops = 2 * nblk;
  const int stage = solve_stage_elems<T>(bw);
  const int n4 = (n + 3) / 4 * 4;
  T* tv = ss;       // running right-hand side
  T* yv = ss + n4;  // y, then x
  const int sbase = 2 * n4;
  const int dinv_off = stage - NB * NB;
  int* sdrop = reinterpret_cast<int*>(ss + sbase + (size_t)S * stage);

  auto issue = [&](int o) {
    const bool fwd = o < nblk;
    const int K = fwd ? o : nops - 1 - o;
    const int rows = min(NB, n - K * NB);
    const uint32_t rb = (uint32_t)((((size_t)rows * ldw * sizeof(T)) + 15) / 16 * 16);
    const uint32_t db = NB * NB * sizeof(T);
    uint64_t* bar = &bars[o % S];
    T* dst = ss + sbase + (size_t)(o % S) * stage;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, rb + db);
    bulk_g2s(dst, (fwd ? lcol : lrow) + (size_t)K * NB * ldw, rb, bar);
    bulk_g2s(dst + dinv_off, dinv + (size_t)K * NB * NB, db, bar);
  };
  if (tid == 0) {
    abort_flag = 0;
    for (int k = 0; k < S; ++k) mbar_init(&bars[k], 1);
    fence_mbar_init();
  }
  __shared__ double bred[FTS / 32];
  double bm = 0.0;
  for (int i = tid; i < n; i += FTS) {
    const int d = dropped[i];
    sdrop[i] = d;
    tv[i] = d ? T(0) : (T)res[i];
    if (first && !d) bm = fmax(bm, fabs(res[i]));
  }
  if (first) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, m));
    if (lane == 0) bred[warp] = bm;
  }
  __syncthreads();
  if (first && tid == 0) {
    double v = 0.0;
    for (int k = 0; k < FTS / 32; ++k) v = fmax(v, bred[k]);
    cstat[0] = (unsigned long long)__double_as_longlong(v);
    cstat[2] = 0ull;
  }
  if (tid == 0) cstat[1] = 0ull;  // the next residual accumulates its max here
  if (tid == 0)
    for (int o = 0; o < S - 1 && o < nops; ++o) issue(o);
  for (int o = 0; o < nops; ++o) {
    const bool fwd = o < nblk;
    const int K = fwd ? o : nops - 1 - o;
    const int r0 = K * NB, r1 = min(r0 + NB, n), nr = r1 - r0;
    if (o == nblk) {
      // the backward pass starts from y
      for (int i = tid; i < n; i += FTS) tv[i] = yv[i];
      __syncthreads();
    }
    if (!mbar_wait_bounded(&bars[o % S], (uint32_t)((o / S) & 1))) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    if (tid == 32 && o + S - 1 < nops) issue(o + S - 1);
    const T* Lb = ss + sbase + (size_t)(o % S) * stage;  // rows of lcol (forward) / lrow (backward) of block K
    const T* X = Lb + dinv_off;
    // (1) block K: y_K = X t_K (forward), x_K = X^T t_K (backward); warp w = row
    if (warp < nr) {
      const int w = warp, c = lane;
      T v = T(0);
      if (c < nr) v = fwd ? (c <= w ? X[w * NB + c] * tv[r0 + c] : T(0)) : (c >= w ? X[c * NB + w] * tv[r0 + c] : T(0));
#pragma unroll
      for (int m = NB / 2; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
      if (lane == 0) yv[r0 + w] = sdrop[r0 + w] ? T(0) : v;
    }
    __syncthreads();
    // (2) subtract block K's contribution from the next bw rows; the block's
    // values sit in registers and two chains share the NB products
    T yb[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) yb[c] = (c < nr) ? yv[r0 + c] : T(0);
    if (fwd) {
      // t_i -= sum_k L[i][k] y_k,  i in [r1, r1 + bw), L[i][k] = lcol[k][i - k]
      const int iend = min(n, r1 + bw);
      for (int i = r1 + tid; i < iend; i += FTS) {
        T acc0 = T(0), acc1 = T(0);
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          const int d = i - (r0 + c);
          if (c < nr && d <= bw) {
            const T t = Lb[(size_t)c * ldw + d] * yb[c];
            if (c & 1) acc1 += t; else acc0 += t;
          }
        }
        tv[i] -= acc0 + acc1;
      }
    } else {
      // t_i -= sum_k L[k][i] x_k,  i in [r0 - bw, r0), L[k][i] = lrow[k][k - i]
      const int ibeg = max(0, r0 - bw);
      for (int i = ibeg + tid; i < r0; i += FTS) {
        T acc0 = T(0), acc1 = T(0);
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          const int d = r0 + c - i;
          if (c < nr && d <= bw) {
            const T t = Lb[(size_t)c * ldw + d] * yb[c];
            if (c & 1) acc1 += t; else acc0 += t;
          }
        }
        tv[i] -= acc0 + acc1;
      }
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
    const double xi = sdrop[i] ? 0.0 : x[i] + (double)yv[i];
    x[i] = xi;
    a_out[i] = scale[i] * xi;
  }
}

// ---- solves with inverted 64 x 64 diagonal blocks (FP32 factor) ----
constexpr int NBB = 64;   // rows per block of the block substitution
constexpr int LDX = 72;   // row stride of the stored block inverses (conflict-free row reads)
constexpr int LDR = 68;   // row stride of the stored band neighbours (conflict-free 16-byte row reads)
constexpr int FTB = 512;  // threads of the block-substitution CTA

// Per NBB-row block K of the FP32 factor, stored one after another:
//   X_K   = L_KK^-1                         NBB x LDX, lower
//   X_K^T                                   NBB x LDX, upper
//   R_K[q][c] = L[r1 + q][r0 + c]           bw x LDR, the band rows below the block
//   U_K[q][c] = L[r0 + c][r0 - bw + q]      bw x LDR, the band columns left of the block
// (r0 = K NBB, r1 = min(r0 + NBB, n); zero outside the band and the matrix).
__host__ __device__ inline size_t blk_elems(int bw) { return 2 * (size_t)NBB * LDX + 2 * (size_t)bw * LDR; }

// The per-block matrices above from the FP32 factor (row and column layouts);
// rows of X past n are identity rows.  Per block, one CTA of 256 threads
// inverts the diagonal block and three more copy a third of R_K and U_K each.
// Block [r0, r0 + nr) of an n-row factor: part 0 inverts the diagonal block,
// parts 1 .. nparts - 1 copy a share of R_K and U_K each.
__device__ __forceinline__ void blockinv_run(int n, int bw, int r0, int nr, const float* __restrict__ lcol,
                                             float* __restrict__ X, int part_id, int nparts) {
  __shared__ float Ls[NBB][NBB + 1];
  __shared__ float Xs[NBB][NBB + 1];
  const int tid = threadIdx.x;
  const int ldw = bw + 1;
  float* XT = X + NBB * LDX;
  float* R = XT + NBB * LDX;
  float* U = R + (size_t)bw * LDR;
  if (part_id > 0) {
    // R_K and U_K, a share of their rows per CTA
    const int r1 = r0 + nr;
    const int part = (bw + nparts - 2) / (nparts - 1);
    const int qa = (part_id - 1) * part, qb = min(bw, qa + part);
#pragma unroll 4
    for (int idx = qa * LDR + tid; idx < qb * LDR; idx += blockDim.x) {
      const int q = idx / LDR, c = idx % LDR;
      float rv = 0.f, uv = 0.f;
      if (c < nr) {
        const int i = r1 + q, k = r0 + c;  // R: L[i][k], i > k
        if (i < n && i - k <= bw) rv = lcol[(size_t)k * ldw + (i - k)];
        const int iu = r0 - bw + q;        // U: L[k][iu], k > iu (coalesced over c)
        if (iu >= 0 && k - iu <= bw) uv = lcol[(size_t)iu * ldw + (k - iu)];
      }
      R[idx] = rv;
      U[idx] = uv;
    }
    return;
  }
#pragma unroll 8
  for (int idx = tid; idx < NBB * NBB; idx += blockDim.x) {
    const int r = idx / NBB, c = idx % NBB;
    float v = 0.f;
    if (r < nr && c <= r && r - c <= bw) v = lcol[(size_t)(r0 + c) * ldw + (r - c)];
    if (r >= nr && r == c) v = 1.f;
    Ls[r][c] = v;
  }
  __syncthreads();
  // X = L^-1 by 16 x 16 blocks: the four diagonal blocks by column
  // substitution (64 threads, one column each), then block rows i = 1..3:
  //   X_ij = -X_ii sum_{k=j}^{i-1} L_ik X_kj   for all j < i at once
  constexpr int B = 16;
  if (tid < NBB) {
    const int b = tid / B, c = tid % B, o = b * B;
    for (int r = 0; r < B; ++r) {
      float acc = (r == c) ? 1.f : 0.f;
#pragma unroll
      for (int k = 0; k < B; ++k)
        if (k >= c && k < r) acc = fmaf(-Ls[o + r][o + k], Xs[o + k][o + c], acc);
      Xs[o + r][o + c] = r < c ? 0.f : acc / Ls[o + r][o + r];
    }
  }
  __syncthreads();
  __shared__ float Ts[3][B][B + 1];
  const int rr = tid / B, cc = tid % B;
  for (int i = 1; i < NBB / B; ++i) {
    for (int j = 0; j < i; ++j) {
      float acc = 0.f;
      for (int k = j; k < i; ++k) {
#pragma unroll
        for (int m = 0; m < B; ++m) acc = fmaf(Ls[i * B + rr][k * B + m], Xs[k * B + m][j * B + cc], acc);
      }
      Ts[j][rr][cc] = acc;
    }
    __syncthreads();
    for (int j = 0; j < i; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int m = 0; m < B; ++m) acc = fmaf(Xs[i * B + rr][i * B + m], Ts[j][m][cc], acc);
      Xs[i * B + rr][j * B + cc] = -acc;
    }
    __syncthreads();
  }
  // the zero upper blocks
  for (int idx = tid; idx < NBB * NBB; idx += blockDim.x) {
    const int r = idx / NBB, c = idx % NBB;
    if (c / B > r / B) Xs[r][c] = 0.f;
  }
  __syncthreads();
  for (int idx = tid; idx < NBB * LDX; idx += blockDim.x) {
    const int r = idx / LDX, c = idx % LDX;
    X[idx] = c < NBB ? Xs[r][c] : 0.f;
    XT[idx] = c < NBB ? Xs[c][r] : 0.f;
  }
}

__global__ void __launch_bounds__(256) k_coarse_blockinv(int n, int bw, const float* __restrict__ lcol,
                                                         float* __restrict__ xinv, const IterCtl* ctl) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  const int K = blockIdx.x, r0 = K * NBB;
  blockinv_run(n, bw, r0, min(NBB, n - r0), lcol, xinv + (size_t)K * blk_elems(bw), blockIdx.y, gridDim.y);
}

// Batched: one CTA per problem (FP32 band factor on one SM), and the block
// inverses of every problem (item = block K, part).
__global__ void __launch_bounds__(FTF, 1) kb_coarse_factor(const BatchProb* __restrict__ P,
                                                           const BatchItem* __restrict__ items) {
  const BatchItem it = items[blockIdx.x];
  const BatchProb& q = P[it.prob];
  if (q.ctl && *(volatile const int*)&q.ctl->done) return;
  factor_run<float>(q.n_c, q.n_c, q.bw, q.lrow, q.lcol, q.dinv, q.dropped, 0, nullptr, 0);
}
__global__ void __launch_bounds__(256) kb_coarse_blockinv(const BatchProb* __restrict__ P,
                                                          const BatchItem* __restrict__ items) {
  const BatchItem it = items[blockIdx.x];
  const BatchProb& q = P[it.prob];
  if (q.ctl && *(volatile const int*)&q.ctl->done) return;
  const int r0 = it.bx * NBB;
  blockinv_run(q.n_c, q.bw, r0, min(NBB, q.n_c - r0), q.lcol, q.xinv + (size_t)it.bx * blk_elems(q.bw), it.by, it.gy);
}

__host__ __device__ inline int big_stage_elems(int bw) { return bw * LDR + NBB * LDX; }

// One step of the block substitution on the vectors tv (running right-hand
// side) and yv (solution) in shared memory, block rows [r0, r1), nr = r1 - r0.
// (1) 8 threads per row: y_w = sum_c M[w][c] t_c (M is zero outside its triangle)
__device__ __forceinline__ void bsolve_diag(const float* M, const float* tv, float* yv, const int* sdrop, int r0,
                                            int nr, int tid) {
  const int w = tid >> 3, p = tid & 7;
  const float* mr = M + w * LDX;
  float v0 = 0.f, v1 = 0.f;
#pragma unroll
  for (int k = 0; k < NBB / 8; k += 2) {
    const int c0 = p + 8 * k, c1 = c0 + 8;
    const float m0 = mr[c0], m1 = mr[c1];
    const float t0 = c0 < nr ? tv[r0 + c0] : 0.f;
    const float t1 = c1 < nr ? tv[r0 + c1] : 0.f;
    v0 = fmaf(m0, t0, v0);
    v1 = fmaf(m1, t1, v1);
  }
  float v = v0 + v1;
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  if (w < nr && p == 0) yv[r0 + w] = sdrop[r0 + w] ? 0.f : v;
}
// (2) the band rows next to the block, t_i -= sum_c B[q][c] y_c with B = R_K
// (rows i = r1 + q, forward) or U_K (rows i = r0 - bw + q, backward): threads
// h*256 + q take row q and the columns [32h, 32h + 32) by 16-byte loads (r0 is
// a multiple of 4; y past the block is finite and meets zero columns of B);
// the two halves meet in shared memory.
__device__ __forceinline__ void bsolve_band(const float* Lb, const float* yv, float* tv, float* hpart, bool fwd,
                                            int r0, int r1, int n, int bw, int tid) {
  const int qlo = fwd ? 0 : max(0, bw - r0);
  const int qhi = fwd ? min(bw, n - r1) : bw;
  const int ioff = fwd ? r1 : r0 - bw;  // i = ioff + q
  const int h = tid >> 8, q0 = tid & 255;
  const int cbase = 32 * h;
  float yb[32];
#pragma unroll
  for (int c4 = 0; c4 < 32; c4 += 4) {
    const float4 y4 = *reinterpret_cast<const float4*>(yv + r0 + cbase + c4);
    yb[c4] = y4.x, yb[c4 + 1] = y4.y, yb[c4 + 2] = y4.z, yb[c4 + 3] = y4.w;
  }
  for (int qb = qlo; qb < qhi; qb += 256) {
    const int q = qb + q0;
    const int i = ioff + q;
    float acc0 = 0.f, acc1 = 0.f;
    if (q < qhi) {
      const float* br = Lb + (size_t)q * LDR + cbase;
#pragma unroll
      for (int c4 = 0; c4 < 32; c4 += 4) {
        const float4 l4 = *reinterpret_cast<const float4*>(br + c4);
        acc0 = fmaf(l4.x, yb[c4], acc0);
        acc1 = fmaf(l4.y, yb[c4 + 1], acc1);
        acc0 = fmaf(l4.z, yb[c4 + 2], acc0);
        acc1 = fmaf(l4.w, yb[c4 + 3], acc1);
      }
    }
    const float part = acc0 + acc1;
    hpart[h * 256 + q0] = part;
    __syncthreads();
    if (h == 0 && q < qhi) tv[i] -= hpart[q0] + hpart[256 + q0];
    if (qb + 256 < qhi) __syncthreads();
  }
}

// Block forward / back substitution with the FP32 factor, NBB rows per step:
//   forward   y_K = X_K t_K,     t_i -= sum_c R_K[i - r1][c] y_c        (the next bw rows)
//   backward  x_K = X_K^T t_K,   t_i -= sum_c U_K[i - r0 + bw][c] x_c   (the previous bw rows)
// then x += y in FP64 and a = D^-1/2 x; the same refinement control as
// k_coarse_solve.  Each step's R_K (U_K) and X_K (X_K^T) are staged by bulk
// copies S - 1 steps ahead.
template <int S>
__device__ __forceinline__ void solve_big_body(int n, int bw, const float* __restrict__ xinv,
                                               const int* __restrict__ dropped, const double* __restrict__ res,
                                               double* __restrict__ x, const double* __restrict__ scale,
                                               double* __restrict__ a_out, unsigned long long* cstat, int first,
                                               const IterCtl* ctl, int* err) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  // first: bit 0 = the solve of b, bit 1 = the last solve the update allows
  const bool last = (first & 2) != 0;
  first &= 1;
  __shared__ int skip;
  if (threadIdx.x == 0) {
    if (first) {
      skip = 0;
    } else {
      const double bmax = __longlong_as_double((long long)cstat[0]);
      const double rmax = __longlong_as_double((long long)cstat[1]);
      skip = (cstat[2] != 0ull) || !(rmax > 1e-14 * bmax);
      if (skip) cstat[2] = 1ull;
      else if (last) atomicAdd(&cstat[3], 1ull);  // refinement used every solve it may
    }
  }
  __syncthreads();
  if (skip) return;
  extern __shared__ __align__(16) unsigned char ssraw[];
  float* ss = reinterpret_cast<float*>(ssraw);
  __shared__ uint64_t bars[S];
  __shared__ int abort_flag;
  __shared__ double bred[FTB / 32];
  __shared__ float hpart[512];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nblk = (n + NBB - 1) / NBB;
  const int nops = 2 * nblk;
  const int stage = big_stage_elems(bw);
  const int xoff = stage - NBB * LDX;
  const int n4 = (n + 3) / 4 * 4;
  float* tv = ss;       // running right-hand side
  float* yv = ss + n4;  // y, then x
  const int sbase = 2 * n4 + NBB;  // yv keeps NBB spare entries for the vector loads of the last block
  int* sdrop = reinterpret_cast<int*>(ss + sbase + (size_t)S * stage);

  auto issue = [&](int o) {
    const bool fwd = o < nblk;
    const int K = fwd ? o : nops - 1 - o;
    const uint32_t rb = (uint32_t)((size_t)bw * LDR * sizeof(float));
    const uint32_t xb = NBB * LDX * sizeof(float);
    uint64_t* bar = &bars[o % S];
    float* dst = ss + sbase + (size_t)(o % S) * stage;
    const float* blk = xinv + (size_t)K * blk_elems(bw);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, rb + xb);
    bulk_g2s(dst, blk + 2 * NBB * LDX + (fwd ? 0 : (size_t)bw * LDR), rb, bar);
    bulk_g2s(dst + xoff, blk + (fwd ? 0 : NBB * LDX), xb, bar);
  };
  if (tid == 0) {
    abort_flag = 0;
    for (int k = 0; k < S; ++k) mbar_init(&bars[k], 1);
    fence_mbar_init();
  }
  double bm = 0.0;
  for (int i = tid; i < n; i += FTB) {
    const int d = dropped[i];
    sdrop[i] = d;
    tv[i] = d ? 0.f : (float)res[i];
    if (first && !d) bm = fmax(bm, fabs(res[i]));
  }
  for (int i = n + tid; i < n4 + NBB; i += FTB) yv[i] = 0.f;
  if (first) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, m));
    if (lane == 0) bred[warp] = bm;
  }
  __syncthreads();
  if (first && tid == 0) {
    double v = 0.0;
    for (int k = 0; k < FTB / 32; ++k) v = fmax(v, bred[k]);
    cstat[0] = (unsigned long long)__double_as_longlong(v);
    cstat[2] = 0ull;
  }
  if (tid == 0) cstat[1] = 0ull;  // the next residual accumulates its max here
  if (tid == 0)
    for (int o = 0; o < S - 1 && o < nops; ++o) issue(o);
  for (int o = 0; o < nops; ++o) {
    const bool fwd = o < nblk;
    const int K = fwd ? o : nops - 1 - o;
    const int r0 = K * NBB, r1 = min(r0 + NBB, n), nr = r1 - r0;
    if (o == nblk) {
      for (int i = tid; i < n; i += FTB) tv[i] = yv[i];
      __syncthreads();
    }
    if (!mbar_wait_bounded(&bars[o % S], (uint32_t)((o / S) & 1))) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    if (tid == 32 && o + S - 1 < nops) issue(o + S - 1);
    const float* Lb = ss + sbase + (size_t)(o % S) * stage;
    const float* M = Lb + xoff;  // X_K (forward) or X_K^T (backward), rows of LDX
    bsolve_diag(M, tv, yv, sdrop, r0, nr, tid);
    __syncthreads();
    bsolve_band(Lb, yv, tv, hpart, fwd, r0, r1, n, bw, tid);
  }
  if (abort_flag) {
    if (tid == 0) {
      for (int b2 = 0; b2 < S; ++b2) mbar_wait_bounded(&bars[b2], 0u), mbar_wait_bounded(&bars[b2], 1u);
      if (err) atomicOr(err, (int)DEVERR_TIMEOUT);
    }
    return;
  }
  for (int i = tid; i < n; i += FTB) {
    const double xi = sdrop[i] ? 0.0 : x[i] + (double)yv[i];
    x[i] = xi;
    a_out[i] = scale[i] * xi;
  }
}

template <int S>
__global__ void __launch_bounds__(FTB) k_coarse_solve_big(int n, int bw, const float* __restrict__ xinv,
                                                          const int* __restrict__ dropped,
                                                          const double* __restrict__ res, double* __restrict__ x,
                                                          const double* __restrict__ scale,
                                                          double* __restrict__ a_out, unsigned long long* cstat,
                                                          int first, const IterCtl* ctl, int* err) {
  solve_big_body<S>(n, bw, xinv, dropped, res, x, scale, a_out, cstat, first, ctl, err);
}

// Batched: one CTA per problem; first = the solve of b, else of the
// refinement residual.
template <int S>
__global__ void __launch_bounds__(FTB) kb_coarse_solve_big(const BatchProb* __restrict__ P,
                                                           const BatchItem* __restrict__ items, int first) {
  const BatchItem it = items[blockIdx.x];
  const BatchProb& q = P[it.prob];
  solve_big_body<S>(q.n_c, q.bw, q.xinv, q.dropped, first ? q.b : q.res, q.x, q.scale, q.a, q.cstat, first, q.ctl,
                    q.err);
}

// ---- two-sided factor and solve (FP32): two SMs, a cluster of 2 CTAs ----
//
// The n unknowns split as [0, m0) (top), the separator [m0, m0 + s) and
// [m0 + s, n) (bottom, m1 rows), with s > bw, so top and bottom do not
// couple.  Side 0 works in the natural order on top + separator, side 1 in
// reversed order (row i of its frame = row n - 1 - i) on bottom + separator;
// each side's frame is a band matrix of bws = s - 1 >= bw (a reversed
// symmetric band matrix is one).  Eliminating a side's segment leaves its
// Schur contribution in the separator block; with both contributions,
//   S = A_MM - L_MT L_MT^T - L_MB L_MB^T,
// each side factors S in its own frame and holds the Cholesky factor of
// [[A_SS, A_SM], [A_MS, S + L_MS L_MS^T]], which with the other side's
// segment contribution is the factor of A in the order (T, B, M).  The chain
// of dependent pivots is max(m0, m1) + s instead of n.
struct FactorSide {
  float* lin;     // (m + s) x (bws + 1) row band of the side's frame: [i][kk] = A[i][i - kk]
  float* lcol;    // L of the side's frame, column layout [c][kk] = L[c + kk][c]
  float* dinv;    // scratch: inverted 16 x 16 diagonal blocks
  int* dropped;   // m + s drop flags of the side's frame
  float* delta;   // s x s, lower: the segment's change of the separator block
  float* srow;    // s x (bws + 1): S in the side's frame, row band
  int m;          // rows of the segment
};

// Both sides' row bands and drop flags from the scaled FP64 band (column layout).
__global__ void k_side_bands(int n, int bw, int bws, int s, int m0, int m1, const double* __restrict__ sband,
                             const int* __restrict__ dropped, float* __restrict__ lin0, float* __restrict__ lin1,
                             int* __restrict__ d0, int* __restrict__ d1, const IterCtl* ctl) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  const int ldw = bws + 1, ld = bw + 1;
  const size_t t0 = (size_t)(m0 + s) * ldw, t1 = (size_t)(m1 + s) * ldw;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < t0 + t1; q += (size_t)gridDim.x * blockDim.x) {
    const bool side1 = q >= t0;
    const size_t ql = side1 ? q - t0 : q;
    const int i = (int)(ql / ldw), kk = (int)(ql % ldw);
    float v = 0.f;
    if (!side1) {
      // A[i][i - kk] = column i - kk, offset kk
      if (kk <= bw && kk <= i) v = (float)sband[(size_t)(i - kk) * ld + kk];
      lin0[ql] = v;
      if (kk == 0) d0[i] = dropped[i];
    } else {
      // A'[i][i - kk] = A[n - 1 - i][n - 1 - i + kk] = column n - 1 - i, offset kk
      const int c = n - 1 - i;
      if (kk <= bw && c + kk < n) v = (float)sband[(size_t)c * ld + kk];
      lin1[ql] = v;
      if (kk == 0) d1[i] = dropped[c];
    }
  }
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(FTF, 1)
    k_coarse_factor_2s(int s, int bws, FactorSide f0, FactorSide f1, const IterCtl* ctl) {
  if (ctl && *(volatile const int*)&ctl->done) return;  // the same for both CTAs
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const FactorSide me = rank ? f1 : f0, ot = rank ? f0 : f1;
  const int ldw = bws + 1;
  // the segment; its change of the separator block to me.delta
  factor_run<float>(me.m + s, me.m, bws, me.lin, me.lcol, me.dinv, me.dropped, 0, me.delta, s);
  __threadfence();
  cl.sync();
  // S in this side's frame; separator row i here is row s - 1 - i of the other frame
  for (int q = threadIdx.x; q < s * ldw; q += FTF) {
    const int i = q / ldw, kk = q - (q / ldw) * ldw, j = i - kk;
    float v = 0.f;
    if (j >= 0)
      v = me.lin[(size_t)(me.m + i) * ldw + kk] - __ldcg(me.delta + (size_t)i * s + j) -
          __ldcg(ot.delta + (size_t)(s - 1 - j) * s + (s - 1 - i));
    me.srow[q] = v;
  }
  __syncthreads();
  factor_run<float>(s, s, bws, me.srow, me.lcol + (size_t)me.m * ldw, me.dinv + (size_t)((me.m + NB - 1) / NB) * NB * NB,
                    me.dropped + me.m, 0, nullptr, 0);
}

// Block partition of a side: 64-row blocks over the segment [0, m) (the last
// one possibly short), then over the separator [m, m + s).
__host__ __device__ inline void side_block(int K, int m, int s, int& r0, int& r1) {
  const int nbT = (m + NBB - 1) / NBB;
  if (K < nbT) {
    r0 = K * NBB;
    r1 = min(r0 + NBB, m);
  } else {
    r0 = m + (K - nbT) * NBB;
    r1 = min(r0 + NBB, m + s);
  }
}
__host__ __device__ inline int side_blocks(int m, int s) { return (m + NBB - 1) / NBB + (s + NBB - 1) / NBB; }

__global__ void __launch_bounds__(256) k_coarse_blockinv_2s(int s, int bws, const float* __restrict__ lcol0,
                                                            const float* __restrict__ lcol1, float* __restrict__ x0,
                                                            float* __restrict__ x1, int m0, int m1,
                                                            const IterCtl* ctl) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  const int nb0 = side_blocks(m0, s);
  const bool side1 = (int)blockIdx.x >= nb0;
  const int K = side1 ? blockIdx.x - nb0 : blockIdx.x;
  const int m = side1 ? m1 : m0;
  int r0, r1;
  side_block(K, m, s, r0, r1);
  blockinv_run(m + s, bws, r0, r1 - r0, side1 ? lcol1 : lcol0,
               (side1 ? x1 : x0) + (size_t)K * blk_elems(bws), blockIdx.y, gridDim.y);
}

struct SolveSide {
  const float* xinv;    // per-block matrices of the side's factor
  const int* dropped;   // drop flags of the side's frame
  const float* lcol;    // the side's factor, column layout (side 1: L_MB^T x_M)
  int m;                // rows of the segment
};

// The block substitution of k_coarse_solve_big on each side's frame.  After
// the forward steps over its segment, each side's separator rows hold b_M
// minus its own segment's contribution; side 0 reads side 1's through
// distributed shared memory (b_M - both contributions) and solves the
// separator with its own factor of S, forward and back.  Side 1 then takes
// x_M from side 0, subtracts L_MB^T x_M from its segment rows and goes back
// through its segment.  One separator solution serves both sides, so they
// agree even where the two frames' FP32 factors of S drop different pivots.
// Side 0 writes the top and the separator, side 1 the bottom.
template <int S>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(FTB)
    k_coarse_solve_2s(int n, int s, int bws, SolveSide s0, SolveSide s1, const double* __restrict__ res,
                      double* __restrict__ x, const double* __restrict__ scale, double* __restrict__ a_out,
                      int* __restrict__ dropped_out, unsigned long long* cstat, int first, const IterCtl* ctl,
                      int* err) {
  if (ctl && *(volatile const int*)&ctl->done) return;  // the same for both CTAs
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const SolveSide sd = rank ? s1 : s0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // first: bit 0 = the solve of b, bit 1 = the last solve the update allows
  const bool last = (first & 2) != 0;
  first &= 1;
  __shared__ int skip;
  if (tid == 0) {
    if (first) {
      skip = 0;
    } else {
      const double bmax = __longlong_as_double((long long)cstat[0]);
      const double rmax = __longlong_as_double((long long)cstat[1]);
      skip = (cstat[2] != 0ull) || !(rmax > 1e-14 * bmax);
      if (!skip && last && rank == 0) atomicAdd(&cstat[3], 1ull);  // refinement used every solve it may
    }
  }
  cl.sync();  // both CTAs have read cstat
  if (skip) {
    if (rank == 0 && tid == 0) cstat[2] = 1ull;
    return;
  }
  if (rank == 0 && tid == 0) cstat[1] = 0ull;  // the next residual accumulates its max here
  extern __shared__ __align__(16) unsigned char ssraw[];
  float* ss = reinterpret_cast<float*>(ssraw);
  __shared__ uint64_t bars[S];
  __shared__ int abort_flag;
  __shared__ double bred[FTB / 32];
  __shared__ double bm_cta;
  __shared__ float hpart[512];
  const int m = sd.m, nside = m + s;
  const int nbT = (m + NBB - 1) / NBB;
  const int nblk = side_blocks(m, s);
  const int nops = 2 * nblk;
  const int stage = big_stage_elems(bws);
  const int xoff = stage - NBB * LDX;
  const int n4 = (nside + 3) / 4 * 4;
  float* tv = ss;
  float* yv = ss + n4;
  const int sbase = 2 * n4 + NBB;
  int* sdrop = reinterpret_cast<int*>(ss + sbase + (size_t)S * stage);
  auto orig = [&](int i) { return rank ? n - 1 - i : i; };

  auto issue = [&](int o) {
    const bool fwd = o < nblk;
    const int K = fwd ? o : nops - 1 - o;
    const uint32_t rb = (uint32_t)((size_t)bws * LDR * sizeof(float));
    const uint32_t xb = NBB * LDX * sizeof(float);
    uint64_t* bar = &bars[o % S];
    float* dst = ss + sbase + (size_t)(o % S) * stage;
    const float* blk = sd.xinv + (size_t)K * blk_elems(bws);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, rb + xb);
    bulk_g2s(dst, blk + 2 * NBB * LDX + (fwd ? 0 : (size_t)bws * LDR), rb, bar);
    bulk_g2s(dst + xoff, blk + (fwd ? 0 : NBB * LDX), xb, bar);
  };
  if (tid == 0) {
    abort_flag = 0;
    for (int k = 0; k < S; ++k) mbar_init(&bars[k], 1);
    fence_mbar_init();
  }
  // the rows this side writes: top and separator (side 0), bottom (side 1)
  const int nown = rank ? m : nside;
  double bm = 0.0;
  for (int i = tid; i < nside; i += FTB) {
    const int d = sd.dropped[i];
    const double bi = res[orig(i)];
    sdrop[i] = d;
    tv[i] = d ? 0.f : (float)bi;
    if (first && !d && i < nown) bm = fmax(bm, fabs(bi));
  }
  for (int i = tid; i < n4 + NBB; i += FTB) yv[i] = 0.f;
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, k));
  if (lane == 0) bred[warp] = bm;
  __syncthreads();
  if (tid == 0) {
    double v = 0.0;
    for (int k = 0; k < FTB / 32; ++k) v = fmax(v, bred[k]);
    bm_cta = v;
  }
  if (tid == 0)
    for (int o = 0; o < S - 1 && o < nops; ++o) issue(o);
  const int oM = 2 * nblk - nbT;  // first backward op over the segment
  for (int o = 0; o < nops; ++o) {
    const bool fwd = o < nblk;
    const int K = fwd ? o : nops - 1 - o;
    int r0, r1;
    side_block(K, m, s, r0, r1);
    const int nr = r1 - r0;
    if (o == oM) {
      // side 0 holds x_M; side 1 takes it (both CTAs come here, aborted or not)
      __syncthreads();
      cl.sync();
      if (rank == 1) {
        const int on4 = (s0.m + s + 3) / 4 * 4;
        const float* oyv = cl.map_shared_rank(ss, 0) + on4;
        for (int i = tid; i < s; i += FTB) yv[m + i] = oyv[s0.m + s - 1 - i];
      }
      cl.sync();  // no reads of the other CTA's shared memory after this
      if (rank == 1 && !abort_flag) {
        // t_i -= sum_{j in M} L[j][i] x_j over the segment's last bws rows, one warp per row
        const int ldw = bws + 1;
        for (int i = max(0, m - bws) + warp; i < m; i += FTB / 32) {
          float acc = 0.f;
          for (int q = lane; q < s && m + q - i <= bws; q += 32)
            acc = fmaf(sd.lcol[(size_t)i * ldw + (m + q - i)], yv[m + q], acc);
#pragma unroll
          for (int k = 16; k > 0; k >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, k);
          if (lane == 0) tv[i] -= acc;
        }
        __syncthreads();
      }
    }
    if (o == nbT) {
      // exchange of the separator rows; both CTAs come here, aborted or not
      __syncthreads();
      cl.sync();
      // the other CTA's layout: tv at 0, its drop flags after its own vectors
      const int mo = rank ? s0.m : s1.m;
      const int on4 = (mo + s + 3) / 4 * 4;
      const float* otv = cl.map_shared_rank(tv, rank ^ 1);
      const int* osd = reinterpret_cast<const int*>(otv + 2 * on4 + NBB + (size_t)S * stage);
      float ov[4] = {0.f, 0.f, 0.f, 0.f};
      bool od[4] = {false, false, false, false};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = tid + u * FTB;
        if (i < s) {
          ov[u] = otv[mo + s - 1 - i];
          od[u] = osd[mo + s - 1 - i] != 0;
        }
      }
      double obm = 0.0;
      if (tid == 0) obm = *cl.map_shared_rank(&bm_cta, rank ^ 1);
      cl.sync();  // no reads of the other CTA's shared memory after this
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = tid + u * FTB;
        // the other side started this row from b (0 if it dropped the row)
        if (i < s && !sdrop[m + i]) tv[m + i] += ov[u] - (od[u] ? 0.f : (float)res[orig(m + i)]);
      }
      if (first && rank == 0 && tid == 0) {
        cstat[0] = (unsigned long long)__double_as_longlong(fmax(bm_cta, obm));
        cstat[2] = 0ull;
      }
      __syncthreads();
    }
    if (abort_flag) {
      if (o >= oM) break;
      continue;
    }
    if (o == nblk) {
      for (int i = tid; i < nside; i += FTB) tv[i] = yv[i];
      __syncthreads();
    }
    if (!mbar_wait_bounded(&bars[o % S], (uint32_t)((o / S) & 1))) abort_flag = 1;
    __syncthreads();
    if (abort_flag) {
      if (o >= oM) break;
      continue;
    }
    if (tid == 32 && o + S - 1 < nops) issue(o + S - 1);
    if (rank == 1 && K >= nbT) continue;  // the separator is side 0's (its copies still pass through)
    const float* Lb = ss + sbase + (size_t)(o % S) * stage;
    const float* Mx = Lb + xoff;
    bsolve_diag(Mx, tv, yv, sdrop, r0, nr, tid);
    __syncthreads();
    bsolve_band(Lb, yv, tv, hpart, fwd, r0, r1, nside, bws, tid);
  }
  if (abort_flag) {
    if (tid == 0) {
      for (int b2 = 0; b2 < S; ++b2) mbar_wait_bounded(&bars[b2], 0u), mbar_wait_bounded(&bars[b2], 1u);
      if (err) atomicOr(err, (int)DEVERR_TIMEOUT);
    }
    return;
  }
  for (int i = tid; i < nown; i += FTB) {
    const int g = orig(i);
    const double xi = sdrop[i] ? 0.0 : x[g] + (double)yv[i];
    x[g] = xi;
    a_out[g] = scale[g] * xi;
    if (first) dropped_out[g] = sdrop[i];
  }
}


__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// res = b - A x in FP64 (A symmetric band: column layout sband, row layout sbandR).
__device__ __forceinline__ void coarse_residual_body(int n, int bw, const double* __restrict__ sband,
                                                     const double* __restrict__ sbandR, const double* __restrict__ b,
                                                     const double* __restrict__ x, const int* __restrict__ dropped,
                                                     double* __restrict__ res, unsigned long long* cstat,
                                                     const IterCtl* ctl, int bx) {
  if (ctl && *(volatile const int*)&ctl->done) return;
  if (*(volatile unsigned long long*)&cstat[2]) return;
  const int lane = threadIdx.x & 31;
  const int row = (bx * blockDim.x + threadIdx.x) >> 5;
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
  if (lane == 0) {
    const double rv = dropped[row] ? 0.0 : b[row] - acc;
    res[row] = rv;
    // max |res| by the order of non-negative doubles' bit patterns
    atomicMax(&cstat[1], (unsigned long long)__double_as_longlong(fabs(rv)));
  }
}

__global__ void k_coarse_residual(int n, int bw, const double* __restrict__ sband,
                                  const double* __restrict__ sbandR, const double* __restrict__ b,
                                  const double* __restrict__ x, const int* __restrict__ dropped,
                                  double* __restrict__ res, unsigned long long* cstat, const IterCtl* ctl) {
  coarse_residual_body(n, bw, sband, sbandR, b, x, dropped, res, cstat, ctl, blockIdx.x);
}
__global__ void kb_coarse_residual(const BatchProb* __restrict__ P, const BatchItem* __restrict__ items) {
  const BatchItem it = items[blockIdx.x];
  const BatchProb& q = P[it.prob];
  coarse_residual_body(q.n_c, q.bw, q.sband, q.sband + (size_t)q.n_c * (q.bw + 1), q.b, q.x, q.dropped, q.res,
                       q.cstat, q.ctl, it.bx);
}

}  // namespace

size_t big_solve_smem_bytes(int n, int bw, int S) {
  const size_t n4 = ((size_t)n + 3) / 4 * 4;
  return (2 * n4 + NBB + (size_t)S * big_stage_elems(bw)) * sizeof(float) + (size_t)n * sizeof(int);
}

cudaError_t configure_coarse_solve(int max_smem) {
  cudaError_t e;
  if ((e = set_max_dynamic_smem(k_coarse_factor_2s, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(kb_coarse_factor, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(kb_coarse_solve_big<2>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(kb_coarse_solve_big<3>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_coarse_solve_2s<2>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_coarse_solve_2s<3>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_coarse_factor<float>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_coarse_factor<double>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_coarse_solve<float>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_coarse_solve_big<2>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_coarse_solve_big<3>, max_smem)) != cudaSuccess) return e;
  return set_max_dynamic_smem(k_coarse_solve<double>, max_smem);
}

size_t coarse_factor_smem_bytes(int n, int bw, bool fp64) {
  if (bw + 1 > 7 * 32) return (size_t)1 << 30;  // beyond the row prefetch of the window slide
  const size_t typed =
      fp64 ? factor_layout<double>(bw).total * sizeof(double) : factor_layout<float>(bw).total * sizeof(float);
  return typed + (size_t)n * sizeof(int) + (size_t)factor_tile_pairs(bw) * 2 * sizeof(unsigned short);
}
size_t coarse_solve_smem_bytes(int n, int bw, bool fp64) {
  const size_t flags = (size_t)n * sizeof(int);
  if (fp64)
    return (2 * (((size_t)n + 3) / 4 * 4) + (size_t)Stages<double>::v * solve_stage_elems<double>(bw)) * sizeof(double) +
           flags;
  return (2 * (((size_t)n + 3) / 4 * 4) + (size_t)Stages<float>::v * solve_stage_elems<float>(bw)) * sizeof(float) +
         flags;
}
int coarse_dinv_size(int n) { return ((n + NB - 1) / NB) * NB * NB; }
size_t coarse_xinv_elems(int n, int bw) { return (size_t)((n + NBB - 1) / NBB) * blk_elems(bw); }

int coarse_big_stages(int n, int bw, int max_smem) {
  for (int S = 3; S >= 2; --S)
    if (big_solve_smem_bytes(n, bw, S) + 4096 <= (size_t)max_smem) return S;
  return 0;
}

cudaError_t launch_coarse_blockinv(cudaStream_t s, int n, int bw, const void* lcol, const void* lrow, float* xinv,
                                   const IterCtl* ctl) {
  (void)lrow;
  k_coarse_blockinv<<<dim3((n + NBB - 1) / NBB, 4), 256, 0, s>>>(n, bw, (const float*)lcol, xinv, ctl);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve_big(cudaStream_t s, int stages, int n, int bw, const void* lcol, const void* lrow,
                                    const float* xinv, const int* dropped, const double* res, double* x,
                                    const double* scale, double* a_out, unsigned long long* cstat, int flags,
                                    const IterCtl* ctl, int* err) {
  const size_t smem = big_solve_smem_bytes(n, bw, stages);
  if (stages >= 3)
    k_coarse_solve_big<3><<<1, FTB, smem, s>>>(n, bw, xinv, dropped, res, x, scale, a_out, cstat, flags,
                                               ctl, err);
  else
    k_coarse_solve_big<2><<<1, FTB, smem, s>>>(n, bw, xinv, dropped, res, x, scale, a_out, cstat, flags,
                                               ctl, err);
  return cudaGetLastError();
}

cudaError_t launch_coarse_factor(cudaStream_t s, int n, int bw, bool fp64, void* lrow, void* lcol, void* dinv,
                                 int* dropped, bool write_lrow, const IterCtl* ctl) {
  const size_t smem = coarse_factor_smem_bytes(n, bw, fp64);
  if (fp64)
    k_coarse_factor<double><<<1, FTF, smem, s>>>(n, bw, (double*)lrow, (double*)lcol, (double*)dinv, dropped,
                                                 write_lrow ? 1 : 0, ctl);
  else
    k_coarse_factor<float><<<1, FTF, smem, s>>>(n, bw, (float*)lrow, (float*)lcol, (float*)dinv, dropped,
                                                write_lrow ? 1 : 0, ctl);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve(cudaStream_t s, int n, int bw, bool fp64, const void* lcol, const void* lrow,
                                const void* dinv, const int* dropped, const double* res, double* x,
                                const double* scale, double* a_out, unsigned long long* cstat, int flags,
                                const IterCtl* ctl, int* err) {
  const size_t smem = coarse_solve_smem_bytes(n, bw, fp64);
  if (fp64)
    k_coarse_solve<double><<<1, FTS, smem, s>>>(n, bw, (const double*)lcol, (const double*)lrow,
                                                (const double*)dinv, dropped, res, x, scale, a_out, cstat,
                                                flags, ctl, err);
  else
    k_coarse_solve<float><<<1, FTS, smem, s>>>(n, bw, (const float*)lcol, (const float*)lrow, (const float*)dinv,
                                               dropped, res, x, scale, a_out, cstat, flags, ctl, err);
  return cudaGetLastError();
}

cudaError_t launch_batch_factor(cudaStream_t s, size_t smem, const BatchProb* P, const BatchItem* it, int n) {
  if (n <= 0) return cudaSuccess;
  kb_coarse_factor<<<n, FTF, smem, s>>>(P, it);
  return cudaGetLastError();
}
cudaError_t launch_batch_blockinv(cudaStream_t s, const BatchProb* P, const BatchItem* it, int n) {
  if (n <= 0) return cudaSuccess;
  kb_coarse_blockinv<<<n, 256, 0, s>>>(P, it);
  return cudaGetLastError();
}
cudaError_t launch_batch_solve(cudaStream_t s, int stages, size_t smem, const BatchProb* P, const BatchItem* it,
                               int n, bool first) {
  if (n <= 0) return cudaSuccess;
  if (stages >= 3) kb_coarse_solve_big<3><<<n, FTB, smem, s>>>(P, it, first ? 1 : 0);
  else kb_coarse_solve_big<2><<<n, FTB, smem, s>>>(P, it, first ? 1 : 0);
  return cudaGetLastError();
}
cudaError_t launch_batch_coarse_residual(cudaStream_t s, const BatchProb* P, const BatchItem* it, int n) {
  if (n <= 0) return cudaSuccess;
  kb_coarse_residual<<<n, 256, 0, s>>>(P, it);
  return cudaGetLastError();
}
int coarse_residual_blocks(int n) { return (int)(((size_t)n * 32 + 255) / 256); }

cudaError_t launch_coarse_residual(cudaStream_t s, int n, int bw, const double* sband, const double* b,
                                   const double* x, const int* dropped, double* res, unsigned long long* cstat,
                                   const IterCtl* ctl) {
  const double* sbandR = sband + (size_t)n * (bw + 1);
  const int threads = 256;
  const int blocks = (int)(((size_t)n * 32 + threads - 1) / threads);
  k_coarse_residual<<<blocks, threads, 0, s>>>(n, bw, sband, sbandR, b, x, dropped, res, cstat, ctl);
  return cudaGetLastError();
}

// Split for the two-sided factor: s = bw + 1 .. bw + 4 separator rows, both
// segments multiples of 4 rows (the factor's 16-byte words) and at least one
// 64-row block.
bool coarse_two_sided_split(int n, int bw, int* m0, int* m1, int* s) {
  const int s0 = bw + 1, rem = n - s0;
  if (rem < 2 * NBB) return false;
  const int a = (rem / 2) / 4 * 4, b = (rem - a) / 4 * 4;
  *m0 = a;
  *m1 = b;
  *s = n - a - b;
  return a >= NBB && b >= NBB && *s <= 7 * 32;  // the window's row loads take ldw <= 224
}
TwoSidedSizes coarse_two_sided_sizes(int m, int s) {
  const int bws = s - 1;
  TwoSidedSizes z;
  z.lin = (size_t)(m + s) * (bws + 1) + 16;
  z.lcol = (size_t)(m + s) * (bws + 1) + 16;
  z.dinv = (size_t)((m + NB - 1) / NB + (s + NB - 1) / NB) * NB * NB;
  z.dropped = (size_t)(m + s);
  z.delta = (size_t)s * s;
  z.srow = (size_t)s * (bws + 1);
  z.xinv = (size_t)side_blocks(m, s) * blk_elems(bws);
  return z;
}
size_t coarse_two_sided_factor_smem(int m0, int m1, int s) {
  return coarse_factor_smem_bytes((m0 > m1 ? m0 : m1) + s, s - 1, false);
}
int coarse_two_sided_stages(int m0, int m1, int s, int max_smem) {
  return coarse_big_stages((m0 > m1 ? m0 : m1) + s, s - 1, max_smem);
}
cudaError_t launch_coarse_factor_2s(cudaStream_t st, int n, int bw, const TwoSided& t, const double* sband,
                                    const int* dropped, const IterCtl* ctl) {
  const int s = t.s, bws = s - 1;
  {
    const size_t total = (size_t)(t.m[0] + t.m[1] + 2 * s) * (bws + 1);
    const int g = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    k_side_bands<<<g, 256, 0, st>>>(n, bw, bws, s, t.m[0], t.m[1], sband, dropped, t.lin[0], t.lin[1],
                                    t.dropped[0], t.dropped[1], ctl);
  }
  FactorSide f[2];
  for (int k = 0; k < 2; ++k)
    f[k] = FactorSide{t.lin[k], t.lcol[k], t.dinv[k], t.dropped[k], t.delta[k], t.srow[k], t.m[k]};
  k_coarse_factor_2s<<<2, FTF, coarse_two_sided_factor_smem(t.m[0], t.m[1], s), st>>>(s, bws, f[0], f[1], ctl);
  const int nb = side_blocks(t.m[0], s) + side_blocks(t.m[1], s);
  k_coarse_blockinv_2s<<<dim3(nb, 4), 256, 0, st>>>(s, bws, t.lcol[0], t.lcol[1], t.xinv[0], t.xinv[1], t.m[0],
                                                    t.m[1], ctl);
  return cudaGetLastError();
}
cudaError_t launch_coarse_solve_2s(cudaStream_t st, int n, const TwoSided& t, const double* res, double* x,
                                   const double* scale, double* a_out, int* dropped_out, unsigned long long* cstat,
                                   int flags, const IterCtl* ctl, int* err) {
  const int s = t.s, bws = s - 1;
  const SolveSide a{t.xinv[0], t.dropped[0], t.lcol[0], t.m[0]}, b{t.xinv[1], t.dropped[1], t.lcol[1], t.m[1]};
  const size_t smem = big_solve_smem_bytes((t.m[0] > t.m[1] ? t.m[0] : t.m[1]) + s, bws, t.stages);
  if (t.stages >= 3)
    k_coarse_solve_2s<3><<<2, FTB, smem, st>>>(n, s, bws, a, b, res, x, scale, a_out, dropped_out, cstat,
                                               flags, ctl, err);
  else
    k_coarse_solve_2s<2><<<2, FTB, smem, st>>>(n, s, bws, a, b, res, x, scale, a_out, dropped_out, cstat,
                                               flags, ctl, err);
  return cudaGetLastError();
}

}  // namespace hms
