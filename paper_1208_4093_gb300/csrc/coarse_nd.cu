// K4 by nested dissection: the upper-level solve of Eq. 8 with its work
// spread over the SMs, for set grids of any width.
//
// The band factorisations (coarse_solve.cu) are one dependency chain down the
// band: n / 16 block steps on one or two SMs, and a band window that must fit
// in shared memory (set grids up to about 22 sets across).  Here the unknowns
// are ordered by nested dissection of the set grid instead.  A box of sets is
// cut by its middle column of sets (or middle row, if it is taller than wide);
// the two halves share no bar (K_aa couples a set only to its eight
// neighbours), so they are eliminated independently and the separator last.
// The recursion stops at boxes of at most 2 x 2 sets.  Every tree node is a
// dense "front" over its own sets S (the separator, or the whole leaf box)
// and its boundary B: the sets around its box, which all lie on ancestor
// separators.  Fronts of one tree level are independent, one CTA each:
//
//   factor, leaves first: F = [A_SS A_SB; A_BS 0] + (children's update
//     matrices, added at their sets' places), then the partial Cholesky
//     L_SS L_SS^T = F_SS, L_BS = F_BS L_SS^-T, U = F_BB - L_BS L_BS^T in 32-
//     column panels; U stays in the front for the parent.  The diagonal
//     32 x 32 blocks of L_SS are stored inverted.
//   forward solve, leaves first: f = [r_S; 0] + children's update vectors,
//     y_S = L_SS^-1 f_S block by block, w = f_B - L_BS y_S for the parent.
//   back substitution, root first: x_S = L_SS^-T (y_S - L_BS^T x_B) with x_B
//     from the ancestors.
//
// The matrix is the Jacobi-scaled one the band path factors, read from the
// blocks of K_aa (coarse_blocks.cu) with the scale and drop flags of
// k_blk_diag and rounded to FP32 as the band path rounds it, so modes dropped
// in FP64 are unit rows already; the factor and solves run in FP32 and the
// FP64 refinement of Eq. 8 (k_blk_residual) works on the same scaled system.
//
// Fronts of at least ND_BIG (300) unknowns (all but the lowest levels of large
// set grids, up to several thousand unknowns) are factored by many CTAs
// instead: one launch assembles every wide front of a level, then per two
// 32-column panels one launch factors the diagonal blocks (one warp per
// front), one forms the panels below them and one applies both panels' rank-32
// updates to the trailing lower triangles in 64 x 64 tiles, so the trailing
// triangle is read and written once per 64 columns.  Their solves hand the
// rectangular parts (the
// boundary rows' products) to many-CTA kernels.  Each step does the arithmetic
// of the one-CTA kernels in the same order, so a front gets the same factor
// and the same solves either way; the threshold only changes the time.
//
// Every sum runs in a fixed order (children in order, rows in order), so
// results are the same on every run.
#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <vector>

#include "coarse_common.cuh"
#include "hms_internal.cuh"

namespace hms {
namespace {

constexpr int NDT = 512;          // threads per front CTA
constexpr int NDW = NDT / 32;     // warps
constexpr int PB = 32;            // panel width (pivots per step)
constexpr float ND_TAU = 1e-6f;   // FP32 pivot below which a mode is dropped (as the band factors)

__device__ inline bool nd_done(const IterCtl* ctl) { return ctl && *(volatile const int*)&ctl->done; }

// global unknown of front position p: set st[p / nm], mode p % nm (nm modes per set)
__device__ inline int nd_glob(const int* st, int p, int nm) { return st[p / nm] * nm + p % nm; }

// Entry (gi, gj) of the scaled matrix, from the blocks of K_aa: 1 on the
// diagonal, 0 in the rows and columns of dropped modes, else s_hi K s_lo in
// FP64 (the larger index's scale first) rounded to FP32.
struct BlkSrc {
  const double* blk;
  const double* scale;
  const int* dropped;
  int Mx, nm;
  __device__ float operator()(int gi, int gj) const {
    if (gi == gj) return 1.f;
    if (dropped[gi] || dropped[gj]) return 0.f;
    const int hi = gi > gj ? gi : gj, lo = gi > gj ? gj : gi;
    const int J = hi / nm, l = hi % nm, I = lo / nm, m = lo % nm;  // J >= I
    const size_t bs = (size_t)nm * nm;
    double k;
    if (J == I) {
      k = blk[(size_t)I * NBLK * bs + (size_t)l * nm + m];
    } else {
      const int b = blk_of(J % Mx - I % Mx, J / Mx - I / Mx);
      if (b <= 0) return 0.f;
      k = blk[((size_t)I * NBLK + b) * bs + (size_t)l * nm + m];
    }
    return (float)(scale[hi] * k * scale[lo]);
  }
};

__device__ inline float warp_sum_f(float v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// ---------------------------------------------------------------- factor
// Cholesky of a kb x kb diagonal block held by one warp (lane = row, a[c] =
// entry (lane, c); rows >= kb zero).  A pivot at or below ND_TAU drops its
// mode: unit diagonal, zero row and column.  Fully unrolled: every index is a
// compile-time constant, so the block stays in registers.
__device__ __forceinline__ unsigned nd_diag_factor(float (&a)[PB], int kb, int lane) {
  constexpr unsigned FULL = 0xffffffffu;
  unsigned dm = 0u;
#pragma unroll
  for (int c = 0; c < PB; ++c) {
    if (c < kb) {
      const float piv = __shfl_sync(FULL, a[c], c);
      const bool drop = !(piv > ND_TAU);
      const float inv = drop ? 0.f : rsqrtf(piv);
      const float d = drop ? 1.f : piv * inv;
      if (lane == c) a[c] = d;
      else if (lane > c) a[c] = a[c] * inv;
      if (drop) {
        dm |= 1u << c;
#pragma unroll
        for (int j = 0; j < c; ++j)
          if (lane == c) a[j] = 0.f;
      }
      const float lc = a[c];
#pragma unroll
      for (int j = c + 1; j < PB; ++j) {
        const float ljc = __shfl_sync(FULL, lc, j);
        if (lane > c) a[j] = fmaf(-lc, ljc, a[j]);
      }
    }
  }
  return dm;
}

// Inverse of a lower-triangular kb x kb block held by one warp (lane = row r,
// a[c] = L[r][c]): by columns, lane j computing x[r] = (inverse)[r][j].
__device__ __forceinline__ void nd_tri_invert(const float (&a)[PB], float (&x)[PB], int kb, int lane) {
  constexpr unsigned FULL = 0xffffffffu;
#pragma unroll
  for (int r = 0; r < PB; ++r) {
    if (r < kb) {
      float sacc = (r == lane) ? 1.f : 0.f;
#pragma unroll
      for (int t = 0; t < r; ++t) sacc = fmaf(-__shfl_sync(FULL, a[t], r), x[t], sacc);
      const float lrr = __shfl_sync(FULL, a[r], r);
      x[r] = (r >= lane) ? sacc / lrr : 0.f;
    } else {
      x[r] = 0.f;
    }
  }
}

// The front of one tree node, factored where it is stored: SM = true keeps it
// in shared memory (packed lower rows, row i from i(i+1)/2) and writes it out
// at the end; SM = false works on the global copy (row-major, nf x nf) with
// the panel staged in shared memory.  Per PB-column panel: warp 0 factors the
// diagonal block and inverts it in registers (the inverse replaces the block:
// the solves multiply by it); every row below is multiplied by the inverse's
// transpose (one warp per row); the trailing lower triangle takes the rank-PB
// update.
template <bool SM, int NT>
__device__ __forceinline__ void nd_factor_body(const NDNode& nd, const NDNode* __restrict__ nodes,
                                               const int* __restrict__ sets, const int* __restrict__ maps,
                                               const BlkSrc& src, float* __restrict__ F,
                                               int* __restrict__ dropped, float* sm, int* gidx, int* cpos,
                                               float (&Dinv)[PB][PB + 1], unsigned& dmask) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nm = nd.nm, nS = nm * nd.ns, nf = nm * (nd.ns + nd.nb);
  float* fg = F + nd.f_off;
  const int* st = sets + nd.s_off;
  auto at = [&](int i, int j) -> float& {
    if constexpr (SM) return sm[(size_t)i * (i + 1) / 2 + j];
    else return fg[(size_t)i * nf + j];
  };
  // the global unknown of every front position
  for (int p = tid; p < nf; p += NT) gidx[p] = nd_glob(st, p, nm);
  __syncthreads();

  // ---- assemble: original entries of the S columns, zero B x B (NU loads in flight per lane) ----
  constexpr int NU = 4;
  for (int p = warp; p < nf; p += (NT / 32)) {
    const int gp = gidx[p];
    for (int q0 = lane; q0 <= p; q0 += 32 * NU) {
      float v[NU];
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        const int q = q0 + 32 * u;
        v[u] = (q <= p && q < nS) ? src(gp, gidx[q]) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        const int q = q0 + 32 * u;
        if (q <= p) at(p, q) = v[u];
      }
    }
  }
  __syncthreads();
  // ---- extend-add of the children's update matrices (one child after the other) ----
  for (int c = 0; c < nd.nchild; ++c) {
    const NDNode ch = nodes[nd.child[c]];
    const int nSc = nm * ch.ns, nbc = nm * ch.nb, nfc = nSc + nbc;
    const float* U = F + ch.f_off + (size_t)nSc * nfc + nSc;
    const int* mp = maps + nd.map_off[c];
    for (int k = tid; k < nbc; k += NT) cpos[k] = nm * mp[k / nm] + k % nm;
    __syncthreads();
    for (int k = warp; k < nbc; k += (NT / 32)) {
      const int pk = cpos[k];
      const float* Uk = U + (size_t)k * nfc;
      for (int l0 = lane; l0 <= k; l0 += 32 * NU) {
        float v[NU];
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          const int l = l0 + 32 * u;
          v[u] = l <= k ? Uk[l] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          const int l = l0 + 32 * u;
          if (l <= k) {
            const int pl = cpos[l];
            at(pk > pl ? pk : pl, pk > pl ? pl : pk) += v[u];
          }
        }
      }
    }
    __syncthreads();
  }

  // ---- partial Cholesky of the first nS columns, PB columns at a time ----
  float* panel = sm;  // global mode: rows below the diagonal block, [nf - k0 - kb][PB + 1]
  for (int k0 = 0; k0 < nS; k0 += PB) {
    const int kb = min(PB, nS - k0);
    // (a) diagonal block: Cholesky and its inverse in warp 0's registers; the
    // inverse is stored in the block's place (the solves multiply by it)
    if (warp == 0) {
      float a[PB], x[PB];
#pragma unroll
      for (int c = 0; c < PB; ++c) a[c] = (lane < kb && c <= lane) ? at(k0 + lane, k0 + c) : 0.f;
      const unsigned dm = nd_diag_factor(a, kb, lane);
      nd_tri_invert(a, x, kb, lane);
#pragma unroll
      for (int r = 0; r < PB; ++r) Dinv[r][lane] = x[r];
      __syncwarp();
      for (int r = 0; r < kb; ++r)
        if (lane <= r) at(k0 + r, k0 + lane) = Dinv[r][lane];
      // a dropped mode's earlier L row is zeroed and its flag raised
      for (int c = 0; c < kb; ++c)
        if ((dm >> c) & 1u) {
          for (int j = lane; j < k0; j += 32) at(k0 + c, j) = 0.f;
          if (lane == 0) dropped[gidx[k0 + c]] = 1;
        }
      if (lane == 0) dmask = dm;
    }
    __syncthreads();
    // (b) the panel below: L[i][blk] = F[i][blk] Dinv^T, one warp per row (lane = column)
    const unsigned dmk = dmask;
    const int r0 = k0 + kb, m = nf - r0;
    for (int ii = warp; ii < m; ii += (NT / 32)) {
      const float fv = lane < kb ? at(r0 + ii, k0 + lane) : 0.f;
      float sacc = 0.f;
#pragma unroll
      for (int u = 0; u < PB; ++u) sacc = fmaf(__shfl_sync(0xffffffffu, fv, u), Dinv[lane][u], sacc);
      if ((dmk >> lane) & 1u) sacc = 0.f;
      if (lane < kb) {
        at(r0 + ii, k0 + lane) = sacc;
        if constexpr (!SM) panel[(size_t)ii * (PB + 1) + lane] = sacc;
      }
    }
    __syncthreads();
    // (c) trailing update of the lower triangle below the block, 4 x 4 tiles
    const int T = (m + 3) / 4;
    const int ntile = T * (T + 1) / 2;
    for (int t = tid; t < ntile; t += NT) {
      int ti = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
      while (ti * (ti + 1) / 2 > t) --ti;
      while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
      const int tj = t - ti * (ti + 1) / 2;
      float acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
      for (int u = 0; u < kb; ++u) {
        float pa[4], pb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int ia = 4 * ti + a, jb = 4 * tj + a;
          if constexpr (SM) {
            pa[a] = ia < m ? at(r0 + ia, k0 + u) : 0.f;
            pb[a] = jb < m ? at(r0 + jb, k0 + u) : 0.f;
          } else {
            pa[a] = ia < m ? panel[(size_t)ia * (PB + 1) + u] : 0.f;
            pb[a] = jb < m ? panel[(size_t)jb * (PB + 1) + u] : 0.f;
          }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(pa[a], pb[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int i = 4 * ti + a;
        if (i >= m) break;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int j = 4 * tj + b;
          if (j <= i) at(r0 + i, r0 + j) -= acc[a][b];
        }
      }
    }
    __syncthreads();
  }
  if constexpr (SM) {
    // the factored front out to its global copy (the solves and the parent read it there)
    for (int p = warp; p < nf; p += (NT / 32))
      for (int q = lane; q <= p; q += 32) fg[(size_t)p * nf + q] = sm[(size_t)p * (p + 1) / 2 + q];
  }
}

// One CTA per front of a tree level.  cap = the launch's dynamic shared
// memory in floats: a front whose packed lower triangle fits is factored in
// shared memory.
template <int NT>
__global__ void __launch_bounds__(NT) k_nd_factor(const NDNode* __restrict__ nodes, const int* __restrict__ lvl,
                                                   int lbeg, const int* __restrict__ sets,
                                                   const int* __restrict__ maps, BlkSrc src,
                                                   float* __restrict__ F, int* __restrict__ dropped,
                                                   long long cap, const IterCtl* ctl) {
  if (nd_done(ctl)) return;
  extern __shared__ __align__(16) float ndsm[];
  __shared__ float Dinv[PB][PB + 1];
  __shared__ unsigned dmask;
  const NDNode nd = nodes[lvl[lbeg + blockIdx.x]];
  const long long nf = nd.nm * (long long)(nd.ns + nd.nb);
  // the last 2 nf floats of the region hold the front's unknown indices and a child's positions
  int* gidx = reinterpret_cast<int*>(ndsm + (cap - 2 * nf));
  int* cpos = gidx + nf;
  if (nf * (nf + 1) / 2 + 2 * nf <= cap)
    nd_factor_body<true, NT>(nd, nodes, sets, maps, src, F, dropped, ndsm, gidx, cpos, Dinv, dmask);
  else
    nd_factor_body<false, NT>(nd, nodes, sets, maps, src, F, dropped, ndsm, gidx, cpos, Dinv, dmask);
}

// ---------------------------------------------------------------- wide fronts
// Assembly of the wide fronts of a level: CTA (x, y) takes rows 32x .. 32x+31
// of front y (one warp per row, lane = column): the original entries of the S
// columns, then each child's update matrix added at its sets' places, child
// after child (the order of the one-CTA extend-add).
__global__ void __launch_bounds__(256) k_ndb_assemble(const NDNode* __restrict__ nodes, const NDBig* __restrict__ bigs,
                                                      const int* __restrict__ sets, const int* __restrict__ inv,
                                                      BlkSrc src, float* __restrict__ F, const IterCtl* ctl) {
  if (nd_done(ctl)) return;
  const NDBig bg = bigs[blockIdx.y];
  const NDNode nd = nodes[bg.node];
  const int nm = nd.nm, nS = nm * nd.ns, nf = nm * (nd.ns + nd.nb);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int* st = sets + nd.s_off;
  float* fg = F + nd.f_off;
  // the children's front shapes (at most two; indices fixed at compile time so
  // that they stay in registers)
  long long cf_off[2] = {0, 0};
  int cnS[2] = {0, 0}, cnf[2] = {0, 0};
#pragma unroll
  for (int c = 0; c < 2; ++c)
    if (c < nd.nchild) {
      const NDNode chn = nodes[nd.child[c]];
      cf_off[c] = chn.f_off;
      cnS[c] = chn.nm * chn.ns;
      cnf[c] = cnS[c] + chn.nm * chn.nb;
    }
  for (int p = blockIdx.x * 32 + warp; p < nf && p < blockIdx.x * 32 + 32; p += 8) {
    const int gp = nd_glob(st, p, nm);
    int kp[2] = {-1, -1};
#pragma unroll
    for (int c = 0; c < 2; ++c)
      if (c < nd.nchild) {
        const int t = inv[bg.inv_off[c] + p / nm];
        kp[c] = t < 0 ? -1 : nm * t + p % nm;
      }
    // AU columns per lane at a time: their loads are independent, so they are
    // all issued before the stores (the same value per entry, added in the
    // same order)
    constexpr int AU = 4;
    for (int q0 = lane; q0 <= p; q0 += 32 * AU) {
      float v[AU];
#pragma unroll
      for (int k = 0; k < AU; ++k) {
        const int q = q0 + 32 * k;
        v[k] = (q <= p && q < nS) ? src(gp, nd_glob(st, q, nm)) : 0.f;
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (c >= nd.nchild || kp[c] < 0) continue;
        const int nSc = cnS[c], nfc = cnf[c];
        float add[AU];
#pragma unroll
        for (int k = 0; k < AU; ++k) {
          const int q = q0 + 32 * k;
          add[k] = 0.f;
          const int t = q <= p ? inv[bg.inv_off[c] + q / nm] : -1;
          if (t >= 0) {
            const int kq = nm * t + q % nm;
            const int a = kp[c] > kq ? kp[c] : kq, b = kp[c] > kq ? kq : kp[c];
            add[k] = F[cf_off[c] + (size_t)(nSc + a) * nfc + nSc + b];
          }
        }
#pragma unroll
        for (int k = 0; k < AU; ++k) {
          const int q = q0 + 32 * k;
          if (q <= p && inv[bg.inv_off[c] + q / nm] >= 0) v[k] += add[k];
        }
      }
#pragma unroll
      for (int k = 0; k < AU; ++k) {
        const int q = q0 + 32 * k;
        if (q <= p) fg[(size_t)p * nf + q] = v[k];
      }
    }
  }
}

// Two 32-column panels per step (A = [k0, k0+32), B = [k0+32, k0+64)), with
// the arithmetic of two one-panel steps in their order, so that the trailing
// triangle is read and written once per 64 columns.
//
// (a, b) One CTA of 8 warps per front: warp 0 factors A's diagonal block
// (factor, inverse, drops); all warps form the rows of B below it (L21 =
// F[B][A] Dinv_A^T, a warp per row) and update B's diagonal block by L21
// L21^T (a thread per entry); warp 0 factors B's diagonal block.
__global__ void __launch_bounds__(256) k_ndb_diag2(const NDNode* __restrict__ nodes, const NDBig* __restrict__ bigs,
                                                   const int* __restrict__ sets, float* __restrict__ F,
                                                   int* __restrict__ dropped, int* __restrict__ dmask_out, int k0,
                                                   const IterCtl* ctl) {
  if (nd_done(ctl)) return;
  const NDNode nd = nodes[bigs[blockIdx.x].node];
  const int nm = nd.nm, nS = nm * nd.ns, nf = nm * (nd.ns + nd.nb);
  if (k0 >= nS) return;
  __shared__ float DA[PB][PB + 1];
  __shared__ float L21[PB][PB + 1];
  __shared__ unsigned dmAs;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int kbA = min(PB, nS - k0), kB = k0 + PB, kbB = min(PB, nS - kB);
  float* fg = F + nd.f_off;
  const int* st = sets + nd.s_off;
  if (warp == 0) {
    // A: the one-panel step (a)
    float a[PB], x[PB];
#pragma unroll
    for (int c = 0; c < PB; ++c) a[c] = (lane < kbA && c <= lane) ? fg[(size_t)(k0 + lane) * nf + k0 + c] : 0.f;
    const unsigned dm = nd_diag_factor(a, kbA, lane);
    nd_tri_invert(a, x, kbA, lane);
#pragma unroll
    for (int r = 0; r < PB; ++r) {
      DA[r][lane] = x[r];
      if (r < kbA && lane <= r) fg[(size_t)(k0 + r) * nf + k0 + lane] = x[r];
    }
    for (int c = 0; c < kbA; ++c)
      if ((dm >> c) & 1u) {
        for (int jj = lane; jj < k0; jj += 32) fg[(size_t)(k0 + c) * nf + jj] = 0.f;
        if (lane == 0) dropped[nd_glob(st, k0 + c, nm)] = 1;
      }
    if (lane == 0) dmAs = dm;
  }
  __syncthreads();
  const unsigned dmA = dmAs;
  unsigned dmB = 0u;
  if (kbB > 0) {
    // B's rows of A's panel (the one-panel step (b) on those rows)
    for (int r = warp; r < kbB; r += 8) {
      float* row = fg + (size_t)(kB + r) * nf + k0;
      const float fv = lane < kbA ? row[lane] : 0.f;
      float sacc = 0.f;
#pragma unroll
      for (int u = 0; u < PB; ++u) sacc = fmaf(__shfl_sync(0xffffffffu, fv, u), DA[lane][u], sacc);
      if ((dmA >> lane) & 1u) sacc = 0.f;
      L21[r][lane] = lane < kbA ? sacc : 0.f;
      if (lane < kbA) row[lane] = sacc;
    }
    __syncthreads();
    // B's diagonal block takes A's rank-kbA update (the one-panel step (c) there)
    for (int e = tid; e < PB * PB; e += 256) {
      const int i = e / PB, jj = e % PB;
      if (i < kbB && jj <= i) {
        float acc = 0.f;
        for (int u = 0; u < kbA; ++u) acc = fmaf(L21[i][u], L21[jj][u], acc);
        fg[(size_t)(kB + i) * nf + kB + jj] -= acc;
      }
    }
    __syncthreads();
    if (warp == 0) {
      // B: the one-panel step (a)
      float a[PB], x[PB];
#pragma unroll
      for (int c = 0; c < PB; ++c) a[c] = (lane < kbB && c <= lane) ? fg[(size_t)(kB + lane) * nf + kB + c] : 0.f;
      dmB = nd_diag_factor(a, kbB, lane);
      nd_tri_invert(a, x, kbB, lane);
#pragma unroll
      for (int r = 0; r < PB; ++r)
        if (r < kbB && lane <= r) fg[(size_t)(kB + r) * nf + kB + lane] = x[r];
      for (int c = 0; c < kbB; ++c)
        if ((dmB >> c) & 1u) {
          for (int jj = lane; jj < kB; jj += 32) fg[(size_t)(kB + c) * nf + jj] = 0.f;
          if (lane == 0) dropped[nd_glob(st, kB + c, nm)] = 1;
        }
    }
  }
  if (tid == 0) {
    dmask_out[2 * blockIdx.x] = (int)dmA;
    dmask_out[2 * blockIdx.x + 1] = (int)dmB;
  }
}

// (c) The rows below both panels, one warp per row (lane = column): L[i][A] =
// F[i][A] Dinv_A^T; F[i][B] takes A's update; L[i][B] = F[i][B] Dinv_B^T.
// CTA (x, y): rows r0 + 64x .. of front y, r0 = k0 + kbA + kbB.
__global__ void __launch_bounds__(256) k_ndb_panel2(const NDNode* __restrict__ nodes, const NDBig* __restrict__ bigs,
                                                    float* __restrict__ F, const int* __restrict__ dmask, int k0,
                                                    const IterCtl* ctl) {
  if (nd_done(ctl)) return;
  const NDNode nd = nodes[bigs[blockIdx.y].node];
  const int nm = nd.nm, nS = nm * nd.ns, nf = nm * (nd.ns + nd.nb);
  if (k0 >= nS) return;
  const int kbA = min(PB, nS - k0), kB = k0 + PB, kbB = max(0, min(PB, nS - kB));
  const int r0 = k0 + kbA + kbB;
  const int rbeg = r0 + 64 * blockIdx.x;
  if (rbeg >= nf) return;
  __shared__ float DA[PB][PB + 1], DB[PB][PB + 1], L21[PB][PB + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* fg = F + nd.f_off;
  for (int e = tid; e < PB * PB; e += 256) {
    const int r = e / PB, c = e % PB;
    DA[r][c] = (r < kbA && c <= r) ? fg[(size_t)(k0 + r) * nf + k0 + c] : 0.f;
    DB[r][c] = (r < kbB && c <= r) ? fg[(size_t)(kB + r) * nf + kB + c] : 0.f;
    L21[r][c] = (r < kbB && c < kbA) ? fg[(size_t)(kB + r) * nf + k0 + c] : 0.f;
  }
  __syncthreads();
  const unsigned dmA = (unsigned)dmask[2 * blockIdx.y], dmB = (unsigned)dmask[2 * blockIdx.y + 1];
  // this warp's eight rows, their entries of both panels loaded first (latency)
  float fa[8], fbv[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int i = rbeg + warp + 8 * q;
    const bool in = i < nf;
    fa[q] = (in && lane < kbA) ? fg[(size_t)i * nf + k0 + lane] : 0.f;
    fbv[q] = (in && lane < kbB) ? fg[(size_t)i * nf + kB + lane] : 0.f;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int i = rbeg + warp + 8 * q;
    if (i >= nf) break;
    float* row = fg + (size_t)i * nf;
    const float fv = fa[q];
    float sA = 0.f;
#pragma unroll
    for (int u = 0; u < PB; ++u) sA = fmaf(__shfl_sync(0xffffffffu, fv, u), DA[lane][u], sA);
    if ((dmA >> lane) & 1u) sA = 0.f;
    if (lane < kbA) row[k0 + lane] = sA;
    if (kbB > 0) {
      float acc = 0.f;
      for (int u = 0; u < kbA; ++u) acc = fmaf(__shfl_sync(0xffffffffu, sA, u), L21[lane][u], acc);
      const float fb = lane < kbB ? fbv[q] - acc : 0.f;
      float sB = 0.f;
#pragma unroll
      for (int u = 0; u < PB; ++u) sB = fmaf(__shfl_sync(0xffffffffu, fb, u), DB[lane][u], sB);
      if ((dmB >> lane) & 1u) sB = 0.f;
      if (lane < kbB) row[kB + lane] = sB;
    }
  }
}

constexpr int ULD = 68;  // padded row of the transposed panels (16-byte multiple)

// (d) The trailing lower triangle below both panels, rows and columns from r0
// = k0 + kbA + kbB, in 64 x 64 tiles: F[i][j] takes A's rank-kbA update, then
// B's, each sum over u in order from 0 (the two one-panel updates).
__global__ void __launch_bounds__(256) k_ndb_update2(const NDNode* __restrict__ nodes, const NDBig* __restrict__ bigs,
                                                     float* __restrict__ F, int k0, const IterCtl* ctl) {
  if (nd_done(ctl)) return;
  const NDNode nd = nodes[bigs[blockIdx.y].node];
  const int nm = nd.nm, nS = nm * nd.ns, nf = nm * (nd.ns + nd.nb);
  if (k0 >= nS) return;
  const int kbA = min(PB, nS - k0), kB = k0 + PB, kbB = max(0, min(PB, nS - kB));
  const int r0 = k0 + kbA + kbB, m = nf - r0;
  const int T = (m + 63) / 64;
  const int t = blockIdx.x;
  if (t >= T * (T + 1) / 2) return;
  int ti = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while (ti * (ti + 1) / 2 > t) --ti;
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  const int tj = t - ti * (ti + 1) / 2;
  __shared__ __align__(16) float La[2][PB][ULD];
  __shared__ __align__(16) float Lb[2][PB][ULD];
  float* fg = F + nd.f_off;
  const int tid = threadIdx.x;
  {
    // all the tile's loads issued before the shared-memory stores (latency)
    constexpr int NE = 64 * 2 * PB / 256;
    float va[NE], vb[NE];
#pragma unroll
    for (int q0 = 0; q0 < NE; ++q0) {
      const int e = tid + 256 * q0;
      const int r = e / (2 * PB), q = e % (2 * PB), pnl = q / PB, u = q % PB;
      const int kbq = pnl == 0 ? kbA : kbB, kq = pnl == 0 ? k0 : kB;
      const int ia = 64 * ti + r, jb = 64 * tj + r;
      va[q0] = (ia < m && u < kbq) ? fg[(size_t)(r0 + ia) * nf + kq + u] : 0.f;
      vb[q0] = (jb < m && u < kbq) ? fg[(size_t)(r0 + jb) * nf + kq + u] : 0.f;
    }
#pragma unroll
    for (int q0 = 0; q0 < NE; ++q0) {
      const int e = tid + 256 * q0;
      const int r = e / (2 * PB), q = e % (2 * PB), pnl = q / PB, u = q % PB;
      La[pnl][u][r] = va[q0];
      Lb[pnl][u][r] = vb[q0];
    }
  }
  __syncthreads();
  const int ty = tid / 16, tx = tid % 16;
  // this thread's 4 x 4 entries of F, fetched before the products (latency)
  float cur[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = 64 * ti + 4 * ty + a, j = 64 * tj + 4 * tx + b;
      cur[a][b] = (i < m && j <= i) ? fg[(size_t)(r0 + i) * nf + r0 + j] : 0.f;
    }
  float acc[4][4], acc2[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f, acc2[a][b] = 0.f;
  for (int u = 0; u < kbA; ++u) {
    const float4 qa = *reinterpret_cast<const float4*>(&La[0][u][4 * ty]);
    const float4 qb = *reinterpret_cast<const float4*>(&Lb[0][u][4 * tx]);
    const float pa[4] = {qa.x, qa.y, qa.z, qa.w}, pb[4] = {qb.x, qb.y, qb.z, qb.w};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(pa[a], pb[b], acc[a][b]);
  }
  for (int u = 0; u < kbB; ++u) {
    const float4 qa = *reinterpret_cast<const float4*>(&La[1][u][4 * ty]);
    const float4 qb = *reinterpret_cast<const float4*>(&Lb[1][u][4 * tx]);
    const float pa[4] = {qa.x, qa.y, qa.z, qa.w}, pb[4] = {qb.x, qb.y, qb.z, qb.w};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc2[a][b] = fmaf(pa[a], pb[b], acc2[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = 64 * ti + 4 * ty + a;
    if (i >= m) break;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = 64 * tj + 4 * tx + b;
      if (j <= i) {
        float v = cur[a][b] - acc[a][b];
        if (kbB > 0) v -= acc2[a][b];
        fg[(size_t)(r0 + i) * nf + r0 + j] = v;
      }
    }
  }
}

// ---------------------------------------------------------------- solves
// Begins a solve: q = 0 takes max |b| (non-dropped rows) for the refinement
// test and clears the converged flag; later solves decide whether refinement
// has converged (cstat[2] = 1: the level kernels and residuals return at once).
// flags: bit 0 = the solve of b, bit 1 = the last solve the update allows.
__global__ void __launch_bounds__(1024) k_nd_solve_begin(int n, const double* __restrict__ rhs,
                                                         const int* __restrict__ dropped, unsigned long long* cstat,
                                                         int flags, const IterCtl* ctl) {
  if (nd_done(ctl)) return;
  __shared__ double red[32];
  const int tid = threadIdx.x;
  if (flags & 1) {
    double bm = 0.0;
    for (int i = tid; i < n; i += blockDim.x)
      if (!dropped[i]) bm = fmax(bm, fabs(rhs[i]));
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, m));
    if ((tid & 31) == 0) red[tid >> 5] = bm;
    __syncthreads();
    if (tid == 0) {
      double v = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v = fmax(v, red[k]);
      cstat[0] = (unsigned long long)__double_as_longlong(v);
      cstat[2] = 0ull;
      cstat[1] = 0ull;
    }
    return;
  }
  if (tid == 0) {
    const double bmax = __longlong_as_double((long long)cstat[0]);
    const double rmax = __longlong_as_double((long long)cstat[1]);
    const bool skip = (cstat[2] != 0ull) || !(rmax > 1e-14 * bmax);
    if (skip) cstat[2] = 1ull;
    else if (flags & 2) atomicAdd(&cstat[3], 1ull);  // refinement used every solve it may
    cstat[1] = 0ull;  // the next residual accumulates its max here
  }
}

// rows per warp in flight in the forward solve's row products: 4 for the
// one-CTA fronts (fewer registers, more CTAs per SM), 16 for the wide ones
constexpr int RU_SMALL = 4, RU_WIDE = 16;
constexpr int NDQ = 12;   // columns per lane and pass in the back substitution's first product

// Shared memory of a solve CTA (floats): the front's vector (nf), the warps'
// partial sums (NDW x nS) and the front's unknown indices (nf ints).  The
// factor is read where it lies (global, L2-resident): staging it first cost
// more than the reads themselves, the fronts being small.
__device__ __host__ inline long long nd_solve_need(long long nS, long long nf) {
  return nf + (nf > nS ? NDW * nS : 0) + nf;
}

template <int RU>
__global__ void __launch_bounds__(NDT) k_nd_forward(const NDNode* __restrict__ nodes, const int* __restrict__ lvl,
                                                    int lbeg, const int* __restrict__ sets,
                                                    const int* __restrict__ maps, const float* __restrict__ F,
                                                    float* __restrict__ W, const double* __restrict__ rhs,
                                                    const int* __restrict__ dropped, float* __restrict__ y,
                                                    long long cap, const unsigned long long* cstat,
                                                    const IterCtl* ctl) {
  if (nd_done(ctl) || *(volatile const unsigned long long*)&cstat[2]) return;
  extern __shared__ __align__(16) float ndsm[];
  __shared__ float yb[PB];
  const NDNode nd = nodes[lvl[lbeg + blockIdx.x]];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nm = nd.nm, nS = nm * nd.ns, nf = nm * (nd.ns + nd.nb);
  // a wide front's boundary rows are updated by k_ndb_fwd_rect, after this kernel
  const int nrow = nf >= ND_BIG ? nS : nf;
  const float* f = F + nd.f_off;
  const int* st = sets + nd.s_off;
  float* fv = ndsm;
  int* gidx = reinterpret_cast<int*>(ndsm + (cap - nf));
  const float* Lp = f;
  const int ld = nf;
  for (int p = tid; p < nf; p += NDT) gidx[p] = nd_glob(st, p, nm);
  __syncthreads();
  for (int p = tid; p < nf; p += NDT) {
    float v = 0.f;
    if (p < nS) {
      const int g = gidx[p];
      v = dropped[g] ? 0.f : (float)rhs[g];
    }
    fv[p] = v;
  }
  __syncthreads();
  for (int c = 0; c < nd.nchild; ++c) {
    const NDNode ch = nodes[nd.child[c]];
    const int nbc = nm * ch.nb;
    const int* mp = maps + nd.map_off[c];
    for (int k = tid; k < nbc; k += NDT) fv[nm * mp[k / nm] + k % nm] += W[ch.w_off + k];
    __syncthreads();
  }
  for (int k0 = 0; k0 < nS; k0 += PB) {
    const int kb = min(PB, nS - k0);
    const float fl = lane < kb ? fv[k0 + lane] : 0.f;
    // y_blk = Dinv f_blk: two rows per warp, lane = column
    for (int t = warp; t < kb; t += NDW) {
      const float v = lane <= t ? Lp[(size_t)(k0 + t) * ld + k0 + lane] * fl : 0.f;
      const float sum = warp_sum_f(v);
      if (lane == 0) yb[t] = sum;
    }
    __syncthreads();
    const float yl = lane < kb ? yb[lane] : 0.f;
    if (tid < kb) fv[k0 + tid] = yb[tid];
    // rows below: f_i -= L[i][blk] y_blk, RU rows per warp at once
    for (int i0 = k0 + kb + RU * warp; i0 < nrow; i0 += RU * NDW) {
      float v[RU];
#pragma unroll
      for (int q = 0; q < RU; ++q) {
        const int i = i0 + q;
        v[q] = (i < nrow && lane < kb) ? Lp[(size_t)i * ld + k0 + lane] * yl : 0.f;
      }
#pragma unroll
      for (int q = 0; q < RU; ++q) v[q] = warp_sum_f(v[q]);
      if (lane < RU && i0 + lane < nrow) {
        float mine = v[0];
#pragma unroll
        for (int q = 1; q < RU; ++q) mine = lane == q ? v[q] : mine;
        fv[i0 + lane] -= mine;
      }
    }
    __syncthreads();
  }
  for (int p = tid; p < nf; p += NDT) {
    if (p < nS) y[gidx[p]] = fv[p];
    else W[nd.w_off + (p - nS)] = fv[p];
  }
}

template <int PRE>
__global__ void __launch_bounds__(NDT) k_nd_backward(const NDNode* __restrict__ nodes, const int* __restrict__ lvl,
                                                     int lbeg, const int* __restrict__ sets,
                                                     const float* __restrict__ F, const float* __restrict__ y,
                                                     float* __restrict__ xc, const int* __restrict__ dropped,
                                                     double* __restrict__ x, const double* __restrict__ scale,
                                                     double* __restrict__ a_out, long long cap,
                                                     const unsigned long long* cstat, const IterCtl* ctl) {
  if (nd_done(ctl) || *(volatile const unsigned long long*)&cstat[2]) return;
  extern __shared__ __align__(16) float ndsm[];
  __shared__ float xb[PB];
  const NDNode nd = nodes[lvl[lbeg + blockIdx.x]];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nm = nd.nm, nS = nm * nd.ns, nB = nm * nd.nb, nf = nS + nB;
  const float* f = F + nd.f_off;
  const int* st = sets + nd.s_off;
  float* tv = ndsm;                 // nS
  float* xB = ndsm + nS;            // nB: the ancestors' corrections
  float* part = ndsm + nf;          // NDW x nS partial sums
  int* gidx = reinterpret_cast<int*>(ndsm + (cap - nf));
  const float* Lp = f;
  const int ld = nf;
  for (int p = tid; p < nf; p += NDT) gidx[p] = nd_glob(st, p, nm);
  __syncthreads();
  for (int k = tid; k < nB; k += NDT) xB[k] = xc[gidx[nS + k]];
  __syncthreads();
  // t = y_S - L_BS^T x_B: warp w sums the rows k = w, w + NDW, ... (lane: columns
  // lane + 32 q), then the warps' partial sums are added in warp order
  // (a wide front's t was formed by k_ndb_bwd_rect, in the same order, into y)
  const bool rect = nB > 0 && nf < ND_BIG;
  for (int jb = 0; rect && jb < nS; jb += 32 * NDQ) {
    float acc[NDQ];
#pragma unroll
    for (int q = 0; q < NDQ; ++q) acc[q] = 0.f;
    for (int k = warp; k < nB; k += NDW) {
      const float xk = xB[k];
      const float* row = Lp + (size_t)(nS + k) * ld + jb;
#pragma unroll
      for (int q = 0; q < NDQ; ++q) {
        const int j = lane + 32 * q;
        if (jb + j < nS) acc[q] = fmaf(row[j], xk, acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < NDQ; ++q) {
      const int j = jb + lane + 32 * q;
      if (j < nS) part[warp * nS + j] = acc[q];
    }
  }
  __syncthreads();
  for (int j = tid; j < nS; j += NDT) {
    float sacc = y[gidx[j]];
    if (rect)
      for (int w = 0; w < NDW; ++w) sacc -= part[w * nS + j];
    tv[j] = sacc;
  }
  __syncthreads();
  const int nblk = (nS + PB - 1) / PB;
  for (int b = nblk - 1; b >= 0; --b) {
    const int k0 = b * PB, kb = min(PB, nS - k0);
    if (warp == 0) {
      // x_blk = Dinv^T t_blk: lane c sums rows r >= c of column c
      float sacc = 0.f;
#pragma unroll 8
      for (int r = 0; r < kb; ++r) {
        const float dv = (lane <= r) ? Lp[(size_t)(k0 + r) * ld + k0 + lane] : 0.f;
        sacc = fmaf(dv, tv[k0 + r], sacc);
      }
      if (lane < kb) xb[lane] = sacc;
    }
    __syncthreads();
    if (tid < kb) tv[k0 + tid] = xb[tid];
    // earlier columns: t_j -= sum_r L[k0 + r][j] x_r
    // PRE entries of the column loaded ahead of their products (same order)
    for (int j = tid; j < k0; j += NDT) {
      float sacc = tv[j];
      for (int r0 = 0; r0 < kb; r0 += PRE) {
        float lv[PRE];
#pragma unroll
        for (int q = 0; q < PRE; ++q) lv[q] = r0 + q < kb ? Lp[(size_t)(k0 + r0 + q) * ld + j] : 0.f;
#pragma unroll
        for (int q = 0; q < PRE; ++q)
          if (r0 + q < kb) sacc = fmaf(-lv[q], xb[r0 + q], sacc);
      }
      tv[j] = sacc;
    }
    __syncthreads();
  }
  for (int j = tid; j < nS; j += NDT) {
    const int g = gidx[j];
    const float v = dropped[g] ? 0.f : tv[j];
    xc[g] = v;
    const double xi = dropped[g] ? 0.0 : x[g] + (double)v;
    x[g] = xi;
    a_out[g] = scale[g] * xi;
  }
}

// Forward solve of a wide front, its boundary rows: W_k -= L[nS+k][blk] y_blk
// panel by panel, each panel's products summed by the warp tree of
// k_nd_forward, in its order (so the result is the one-CTA solve's).  CTA
// (x, y): rows nS + 32x .. + 31 of front y, four per warp.
__global__ void __launch_bounds__(256) k_ndb_fwd_rect(const NDNode* __restrict__ nodes, const NDBig* __restrict__ bigs,
                                                      const int* __restrict__ sets, const float* __restrict__ F,
                                                      const float* __restrict__ y, float* __restrict__ W,
                                                      const unsigned long long* cstat, const IterCtl* ctl) {
  if (nd_done(ctl) || *(volatile const unsigned long long*)&cstat[2]) return;
  extern __shared__ __align__(16) float ndsm[];  // y_S of the front
  const NDNode nd = nodes[bigs[blockIdx.y].node];
  const int nm = nd.nm, nS = nm * nd.ns, nB = nm * nd.nb, nf = nS + nB;
  const int kbeg = 32 * blockIdx.x;
  if (kbeg >= nB) return;
  const int* st = sets + nd.s_off;
  for (int j = threadIdx.x; j < nS; j += blockDim.x) ndsm[j] = y[nd_glob(st, j, nm)];
  __syncthreads();
  const float* f = F + nd.f_off;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = kbeg + warp; k < nB && k < kbeg + 32; k += 8) {
    const float* row = f + (size_t)(nS + k) * nf;
    float acc = W[nd.w_off + k];
    for (int k0 = 0; k0 < nS; k0 += PB) {
      const int kb = min(PB, nS - k0);
      const float v = lane < kb ? row[k0 + lane] * ndsm[k0 + lane] : 0.f;
      acc -= warp_sum_f(v);
    }
    if (lane == 0) W[nd.w_off + k] = acc;
  }
}

// Back substitution of a wide front, t = y_S - L_BS^T x_B: per column j the
// NDW partial sums over the boundary rows k = w, w + NDW, ... and their
// difference from y in w order, as k_nd_backward forms them; written into y.
// CTA (x, y): columns 32x .. 32x + 31 of front y; warp w forms the partial sum
// w of every column (lane = column), then warp 0 combines them in order.
__global__ void __launch_bounds__(NDT) k_ndb_bwd_rect(const NDNode* __restrict__ nodes, const NDBig* __restrict__ bigs,
                                                      const int* __restrict__ sets, const float* __restrict__ F,
                                                      const float* __restrict__ xc, float* __restrict__ y,
                                                      const unsigned long long* cstat, const IterCtl* ctl) {
  static_assert(NDT == 32 * NDW, "one warp per partial sum");
  if (nd_done(ctl) || *(volatile const unsigned long long*)&cstat[2]) return;
  extern __shared__ __align__(16) float ndsm[];  // x_B of the front
  __shared__ float part[NDW][32];
  const NDNode nd = nodes[bigs[blockIdx.y].node];
  const int nm = nd.nm, nS = nm * nd.ns, nB = nm * nd.nb, nf = nS + nB;
  if (nB == 0 || 32 * (int)blockIdx.x >= nS) return;
  const int* st = sets + nd.s_off;
  for (int k = threadIdx.x; k < nB; k += blockDim.x) ndsm[k] = xc[nd_glob(st, nS + k, nm)];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = 32 * blockIdx.x + lane;
  float acc = 0.f;
  if (j < nS) {
    const float* col = F + nd.f_off + (size_t)nS * nf + j;
#pragma unroll 4
    for (int k = warp; k < nB; k += NDW) acc = fmaf(col[(size_t)k * nf], ndsm[k], acc);
  }
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && j < nS) {
    const int g = nd_glob(st, j, nm);
    float sacc = y[g];
#pragma unroll
    for (int w = 0; w < NDW; ++w) sacc -= part[w][lane];
    y[g] = sacc;
  }
}

}  // namespace

// ---------------------------------------------------------------- host plan
namespace {
struct HNode {
  int x0, y0, w, h;
  std::vector<int> S, B;
  int child[2] = {-1, -1};
  int nchild = 0;
  int height = 0;
};

int nd_build(std::vector<HNode>& out, int Mx, int My, int x0, int y0, int w, int h) {
  HNode nd;
  nd.x0 = x0, nd.y0 = y0, nd.w = w, nd.h = h;
  int kids[2] = {-1, -1}, nk = 0;
  if (w <= 2 && h <= 2) {
    for (int y = y0; y < y0 + h; ++y)
      for (int x = x0; x < x0 + w; ++x) nd.S.push_back(y * Mx + x);
  } else if (w >= h) {
    const int c = x0 + w / 2;
    for (int y = y0; y < y0 + h; ++y) nd.S.push_back(y * Mx + c);
    if (c > x0) kids[nk++] = nd_build(out, Mx, My, x0, y0, c - x0, h);
    if (x0 + w - c - 1 > 0) kids[nk++] = nd_build(out, Mx, My, c + 1, y0, x0 + w - c - 1, h);
  } else {
    const int r = y0 + h / 2;
    for (int x = x0; x < x0 + w; ++x) nd.S.push_back(r * Mx + x);
    if (r > y0) kids[nk++] = nd_build(out, Mx, My, x0, y0, w, r - y0);
    if (y0 + h - r - 1 > 0) kids[nk++] = nd_build(out, Mx, My, x0, r + 1, w, y0 + h - r - 1);
  }
  // the ring of sets around the box, inside the grid (all on ancestor separators)
  for (int y = y0 - 1; y <= y0 + h; ++y)
    for (int x = x0 - 1; x <= x0 + w; ++x) {
      if (x < 0 || y < 0 || x >= Mx || y >= My) continue;
      if (x >= x0 && x < x0 + w && y >= y0 && y < y0 + h) continue;
      nd.B.push_back(y * Mx + x);
    }
  std::sort(nd.B.begin(), nd.B.end());
  nd.nchild = nk;
  for (int k = 0; k < nk; ++k) {
    nd.child[k] = kids[k];
    nd.height = std::max(nd.height, out[kids[k]].height + 1);
  }
  out.push_back(nd);
  return (int)out.size() - 1;
}
}  // namespace

bool nd_plan_build(const LatView& lv, NDPlanHost* P) {
  std::vector<HNode> hn;
  hn.reserve(4 * (size_t)lv.M + 8);
  nd_build(hn, lv.Mx, lv.My, 0, 0, lv.Mx, lv.My);
  const int nn = (int)hn.size();
  int H = 0;
  for (const HNode& h : hn) H = std::max(H, h.height);
  P->nodes.assign(nn, NDNode{});
  P->sets.clear();
  P->maps.clear();
  P->level_begin.assign(H + 2, 0);
  P->lvl_nodes.clear();
  P->f_elems = 0;
  P->w_elems = 0;
  P->max_front = 0;
  P->max_level_nodes = 0;
  // sets of every node, S then B
  for (int k = 0; k < nn; ++k) {
    NDNode& d = P->nodes[k];
    d.ns = (int)hn[k].S.size();
    d.nb = (int)hn[k].B.size();
    d.s_off = (int)P->sets.size();
    P->sets.insert(P->sets.end(), hn[k].S.begin(), hn[k].S.end());
    P->sets.insert(P->sets.end(), hn[k].B.begin(), hn[k].B.end());
    d.nm = lv.q;
    const long long nf = (long long)d.nm * (d.ns + d.nb);
    d.f_off = (long long)P->f_elems;
    P->f_elems += (size_t)(nf * nf);
    d.w_off = (long long)P->w_elems;
    P->w_elems += (size_t)d.nm * d.nb;
    P->max_front = std::max(P->max_front, (int)nf);
    d.nchild = hn[k].nchild;
  }
  // children's boundary sets -> their place in the parent's front
  for (int k = 0; k < nn; ++k) {
    NDNode& d = P->nodes[k];
    const HNode& h = hn[k];
    for (int c = 0; c < h.nchild; ++c) {
      const int ch = h.child[c];
      d.child[c] = ch;
      d.map_off[c] = (int)P->maps.size();
      for (int J : hn[ch].B) {
        int pos = -1;
        for (size_t q = 0; q < h.S.size() && pos < 0; ++q)
          if (h.S[q] == J) pos = (int)q;
        for (size_t q = 0; q < h.B.size() && pos < 0; ++q)
          if (h.B[q] == J) pos = (int)(h.S.size() + q);
        if (pos < 0) return false;  // not reachable for boxes cut by full separators
        P->maps.push_back(pos);
      }
    }
  }
  // nodes by height, leaves first; in a level the one-CTA fronts, then the wide ones
  std::vector<std::vector<int>> byh(H + 1);
  for (int k = 0; k < nn; ++k) byh[hn[k].height].push_back(k);
  P->level_split.assign(H + 1, 0);
  P->big_begin.assign(H + 2, 0);
  P->level_big_ns.assign(H + 1, 0);
  P->level_big_nf.assign(H + 1, 0);
  P->level_big_nb.assign(H + 1, 0);
  P->level_small_nf.assign(H + 1, 0);
  P->bigs.clear();
  P->inv.clear();
  P->max_level_bigs = 0;
  auto nf_of = [&](int k) { return (long long)P->nodes[k].nm * (P->nodes[k].ns + P->nodes[k].nb); };
  for (int h = 0; h <= H; ++h) {
    P->level_begin[h] = (int)P->lvl_nodes.size();
    P->level_small_nf[h] = 0;
    for (int k : byh[h])
      if (nf_of(k) < ND_BIG) {
        P->lvl_nodes.push_back(k);
        P->level_small_nf[h] = std::max(P->level_small_nf[h], (int)nf_of(k));
      }
    P->level_split[h] = (int)P->lvl_nodes.size();
    P->big_begin[h] = (int)P->bigs.size();
    for (int k : byh[h]) {
      if (nf_of(k) < ND_BIG) continue;
      P->lvl_nodes.push_back(k);
      NDBig b{};
      b.node = k;
      // per child: place of each of this front's sets in the child's boundary list
      const HNode& hk = hn[k];
      for (int c = 0; c < hk.nchild; ++c) {
        std::unordered_map<int, int> where;
        const std::vector<int>& cb = hn[hk.child[c]].B;
        for (size_t q = 0; q < cb.size(); ++q) where[cb[q]] = (int)q;
        b.inv_off[c] = (int)P->inv.size();
        for (int J : hk.S) {
          auto it = where.find(J);
          P->inv.push_back(it == where.end() ? -1 : it->second);
        }
        for (int J : hk.B) {
          auto it = where.find(J);
          P->inv.push_back(it == where.end() ? -1 : it->second);
        }
      }
      P->bigs.push_back(b);
      P->level_big_ns[h] = std::max(P->level_big_ns[h], P->nodes[k].nm * P->nodes[k].ns);
      P->level_big_nf[h] = std::max(P->level_big_nf[h], (int)nf_of(k));
      P->level_big_nb[h] = std::max(P->level_big_nb[h], P->nodes[k].nm * P->nodes[k].nb);
    }
    P->max_level_nodes = std::max(P->max_level_nodes, (int)byh[h].size());
    P->max_level_bigs = std::max(P->max_level_bigs, (int)P->bigs.size() - P->big_begin[h]);
  }
  P->level_begin[H + 1] = (int)P->lvl_nodes.size();
  P->big_begin[H + 1] = (int)P->bigs.size();
  P->nlevels = H + 1;
  return true;
}

// Shared memory of the factor launch of a level: per front its packed lower
// triangle where that fits in `cap` floats, else the global path's panel.
static long long nd_factor_need(long long nf, long long cap) {
  const long long packed = nf * (nf + 1) / 2 + 2 * nf;
  return packed <= cap ? packed : nf * (PB + 1) + 2 * nf;
}

bool nd_plan_smem(NDPlanHost* P, int max_smem) {
  // dynamic shared memory of the ND kernels: what the device offers beside
  // their static shared memory (a few KB)
  const long long cap = ((long long)max_smem - 8 * 1024) / (long long)sizeof(float);
  P->level_smem_factor.assign(P->nlevels, 0);
  P->level_smem_solve.assign(P->nlevels, 0);
  for (int h = 0; h < P->nlevels; ++h) {
    long long nfac = 0, nsol = 0;
    for (int k = P->level_begin[h]; k < P->level_begin[h + 1]; ++k) {
      const NDNode& d = P->nodes[P->lvl_nodes[k]];
      const long long nS = (long long)d.nm * d.ns, nf = (long long)d.nm * (d.ns + d.nb);
      // wide fronts are factored by the panel kernels (static shared memory only)
      const long long fneed = k < P->level_split[h] ? nd_factor_need(nf, cap) : 0;
      const long long sneed = nd_solve_need(nS, nf);
      if (fneed > cap || sneed > cap) return false;
      nfac = std::max(nfac, fneed);
      nsol = std::max(nsol, sneed);
    }
    P->level_smem_factor[h] = (size_t)nfac * sizeof(float);
    P->level_smem_solve[h] = (size_t)nsol * sizeof(float);
  }
  return true;
}

cudaError_t launch_nd_factor(cudaStream_t s, const LatView& lv, const NDPlanHost& P, const NDPlanDev& D,
                             const double* blk, const double* scale, int* dropped, const IterCtl* ctl) {
  BlkSrc src;
  src.blk = blk;
  src.scale = scale;
  src.dropped = dropped;
  src.Mx = lv.Mx;
  src.nm = lv.q;
  cudaError_t e;
  for (int h = 0; h < P.nlevels; ++h) {
    const int b = P.level_begin[h], n = P.level_split[h] - b;
    if (n > 0) {
      const size_t smem = P.level_smem_factor[h];
      // levels of many tiny fronts (at most 200 unknowns): 256-thread CTAs, so
      // that several fronts share an SM and one front's serial steps overlap
      // another's (the same arithmetic either way)
      if (P.level_small_nf[h] <= 200)
        k_nd_factor<NDT / 2><<<n, NDT / 2, smem, s>>>(D.nodes, D.lvl_nodes, b, D.sets, D.maps, src, D.F, dropped,
                                                      (long long)(smem / sizeof(float)), ctl);
      else
        k_nd_factor<NDT><<<n, NDT, smem, s>>>(D.nodes, D.lvl_nodes, b, D.sets, D.maps, src, D.F, dropped,
                                              (long long)(smem / sizeof(float)), ctl);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int nb = P.big_begin[h + 1] - P.big_begin[h];
    if (nb <= 0) continue;
    const NDBig* bg = D.bigs + P.big_begin[h];
    const int maxnf = P.level_big_nf[h];
    k_ndb_assemble<<<dim3((maxnf + 31) / 32, nb), 256, 0, s>>>(D.nodes, bg, D.sets, D.inv, src, D.F, ctl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int k0 = 0; k0 < P.level_big_ns[h]; k0 += 2 * PB) {
      k_ndb_diag2<<<nb, 256, 0, s>>>(D.nodes, bg, D.sets, D.F, dropped, D.dmask, k0, ctl);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      // the largest trailing size over the level's fronts that still have pivots
      const long long m = (long long)maxnf - k0 - 1;
      const int rows = (int)((m + 63) / 64);
      const long long T = (m + 63) / 64;
      k_ndb_panel2<<<dim3(std::max(rows, 1), nb), 256, 0, s>>>(D.nodes, bg, D.F, D.dmask, k0, ctl);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      k_ndb_update2<<<dim3((unsigned)std::max(T * (T + 1) / 2, 1LL), nb), 256, 0, s>>>(D.nodes, bg, D.F, k0, ctl);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_nd_solve(cudaStream_t s, int n, const NDPlanHost& P, const NDPlanDev& D, const double* rhs,
                            double* x, const double* scale, double* a_out, const int* dropped,
                            unsigned long long* cstat, int flags, const IterCtl* ctl) {
  k_nd_solve_begin<<<1, 1024, 0, s>>>(n, rhs, dropped, cstat, flags, ctl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int h = 0; h < P.nlevels; ++h) {
    const int b = P.level_begin[h], m = P.level_begin[h + 1] - b;
    if (m <= 0) continue;
    const size_t smem = P.level_smem_solve[h];
    const int msmall = P.level_split[h] - b, mwide = m - msmall;
    if (msmall > 0)
      k_nd_forward<RU_SMALL><<<msmall, NDT, smem, s>>>(D.nodes, D.lvl_nodes, b, D.sets, D.maps, D.F, D.W, rhs, dropped,
                                                      D.y, (long long)(smem / sizeof(float)), cstat, ctl);
    if (mwide > 0)
      k_nd_forward<RU_WIDE><<<mwide, NDT, smem, s>>>(D.nodes, D.lvl_nodes, b + msmall, D.sets, D.maps, D.F, D.W, rhs,
                                                    dropped, D.y, (long long)(smem / sizeof(float)), cstat, ctl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int nb = P.big_begin[h + 1] - P.big_begin[h];
    if (nb > 0 && P.level_big_nb[h] > 0) {
      k_ndb_fwd_rect<<<dim3((P.level_big_nb[h] + 31) / 32, nb), 256, (size_t)P.level_big_ns[h] * sizeof(float), s>>>(
          D.nodes, D.bigs + P.big_begin[h], D.sets, D.F, D.y, D.W, cstat, ctl);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  for (int h = P.nlevels - 1; h >= 0; --h) {
    const int b = P.level_begin[h], m = P.level_begin[h + 1] - b;
    if (m <= 0) continue;
    const int nb = P.big_begin[h + 1] - P.big_begin[h];
    if (nb > 0 && P.level_big_nb[h] > 0) {
      k_ndb_bwd_rect<<<dim3((P.level_big_ns[h] + 31) / 32, nb), NDT, (size_t)P.level_big_nb[h] * sizeof(float), s>>>(
          D.nodes, D.bigs + P.big_begin[h], D.sets, D.F, D.xc, D.y, cstat, ctl);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const size_t smem = P.level_smem_solve[h];
    const int msmall = P.level_split[h] - b, mwide = m - msmall;
    if (msmall > 0)
      k_nd_backward<8><<<msmall, NDT, smem, s>>>(D.nodes, D.lvl_nodes, b, D.sets, D.F, D.y, D.xc, dropped, x, scale,
                                                 a_out, (long long)(smem / sizeof(float)), cstat, ctl);
    if (mwide > 0)
      k_nd_backward<PB><<<mwide, NDT, smem, s>>>(D.nodes, D.lvl_nodes, b + msmall, D.sets, D.F, D.y, D.xc, dropped, x,
                                                 scale, a_out, (long long)(smem / sizeof(float)), cstat, ctl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t configure_coarse_nd(int max_smem) {
  cudaError_t e = set_max_dynamic_smem(k_nd_factor<NDT>, max_smem);
  if (e != cudaSuccess) return e;
  e = set_max_dynamic_smem(k_nd_factor<NDT / 2>, max_smem);
  if (e != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_nd_forward<RU_SMALL>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_nd_forward<RU_WIDE>, max_smem)) != cudaSuccess) return e;
  if ((e = set_max_dynamic_smem(k_nd_backward<8>, max_smem)) != cudaSuccess) return e;
  return set_max_dynamic_smem(k_nd_backward<PB>, max_smem);
}

}  // namespace hms
