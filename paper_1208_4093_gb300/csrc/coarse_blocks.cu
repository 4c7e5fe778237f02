// K_aa of Eq. 6 stored by blocks of the set grid, for the nested-dissection
// solve of Eq. 8 (coarse_nd.cu): no band, so the upper level's storage and
// every pass over it grow with the number of sets, not with sets x band width.
//
// K_aa couples a set only to its eight neighbours (a bar joins two nodes of
// the same or of adjacent sets).  Per set I the blocks kept are its diagonal
// block and the blocks of its four "later" neighbours J > I (row-major set
// order): E (I+1), NW (I+Mx-1), N (I+Mx), NE (I+Mx+1); block b holds K_aa[J
// modes][I modes].  The other four neighbours' blocks are their transposes,
// kept by those neighbours.  Every entry is summed from the slots of
// coarse_assemble.cu in the order the band assembly uses, so it has the same
// value as the band entry.
//
// On top of the blocks:
//   k_blk_diag      Jacobi scaling, right-hand side and the modes that take no
//                   part (mode mask, vanishing diagonal, the per-set FP64 drop
//                   rule), with the same arithmetic as the band path;
//   k_blk_residual  the FP64 refinement residual res = b - A x of the scaled
//                   system (Eq. 8), one thread per unknown over its nine
//                   neighbour sets;
// and the dense conversions of the step entry points.
#include "hms_internal.cuh"

namespace hms {
namespace {

__device__ inline bool done_(const IterCtl* ctl) { return ctl && *(volatile const int*)&ctl->done; }

__device__ inline double slot_val(const double* base, const double* it, int nm, int I, int slot, int p, int c) {
  const size_t o = ((size_t)I * NSLOTS + slot) * slot_size(nm) + (size_t)p * slot_dim(nm) + c;
  return base[o] + it[o];
}

// entry (J mode l, I mode m) of K_aa, J the neighbour b of I (b = 0: J = I);
// 0 if J lies outside the set grid
__device__ inline double blk_entry(const LatView& lv, const double* base, const double* it, int I, int b, int l,
                                   int m) {
  const int nm = lv.q;
  const int Ix = I % lv.Mx, Iy = I / lv.Mx;
  if (b == BLK_SELF) {
    double v = slot_val(base, it, nm, I, SLOT_SELF, l, m);
    for (int s = SLOT_E; s < NSLOTS; ++s) v += slot_val(base, it, nm, I, s, l, m);
    // neighbours that own bars into I
    const int kx[5] = {-1, 1, 0, -1, 1};  // owner offset for E, W, N, NE, NW
    const int ky[5] = {0, 0, -1, -1, -1};
    for (int s = 0; s < 5; ++s) {
      const int Kx = Ix + kx[s], Ky = Iy + ky[s];
      if (Kx < 0 || Kx >= lv.Mx || Ky < 0 || Ky >= lv.My) continue;
      v += slot_val(base, it, nm, Ky * lv.Mx + Kx, SLOT_E + s, nm + l, nm + m);
    }
    return v;
  }
  const int dx = blk_dx(b), dy = blk_dy(b);
  const int Jx = Ix + dx, Jy = Iy + dy;
  if (Jx < 0 || Jx >= lv.Mx || Jy >= lv.My) return 0.0;
  const int J = Jy * lv.Mx + Jx;
  if (b == BLK_E) return slot_val(base, it, nm, I, SLOT_E, nm + l, m) + slot_val(base, it, nm, J, SLOT_W, l, nm + m);
  if (b == BLK_N) return slot_val(base, it, nm, I, SLOT_N, nm + l, m);
  if (b == BLK_NE) return slot_val(base, it, nm, I, SLOT_NE, nm + l, m);
  return slot_val(base, it, nm, I, SLOT_NW, nm + l, m);
}

__global__ void k_blocks_from_slots(LatView lv, const double* __restrict__ base, const double* __restrict__ it,
                                    double* __restrict__ blk, const IterCtl* ctl) {
  if (done_(ctl)) return;
  const int nm = lv.q, bs = nm * nm;
  const size_t total = (size_t)lv.M * NBLK * bs;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int I = (int)(e / ((size_t)NBLK * bs));
    const int r = (int)(e % ((size_t)NBLK * bs));
    const int b = r / bs, l = (r % bs) / nm, m = r % nm;
    blk[e] = blk_entry(lv, base, it, I, b, l, m);
  }
}

// Per set: scale s_i = D_ii^-1/2, b = s P, x = 0 and the modes that take no
// part -- left out by the mode mask, D_ii <= 1e-300 or <= 1e-28 times the
// largest kept diagonal of the set, or a pivot <= 1e-14 in the FP64 Cholesky
// of the scaled diagonal block in mode order (the rules of the band path,
// k_coarse_diag and k_coarse_set_drops, on the same values).
template <int Q>
__global__ void k_blk_diag(int nsets, const double* __restrict__ blk, const double* __restrict__ P,
                           double* __restrict__ scale, double* __restrict__ b, double* __restrict__ x,
                           int* __restrict__ dropped, unsigned mode_mask, const IterCtl* ctl) {
  if (done_(ctl)) return;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nsets) return;
  const double* S = blk + (size_t)I * NBLK * Q * Q;  // diagonal block [l][m]
  double sc[Q];
  bool dr[Q];
  double dmax = 0.0;
#pragma unroll
  for (int m = 0; m < Q; ++m)
    if ((mode_mask >> m) & 1u) dmax = fmax(dmax, S[m * Q + m]);
#pragma unroll
  for (int m = 0; m < Q; ++m) {
    const double D = S[m * Q + m];
    dr[m] = !((mode_mask >> m) & 1u) || !(D > 1e-300) || !(D > 1e-28 * dmax);
    sc[m] = dr[m] ? 0.0 : 1.0 / sqrt(D);
  }
  double A[Q][Q];
#pragma unroll
  for (int m = 0; m < Q; ++m)
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const int lo = l < m ? l : m, hi = l < m ? m : l;
      A[m][l] = sc[m] * S[hi * Q + lo] * sc[l];
    }
#pragma unroll
  for (int m = 0; m < Q; ++m) {
    if (dr[m]) continue;
    double piv = A[m][m];
#pragma unroll
    for (int k = 0; k < m; ++k) piv -= A[m][k] * A[m][k];
    if (!(piv > 1e-14)) {
      dr[m] = true;
#pragma unroll
      for (int l = m + 1; l < Q; ++l) A[l][m] = 0.0;
      continue;
    }
    const double d = sqrt(piv);
    A[m][m] = d;
#pragma unroll
    for (int l = m + 1; l < Q; ++l) {
      if (dr[l]) continue;
      double v = A[l][m];
#pragma unroll
      for (int k = 0; k < m; ++k) v -= A[l][k] * A[m][k];
      A[l][m] = v / d;
    }
  }
#pragma unroll
  for (int m = 0; m < Q; ++m) {
    const int i = Q * I + m;
    scale[i] = sc[m];
    b[i] = dr[m] ? 0.0 : sc[m] * P[i];
    x[i] = 0.0;
    dropped[i] = dr[m] ? 1 : 0;
  }
}

// res = b - A x of the scaled system, A_ij = s_i K_ij s_j (s of the larger
// index first, as the band path rounds it), A_ii = 1, rows and columns of
// dropped modes zero; max |res| into cstat[1].  Skipped once refinement has
// converged (cstat[2]).
__global__ void __launch_bounds__(256) k_blk_residual(LatView lv, const double* __restrict__ blk,
                                                      const double* __restrict__ scale,
                                                      const int* __restrict__ dropped, const double* __restrict__ bv,
                                                      const double* __restrict__ x, double* __restrict__ res,
                                                      unsigned long long* cstat, const IterCtl* ctl) {
  if (done_(ctl)) return;
  if (*(volatile unsigned long long*)&cstat[2]) return;
  const int nm = lv.q, n = nm * lv.M;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double rv = 0.0;
  if (i < n && !dropped[i]) {
    const int I = i / nm, l = i % nm;
    const int Ix = I % lv.Mx, Iy = I / lv.Mx;
    const size_t bs = (size_t)nm * nm;
    double acc = 0.0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int Jx = Ix + dx, Jy = Iy + dy;
        if (Jx < 0 || Jx >= lv.Mx || Jy < 0 || Jy >= lv.My) continue;
        const int J = Jy * lv.Mx + Jx;
        for (int m = 0; m < nm; ++m) {
          const int j = nm * J + m;
          if (dropped[j]) continue;
          double a;
          if (j == i) {
            a = 1.0;
          } else {
            // K_ij from the block kept by the earlier of the two sets
            double k;
            if (J == I) {
              k = blk[(size_t)I * NBLK * bs + (size_t)(l > m ? l : m) * nm + (l > m ? m : l)];
            } else if (J > I) {
              k = blk[((size_t)I * NBLK + blk_of(dx, dy)) * bs + (size_t)m * nm + l];
            } else {
              k = blk[((size_t)J * NBLK + blk_of(-dx, -dy)) * bs + (size_t)l * nm + m];
            }
            a = i > j ? scale[i] * k * scale[j] : scale[j] * k * scale[i];
          }
          acc = fma(a, x[j], acc);
        }
      }
    rv = bv[i] - acc;
    res[i] = rv;
  } else if (i < n) {
    res[i] = 0.0;
  }
  // max |res|: warp maximum, one atomic per warp (order of non-negative doubles' bit patterns)
  double am = fabs(rv);
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) am = fmax(am, __shfl_xor_sync(0xffffffffu, am, s));
  if ((threadIdx.x & 31) == 0) atomicMax(&cstat[1], (unsigned long long)__double_as_longlong(am));
}

__global__ void k_blocks_from_dense(LatView lv, const double* __restrict__ dense, double* __restrict__ blk) {
  const int nm = lv.q, bs = nm * nm, n = nm * lv.M;
  const size_t total = (size_t)lv.M * NBLK * bs;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int I = (int)(e / ((size_t)NBLK * bs));
    const int r = (int)(e % ((size_t)NBLK * bs));
    const int b = r / bs, l = (r % bs) / nm, m = r % nm;
    const int Jx = I % lv.Mx + blk_dx(b), Jy = I / lv.Mx + blk_dy(b);
    double v = 0.0;
    if (Jx >= 0 && Jx < lv.Mx && Jy < lv.My) {
      const int J = Jy * lv.Mx + Jx;
      v = dense[(size_t)(nm * J + l) * n + nm * I + m];
    }
    blk[e] = v;
  }
}

__global__ void k_dense_from_blocks(LatView lv, const double* __restrict__ blk, double* __restrict__ dense) {
  const int nm = lv.q, n = nm * lv.M;
  const size_t bs = (size_t)nm * nm;
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    if (i < j) {
      const int t = i;
      i = j;
      j = t;
    }
    const int I = j / nm, m = j % nm, J = i / nm, l = i % nm;  // J >= I
    const int dx = J % lv.Mx - I % lv.Mx, dy = J / lv.Mx - I / lv.Mx;
    double v = 0.0;
    if (J == I) v = blk[(size_t)I * NBLK * bs + (size_t)l * nm + m];
    else if (dy >= 0 && dy <= 1 && dx >= -1 && dx <= 1 && blk_of(dx, dy) > 0)
      v = blk[((size_t)I * NBLK + blk_of(dx, dy)) * bs + (size_t)l * nm + m];
    dense[e] = v;
  }
}

int grid_for_(size_t total) {
  size_t g = (total + 255) / 256;
  if (g > 8192) g = 8192;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

size_t coarse_blocks_elems(const LatView& lv) { return (size_t)lv.M * NBLK * lv.q * lv.q; }

cudaError_t launch_blocks_from_slots(cudaStream_t s, const LatView& lv, const double* base, const double* slots,
                                     double* blk, const IterCtl* ctl) {
  k_blocks_from_slots<<<grid_for_(coarse_blocks_elems(lv)), 256, 0, s>>>(lv, base, slots, blk, ctl);
  return cudaGetLastError();
}

cudaError_t launch_blk_diag(cudaStream_t s, const LatView& lv, const double* blk, const double* P, double* scale,
                            double* b, double* x, int* dropped, unsigned mode_mask, const IterCtl* ctl) {
  const int g = (lv.M + 127) / 128;
  if (lv.q == NMODES_RF) k_blk_diag<NMODES_RF><<<g, 128, 0, s>>>(lv.M, blk, P, scale, b, x, dropped, mode_mask, ctl);
  else k_blk_diag<NMODES><<<g, 128, 0, s>>>(lv.M, blk, P, scale, b, x, dropped, mode_mask, ctl);
  return cudaGetLastError();
}

cudaError_t launch_blk_residual(cudaStream_t s, const LatView& lv, const double* blk, const double* scale,
                                const int* dropped, const double* b, const double* x, double* res,
                                unsigned long long* cstat, const IterCtl* ctl) {
  const int n = lv.q * lv.M;
  k_blk_residual<<<(n + 255) / 256, 256, 0, s>>>(lv, blk, scale, dropped, b, x, res, cstat, ctl);
  return cudaGetLastError();
}

cudaError_t launch_blocks_from_dense(cudaStream_t s, const LatView& lv, const double* dense, double* blk) {
  k_blocks_from_dense<<<grid_for_(coarse_blocks_elems(lv)), 256, 0, s>>>(lv, dense, blk);
  return cudaGetLastError();
}

cudaError_t launch_dense_from_blocks(cudaStream_t s, const LatView& lv, const double* blk, double* dense) {
  const size_t n = (size_t)lv.q * lv.M;
  k_dense_from_blocks<<<grid_for_(n * n), 256, 0, s>>>(lv, blk, dense);
  return cudaGetLastError();
}

}  // namespace hms
