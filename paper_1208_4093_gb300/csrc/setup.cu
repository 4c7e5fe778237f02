// K2f: factor every set's k^Inner once (end of Sec. 2.2: the local matrices of
// Eq. 12 do not change during the iteration, so they are factored in the
// first iteration and the factors are reused).
//
// k^Inner_I is K restricted to the free DOFs of set I's relaxation region
// (the set, or its tile grown by lv.ov nodes: Sec. 2.2's extended region; Eq.
// 11: its entries are those of the global matrix).  Constrained DOFs are kept as identity
// rows/columns so that every set row has the same layout; their right-hand
// side is always 0, which leaves the free-DOF solution unchanged.
//
// Ordered row by row of the set (DOF 2*il + c of lattice row jj), k^Inner is
// block tridiagonal with one block row per lattice row (nb = 2w DOFs), so its
// Cholesky factor is block bidiagonal: L_jj (dense lower) and
// B_j = L_{j,j-1}, whose row r is zero left of column r - 3 (the band of
// k^Inner reaches 2w + 3 DOFs back).  Stored per set: Linv_j = L_jj^-1 and
// B_j, so the solves of relax.cu are matrix-vector products only, and a
// second copy of both stored by columns for the back substitution.
//
// One CTA per set (grid-stride over sets), FP64 throughout; the FP32 copy for
// the mixed path is rounded from the FP64 factor.
//
// CUT = true factors k^Inner + Delta k of Eq. 15 instead: Delta k adds to each
// inner node's diagonal block the blocks k_il of the bars to nodes l outside
// the set, which cancels their stiffness, so the matrix is that of the set's
// own bars (the set cut free).  The diagonal blocks then sum only the bars whose
// other end lies in the region; the couplings are inner bars already.  A set
// clear of the supports floats (rigid motions); the caller marks as
// constrained, besides the supports, as many DOFs as the set has free rigid
// motions ("pinned", chosen so that no rigid motion vanishes on them), which
// makes the matrix nonsingular (see force.cu for the use of its solution).
#include "hms_internal.cuh"

namespace hms {
namespace {

constexpr int NT = 256;
constexpr double SQ3_4 = 0.43301270189221932338;  // sqrt(3)/4

__device__ inline long long pk(int r, int c) { return (long long)r * (r + 1) / 2 + c; }

// 2x2 diagonal block of K at node (i, j): sum over its six bars of (EA/L) e e^T
// (CUT: only the bars whose other end lies in the region R).
template <bool CUT>
__device__ inline void node_diag(const LatView& lv, int i, int j, const Region& R, double& dxx, double& dxy,
                                 double& dyy) {
  const int off = j & 1;
  auto in = [&](int ii, int jj) {
    return !CUT || (ii >= R.i0 && ii < R.i0 + R.w && jj >= R.j0 && jj < R.j0 + R.h);
  };
  const double kE = in(i + 1, j) ? bar_k(lv, i, j, 0) : 0.0;
  const double kW = in(i - 1, j) ? bar_k(lv, i - 1, j, 0) : 0.0;
  const double kNE = in(i + off, j + 1) ? bar_k(lv, i, j, 1) : 0.0;
  const double kSW = in(i - 1 + off, j - 1) ? bar_k(lv, i - 1 + off, j - 1, 1) : 0.0;
  const double kNW = in(i - 1 + off, j + 1) ? bar_k(lv, i, j, 2) : 0.0;
  const double kSE = in(i + off, j - 1) ? bar_k(lv, i + off, j - 1, 2) : 0.0;
  const double sne = kNE + kSW, snw = kNW + kSE;
  dxx = kE + kW + 0.25 * (sne + snw);
  dxy = SQ3_4 * (sne - snw);
  dyy = 0.75 * (sne + snw);
}

template <bool CUT>
__global__ void __launch_bounds__(NT) k_set_factor(LatView lv, const long long* __restrict__ set_off,
                                                   double* __restrict__ f64, float* __restrict__ f32,
                                                   double* __restrict__ scratch, int* err,
                                                   const int* __restrict__ list, int nlist) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* Bprev = scratch + (size_t)blockIdx.x * b_size(MAX_NB);
  __shared__ int bad;
  __shared__ double diag0[MAX_NB];

  // every set, or the sets list[0 .. nlist) (factor t at set_off[t])
  const int nwork = list ? nlist : lv.M;
  for (int t = blockIdx.x; t < nwork; t += gridDim.x) {
    const int I = list ? list[t] : t;
    // the set's relaxation region (the set itself without overlap)
    const Region R = relax_region(lv, I);
    const int i0 = R.i0, j0 = R.j0, w = R.w, h = R.h;
    const int nb = 2 * w;
    const long long npk = pk(nb - 1, nb - 1) + 1;
    double* S = sm;          // packed lower nb x nb
    double* Li = sm + npk;   // packed lower nb x nb
    const long long base = set_off[t];
    const long long tr_base = set_factor_size(nb, h);  // the column-stored copy
    if (tid == 0) bad = 0;

    for (int jj = 0; jj < h; ++jj) {
      const int j = j0 + jj;
      // 1. S = K_jj
      for (long long q = tid; q < npk; q += NT) S[q] = 0.0;
      __syncthreads();
      for (int il = tid; il < w; il += NT) {
        const int i = i0 + il;
        double dxx, dxy, dyy;
        node_diag<CUT>(lv, i, j, R, dxx, dxy, dyy);
        S[pk(2 * il, 2 * il)] = dxx;
        S[pk(2 * il + 1, 2 * il)] = dxy;
        S[pk(2 * il + 1, 2 * il + 1)] = dyy;
        if (il + 1 < w) S[pk(2 * il + 2, 2 * il)] = -bar_k(lv, i, j, 0);  // E bar, xx only
      }
      __syncthreads();
      // constrained DOFs: identity row / column
      for (int il = tid; il < w; il += NT) {
        const unsigned fm = lv.fix[(size_t)j * lv.nx + i0 + il];
        for (int c = 0; c < 2; ++c) {
          if (!(fm & (1u << c))) continue;
          const int d = 2 * il + c;
          for (int k = 0; k < d; ++k) S[pk(d, k)] = 0.0;
          for (int k = d + 1; k < nb; ++k) S[pk(k, d)] = 0.0;
          S[pk(d, d)] = 1.0;
        }
      }
      __syncthreads();
      for (int k = tid; k < nb; k += NT) diag0[k] = S[pk(k, k)];
      __syncthreads();
      // 2. Schur update S -= B_j B_j^T  (B_j = L_{j,j-1} from the previous row)
      if (jj > 0) {
        for (int r = warp; r < nb; r += NT / 32) {
          const int lo = b_lo(r);
          const double* br = Bprev + b_row_off(nb, r) - lo;
          for (int c = lane; c <= r; c += 32) {
            const double* bc = Bprev + b_row_off(nb, c) - b_lo(c);
            double acc = 0.0;
            for (int k = lo; k < nb; ++k) acc = fma(br[k], bc[k], acc);
            S[pk(r, c)] -= acc;
          }
        }
        __syncthreads();
      }
      // 3. Cholesky of S in place; a pivot below 1e-12 of the DOF's own
      //    stiffness K_kk means k^Inner is singular to working precision
      for (int k = 0; k < nb; ++k) {
        if (tid == 0) {
          double piv = S[pk(k, k)];
          if (!(piv > 1e-12 * diag0[k])) {
            bad = 1;
            piv = 1.0;
          }
          S[pk(k, k)] = sqrt(piv);
        }
        __syncthreads();
        const double dk = S[pk(k, k)];
        for (int i = k + 1 + tid; i < nb; i += NT) S[pk(i, k)] /= dk;
        __syncthreads();
        for (int i = k + 1 + warp; i < nb; i += NT / 32) {
          const double lik = S[pk(i, k)];
          for (int l = k + 1 + lane; l <= i; l += 32) S[pk(i, l)] = fma(-lik, S[pk(l, k)], S[pk(i, l)]);
        }
        __syncthreads();
      }
      // 4. Li = S^-1 (lower triangular), one column per thread
      for (int c = tid; c < nb; c += NT) {
        for (int r = c; r < nb; ++r) {
          double acc = (r == c) ? 1.0 : 0.0;
          for (int k = c; k < r; ++k) acc = fma(-S[pk(r, k)], Li[pk(k, c)], acc);
          Li[pk(r, c)] = acc / S[pk(r, r)];
        }
      }
      __syncthreads();
      // 5. store Linv_j, and Linv_j^T by rows (= Linv_j by columns)
      {
        const long long o = base + mat_off(nb, 2 * jj);
        for (long long q = tid; q < npk; q += NT) {
          if (f64) f64[o + q] = Li[q];
          if (f32) f32[o + q] = (float)Li[q];
        }
        const long long ot = base + tr_base + mat_off(nb, 2 * jj);
        for (int c = warp; c < nb; c += NT / 32)
          for (int r = c + lane; r < nb; r += 32) {
            const long long q = ot + lt_row_off(nb, c) + (r - c);
            const double v = Li[pk(r, c)];
            if (f64) f64[q] = v;
            if (f32) f32[q] = (float)v;
          }
      }
      // 6. B_{j+1} = K_{j+1,j} Linv_j^T
      if (jj + 1 < h) {
        const int ja = j + 1, offa = ja & 1;
        const long long o = base + mat_off(nb, 2 * jj + 1);
        const long long ot = base + tr_base + mat_off(nb, 2 * jj + 1);
        for (int r = warp; r < nb; r += NT / 32)
          for (int c = b_lo(r) + lane; c < nb; c += 32) {
          const long long q = b_row_off(nb, r) + (c - b_lo(r));
          const int il = r >> 1, comp = r & 1;
          const int ia = i0 + il;
          const unsigned fma_ = lv.fix[(size_t)ja * lv.nx + ia];
          double acc = 0.0;
          if (!(fma_ & (1u << comp))) {
            // SW neighbour via its NE bar, SE neighbour via its NW bar
            for (int nbi = 0; nbi < 2; ++nbi) {
              const int ilb = (nbi == 0) ? il - 1 + offa : il + offa;
              if (ilb < 0 || ilb >= w) continue;
              const int ib = i0 + ilb;
              const double kb = (nbi == 0) ? bar_k(lv, ib, j, 1) : bar_k(lv, ib, j, 2);
              const double ex = (nbi == 0) ? 0.5 : -0.5;
              const unsigned fmb = lv.fix[(size_t)j * lv.nx + ib];
              for (int cb = 0; cb < 2; ++cb) {
                const int kcol = 2 * ilb + cb;
                if (kcol > c || (fmb & (1u << cb))) continue;
                const double ea = comp ? SQ3_2 : ex, eb = cb ? SQ3_2 : ex;
                acc = fma(-kb * ea * eb, Li[pk(c, kcol)], acc);
              }
            }
          }
          Bprev[q] = acc;
          if (f64) f64[o + q] = acc, f64[ot + bt_row_off(nb, c) + r] = acc;
          if (f32) f32[o + q] = (float)acc, f32[ot + bt_row_off(nb, c) + r] = (float)acc;
        }
      }
      __syncthreads();
    }
    if (tid == 0 && bad) atomicOr(err, (int)DEVERR_NOT_SPD);
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_set_factor(cudaStream_t s, const LatView& lv, const long long* set_off,
                              double* f64, float* f32, double* scratch, int grid, int* err, bool cut,
                              const int* list, int nlist) {
  const int nb = 2 * region_w_max(lv);
  const size_t smem = 2 * (size_t)((long long)nb * (nb + 1) / 2) * sizeof(double);
  if (cut) k_set_factor<true><<<grid, NT, smem, s>>>(lv, set_off, f64, f32, scratch, err, list, nlist);
  else k_set_factor<false><<<grid, NT, smem, s>>>(lv, set_off, f64, f32, scratch, err, list, nlist);
  return cudaGetLastError();
}

cudaError_t configure_setup(int max_smem) {
  cudaError_t e = set_max_dynamic_smem(k_set_factor<false>, max_smem);
  if (e != cudaSuccess) return e;
  return set_max_dynamic_smem(k_set_factor<true>, max_smem);
}

}  // namespace hms
