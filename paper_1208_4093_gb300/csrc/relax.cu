// K2: displacement-controlled local relaxation of every set (Eqs. 11-13) and
// the upper-level force P = V^T r (Eq. 7).
//
// Eq. 12 fixes the outer displacements at their old values and solves
//   k^Inner u^RD = p^Inner - k^Outer u^Outer-old.
// Subtracting k^Inner u^Inner-old from both sides gives the increment of
// Eq. 13 directly from the global residual:
//   k^Inner (u^RD - u^old) = p^Inner - k^Outer u^Outer-old - k^Inner u^Inner-old = r_I,
// so delta_I = (k^Inner_I)^-1 r_I, all sets from the same u (every set relaxes
// against its neighbours' old displacements).
//
// One CTA per set.  The set's block-bidiagonal factor (setup.cu) is a stream
// of matrices Linv_0, B_1, Linv_1, ..., consumed in order by the forward
// substitution and in reverse order by the back substitution:
//   forward  y_j = Linv_j (r_j - B_j y_{j-1})
//   backward x_j = Linv_j^T (y_j - B_{j+1}^T x_{j+1})
// Each matrix is staged in shared memory by a 1-D bulk copy (cp.async.bulk,
// completion on an mbarrier), double-buffered so the next matrix streams in
// while the current one is applied.  The solve runs in T = double (FP64
// path) or T = float (mixed path, FP32 factor).  While x_j = delta is
// finalised, each thread accumulates its DOF's share of the nine sums of
// P_I = V_I^T r_I in FP64.
#include "hms_internal.cuh"
#include "ptx.cuh"

namespace hms {
namespace {

constexpr int NT = 256, NW = NT / 32;

__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}
__device__ inline float warp_sum_f(float v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}
__device__ inline double wsum(double v) { return warp_sum_d(v); }
__device__ inline float wsum(float v) { return warp_sum_f(v); }

constexpr int NSLOT = 3;  // matrices staged in shared memory (two in flight while one is applied)

struct RelaxSmem {
  size_t slot_elems, ycur_off, z_off, w_off, x_off, part_off, total_elems;
};

template <typename T>
__host__ __device__ inline RelaxSmem relax_layout(int nb) {
  RelaxSmem L;
  long long ls = linv_size(nb), bs = b_size(nb);
  L.slot_elems = (size_t)(ls > bs ? ls : bs);
  const size_t a = 16 / sizeof(T);  // keep every region 16-byte aligned
  auto up = [a](size_t n) { return (n + a - 1) / a * a; };
  L.ycur_off = up(NSLOT * L.slot_elems);
  L.z_off = up(L.ycur_off + nb);
  L.w_off = up(L.z_off + nb);
  L.x_off = up(L.w_off + nb);
  L.part_off = up(L.x_off + nb);
  L.total_elems = up(L.part_off + (size_t)NW * nb);
  return L;
}

template <typename T>
__global__ void __launch_bounds__(NT) k_relax(LatView lv, const long long* __restrict__ set_off,
                                              const T* __restrict__ fac, const double2* __restrict__ r,
                                              T* __restrict__ delta, double* __restrict__ P,
                                              T* __restrict__ yglob, long long ystride, const IterCtl* ctl,
                                              int* err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint64_t bars[NSLOT];
  __shared__ double pred[NW * NMODES];
  __shared__ int abort_flag;
  if (ctl && *(volatile const int*)&ctl->done) return;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int I = blockIdx.x;
  const int Ix = I % lv.Mx, Iy = I / lv.Mx;
  const int i0 = Ix * lv.sx, j0 = Iy * lv.sy;
  const int w = min(lv.sx, lv.nx - i0), h = min(lv.sy, lv.ny - j0);
  const int nb = 2 * w;
  const RelaxSmem LY = relax_layout<T>(nb);
  T* sm = reinterpret_cast<T*>(smraw);
  T* ycur = sm + LY.ycur_off;  // the latest y_j of the forward pass
  T* zbuf = sm + LY.z_off;
  T* wbuf = sm + LY.w_off;
  T* xbuf = sm + LY.x_off;
  T* part = sm + LY.part_off;
  T* yg = yglob + (size_t)I * ystride;  // all y_j, read back by the backward pass
  const T* fset = fac + set_off[I];
  const double* rg = reinterpret_cast<const double*>(r);
  const int nmat = 2 * h - 1;
  const int nops = 2 * nmat;

  auto mat_of_op = [&](int o) { return o < nmat ? o : 2 * nmat - 1 - o; };
  auto issue = [&](int o) {
    const int k = mat_of_op(o);
    uint64_t* bar = &bars[o % NSLOT];
    const uint32_t bytes = (uint32_t)(((k & 1) ? b_size(nb) : linv_size(nb)) * sizeof(T));
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(sm + (size_t)(o % NSLOT) * LY.slot_elems, fset + mat_off(nb, k), bytes, bar);
  };

  if (tid == 0) {
    abort_flag = 0;
    for (int k = 0; k < NSLOT; ++k) mbar_init(&bars[k], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int o = 0; o < NSLOT - 1 && o < nops; ++o) issue(o);
  // z = r_0
  const size_t rowbase0 = 2 * ((size_t)j0 * lv.nx + i0);
  for (int t = tid; t < nb; t += NT) zbuf[t] = (T)rg[rowbase0 + t];

  double pacc[NMODES];
#pragma unroll
  for (int m = 0; m < NMODES; ++m) pacc[m] = 0.0;
  const double2 rep = lv.rep[I];

  for (int o = 0; o < nops; ++o) {
    const int k = mat_of_op(o);
    const bool is_b = (k & 1) != 0;
    const int j = is_b ? (k + 1) / 2 : k / 2;
    if (!mbar_wait_bounded(&bars[o % NSLOT], (uint32_t)((o / NSLOT) & 1))) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    // the slot of op o - 1 is free: stream op o + NSLOT - 1 into it
    if (tid == 0 && o + NSLOT - 1 < nops) issue(o + NSLOT - 1);
    const T* M = sm + (size_t)(o % NSLOT) * LY.slot_elems;
    if (o < nmat) {
      // ---------------- forward: a quad of threads per pair of rows ----------------
      // Rows r and nb-1-r (together nb+1 entries of Linv, about nb+7 of B) go
      // to one quad; its threads take every fourth column, so a row costs two
      // shuffles instead of a warp-wide reduction.
      const T* vin = is_b ? ycur : zbuf;
      const int npair = (nb + 1) / 2;
      const int sub = tid & 3;
      const size_t rowbase = 2 * ((size_t)(j0 + j) * lv.nx + i0);
      for (int base = 0; base < npair; base += NT / 4) {
        const int pq = base + (tid >> 2);
        const bool active = pq < npair;
        const int ra = active ? pq : 0, rb2 = nb - 1 - ra;
        T acc_a = 0, acc_b = 0;
        if (active) {
          {
            const int lo = is_b ? b_lo(ra) : 0, hi = is_b ? nb - 1 : ra;
            const T* row = is_b ? M + b_row_off(nb, ra) - lo : M + linv_row_off(ra);
            for (int c = lo + sub; c <= hi; c += 4) acc_a = fma(row[c], vin[c], acc_a);
          }
          if (rb2 != ra) {
            const int lo = is_b ? b_lo(rb2) : 0, hi = is_b ? nb - 1 : rb2;
            const T* row = is_b ? M + b_row_off(nb, rb2) - lo : M + linv_row_off(rb2);
            for (int c = lo + sub; c <= hi; c += 4) acc_b = fma(row[c], vin[c], acc_b);
          }
        }
        acc_a += __shfl_xor_sync(0xffffffffu, acc_a, 1);
        acc_b += __shfl_xor_sync(0xffffffffu, acc_b, 1);
        acc_a += __shfl_xor_sync(0xffffffffu, acc_a, 2);
        acc_b += __shfl_xor_sync(0xffffffffu, acc_b, 2);
        if (active && sub == 0) {
          if (is_b) {
            zbuf[ra] = (T)rg[rowbase + ra] - acc_a;
            if (rb2 != ra) zbuf[rb2] = (T)rg[rowbase + rb2] - acc_b;
          } else {
            part[ra] = acc_a;  // y_j, copied to ycur below
            if (rb2 != ra) part[rb2] = acc_b;
          }
        }
      }
      __syncthreads();
      if (!is_b) {
        for (int c = tid; c < nb; c += NT) {
          const T v = part[c];
          ycur[c] = v;
          yg[(size_t)j * nb + c] = v;
        }
        __syncthreads();
      }
    } else {
      // ---------------- backward ----------------
      T acc[MAX_NB / 32];
#pragma unroll
      for (int q = 0; q < MAX_NB / 32; ++q) acc[q] = 0;
      if (!is_b) {
        // x_j = Linv_j^T w  (w = y_{h-1} for the last row)
        const T* wv = (j == h - 1) ? ycur : wbuf;
        for (int rr = warp; rr < nb; rr += NW) {
          const T* row = M + linv_row_off(rr);
          const T v = wv[rr];
#pragma unroll
          for (int q = 0; q < MAX_NB / 32; ++q) {
            if (32 * q > rr) break;  // warp-uniform: the rest of the row is beyond the diagonal
            const int c = lane + 32 * q;
            if (c <= rr) acc[q] = fma(row[c], v, acc[q]);
          }
        }
      } else {
        // w = y_{j-1} - B_j^T x_j
        for (int rr = warp; rr < nb; rr += NW) {
          const int lo = b_lo(rr);
          const T* row = M + b_row_off(nb, rr) - lo;
          const T v = xbuf[rr];
#pragma unroll
          for (int q = 0; q < MAX_NB / 32; ++q) {
            if (32 * q >= nb) break;
            if (32 * q + 31 < lo) continue;  // warp-uniform: chunk left of the row's profile
            const int c = lane + 32 * q;
            if (c >= lo && c < nb) acc[q] = fma(row[c], v, acc[q]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < MAX_NB / 32; ++q) {
        const int c = lane + 32 * q;
        if (c < nb) part[warp * nb + c] = acc[q];
      }
      __syncthreads();
      if (!is_b) {
        const size_t node0 = (size_t)(j0 + j) * lv.nx + i0;
        const size_t rowbase = 2 * node0;
        const double eta = lv.L * SQ3_2 * (double)(j0 + j) - rep.y;
        for (int c = tid; c < nb; c += NT) {
          T s = 0;
#pragma unroll
          for (int ww = 0; ww < NW; ++ww) s += part[ww * nb + c];
          xbuf[c] = s;
          delta[rowbase + c] = s;
          // P = V^T r (Eq. 7) for this DOF
          const int il = c >> 1, comp = c & 1;
          const double rv = rg[rowbase + c];
          const double xi = lv.L * ((double)(i0 + il) + 0.5 * (double)((j0 + j) & 1)) - rep.x;
          const double dr = (double)s * rv;
          if (comp == 0) {
            pacc[0] += rv;
            pacc[2] = fma(xi, rv, pacc[2]);
            pacc[3] = fma(eta, rv, pacc[3]);
          } else {
            pacc[1] += rv;
            pacc[4] = fma(xi, rv, pacc[4]);
            pacc[5] = fma(eta, rv, pacc[5]);
          }
          pacc[6] += dr;
          pacc[7] = fma(xi, dr, pacc[7]);
          pacc[8] = fma(eta, dr, pacc[8]);
        }
      } else {
        const T* yp = yg + (size_t)(j - 1) * nb;
        for (int c = tid; c < nb; c += NT) {
          T s = 0;
#pragma unroll
          for (int ww = 0; ww < NW; ++ww) s += part[ww * nb + c];
          wbuf[c] = yp[c] - s;
        }
      }
      __syncthreads();
    }
  }
  if (abort_flag) {
    // let copies still in flight land before the CTA exits
    if (tid == 0) {
      for (int b2 = 0; b2 < NSLOT; ++b2) mbar_wait_bounded(&bars[b2], 0u), mbar_wait_bounded(&bars[b2], 1u);
      atomicOr(err, (int)DEVERR_TIMEOUT);
    }
    return;
  }
  // deterministic block reduction of the nine P sums
#pragma unroll
  for (int m = 0; m < NMODES; ++m) {
    const double v = warp_sum_d(pacc[m]);
    if (lane == 0) pred[warp * NMODES + m] = v;
  }
  __syncthreads();
  if (tid < NMODES) {
    double s = 0.0;
    for (int ww = 0; ww < NW; ++ww) s += pred[ww * NMODES + tid];
    P[(size_t)NMODES * I + tid] = s;
  }
}

}  // namespace

size_t relax_smem_bytes(const LatView& lv, bool fp32) {
  const int w = lv.sx < lv.nx ? lv.sx : lv.nx;
  return fp32 ? relax_layout<float>(2 * w).total_elems * sizeof(float)
              : relax_layout<double>(2 * w).total_elems * sizeof(double);
}

long long relax_y_stride(const LatView& lv) {
  const int w = lv.sx < lv.nx ? lv.sx : lv.nx;
  const int h = lv.sy < lv.ny ? lv.sy : lv.ny;
  return 2LL * w * h;
}

cudaError_t launch_relax(cudaStream_t s, const LatView& lv, const long long* set_off,
                         const double* f64, const float* f32, const double2* r, void* delta,
                         double* P, void* yscratch, const IterCtl* ctl, int* err) {
  const bool fp32 = (f32 != nullptr);
  const size_t smem = relax_smem_bytes(lv, fp32);
  const long long ys = relax_y_stride(lv);
  if (fp32)
    k_relax<float><<<lv.M, NT, smem, s>>>(lv, set_off, f32, r, (float*)delta, P, (float*)yscratch, ys, ctl, err);
  else
    k_relax<double><<<lv.M, NT, smem, s>>>(lv, set_off, f64, r, (double*)delta, P, (double*)yscratch, ys, ctl,
                                           err);
  return cudaGetLastError();
}

cudaError_t configure_relax(int max_smem) {
  cudaError_t e = set_max_dynamic_smem(k_relax<float>, max_smem);
  if (e != cudaSuccess) return e;
  return set_max_dynamic_smem(k_relax<double>, max_smem);
}

}  // namespace hms
