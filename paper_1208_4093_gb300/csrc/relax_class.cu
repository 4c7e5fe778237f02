// K2 with factors shared by classes of identical sets: the displacement-
// controlled relaxation of Eqs. 11-13 and the forces P = V^T r of Eq. 7 for
// lattices too large to hold one factor per set.
//
// With a uniform bar stiffness, k^Inner of a set depends only on its width and
// height, the parity of its first row (the row offset of the triangle
// lattice), which lattice edges it touches (bars to nodes outside the lattice
// are absent) and its constrained DOFs.  Sets that agree in all of these have
// the same k^Inner, so one factor (setup.cu, factored for the class's first
// set) serves the whole class, and the solves of many sets become products of
// one matrix with many right-hand sides:
//   forward  Y_j = Linv_j (R_j - B_j Y_{j-1}),
//   backward X_j = Linv_j^T (Y_j - B_{j+1}^T X_{j+1}),
// with the columns of R_j, Y_j, X_j the sets of a batch (TS = 32 or 64 sets
// per CTA).  Each matrix is applied in 8-row groups: the factor is stored
// again for this kernel ("grouped": per group of 8 output rows, the columns
// the group's rows reach, 8 values per column, zero where a row does not
// reach), so that one column step of a group is 8 broadcast loads of the
// matrix, one load of the sets' vector entries and 8 x SPL FMAs per thread.
// Warp w takes groups w and NG-1-w (NG = nb/8 groups), so that every warp
// runs about the same number of column steps for each of the four kinds of
// matrix (triangles and band blocks); lane l takes sets l*SPL .. l*SPL+SPL-1.
// The matrices stream through shared memory by 1-D bulk copies issued by one
// more warp, NS slots deep, as in relax.cu; the vectors Y_j of the forward
// pass go to a scratch buffer for the backward pass (each thread reads back
// what it wrote).  Every sum runs in a fixed order, so the results are the
// same on every run; they differ from the per-set kernel's (relax.cu) only by
// rounding, the order of the sums being another.
//
// The sums of P_I = V_I^T r_I are formed in FP64 in the backward pass, as each
// row of delta is produced: per thread over its nodes of the row (xi of a node
// is the row's xi0 plus L times its column, eta is the row's), then over the
// rows, then over the warps in order.
#include <type_traits>

#include "hms_internal.cuh"
#include "ptx.cuh"

namespace hms {
namespace {

constexpr int NTC = 256;  // compute threads: 8 warps (one more warp issues the copies)

__device__ inline void ld8(const float* p, float (&m)[8]) {
  const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
  m[0] = a.x, m[1] = a.y, m[2] = a.z, m[3] = a.w, m[4] = b.x, m[5] = b.y, m[6] = b.z, m[7] = b.w;
}
__device__ inline void ld8(const double* p, double (&m)[8]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double2 a = reinterpret_cast<const double2*>(p)[q];
    m[2 * q] = a.x, m[2 * q + 1] = a.y;
  }
}
template <typename T, int SPL>
__device__ inline void ldv(const T* p, T (&v)[SPL]) {
  if constexpr (SPL == 1) {
    v[0] = *p;
  } else {
    static_assert(SPL == 2, "one or two sets per lane");
    using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
    const T2 a = *reinterpret_cast<const T2*>(p);
    v[0] = a.x, v[1] = a.y;
  }
}
template <typename T, int SPL>
__device__ inline void stv(T* p, const T (&v)[SPL]) {
  if constexpr (SPL == 1) {
    *p = v[0];
  } else {
    using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
    T2 a;
    a.x = v[0], a.y = v[1];
    *reinterpret_cast<T2*>(p) = a;
  }
}

// kind and block row of op o of a class of nb-DOF rows and h rows (forward ops
// 0 .. 2h-2: Linv_0, B_1, Linv_1, ..., Linv_{h-1}; backward ops: Linv_{h-1}^T,
// B_{h-1}^T, ..., B_1^T, Linv_0^T)
__device__ inline void op_kind(int h, int o, int& kind, int& j) {
  const int nm = 2 * h - 1;
  if (o < nm) {
    kind = (o & 1) ? GK_B : GK_LINV;
    j = (o & 1) ? (o + 1) / 2 : o / 2;
  } else {
    const int k = o - nm;
    kind = (k & 1) ? GK_BT : GK_LT;
    j = (k & 1) ? h - (k + 1) / 2 : h - 1 - k / 2;
  }
}

// Shared-memory regions: NS matrix slots and two vector panels [nb8max][TS]
// (elements of T), then the P partial sums [8 warps][TS][9] (doubles; each
// thread adds only to its own warp's entries of its own sets)
struct ClassSmem {
  size_t pan0, pan1, red_bytes_off, total_bytes;
};
template <typename T, int SPL, int NS>
__host__ __device__ inline ClassSmem class_layout(size_t slot_elems, int nb8max) {
  constexpr int TS = 32 * SPL;
  ClassSmem L;
  L.pan0 = NS * slot_elems;
  L.pan1 = L.pan0 + (size_t)nb8max * TS;
  const size_t pan_bytes = 2 * (size_t)nb8max * TS * sizeof(T);
  const size_t red_bytes = (size_t)(NTC / 32) * TS * NMODES * sizeof(double);
  L.red_bytes_off = (L.pan0 * sizeof(T) + pan_bytes + 15) / 16 * 16;
  L.total_bytes = L.red_bytes_off + red_bytes;
  return L;
}

template <typename T, int SPL, int NS>
__global__ void __launch_bounds__(NTC + 32, 1) k_relax_class(LatView lv, ClassPlanDev cp, const T* __restrict__ fac,
                                                         const double2* __restrict__ r, T* __restrict__ delta,
                                                         double* __restrict__ P, T* __restrict__ yglob,
                                                         const IterCtl* ctl, int* err, int wait0) {
  constexpr int TS = 32 * SPL;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint64_t bars[NS];
  __shared__ int abort_flag;
  if (ctl && *(volatile const int*)&ctl->done) return;

  using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
  const ClassItem it = cp.items[blockIdx.x];
  const ClassInfo ci = cp.info[it.cls];
  const int w = ci.w, h = ci.h, nb = 2 * w, NG = (nb + 7) / 8;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool producer = tid >= NTC;
  const ClassSmem LY = class_layout<T, SPL, NS>(cp.slot_elems, cp.nb8max);
  T* sm = reinterpret_cast<T*>(smraw);
  T* const pan0 = sm + LY.pan0;
  T* const pan1 = sm + LY.pan1;
  T* ybase = yglob + (size_t)blockIdx.x * cp.ystride;  // Y_j of this batch: [h][nb8max][TS]
  const size_t yrow = (size_t)cp.nb8max * TS;
  const T* fcls = fac + ci.off;

  // this warp's groups: w and NG-1-w while w < NG-1-w, the middle group alone
  // when they coincide, none above (those groups are a lower warp's)
  const int gA = warp, gB = NG - 1 - warp;
  const int ngrp = producer ? 0 : (gA < gB ? 2 : (gA == gB ? 1 : 0));
  // this lane's sets
  size_t nbase[SPL];
  bool valid[SPL];
  int j0p[SPL];
  double xoff[SPL], repx[SPL], repy[SPL];
#pragma unroll
  for (int s = 0; s < SPL; ++s) {
    const int ls = lane * SPL + s;
    valid[s] = ls < it.count;
    const int I = cp.sets[it.first + (valid[s] ? ls : 0)];
    const int i0 = (I % lv.Mx) * lv.sx, j0 = (I / lv.Mx) * lv.sy;
    nbase[s] = (size_t)j0 * lv.nx + i0;
    j0p[s] = j0;
    xoff[s] = (double)i0;
    const double2 rp = lv.rep[I];
    repx[s] = rp.x, repy[s] = rp.y;
  }

  const int nmat = 2 * h - 1, nops = 2 * nmat;
  int issued = 0;
  auto issue = [&](int o) {
    ++issued;
    int kind, j;
    op_kind(h, o, kind, j);
    const uint32_t bytes = (uint32_t)(grp_size(kind, nb) * sizeof(T));
    uint64_t* bar = &bars[o % NS];
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(sm + (size_t)(o % NS) * cp.slot_elems, fcls + class_op_off(nb, h, o), bytes, bar);
  };

  if (tid == 0) {
    abort_flag = 0;
    for (int k = 0; k < NS; ++k) mbar_init(&bars[k], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == NTC)
    for (int o = 0; o < NS - 1 && o < nops; ++o) issue(o);

  // r rows 8g .. 8g+7 of block row j (nodes 4g .. 4g+3 of lattice row j0 + j) of every set of this lane
  auto fetch_r = [&](int g, int j, double2 (&rv)[4][SPL]) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int il = 4 * g + t;
#pragma unroll
      for (int s = 0; s < SPL; ++s)
        rv[t][s] = (valid[s] && il < w) ? r[nbase[s] + (size_t)j * lv.nx + il] : make_double2(0.0, 0.0);
    }
  };

  // z = r_0 in panel 0 (each warp its own rows)
  for (int q = 0; q < ngrp; ++q) {
    const int g = q == 0 ? gA : gB;
    double2 rv[4][SPL];
    fetch_r(g, 0, rv);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      T a[SPL], b[SPL];
#pragma unroll
      for (int s = 0; s < SPL; ++s) a[s] = (T)rv[t][s].x, b[s] = (T)rv[t][s].y;
      stv<T, SPL>(pan0 + (size_t)(8 * g + 2 * t) * TS + lane * SPL, a);
      stv<T, SPL>(pan0 + (size_t)(8 * g + 2 * t + 1) * TS + lane * SPL, b);
    }
  }
  __syncthreads();

  double* red = reinterpret_cast<double*>(smraw + LY.red_bytes_off);  // [8 warps][TS][9]
  if (!producer)
    for (int q = 0; q < SPL * NMODES; ++q) red[((size_t)warp * TS + lane * SPL) * NMODES + q] = 0.0;

  int o_stop = 0;
  for (int o = 0; o < nops; ++o) {
    o_stop = o;
    const uint32_t tries = (o == 0 && wait0 >= 0) ? (uint32_t)wait0 : MBAR_WAIT_TRIES;
    const bool late = !producer && !mbar_wait_bounded(&bars[o % NS], (uint32_t)((o / NS) & 1), tries);
    if (producer) {
      // the slot of op o - 1 is free since the barrier that ended it
      if (tid == NTC && o + NS - 1 < nops) issue(o + NS - 1);
      if (__syncthreads_or(0)) {
        abort_flag = 1;
        break;
      }
      continue;
    }
    int kind, j;
    op_kind(h, o, kind, j);
    const T* M = sm + (size_t)(o % NS) * cp.slot_elems;
    // input and output panels (see the ping-pong in the header of this file)
    const bool from0 = kind == GK_LINV || kind == GK_BT;
    const T* pin = from0 ? pan0 : pan1;
    T* pout = from0 ? pan1 : pan0;
    if (!late) {
      for (int q = 0; q < ngrp; ++q) {
        const int g = q == 0 ? gA : gB;
        // the epilogue's operand, fetched before the products
        double2 rv[4][SPL];
        T yp[8][SPL];
        if (kind == GK_B || kind == GK_LT) fetch_r(g, j, rv);
        if (kind == GK_BT) {
#pragma unroll
          for (int rr = 0; rr < 8; ++rr) ldv<T, SPL>(ybase + (size_t)(j - 1) * yrow + (size_t)(8 * g + rr) * TS + lane * SPL, yp[rr]);
        }
        int lo, hi;
        grp_range(kind, nb, g, lo, hi);
        const T* mg = M + grp_off(kind, nb, g);
        T acc[8][SPL];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr)
#pragma unroll
          for (int s = 0; s < SPL; ++s) acc[rr][s] = T(0);
        // column steps, the loads of column c + 1 issued before the products of c
        T m[8], v[SPL];
        if (lo < hi) {
          ld8(mg, m);
          ldv<T, SPL>(pin + (size_t)lo * TS + lane * SPL, v);
        }
#pragma unroll 2
        for (int c = lo; c + 1 < hi; ++c) {
          T mn[8], vn[SPL];
          ld8(mg + (size_t)(c + 1 - lo) * 8, mn);
          ldv<T, SPL>(pin + (size_t)(c + 1) * TS + lane * SPL, vn);
#pragma unroll
          for (int rr = 0; rr < 8; ++rr)
#pragma unroll
            for (int s = 0; s < SPL; ++s) acc[rr][s] = fma(m[rr], v[s], acc[rr][s]);
#pragma unroll
          for (int rr = 0; rr < 8; ++rr) m[rr] = mn[rr];
#pragma unroll
          for (int s = 0; s < SPL; ++s) v[s] = vn[s];
        }
        if (lo < hi) {
#pragma unroll
          for (int rr = 0; rr < 8; ++rr)
#pragma unroll
            for (int s = 0; s < SPL; ++s) acc[rr][s] = fma(m[rr], v[s], acc[rr][s]);
        }
        // epilogue: rows 8g + rr < nb only
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
          const int row = 8 * g + rr;
          if (row >= nb) break;
          T out[SPL];
#pragma unroll
          for (int s = 0; s < SPL; ++s) {
            if (kind == GK_B) {
              const double rc = (rr & 1) ? rv[rr >> 1][s].y : rv[rr >> 1][s].x;
              out[s] = (T)rc - acc[rr][s];
            } else if (kind == GK_BT) {
              out[s] = yp[rr][s] - acc[rr][s];
            } else {
              out[s] = acc[rr][s];
            }
          }
          stv<T, SPL>(pout + (size_t)row * TS + lane * SPL, out);
          if (kind == GK_LINV) stv<T, SPL>(ybase + (size_t)j * yrow + (size_t)row * TS + lane * SPL, out);
        }
        if (kind == GK_LT) {
          // delta of block row j (lattice row j0 + j) and the P sums of its
          // nodes.  On a row, eta is one value and xi = xi0 + L il, so the row's
          // six sums (r_x, r_y, delta.r and their il-weighted copies) are
          // formed first and the nine modes from them once per row.
#pragma unroll
          for (int s = 0; s < SPL; ++s) {
            if (!valid[s]) continue;
            double sx = 0.0, sy = 0.0, sd = 0.0, six = 0.0, siy = 0.0, sid = 0.0;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const int il = 4 * g + t;
              if (il >= w) break;
              T2 dv;
              dv.x = acc[2 * t][s], dv.y = acc[2 * t + 1][s];
              reinterpret_cast<T2*>(delta)[nbase[s] + (size_t)j * lv.nx + il] = dv;
              const double2 rc = rv[t][s];
              const double dr = fma((double)dv.x, rc.x, (double)dv.y * rc.y);
              const double fil = (double)il;
              sx += rc.x;
              sy += rc.y;
              sd += dr;
              six = fma(fil, rc.x, six);
              siy = fma(fil, rc.y, siy);
              sid = fma(fil, dr, sid);
            }
            const int jg = j0p[s] + j;
            const double xi0 = fma(lv.L, xoff[s] + 0.5 * (double)(jg & 1), -repx[s]);
            const double eta = fma(lv.L * SQ3_2, (double)jg, -repy[s]);
            double* pr = red + ((size_t)warp * TS + lane * SPL + s) * NMODES;
            pr[0] += sx;
            pr[1] += sy;
            pr[2] += fma(xi0, sx, lv.L * six);
            pr[3] = fma(eta, sx, pr[3]);
            pr[4] += fma(xi0, sy, lv.L * siy);
            pr[5] = fma(eta, sy, pr[5]);
            pr[6] += sd;
            pr[7] += fma(xi0, sd, lv.L * sid);
            pr[8] = fma(eta, sd, pr[8]);
          }
        }
      }
    }
    if (__syncthreads_or(late)) {
      abort_flag = 1;
      break;
    }
  }
  if (abort_flag) {
    // the copies in flight are those of ops o_stop .. issued - 1, one per slot
    if (tid == NTC) {
      for (int k = o_stop; k < issued; ++k) mbar_wait_bounded(&bars[k % NS], (uint32_t)((k / NS) & 1));
      atomicOr(err, (int)DEVERR_TIMEOUT);
    }
    return;
  }
  // P_I: the warps' partial sums, added in warp order
  __syncthreads();
  for (int q = tid; q < it.count * NMODES; q += NTC + 32) {
    const int ls = q / NMODES, m = q % NMODES;
    double sum = 0.0;
    for (int ww = 0; ww < NTC / 32; ++ww) sum += red[((size_t)ww * TS + ls) * NMODES + m];
    P[(size_t)lv.q * cp.sets[it.first + ls] + m] = sum;
  }
}

// The grouped copy of one class's factor from its standard layout (setup.cu):
// one thread per stored element of op o's matrix.
template <typename T>
__global__ void k_group_factor(const double* __restrict__ src, int nb, int h, T* __restrict__ dst) {
  const int o = blockIdx.y;
  int kind, j;
  op_kind(h, o, kind, j);
  const long long size = grp_size(kind, nb);
  T* out = dst + class_op_off(nb, h, o);
  const double* lin = src + mat_off(nb, 2 * j);      // Linv_j, rows packed
  const double* bm = src + mat_off(nb, 2 * j - 1);   // B_j (j >= 1), rows packed
  const int NG = (nb + 7) / 8;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < size; e += (long long)gridDim.x * blockDim.x) {
    // group g: the first with grp_off(kind, nb, g + 1) > e
    int g = 0;
    while (g + 1 < NG && grp_off(kind, nb, g + 1) <= e) ++g;
    double v = 0.0;
    const long long go = grp_off(kind, nb, g);
    int lo, hi;
    grp_range(kind, nb, g, lo, hi);
    if (g < NG && e - go < 8LL * (hi - lo)) {
      const int c = lo + (int)((e - go) / 8), row = 8 * g + (int)((e - go) % 8);
      if (row < nb) {
        if (kind == GK_LINV) {
          if (c <= row) v = lin[linv_row_off(row) + c];
        } else if (kind == GK_B) {
          if (c >= b_lo(row)) v = bm[b_row_off(nb, row) + (c - b_lo(row))];
        } else if (kind == GK_LT) {
          if (c >= row) v = lin[linv_row_off(c) + row];  // Linv_j[c][row]
        } else {
          if (row >= b_lo(c)) v = bm[b_row_off(nb, c) + (row - b_lo(c))];  // B_j[c][row]
        }
      }
    }
    out[e] = (T)v;
  }
}

}  // namespace

int class_sets_per_cta(bool fp32) { return fp32 ? 64 : 32; }

size_t relax_class_smem(size_t slot_elems, int nb8max, bool fp32) {
  return fp32 ? class_layout<float, 2, 3>(slot_elems, nb8max).total_bytes
              : class_layout<double, 1, 2>(slot_elems, nb8max).total_bytes;
}

cudaError_t launch_group_factor(cudaStream_t s, const double* src, int nb, int h, double* g64, float* g32) {
  const dim3 grid(32, 2 * (2 * h - 1));
  if (g64) k_group_factor<double><<<grid, 256, 0, s>>>(src, nb, h, g64);
  if (g32) k_group_factor<float><<<grid, 256, 0, s>>>(src, nb, h, g32);
  return cudaGetLastError();
}

cudaError_t launch_relax_class(cudaStream_t s, const LatView& lv, const ClassPlanDev& cp, const double* f64,
                               const float* f32, const double2* r, void* delta, double* P, void* yscratch,
                               const IterCtl* ctl, int* err, int wait0) {
  if (cp.nitems <= 0) return cudaSuccess;
  const bool fp32 = f32 != nullptr;
  const size_t smem = relax_class_smem(cp.slot_elems, cp.nb8max, fp32);
  if (fp32)
    k_relax_class<float, 2, 3><<<cp.nitems, NTC + 32, smem, s>>>(lv, cp, f32, r, (float*)delta, P, (float*)yscratch,
                                                                 ctl, err, wait0);
  else
    k_relax_class<double, 1, 2><<<cp.nitems, NTC + 32, smem, s>>>(lv, cp, f64, r, (double*)delta, P,
                                                                  (double*)yscratch, ctl, err, wait0);
  return cudaGetLastError();
}

cudaError_t configure_relax_class(int max_smem) {
  cudaError_t e = set_max_dynamic_smem(k_relax_class<float, 2, 3>, max_smem);
  if (e != cudaSuccess) return e;
  return set_max_dynamic_smem(k_relax_class<double, 1, 2>, max_smem);
}

}  // namespace hms
