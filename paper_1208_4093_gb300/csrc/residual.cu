// K1: update + matrix-free residual + norms (Eqs. 3, 1, 19, 2).
//
// One CTA per 32 x 8 node tile.  The tile and its one-node halo are staged in
// shared memory; every staged node first gets the upper-level update of
// Eq. 3, u += V a (translations, gradients and the relaxation modes of the
// node's own set), so halo nodes see the same updated values their owners
// write.  Then each node sums the axial forces of its six bars,
//   (K u)_a = sum_b (EA/L)_ab e_ab e_ab^T (u_a - u_b),
// and writes r = p - K u on free DOFs (0 on constrained DOFs), the new u, and
// its share of ||r||_1, ||r||_2^2 and u.(p + r).  The last CTA to finish
// reduces the per-CTA sums in CTA order (deterministic), turns them into the
// relative residuals of Eq. 19 and the energy Pi = 1/2 u.K.u - u.p =
// -1/2 u.(p + r) of Eq. 2, and decides convergence.
//
// In the mixed form (FP32 delta) the increment V a of Eq. 3 is formed in FP32
// and added to the FP64 u: the coefficients of the tile's sets are rounded to
// FP32 once per CTA (with the set's representative point as an offset, so
// that xi and eta are small numbers), and a staged node then costs 4 FP64
// operations (two conversions, two adds) instead of about 17.  The increment
// carries FP32 rounding errors of about 1e-7 of its terms' size, like the FP32
// relaxation's delta it multiplies; the residual that decides convergence
// stays FP64, so the iteration still converges to the FP64 solution (later
// updates correct what an update got wrong).  The FP64 form and the
// force-controlled modes keep the FP64 increment.
#include <type_traits>

#include "hms_internal.cuh"

namespace hms {
namespace {

constexpr int TX = 32, TY = 8, NT = TX * TY;

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// Deterministic block sum of N values per thread over the NT threads of a
// CTA; the sums land in v of thread 0.  The values go through shared memory:
// warp k adds value k of the eight warps lane by lane in warp order, then a
// shuffle tree finishes it.  That is 12 FP64 adds in N warps instead of a
// shuffle tree in every warp.  sred holds N * (NT + 1) doubles.
template <int N>
__device__ inline void block_sum(double (&v)[N], double* sred) {
  static_assert(N <= NT / 32, "one warp per value");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) sred[k * NT + tid] = v[k];
  __syncthreads();
  if (warp < N) {
    const double* c = sred + warp * NT + lane;
    double t = c[0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) t += c[32 * w];
    t = warp_sum(t);
    if (lane == 0) sred[N * NT + warp] = t;
  }
  __syncthreads();
  if (tid == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = sred[N * NT + k];
}

template <typename DT>
__device__ inline double2 load_delta(const DT* d, size_t n);
template <>
__device__ inline double2 load_delta<double2>(const double2* d, size_t n) { return d[n]; }
template <>
__device__ inline double2 load_delta<float2>(const float2* d, size_t n) {
  float2 f = d[n];
  return make_double2((double)f.x, (double)f.y);
}

// Eq. 3 at node (i, j): u += sum_m a_m^(I) uhat_m^(I) with the modes of
// Eqs. 9, 10, 13, 14 (zero on constrained DOFs), and with RF the force-
// controlled modes of Eqs. 17-18 (delta^RF and its gradient-weighted copies).
template <typename DT, bool RF>
__device__ inline double2 apply_update(const LatView& lv, double2 v, int i, int j, const DT* delta,
                                       const DT* delta_rf, const double* __restrict__ a) {
  const size_t n = (size_t)j * lv.nx + i;
  const int I = set_of(lv, i, j);
  const double* aI = a + (size_t)lv.q * I;
  const double2 c = lv.rep[I];
  // xi = x - x^(I), eta = y - y^(I) as one FMA each (the half-column offset of odd
  // rows added to i exactly)
  const double xi = fma(lv.L, (double)i + ((j & 1) ? 0.5 : 0.0), -c.x);
  const double eta = fma(lv.L * SQ3_2, (double)j, -c.y);
  const double2 d = load_delta(delta, n);
  const unsigned fm = lv.fix[n];
  const double cd = fma(__ldg(aI + 8), eta, fma(__ldg(aI + 7), xi, __ldg(aI + 6)));
  if (!(fm & 1u)) v.x += fma(cd, d.x, fma(__ldg(aI + 3), eta, fma(__ldg(aI + 2), xi, __ldg(aI + 0))));
  if (!(fm & 2u)) v.y += fma(cd, d.y, fma(__ldg(aI + 5), eta, fma(__ldg(aI + 4), xi, __ldg(aI + 1))));
  if constexpr (RF) {
    const double2 f = load_delta(delta_rf, n);
    const double cf = fma(__ldg(aI + 11), eta, fma(__ldg(aI + 10), xi, __ldg(aI + 9)));
    if (!(fm & 1u)) v.x = fma(cf, f.x, v.x);
    if (!(fm & 2u)) v.y = fma(cf, f.y, v.y);
  }
  return v;
}

// FP32 increment of the mixed form: the sets a tile's staged nodes (the tile
// and its one-node halo) can fall in, at most F32SETS of them.
constexpr int F32SETS = 32;
constexpr int F32STRIDE = 12;  // a_0 .. a_8, the offsets ox, oy, pad
__host__ __device__ inline bool f32_increment_fits(int sx, int sy) {
  // set columns a span of TX + 2 nodes can touch, times set rows of TY + 2
  return ((TX + 2 + sx - 1) / sx + 1) * ((TY + 2 + sy - 1) / sy + 1) <= F32SETS;
}

// Eq. 3 at node (i, j) with the FP32 coefficients f of its set (origin i0s, j0s):
// xi = L (i - i0s + (j odd ? 1/2 : 0)) + ox, eta = L sqrt3/2 (j - j0s) + oy
// with ox = L i0s - x^(I), oy = L sqrt3/2 j0s - y^(I) rounded to FP32.
__device__ inline double2 apply_update_f32(const LatView& lv, double2 v, int i, int j, int i0s, int j0s,
                                           const float* f, const float2* delta) {
  const size_t n = (size_t)j * lv.nx + i;
  const float L = (float)lv.L;
  const float xi = fmaf(L, (float)(i - i0s) + ((j & 1) ? 0.5f : 0.0f), f[9]);
  const float eta = fmaf(L * (float)SQ3_2, (float)(j - j0s), f[10]);
  const float2 d = delta[n];
  const unsigned fm = lv.fix[n];
  const float cd = fmaf(f[8], eta, fmaf(f[7], xi, f[6]));
  if (!(fm & 1u)) v.x += (double)fmaf(cd, d.x, fmaf(f[3], eta, fmaf(f[2], xi, f[0])));
  if (!(fm & 2u)) v.y += (double)fmaf(cd, d.y, fmaf(f[5], eta, fmaf(f[4], xi, f[1])));
  return v;
}

// The kernel body for tile (bx, by) of a gx x gy grid (the whole lattice).
template <typename DT, bool RF = false>
__device__ __forceinline__ void update_residual_body(
    const LatView lv, const double2* __restrict__ u_in, double2* __restrict__ u_out,
    const double2* __restrict__ p, const DT* __restrict__ delta, const DT* __restrict__ delta_rf,
    const double* __restrict__ a,
    double2* __restrict__ r, double* __restrict__ partials, unsigned* ticket, double* norms_out,
    IterCtl* ctl, double* hist, int hist_cap, int bx, int by, int gx, int gy) {
  __shared__ double2 U[TY + 2][TX + 2];
  __shared__ double sred[3 * (NT + 1)];
  __shared__ bool last;
  int t = 0;
  if (ctl) {
    if (*(volatile int*)&ctl->done) return;
    t = *(volatile int*)&ctl->t;
  }
  const bool upd = (a != nullptr) && (t > 0 || ctl == nullptr);
  const int i0 = bx * TX, j0 = by * TY;
  const int tid = threadIdx.x;

  constexpr bool MIXED = std::is_same<DT, float2>::value && !RF;
  __shared__ float fa[MIXED ? F32SETS * F32STRIDE : 1];
  const bool f32inc = MIXED && upd && f32_increment_fits(lv.sx, lv.sy);
  // the sets of the staged nodes: columns scx0.., rows scy0.. (nscx across)
  const int scx0 = max(i0 - 1, 0) / lv.sx, scy0 = max(j0 - 1, 0) / lv.sy;
  const int nscx = min(i0 + TX, lv.nx - 1) / lv.sx - scx0 + 1;
  if (f32inc) {
    const int nscy = min(j0 + TY, lv.ny - 1) / lv.sy - scy0 + 1;
    for (int q = tid; q < nscx * nscy * F32STRIDE; q += NT) {
      const int sl = q / F32STRIDE, m = q - sl * F32STRIDE;
      const int Ix = scx0 + sl % nscx, Iy = scy0 + sl / nscx;
      const int I = Iy * lv.Mx + Ix;
      float v = 0.0f;
      if (m < NMODES) {
        v = (float)__ldg(a + (size_t)lv.q * I + m);
      } else if (m == 9) {
        v = (float)fma(lv.L, (double)(Ix * lv.sx), -lv.rep[I].x);
      } else if (m == 10) {
        v = (float)fma(lv.L * SQ3_2, (double)(Iy * lv.sy), -lv.rep[I].y);
      }
      fa[q] = v;
    }
    __syncthreads();
  }

  for (int idx = tid; idx < (TX + 2) * (TY + 2); idx += NT) {
    const int lx = idx % (TX + 2), ly = idx / (TX + 2);
    const int i = i0 + lx - 1, j = j0 + ly - 1;
    double2 v = make_double2(0.0, 0.0);
    if (i >= 0 && i < lv.nx && j >= 0 && j < lv.ny) {
      v = u_in[(size_t)j * lv.nx + i];
      if constexpr (MIXED) {
        if (f32inc) {
          const int Ix = i / lv.sx, Iy = j / lv.sy;
          const float* f = fa + ((Iy - scy0) * nscx + (Ix - scx0)) * F32STRIDE;
          v = apply_update_f32(lv, v, i, j, Ix * lv.sx, Iy * lv.sy, f, reinterpret_cast<const float2*>(delta));
        } else if (upd) {
          v = apply_update<DT, RF>(lv, v, i, j, delta, delta_rf, a);
        }
      } else if (upd) {
        v = apply_update<DT, RF>(lv, v, i, j, delta, delta_rf, a);
      }
    }
    U[ly][lx] = v;
  }
  __syncthreads();

  const int tx = tid % TX, ty = tid / TX;
  const int i = i0 + tx, j = j0 + ty;
  double s[3] = {0.0, 0.0, 0.0};
  if (i < lv.nx && j < lv.ny) {
    const size_t n = (size_t)j * lv.nx + i;
    const int lx = tx + 1, ly = ty + 1, off = j & 1;
    const double2 uc = U[ly][lx];
    // E-W bars (e = (1, 0))
    const double kE = bar_k(lv, i, j, 0), kW = bar_k(lv, i - 1, j, 0);
    double fx = kE * (uc.x - U[ly][lx + 1].x) + kW * (uc.x - U[ly][lx - 1].x);
    // NE bar of this node and NE bar of the SW neighbour: e = (1/2, sqrt3/2)
    const double kNE = bar_k(lv, i, j, 1), kSW = bar_k(lv, i - 1 + off, j - 1, 1);
    const double2 une = U[ly + 1][lx + off], usw = U[ly - 1][lx - 1 + off];
    const double d1x = kNE * (uc.x - une.x) + kSW * (uc.x - usw.x);
    const double d1y = kNE * (uc.y - une.y) + kSW * (uc.y - usw.y);
    const double p1 = fma(SQ3_2, d1y, 0.5 * d1x);
    // NW bar of this node and NW bar of the SE neighbour: e = (-1/2, sqrt3/2)
    const double kNW = bar_k(lv, i, j, 2), kSE = bar_k(lv, i + off, j - 1, 2);
    const double2 unw = U[ly + 1][lx - 1 + off], use = U[ly - 1][lx + off];
    const double d2x = kNW * (uc.x - unw.x) + kSE * (uc.x - use.x);
    const double d2y = kNW * (uc.y - unw.y) + kSE * (uc.y - use.y);
    const double p2 = fma(SQ3_2, d2y, -0.5 * d2x);
    fx = fma(0.5, p1 - p2, fx);
    const double fy = SQ3_2 * (p1 + p2);
    const double2 pn = p[n];
    const unsigned fm = lv.fix[n];
    double2 rn;
    rn.x = (fm & 1u) ? 0.0 : pn.x - fx;
    rn.y = (fm & 2u) ? 0.0 : pn.y - fy;
    r[n] = rn;
    u_out[n] = uc;
    s[0] = fabs(rn.x) + fabs(rn.y);
    s[1] = fma(rn.x, rn.x, rn.y * rn.y);
    s[2] = fma(uc.x, pn.x + rn.x, uc.y * (pn.y + rn.y));
  }
  block_sum<3>(s, sred);
  const unsigned nblocks = (unsigned)(gx * gy);
  const unsigned bid = (unsigned)(by * gx + bx);
  if (tid == 0) {
    partials[3 * (size_t)bid + 0] = s[0];
    partials[3 * (size_t)bid + 1] = s[1];
    partials[3 * (size_t)bid + 2] = s[2];
    __threadfence();
    last = (atomicAdd(ticket, 1u) == nblocks - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v[3] = {0.0, 0.0, 0.0};
  for (unsigned b = tid; b < nblocks; b += NT) {
    v[0] += __ldcg(partials + 3 * (size_t)b + 0);
    v[1] += __ldcg(partials + 3 * (size_t)b + 1);
    v[2] += __ldcg(partials + 3 * (size_t)b + 2);
  }
  __syncthreads();
  block_sum<3>(v, sred);
  if (tid == 0) {
    *ticket = 0u;  // ready for the next launch
    if (norms_out) {
      norms_out[0] = v[0];
      norms_out[1] = v[1];
      norms_out[2] = v[2];
    }
    if (ctl) {
      const double R1 = ctl->p1 > 0.0 ? v[0] / ctl->p1 : 0.0;
      const double R2 = ctl->p2 > 0.0 ? sqrt(v[1]) / ctl->p2 : 0.0;
      const double Pi = -0.5 * v[2];
      if (t < hist_cap && hist) {
        hist[3 * t + 0] = R1;
        hist[3 * t + 1] = R2;
        hist[3 * t + 2] = Pi;
      }
      if (!isfinite(R1) || !isfinite(R2) || !isfinite(Pi)) {
        ctl->status = 3;
        ctl->err |= DEVERR_NONFINITE;
        ctl->done = 1;
      } else if (R1 < ctl->tol) {
        ctl->status = 1;
        ctl->done = 1;
      } else if (t >= ctl->max_iter || ctl->err != 0) {
        ctl->status = 2;
        ctl->done = 1;
      }
      ctl->t = t + 1;
    }
  }
}

template <typename DT, bool RF>
__global__ void __launch_bounds__(NT) k_update_residual(
    LatView lv, const double2* __restrict__ u_in, double2* __restrict__ u_out,
    const double2* __restrict__ p, const DT* __restrict__ delta, const DT* __restrict__ delta_rf,
    const double* __restrict__ a, double2* __restrict__ r, double* __restrict__ partials, unsigned* ticket,
    double* norms_out, IterCtl* ctl, double* hist, int hist_cap) {
  update_residual_body<DT, RF>(lv, u_in, u_out, p, delta, delta_rf, a, r, partials, ticket, norms_out, ctl, hist,
                               hist_cap, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
}

// Batched: update k of a CUDA-graph round (u ping-pongs between u[k & 1] and
// u[(k + 1) & 1]) for the tiles of every problem of a batch.
template <typename DT>
__global__ void __launch_bounds__(NT) kb_update_residual(const BatchProb* __restrict__ P,
                                                         const BatchItem* __restrict__ items, int k) {
  const BatchItem it = items[blockIdx.x];
  const BatchProb& q = P[it.prob];
  update_residual_body<DT>(q.lv, q.u[k & 1], q.u[(k + 1) & 1], q.p, (const DT*)q.delta, nullptr, q.a, q.r,
                           q.partials, q.ticket, nullptr, q.ctl, q.hist, q.hist_cap, it.bx, it.by, it.gx, it.gy);
}

// Masks the loads on constrained DOFs and computes ||p||_1, ||p||_2 into ctl.
__global__ void __launch_bounds__(NT) k_load_norms(LatView lv, double2* __restrict__ p,
                                                    double* __restrict__ partials, unsigned* ticket,
                                                    IterCtl* ctl) {
  __shared__ double sred[2 * (NT + 1)];
  __shared__ bool last;
  const size_t nn = (size_t)lv.nx * lv.ny;
  double s[2] = {0.0, 0.0};
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nn;
       n += (size_t)gridDim.x * blockDim.x) {
    double2 v = p[n];
    const unsigned fm = lv.fix[n];
    if (fm & 1u) v.x = 0.0;
    if (fm & 2u) v.y = 0.0;
    p[n] = v;
    s[0] += fabs(v.x) + fabs(v.y);
    s[1] += fma(v.x, v.x, v.y * v.y);
  }
  block_sum<2>(s, sred);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x + 0] = s[0];
    partials[2 * blockIdx.x + 1] = s[1];
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v[2] = {0.0, 0.0};
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    v[0] += __ldcg(partials + 2 * b + 0);
    v[1] += __ldcg(partials + 2 * b + 1);
  }
  __syncthreads();
  block_sum<2>(v, sred);
  if (threadIdx.x == 0) {
    *ticket = 0u;
    ctl->p1 = v[0];
    ctl->p2 = sqrt(v[1]);
  }
}

// K u at every DOF (constrained ones included): the nodal forces of the bars,
// with u read as 0 on constrained DOFs.  One CTA per 32 x 8 node tile and its
// one-node halo in shared memory, the six bars of each node summed as in the
// residual above.
__global__ void __launch_bounds__(NT) k_reactions(LatView lv, const double2* __restrict__ u,
                                                  double2* __restrict__ f) {
  __shared__ double2 U[TY + 2][TX + 2];
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < (TX + 2) * (TY + 2); idx += NT) {
    const int lx = idx % (TX + 2), ly = idx / (TX + 2);
    const int i = i0 + lx - 1, j = j0 + ly - 1;
    double2 v = make_double2(0.0, 0.0);
    if (i >= 0 && i < lv.nx && j >= 0 && j < lv.ny) {
      const size_t n = (size_t)j * lv.nx + i;
      v = u[n];
      const unsigned fm = lv.fix[n];
      if (fm & 1u) v.x = 0.0;
      if (fm & 2u) v.y = 0.0;
    }
    U[ly][lx] = v;
  }
  __syncthreads();
  const int tx = tid % TX, ty = tid / TX;
  const int i = i0 + tx, j = j0 + ty;
  if (i >= lv.nx || j >= lv.ny) return;
  const int lx = tx + 1, ly = ty + 1, off = j & 1;
  const double2 uc = U[ly][lx];
  const double kE = bar_k(lv, i, j, 0), kW = bar_k(lv, i - 1, j, 0);
  double fx = kE * (uc.x - U[ly][lx + 1].x) + kW * (uc.x - U[ly][lx - 1].x);
  const double kNE = bar_k(lv, i, j, 1), kSW = bar_k(lv, i - 1 + off, j - 1, 1);
  const double2 une = U[ly + 1][lx + off], usw = U[ly - 1][lx - 1 + off];
  const double d1x = kNE * (uc.x - une.x) + kSW * (uc.x - usw.x);
  const double d1y = kNE * (uc.y - une.y) + kSW * (uc.y - usw.y);
  const double p1 = fma(SQ3_2, d1y, 0.5 * d1x);
  const double kNW = bar_k(lv, i, j, 2), kSE = bar_k(lv, i + off, j - 1, 2);
  const double2 unw = U[ly + 1][lx - 1 + off], use = U[ly - 1][lx + off];
  const double d2x = kNW * (uc.x - unw.x) + kSE * (uc.x - use.x);
  const double d2y = kNW * (uc.y - unw.y) + kSE * (uc.y - use.y);
  const double p2 = fma(SQ3_2, d2y, -0.5 * d2x);
  fx = fma(0.5, p1 - p2, fx);
  f[(size_t)j * lv.nx + i] = make_double2(fx, SQ3_2 * (p1 + p2));
}

}  // namespace

cudaError_t launch_reactions(cudaStream_t s, const LatView& lv, const double2* u, double2* f) {
  dim3 grid((lv.nx + TX - 1) / TX, (lv.ny + TY - 1) / TY);
  k_reactions<<<grid, NT, 0, s>>>(lv, u, f);
  return cudaGetLastError();
}

int update_residual_blocks(const LatView& lv) {
  return ((lv.nx + TX - 1) / TX) * ((lv.ny + TY - 1) / TY);
}
int update_residual_grid_x(const LatView& lv) { return (lv.nx + TX - 1) / TX; }
int update_residual_grid_y(const LatView& lv) { return (lv.ny + TY - 1) / TY; }

cudaError_t launch_batch_update_residual(cudaStream_t s, bool fp32, const BatchProb* P, const BatchItem* it, int n,
                                         int k) {
  if (n <= 0) return cudaSuccess;
  if (fp32) kb_update_residual<float2><<<n, NT, 0, s>>>(P, it, k);
  else kb_update_residual<double2><<<n, NT, 0, s>>>(P, it, k);
  return cudaGetLastError();
}

cudaError_t launch_update_residual(cudaStream_t s, const LatView& lv, const double2* u_in,
                                   double2* u_out, const double2* p, const void* delta,
                                   bool delta_fp32, const double* a, double2* r, double* partials,
                                   unsigned* ticket, double* norms_out, IterCtl* ctl, double* hist,
                                   int hist_cap, const void* delta_rf) {
  dim3 grid((lv.nx + TX - 1) / TX, (lv.ny + TY - 1) / TY);
  const bool rf = lv.q == NMODES_RF;
  if (delta_fp32) {
    if (rf)
      k_update_residual<float2, true><<<grid, NT, 0, s>>>(lv, u_in, u_out, p, (const float2*)delta,
                                                          (const float2*)delta_rf, a, r, partials, ticket,
                                                          norms_out, ctl, hist, hist_cap);
    else
      k_update_residual<float2, false><<<grid, NT, 0, s>>>(lv, u_in, u_out, p, (const float2*)delta, nullptr, a, r,
                                                           partials, ticket, norms_out, ctl, hist, hist_cap);
  } else {
    if (rf)
      k_update_residual<double2, true><<<grid, NT, 0, s>>>(lv, u_in, u_out, p, (const double2*)delta,
                                                           (const double2*)delta_rf, a, r, partials, ticket,
                                                           norms_out, ctl, hist, hist_cap);
    else
      k_update_residual<double2, false><<<grid, NT, 0, s>>>(lv, u_in, u_out, p, (const double2*)delta, nullptr, a,
                                                            r, partials, ticket, norms_out, ctl, hist, hist_cap);
  }
  return cudaGetLastError();
}

cudaError_t launch_load_norms(cudaStream_t s, const LatView& lv, double2* p, double* partials,
                              unsigned* ticket, IterCtl* ctl) {
  const size_t nn = (size_t)lv.nx * lv.ny;
  int grid = (int)((nn + 255) / 256);
  if (grid > 1024) grid = 1024;
  k_load_norms<<<grid, NT, 0, s>>>(lv, p, partials, ticket, ctl);
  return cudaGetLastError();
}

}  // namespace hms
