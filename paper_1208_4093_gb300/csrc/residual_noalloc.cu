// Residual of Eq. 1 with the sums of Eq. 19 and Eq. 2, computed with scratch
// held in static device memory, so that a call allocates nothing.
//
// The kernel is the residual half of K1 (residual.cu) in the same launch
// shape: one CTA per 32 x 8 node tile with a one-node halo in shared memory,
// r = p - K u summed bar by bar, and per-CTA sums of ||r||_1, ||r||_2^2 and
// u.(p + r) reduced by the last CTA in CTA order.  It reads the caller's u
// and p in place (constrained DOFs of u taken as 0 while staging) and writes
// no displacement.  The per-CTA sums and the completion ticket live in the
// two file-scope arrays below instead of problem-owned buffers.
//
// Scratch contract:
//   g_partials  3 doubles per CTA, at most kMaxTiles CTAs; every slot a launch
//               reads is written by the same launch first, so it needs no
//               initial value.
//   g_ticket    must be 0 when a launch starts.  It is 0 after module load
//               (explicit initialiser) and the last CTA of every launch
//               resets it, so it is 0 again once the launch completes.
// Two launches in flight on one device at the same time share both and race
// (wrong sums, possibly a ticket left non-zero); launches in one stream are
// serialised and do not.
#include <mutex>

#include "../../include/hms.h"
#include "hms_internal.cuh"

namespace hms {

constexpr int kNoallocTX = 32, kNoallocTY = 8, kNoallocNT = kNoallocTX * kNoallocTY;
constexpr int kMaxTiles = HMS_RESIDUAL_NOALLOC_MAX_TILES;
static_assert(kMaxTiles > 0 && kMaxTiles <= (1 << 20), "static scratch size");

static __device__ __align__(256) double g_partials[3 * kMaxTiles];
static __device__ __align__(256) unsigned int g_ticket = 0u;

namespace {

__device__ inline double warp_sum_na(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// Sum of N values per thread over the CTA in fixed order; valid in warp 0.
template <int N>
__device__ inline void block_sum_na(double (&v)[N], double* sred) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = warp_sum_na(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) sred[warp * N + k] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = warp_sum_na(lane < nw ? sred[lane * N + k] : 0.0);
  }
}

__global__ void __launch_bounds__(kNoallocNT)
    k_residual_noalloc(LatView lv, const double2* __restrict__ u, const double2* __restrict__ p,
                       double2* __restrict__ r, double* __restrict__ partials, unsigned* ticket,
                       double* norms_out) {
  constexpr int TX = kNoallocTX, TY = kNoallocTY, NT = kNoallocNT;
  __shared__ double2 U[TY + 2][TX + 2];
  __shared__ double sred[32 * 3];
  __shared__ bool last;
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
  double s[3] = {0.0, 0.0, 0.0};
  if (i < lv.nx && j < lv.ny) {
    const size_t n = (size_t)j * lv.nx + i;
    const int lx = tx + 1, ly = ty + 1, off = j & 1;
    const double2 uc = U[ly][lx];
    // E-W bars, e = (1, 0)
    const double kE = bar_k(lv, i, j, 0), kW = bar_k(lv, i - 1, j, 0);
    double fx = kE * (uc.x - U[ly][lx + 1].x) + kW * (uc.x - U[ly][lx - 1].x);
    // this node's NE bar and the SW neighbour's, e = (1/2, sqrt3/2)
    const double kNE = bar_k(lv, i, j, 1), kSW = bar_k(lv, i - 1 + off, j - 1, 1);
    const double2 une = U[ly + 1][lx + off], usw = U[ly - 1][lx - 1 + off];
    const double d1x = kNE * (uc.x - une.x) + kSW * (uc.x - usw.x);
    const double d1y = kNE * (uc.y - une.y) + kSW * (uc.y - usw.y);
    const double p1 = fma(SQ3_2, d1y, 0.5 * d1x);
    // this node's NW bar and the SE neighbour's, e = (-1/2, sqrt3/2)
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
    s[0] = fabs(rn.x) + fabs(rn.y);
    s[1] = fma(rn.x, rn.x, rn.y * rn.y);
    s[2] = fma(uc.x, pn.x + rn.x, uc.y * (pn.y + rn.y));
  }
  block_sum_na<3>(s, sred);
  const unsigned nblocks = gridDim.x * gridDim.y;
  const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
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
  block_sum_na<3>(v, sred);
  if (tid == 0) {
    *ticket = 0u;
    if (norms_out) {
      norms_out[0] = v[0];
      norms_out[1] = v[1];
      norms_out[2] = v[2];
    }
  }
}

struct StaticScratch {
  bool ready = false;
  double* partials = nullptr;
  unsigned* ticket = nullptr;
};
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
StaticScratch g_scratch[kMaxDevices];

}  // namespace

int residual_noalloc_tiles(const LatView& lv) {
  return ((lv.nx + kNoallocTX - 1) / kNoallocTX) * ((lv.ny + kNoallocTY - 1) / kNoallocTY);
}

// Device addresses of the static scratch on `device`, looked up on the first
// call for that device (which must have it current) and cached.
cudaError_t residual_noalloc_scratch(int device, double** partials, unsigned** ticket) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  StaticScratch& d = g_scratch[device];
  if (!d.ready) {
    void* pp = nullptr;
    void* tp = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&pp, g_partials);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&tp, g_ticket);
    if (e != cudaSuccess) return e;
    d.partials = static_cast<double*>(pp);
    d.ticket = static_cast<unsigned*>(tp);
    d.ready = true;
  }
  *partials = d.partials;
  *ticket = d.ticket;
  return cudaSuccess;
}

cudaError_t launch_residual_noalloc(cudaStream_t s, const LatView& lv, const double2* u, const double2* p,
                                    double2* r, double* partials, unsigned* ticket, double* norms_out) {
  dim3 grid((lv.nx + kNoallocTX - 1) / kNoallocTX, (lv.ny + kNoallocTY - 1) / kNoallocTY);
  k_residual_noalloc<<<grid, kNoallocNT, 0, s>>>(lv, u, p, r, partials, ticket, norms_out);
  return cudaGetLastError();
}

}  // namespace hms
