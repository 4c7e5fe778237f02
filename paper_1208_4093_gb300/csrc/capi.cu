// C ABI of the HMS truss solver: contexts, problem setup, the iteration loop
// (Fig. 3 of the paper as a device-resident CUDA graph) and the single steps.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/hms.h"
#include "hms_internal.cuh"

using namespace hms;

struct hms_context {
  int device = 0;
  int nsm = 0;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> pool;  // streams of hms_solve_batch, created on first use
  std::string err;
  // relaxation launch shape picked by timing, per (set width, set height,
  // precision and copies, overlap, set count where the balanced schedule applies)
  std::map<std::tuple<int, int, int, int, int>, int> relax_tuned;
  int batch_mode = HMS_BATCH_AUTO;
};

// Buffers that stay read-only after setup (lattice description, set
// factors, constant part of K_aa), shared by a problem and its clones and
// freed with the last of them.
struct SharedSetup {
  int refs = 1;
  std::vector<void*> allocs;
};

struct hms_problem {
  hms_context* ctx = nullptr;
  SharedSetup* shared = nullptr;
  LatView lv{};
  int precision = HMS_FP64, nsolve = 4, batch = 16, profile = 0, max_iter = 0;
  unsigned mode_mask = 0x1FFu;  // modes taking part in the upper-level correction
  bool record_history = true;
  int relax_wait0 = -1;         // tries of the relaxation's first copy wait (-1: the usual bound)
  long long refine_cap_hits = 0;  // of the last hms_solve
  bool coarse_fp64 = false;  // factor of the upper-level system in FP64 (else FP32 + FP64 refinement)
  double tol = 1e-8;
  int relax_threads = 256;   // CTA size of the relaxation
  int relax_chunks = 1;      // bulk copies per factor matrix in the relaxation (2: half the shared memory)
  // the relaxation on a balanced schedule (one persistent CTA per SM; relax.cu)
  bool relax_sched = false;
  int sched_grid = 0;
  RelaxSeg* sched_segs = nullptr;
  int* sched_cta = nullptr;
  int* sched_flags = nullptr;  // per set; per instance, as clones run at the same time
  int n_c = 0, bw = 0;
  size_t bytes = 0;
  std::vector<void*> allocs;
  // lattice
  double* kbar = nullptr;
  uint8_t* fix = nullptr;
  double2* rep = nullptr;
  long long* set_off = nullptr;
  // factors: one per set (set_off), or with cls one per class of identical
  // sets in the grouped layout of relax_class.cu (plan in cpd)
  double* f64 = nullptr;
  float* f32 = nullptr;
  bool cls = false;
  ClassPlanDev cpd;
  // force-controlled relaxation (q = 12): cut-free set factors with pinned DOFs,
  // supports | pins, per-set projection onto the free rigid motions (force.cu)
  double* f64F = nullptr;
  float* f32F = nullptr;
  uint8_t* fixF = nullptr;
  double* Mforce = nullptr;
  double2* rproj = nullptr;  // per instance: r projected, 0 at the pins
  void* delta_rf = nullptr;  // per instance: delta^RF of Eq. 17 (double2 or float2)
  // iteration state
  double2* u[2] = {nullptr, nullptr};
  double2* p = nullptr;
  double2* r = nullptr;
  void* delta = nullptr;
  void* yscratch = nullptr;  // forward-substitution vectors of every set
  double* a = nullptr;
  double* P = nullptr;
  double* slots_base = nullptr;
  double* slots_it = nullptr;
  double* band = nullptr;
  double* sband = nullptr;   // column + row layouts
  double* scale = nullptr;
  double* b = nullptr;
  double* x = nullptr;
  double* res = nullptr;
  void* lcol = nullptr;      // L in column layout (float or double)
  void* lrow = nullptr;      // scaled band in row layout, then L in row layout
  void* dinv = nullptr;      // inverted 16 x 16 diagonal blocks of L
  float* xinv = nullptr;     // per 64-row block of the FP32 L: inverted diagonal block and band neighbours
  int big_stages = 0;        // pipeline depth of the 64-row block solve, 0 = 16-row solve
  bool cluster_factor = false;  // FP32 factor on a cluster of 4 CTAs (with the block solve)
  bool two_sided = false;       // FP32 two-sided factor and solve on two SMs
  TwoSided ts;
  bool nd = false;              // nested-dissection factor and solve (coarse_nd.cu) over
  NDPlanHost ndp;               // the blocks of K_aa (coarse_blocks.cu; no band)
  NDPlanDev ndd;
  double* blk = nullptr;
  int* dropped = nullptr;
  unsigned long long* cstat = nullptr;  // refinement state of the upper-level solve
  double* partials = nullptr;
  unsigned* ticket = nullptr;
  IterCtl* ctl = nullptr;
  IterCtl* ctl_host = nullptr;  // pinned
  double* hist = nullptr;
  int hist_cap = 0;
  int* err = nullptr;
  double* norms = nullptr;
  cudaGraphExec_t graph = nullptr;
  float setup_ms = 0.f;
  double ktime[KID_COUNT] = {0};
  long long klaunch[KID_COUNT] = {0};
};

namespace {

hms_status fail(hms_context* c, hms_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

#define CKC(ctx, x)                                                                            \
  do {                                                                                         \
    cudaError_t e_ = (x);                                                                      \
    if (e_ != cudaSuccess)                                                                     \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? HMS_ERR_OOM : HMS_ERR_CUDA,          \
                  std::string(#x) + ": " + cudaGetErrorString(e_));                            \
  } while (0)

template <typename T>
cudaError_t palloc(hms_problem* pr, T** ptr, size_t count) {
  void* p = nullptr;
  const size_t bytes = count * sizeof(T);
  cudaError_t e = cudaMalloc(&p, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) return e;
  pr->allocs.push_back(p);
  pr->bytes += bytes;
  *ptr = (T*)p;
  return cudaSuccess;
}

// allocation of a shared (read-only after setup) buffer; counted in the
// owner's bytes
template <typename T>
cudaError_t salloc(hms_problem* pr, T** ptr, size_t count) {
  void* p = nullptr;
  const size_t bytes = count * sizeof(T);
  cudaError_t e = cudaMalloc(&p, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) return e;
  pr->shared->allocs.push_back(p);
  pr->bytes += bytes;
  *ptr = (T*)p;
  return cudaSuccess;
}

__global__ void k_mask_u(LatView lv, double2* u) {
  const size_t nn = (size_t)lv.nx * lv.ny;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < nn; n += (size_t)gridDim.x * blockDim.x) {
    const unsigned fm = lv.fix[n];
    if (fm) {
      double2 v = u[n];
      if (fm & 1u) v.x = 0.0;
      if (fm & 2u) v.y = 0.0;
      u[n] = v;
    }
  }
}
__global__ void k_d2f(const double* in, float* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void k_f2d(const float* in, double* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

int grid1d(size_t n) {
  size_t g = (n + 255) / 256;
  if (g > 8192) g = 8192;
  return g < 1 ? 1 : (int)g;
}

cudaMemcpyKind kind_in(int mem_kind) {
  return mem_kind == HMS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind kind_out(int mem_kind) {
  return mem_kind == HMS_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

size_t nnodes(const hms_problem* pr) { return (size_t)pr->lv.nx * pr->lv.ny; }
bool fp32(const hms_problem* pr) { return pr->precision == HMS_MIXED; }

// The factor of Eq. 8 (after the scaled band is built) and its per-block
// matrices, by the configured variant.
cudaError_t launch_factor_stage(hms_problem* pr, cudaStream_t s, const IterCtl* ctl) {
  if (pr->nd) return launch_nd_factor(s, pr->lv, pr->ndp, pr->ndd, pr->blk, pr->scale, pr->dropped, ctl);
  if (pr->two_sided) return launch_coarse_factor_2s(s, pr->n_c, pr->bw, pr->ts, pr->sband, pr->dropped, ctl);
  cudaError_t e = pr->cluster_factor
                      ? launch_coarse_factor_cl(s, pr->n_c, pr->bw, pr->lrow, pr->lcol, pr->dinv, pr->dropped, ctl)
                      : launch_coarse_factor(s, pr->n_c, pr->bw, pr->coarse_fp64, pr->lrow, pr->lcol, pr->dinv,
                                             pr->dropped, pr->big_stages == 0, ctl);
  if (e != cudaSuccess || pr->big_stages == 0) return e;
  return launch_coarse_blockinv(s, pr->n_c, pr->bw, pr->lcol, pr->lrow, pr->xinv, ctl);
}
// Solve q (0: of b, then of the refinement residual) with the factor.
cudaError_t launch_solve_stage(hms_problem* pr, cudaStream_t s, int q, const IterCtl* ctl) {
  const double* rhs = q == 0 ? pr->b : pr->res;
  // bit 0: the solve of b; bit 1: the last solve an update allows (the
  // kernels count the updates whose refinement had not converged before it)
  const int flags = (q == 0 ? 1 : 0) | (q == pr->nsolve - 1 ? 2 : 0);
  if (pr->nd)
    return launch_nd_solve(s, pr->n_c, pr->ndp, pr->ndd, rhs, pr->x, pr->scale, pr->a, pr->dropped, pr->cstat, flags,
                           ctl);
  if (pr->two_sided)
    return launch_coarse_solve_2s(s, pr->n_c, pr->ts, rhs, pr->x, pr->scale, pr->a, pr->dropped, pr->cstat, flags,
                                  ctl, pr->err);
  if (pr->big_stages > 0)
    return launch_coarse_solve_big(s, pr->big_stages, pr->n_c, pr->bw, pr->lcol, pr->lrow, pr->xinv, pr->dropped,
                                   rhs, pr->x, pr->scale, pr->a, pr->cstat, flags, ctl, pr->err);
  return launch_coarse_solve(s, pr->n_c, pr->bw, pr->coarse_fp64, pr->lcol, pr->lrow, pr->dinv, pr->dropped, rhs,
                             pr->x, pr->scale, pr->a, pr->cstat, flags, ctl, pr->err);
}

// The displacement-controlled relaxation of every set (K2), with per-set or
// class factors.
cudaError_t launch_relax_main(hms_problem* pr, cudaStream_t s, const IterCtl* ctl) {
  if (pr->cls)
    return launch_relax_class(s, pr->lv, pr->cpd, pr->f64, pr->f32, pr->r, pr->delta, pr->P, pr->yscratch, ctl,
                              pr->err, pr->relax_wait0);
  if (pr->relax_sched)
    return launch_relax_sched(s, pr->lv, pr->set_off, pr->f64, pr->f32, pr->r, pr->delta, pr->P, pr->yscratch, ctl,
                              pr->err, pr->sched_segs, pr->sched_cta, pr->sched_flags, pr->sched_grid,
                              pr->relax_wait0);
  return launch_relax(s, pr->lv, pr->set_off, pr->f64, pr->f32, pr->r, pr->delta, pr->P, pr->yscratch, ctl, pr->err,
                      pr->relax_threads, pr->relax_chunks, pr->relax_wait0);
}

// K_aa from the slots and the scaled system of Eq. 8 (scale, b, x = 0, drop
// flags): by blocks for nested dissection, else as a band.
cudaError_t launch_scaled_system(hms_problem* pr, cudaStream_t s, const IterCtl* ctl) {
  if (pr->nd) {
    cudaError_t e = launch_blocks_from_slots(s, pr->lv, pr->slots_base, pr->slots_it, pr->blk, ctl);
    if (e != cudaSuccess) return e;
    return launch_blk_diag(s, pr->lv, pr->blk, pr->P, pr->scale, pr->b, pr->x, pr->dropped, pr->mode_mask, ctl);
  }
  cudaError_t e = launch_coarse_band_from_slots(s, pr->lv, pr->slots_base, pr->slots_it, pr->band, ctl);
  if (e != cudaSuccess) return e;
  return launch_coarse_scale(s, pr->n_c, pr->bw, pr->coarse_fp64, pr->band, pr->P, pr->sband, pr->lrow, pr->scale,
                             pr->b, pr->x, pr->dropped, pr->mode_mask, pr->lv.q, ctl);
}
// The FP64 refinement residual of Eq. 8, res = b - A x.
cudaError_t launch_refine_residual(hms_problem* pr, cudaStream_t s, const IterCtl* ctl) {
  if (pr->nd)
    return launch_blk_residual(s, pr->lv, pr->blk, pr->scale, pr->dropped, pr->b, pr->x, pr->res, pr->cstat, ctl);
  return launch_coarse_residual(s, pr->n_c, pr->bw, pr->sband, pr->b, pr->x, pr->dropped, pr->res, pr->cstat, ctl);
}

// The force-controlled relaxation of every set (Eqs. 15-17, force.cu) after the
// displacement-controlled one: r projected, the cut-free solve, delta^RF and
// the upper-level forces of the modes 10-12 (P[12 I + 9 .. 11]).
cudaError_t launch_force_relax(hms_problem* pr, cudaStream_t s, const IterCtl* ctl) {
  const LatView& lv = pr->lv;
  cudaError_t e = launch_force_in(s, lv, pr->r, pr->Mforce, pr->fixF, pr->rproj, ctl);
  if (e != cudaSuccess) return e;
  e = launch_relax(s, lv, pr->set_off, pr->f64F, pr->f32F, pr->rproj, pr->delta_rf, nullptr, pr->yscratch, ctl,
                   pr->err, pr->relax_threads, pr->relax_chunks, pr->relax_wait0);
  if (e != cudaSuccess) return e;
  return launch_force_out(s, lv, pr->delta_rf, fp32(pr), pr->Mforce, pr->r, pr->P, ctl);
}

// Launches of one iteration (the body of Fig. 3's loop); k = position in a batch.
cudaError_t launch_iteration(hms_problem* pr, cudaStream_t s, int k, cudaEvent_t* ev) {
  const LatView& lv = pr->lv;
  int ei = 0;
  auto mark = [&]() {
    if (ev) cudaEventRecord(ev[ei++], s);
  };
  cudaError_t e;
  mark();
  e = launch_update_residual(s, lv, pr->u[k & 1], pr->u[(k + 1) & 1], pr->p, pr->delta, fp32(pr), pr->a,
                             pr->r, pr->partials, pr->ticket, nullptr, pr->ctl, pr->hist, pr->hist_cap,
                             pr->delta_rf);
  if (e != cudaSuccess) return e;
  mark();
  e = launch_relax_main(pr, s, pr->ctl);
  if (e != cudaSuccess) return e;
  if (lv.q == NMODES_RF) {
    e = launch_force_relax(pr, s, pr->ctl);
    if (e != cudaSuccess) return e;
  }
  mark();
  e = launch_coarse_slots(s, lv, pr->delta, fp32(pr), false, pr->slots_it, pr->ctl, pr->delta_rf);
  if (e != cudaSuccess) return e;
  mark();
  e = launch_scaled_system(pr, s, pr->ctl);
  if (e != cudaSuccess) return e;
  mark();
  e = launch_factor_stage(pr, s, pr->ctl);
  if (e != cudaSuccess) return e;
  mark();
  for (int q = 0; q < pr->nsolve; ++q) {
    if (q > 0) {
      e = launch_refine_residual(pr, s, pr->ctl);
      if (e != cudaSuccess) return e;
      mark();
    }
    e = launch_solve_stage(pr, s, q, pr->ctl);
    if (e != cudaSuccess) return e;
    mark();
  }
  return cudaSuccess;
}

// kernel id of the interval between event i and i+1 of launch_iteration
int interval_kid(int i) {
  if (i == 0) return KID_UPDATE_RESIDUAL;
  if (i == 1) return KID_RELAX;
  if (i == 2) return KID_COARSE_ASSEMBLE;
  if (i == 3) return KID_COARSE_BAND;
  if (i == 4) return KID_COARSE_FACTOR;
  // then: solve, (residual, solve)*
  return ((i - 5) % 2 == 0) ? KID_COARSE_SOLVE : KID_COARSE_RESIDUAL;
}

hms_status build_graph(hms_problem* pr) {
  hms_context* c = pr->ctx;
  cudaStream_t s = c->stream;
  cudaGraph_t g = nullptr;
  CKC(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < pr->batch && e == cudaSuccess; ++k) e = launch_iteration(pr, s, k, nullptr);
  cudaError_t e2 = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(c, HMS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  CKC(c, e2);
  e = cudaGraphInstantiate(&pr->graph, g, 0);
  cudaGraphDestroy(g);
  CKC(c, e);
  return HMS_OK;
}

hms_status check_dev_err(hms_problem* pr) {
  int herr = 0;
  CKC(pr->ctx, cudaMemcpyAsync(&herr, pr->err, sizeof(int), cudaMemcpyDeviceToHost, pr->ctx->stream));
  CKC(pr->ctx, cudaStreamSynchronize(pr->ctx->stream));
  if (herr) {
    // reported once: the next call starts from a clear flag, and from clear
    // set flags of the balanced relaxation (an aborted launch may leave a
    // head's flag raised with its tail never run)
    CKC(pr->ctx, cudaMemsetAsync(pr->err, 0, sizeof(int), pr->ctx->stream));
    if (pr->sched_flags)
      CKC(pr->ctx, cudaMemsetAsync(pr->sched_flags, 0, (size_t)pr->lv.M * sizeof(int), pr->ctx->stream));
    CKC(pr->ctx, cudaStreamSynchronize(pr->ctx->stream));
  }
  if (herr & DEVERR_NOT_SPD) return fail(pr->ctx, HMS_ERR_NOT_SPD, "non-positive pivot in a local factorisation");
  if (herr & DEVERR_TIMEOUT) return fail(pr->ctx, HMS_ERR_TIMEOUT, "a bounded device wait gave up");
  return HMS_OK;
}

// Upper-level factor precision and substitution of a problem whose lv, n_c,
// bw and precision are set: FP64 for degenerate set shapes (one- or
// two-node-wide tiles give ill-conditioned upper-level systems), else FP32
// with FP64 refinement: two-sided on two SMs for long systems (auto or
// coarse_factor = 5), else solved by 64-row blocks with inverted diagonal
// blocks when that fits in shared memory (coarse_factor = 3 keeps the 16-row
// solve).  False if the band does not fit one CTA's shared memory.
bool choose_band(hms_problem* pr, const hms_options* o, int maxsm) {
  const LatView& lv = pr->lv;
  const int wmin = std::min(lv.sx, lv.nx - (lv.Mx - 1) * lv.sx);
  const int hmin = std::min(lv.sy, lv.ny - (lv.My - 1) * lv.sy);
  const bool degenerate = std::min(wmin, hmin) <= 2;
  auto fits = [&](bool f64) {
    return coarse_factor_smem_bytes(pr->n_c, pr->bw, f64) + 1024 <= (size_t)maxsm &&
           coarse_solve_smem_bytes(pr->n_c, pr->bw, f64) + 1024 <= (size_t)maxsm;
  };
  const int big = coarse_big_stages(pr->n_c, pr->bw, maxsm);
  const bool cl_fits = big > 0 && coarse_factor_cl_smem_bytes(pr->n_c, pr->bw) + 4096 <= (size_t)maxsm;
  if (o->coarse_factor == 2) pr->coarse_fp64 = true;
  else if (o->coarse_factor == 1 || o->coarse_factor >= 3) pr->coarse_fp64 = false;
  else pr->coarse_fp64 = degenerate && fits(true);
  if (pr->coarse_fp64) {
    if (!fits(true)) return false;
    pr->big_stages = 0;
    pr->cluster_factor = false;
    return true;
  }
  // FP32: one SM where the window fits (the block solve unless coarse_factor
  // = 3), else, or with coarse_factor = 1, a cluster of SMs with the block solve
  const bool one_fits = fits(false);
  if (o->coarse_factor == 3) {
    if (!one_fits) return false;
    pr->big_stages = 0;
    pr->cluster_factor = false;
    return true;
  }
  // two-sided: where the split exists and both CTAs' shared memory fits; by
  // default only for systems at least three bands long (a shorter chain
  // gains less than the separator's extra factor costs)
  pr->two_sided = false;
  if (o->coarse_factor == 0 || o->coarse_factor == 5) {
    int m0, m1, s;
    if (coarse_two_sided_split(pr->n_c, pr->bw, &m0, &m1, &s) &&
        (o->coarse_factor == 5 || pr->n_c >= 3 * (pr->bw + 1)) &&
        coarse_two_sided_factor_smem(m0, m1, s) + 1024 <= (size_t)maxsm) {
      const int st = coarse_two_sided_stages(m0, m1, s, maxsm);
      if (st > 0) {
        pr->two_sided = true;
        pr->cluster_factor = false;
        pr->big_stages = 0;
        pr->ts = TwoSided();
        pr->ts.m[0] = m0;
        pr->ts.m[1] = m1;
        pr->ts.s = s;
        pr->ts.stages = st;
        return true;
      }
    }
    if (o->coarse_factor == 5) return false;
  }
  if (o->coarse_factor == 4) pr->cluster_factor = false;
  else pr->cluster_factor = cl_fits && (o->coarse_factor == 1 || !one_fits);
  if (!pr->cluster_factor && !one_fits) return false;
  pr->big_stages = big;
  return true;
}

// The supports of a lattice description, per node (bit 0: x, bit 1: y).
std::vector<uint8_t> fix_pattern(const hms_lattice_desc* d) {
  const size_t nn = (size_t)d->nx * d->ny;
  std::vector<uint8_t> fm(nn, 0);
  if (d->fixed) {
    for (size_t n = 0; n < nn; ++n) fm[n] = (uint8_t)((d->fixed[2 * n] ? 1 : 0) | (d->fixed[2 * n + 1] ? 2 : 0));
  } else if (d->fix_bottom_edge) {
    for (int i = 0; i < d->nx; ++i) fm[i] = 3;
  }
  return fm;
}

// Classes of sets with the same k^Inner under a uniform bar stiffness (the
// relaxation with class factors, relax_class.cu): the same width and height,
// parity of the first row, lattice edges touched and constrained DOFs.  Per
// class: the offset and shape of its grouped factor and its first set (the one
// factored); the sets class by class in index order; and batches of ts sets of
// one class, one CTA each.
struct ClassPlanHost {
  std::vector<ClassInfo> info;
  std::vector<int> rep, sets;
  std::vector<ClassItem> items;
  long long fac_elems = 0;
  int nb8max = 0, hmax = 0;
  size_t slot_elems = 0;
};
void class_plan_build(const LatView& lv, const std::vector<uint8_t>& fix, int ts, ClassPlanHost* P) {
  std::map<std::array<int, 7>, std::vector<int>> by_key;
  std::vector<std::vector<int>> members;
  for (int I = 0; I < lv.M; ++I) {
    const int i0 = (I % lv.Mx) * lv.sx, j0 = (I / lv.Mx) * lv.sy;
    const int w = std::min(lv.sx, lv.nx - i0), h = std::min(lv.sy, lv.ny - j0);
    const std::array<int, 7> key = {w, h, j0 & 1, i0 == 0, i0 + w == lv.nx, j0 == 0, j0 + h == lv.ny};
    std::vector<int>& ids = by_key[key];
    int cls = -1;
    for (int c : ids) {
      const int R = P->rep[c];
      const int ri0 = (R % lv.Mx) * lv.sx, rj0 = (R / lv.Mx) * lv.sy;
      bool same = true;
      for (int jj = 0; jj < h && same; ++jj)
        same = std::memcmp(&fix[(size_t)(j0 + jj) * lv.nx + i0], &fix[(size_t)(rj0 + jj) * lv.nx + ri0], w) == 0;
      if (same) {
        cls = c;
        break;
      }
    }
    if (cls < 0) {
      cls = (int)members.size();
      members.emplace_back();
      P->rep.push_back(I);
      ids.push_back(cls);
      ClassInfo ci;
      ci.off = 0;
      ci.w = w;
      ci.h = h;
      P->info.push_back(ci);
    }
    members[cls].push_back(I);
  }
  for (size_t c = 0; c < members.size(); ++c) {
    ClassInfo& ci = P->info[c];
    const int nb = 2 * ci.w;
    ci.off = P->fac_elems;
    P->fac_elems += class_factor_size(nb, ci.h);
    P->nb8max = std::max(P->nb8max, (nb + 7) / 8 * 8);
    P->hmax = std::max(P->hmax, ci.h);
    for (int k = 0; k < 4; ++k) P->slot_elems = std::max(P->slot_elems, (size_t)grp_size(k, nb));
    const int first = (int)P->sets.size();
    const int cnt = (int)members[c].size();
    P->sets.insert(P->sets.end(), members[c].begin(), members[c].end());
    for (int b = 0; b < cnt; b += ts) {
      ClassItem it;
      it.cls = (int)c;
      it.first = first + b;
      it.count = std::min(ts, cnt - b);
      it.pad = 0;
      P->items.push_back(it);
    }
  }
}

// Nested dissection over the set grid (coarse_nd.cu): the plan of fronts, if
// every front fits the factor kernel's shared memory.
bool choose_nd(hms_problem* pr, int maxsm) {
  pr->coarse_fp64 = false;
  pr->two_sided = false;
  pr->cluster_factor = false;
  pr->big_stages = 0;
  pr->nd = false;
  if (!nd_plan_build(pr->lv, &pr->ndp) || !nd_plan_smem(&pr->ndp, maxsm)) return false;
  pr->nd = true;
  return true;
}

// The factor of Eq. 8: coarse_factor = 6 is nested dissection; otherwise the
// band factors of choose_band, and with coarse_factor = 0 nested dissection
// where no band factor fits (set grids wider than one SM's band window).
bool choose_coarse(hms_problem* pr, const hms_options* o, int maxsm) {
  pr->nd = false;
  if (o->coarse_factor == 6) return choose_nd(pr, maxsm);
  if (choose_band(pr, o, maxsm)) return true;
  return o->coarse_factor == 0 && choose_nd(pr, maxsm);
}

}  // namespace

namespace hms {
cudaError_t launch_mask_u(cudaStream_t s, const LatView& lv, double2* u) {
  k_mask_u<<<grid1d(nnodes_of(lv)), 256, 0, s>>>(lv, u);
  return cudaGetLastError();
}
}  // namespace hms

static std::string g_create_err;  // message of the last failed hms_context_create

extern "C" {

hms_status hms_context_create(int32_t device, hms_context** out) {
  if (!out) return HMS_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || device < 0 || device >= ndev) {
    g_create_err = std::string("no CUDA device ") + std::to_string(device) + ": " + cudaGetErrorString(ce);
    return HMS_ERR_ARG;
  }
  hms_context* c = new hms_context();
  c->device = device;
  if ((ce = cudaSetDevice(device)) != cudaSuccess) {
    g_create_err = std::string("cudaSetDevice: ") + cudaGetErrorString(ce);
    delete c;
    return HMS_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device);
  int maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = configure_setup(maxsm);
  if (e == cudaSuccess) e = configure_relax(maxsm);
  if (e == cudaSuccess) e = configure_relax_class(maxsm);
  if (e == cudaSuccess) e = configure_coarse_assemble(maxsm);
  if (e == cudaSuccess) e = configure_coarse_solve(maxsm);
  if (e == cudaSuccess) e = configure_coarse_factor_cl(maxsm);
  if (e == cudaSuccess) e = configure_coarse_nd(maxsm);
  if (e != cudaSuccess) {
    g_create_err = std::string("context setup: ") + cudaGetErrorString(e);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return HMS_ERR_CUDA;
  }
  *out = c;
  return HMS_OK;
}

void hms_context_destroy(hms_context* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamDestroy(c->stream);
  for (cudaStream_t s : c->pool) cudaStreamDestroy(s);
  delete c;
}

void* hms_context_stream(hms_context* c) { return c ? (void*)c->stream : nullptr; }
const char* hms_last_error(hms_context* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

void hms_problem_destroy(hms_problem* pr) {
  if (!pr) return;
  cudaSetDevice(pr->ctx->device);
  cudaStreamSynchronize(pr->ctx->stream);
  if (pr->graph) cudaGraphExecDestroy(pr->graph);
  for (void* p : pr->allocs) cudaFree(p);
  if (pr->ctl_host) cudaFreeHost(pr->ctl_host);
  if (pr->shared && --pr->shared->refs == 0) {
    for (void* p : pr->shared->allocs) cudaFree(p);
    delete pr->shared;
  }
  delete pr;
}

static cudaError_t alloc_instance(hms_problem* pr);
static cudaError_t setup_relax_sched(hms_problem* pr, bool* ok);

hms_status hms_problem_clone(hms_problem* src, hms_problem** out) {
  if (!src || !out) return HMS_ERR_ARG;
  *out = nullptr;
  hms_context* c = src->ctx;
  CKC(c, cudaSetDevice(c->device));
  hms_problem* pr = new hms_problem();
  pr->ctx = c;
  pr->shared = src->shared;
  ++src->shared->refs;
  pr->lv = src->lv;
  pr->precision = src->precision;
  pr->nsolve = src->nsolve;
  pr->batch = src->batch;
  pr->profile = src->profile;
  pr->max_iter = src->max_iter;
  pr->mode_mask = src->mode_mask;
  pr->record_history = src->record_history;
  pr->relax_wait0 = src->relax_wait0;
  pr->coarse_fp64 = src->coarse_fp64;
  pr->tol = src->tol;
  pr->n_c = src->n_c;
  pr->bw = src->bw;
  pr->big_stages = src->big_stages;
  pr->cluster_factor = src->cluster_factor;
  pr->relax_threads = src->relax_threads;
  pr->relax_chunks = src->relax_chunks;
  pr->relax_sched = src->relax_sched;
  pr->two_sided = src->two_sided;
  pr->nd = src->nd;
  pr->ndp = src->ndp;
  pr->ts = TwoSided();
  pr->ts.m[0] = src->ts.m[0];
  pr->ts.m[1] = src->ts.m[1];
  pr->ts.s = src->ts.s;
  pr->ts.stages = src->ts.stages;
  pr->kbar = src->kbar;
  pr->fix = src->fix;
  pr->rep = src->rep;
  pr->set_off = src->set_off;
  pr->f64 = src->f64;
  pr->f32 = src->f32;
  pr->cls = src->cls;
  pr->cpd = src->cpd;
  pr->f64F = src->f64F;
  pr->f32F = src->f32F;
  pr->fixF = src->fixF;
  pr->Mforce = src->Mforce;
  pr->slots_base = src->slots_base;
  cudaError_t e = alloc_instance(pr);
  if (e == cudaSuccess && pr->relax_sched) {
    bool ok = false;  // the clone's own flags (same plan)
    e = setup_relax_sched(pr, &ok);
    if (e == cudaSuccess && !ok) e = cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    const hms_status st = fail(c, e == cudaErrorMemoryAllocation ? HMS_ERR_OOM : HMS_ERR_CUDA,
                               std::string("hms_problem_clone: ") + cudaGetErrorString(e));
    hms_problem_destroy(pr);
    return st;
  }
  if (!pr->profile) {
    const hms_status st = build_graph(pr);
    if (st != HMS_OK) {
      hms_problem_destroy(pr);
      return st;
    }
  }
  *out = pr;
  return HMS_OK;
}

size_t hms_problem_device_bytes(const hms_problem* pr) { return pr ? pr->bytes : 0; }
int32_t hms_problem_relax_threads(const hms_problem* pr) { return pr ? pr->relax_threads : 0; }
int32_t hms_problem_relax_copies(const hms_problem* pr) { return pr ? pr->relax_chunks : 0; }
int32_t hms_problem_relax_balanced(const hms_problem* pr) { return pr && pr->relax_sched ? 1 : 0; }

int32_t hms_set_classes(const hms_lattice_desc* d, int32_t* class_out, int32_t cap) {
  if (!d || !class_out || d->ea || d->nx < 2 || d->ny < 2 || d->set_sx < 1 || d->set_sx > MAX_SX || d->set_sy < 1)
    return -1;
  LatView lv{};
  lv.nx = d->nx;
  lv.ny = d->ny;
  lv.sx = d->set_sx;
  lv.sy = d->set_sy;
  lv.Mx = (lv.nx + lv.sx - 1) / lv.sx;
  lv.My = (lv.ny + lv.sy - 1) / lv.sy;
  if ((long long)lv.Mx * lv.My > cap) return -1;
  lv.M = lv.Mx * lv.My;
  ClassPlanHost P;
  class_plan_build(lv, fix_pattern(d), 1, &P);  // one set per item
  for (const ClassItem& it : P.items) class_out[P.sets[it.first]] = it.cls;
  return (int32_t)P.info.size();
}

int32_t hms_nd_plan(int32_t mx, int32_t my, int32_t* nodes_out, int32_t node_cap, int32_t* sets_out,
                    int32_t sets_cap) {
  if (mx < 1 || my < 1 || (long long)mx * my > (1LL << 24) || !nodes_out || !sets_out) return -1;
  LatView lv{};
  lv.Mx = mx;
  lv.My = my;
  lv.M = mx * my;
  NDPlanHost P;
  if (!nd_plan_build(lv, &P)) return -1;
  if ((long long)P.nodes.size() > node_cap || (long long)P.sets.size() > sets_cap) return -1;
  for (size_t k = 0; k < P.nodes.size(); ++k) {
    const NDNode& d = P.nodes[k];
    int32_t* o = nodes_out + 6 * k;
    o[0] = d.ns;
    o[1] = d.nb;
    o[2] = d.s_off;
    o[3] = d.nchild;
    o[4] = d.nchild > 0 ? d.child[0] : -1;
    o[5] = d.nchild > 1 ? d.child[1] : -1;
  }
  for (size_t q = 0; q < P.sets.size(); ++q) sets_out[q] = P.sets[q];
  return (int32_t)P.nodes.size();
}

int32_t hms_relax_schedule(int32_t nx, int32_t ny, int32_t set_sx, int32_t set_sy, int32_t ctas,
                           int32_t* segs_out, int32_t cap, int32_t* cta_out) {
  if (nx < 2 || ny < 2 || set_sx < 1 || set_sx > MAX_SX || set_sy < 1 || ctas < 1 || cap < 0 || !cta_out)
    return -1;
  LatView lv{};
  lv.nx = nx;
  lv.ny = ny;
  lv.sx = set_sx;
  lv.sy = set_sy;
  lv.Mx = (nx + set_sx - 1) / set_sx;
  lv.My = (ny + set_sy - 1) / set_sy;
  if ((long long)lv.Mx * lv.My > (1LL << 30)) return -1;
  lv.M = lv.Mx * lv.My;
  lv.ov = 0;
  std::vector<RelaxSeg> segs;
  std::vector<int> cta;
  if (!relax_sched_plan(lv, ctas, segs, cta)) return 0;
  if ((long long)segs.size() > cap || !segs_out) return -1;
  for (size_t k = 0; k < segs.size(); ++k) {
    segs_out[3 * k] = segs[k].I;
    segs_out[3 * k + 1] = segs[k].o0;
    segs_out[3 * k + 2] = segs[k].o1;
  }
  for (size_t g = 0; g < cta.size(); ++g) cta_out[g] = cta[g];
  return (int32_t)segs.size();
}
double hms_problem_setup_ms(const hms_problem* pr) { return pr ? (double)pr->setup_ms : 0.0; }

// The per-instance buffers of a problem whose configuration (lv, n_c, bw,
// precision, coarse choice, max_iter) is set: iteration state, upper-level
// system and control block.
static cudaError_t alloc_instance(hms_problem* pr) {
#define CKI(x)                        \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)
  const LatView& lv = pr->lv;
  cudaStream_t s = pr->ctx->stream;
  const size_t nn = (size_t)lv.nx * lv.ny;
  CKI(palloc(pr, &pr->u[0], nn));
  CKI(palloc(pr, &pr->u[1], nn));
  CKI(palloc(pr, &pr->p, nn));
  CKI(palloc(pr, &pr->r, nn));
  if (fp32(pr)) {
    float2* dl;
    CKI(palloc(pr, &dl, nn));
    pr->delta = dl;
    CKI(cudaMemsetAsync(dl, 0, nn * sizeof(float2), s));
  } else {
    double2* dl;
    CKI(palloc(pr, &dl, nn));
    pr->delta = dl;
    CKI(cudaMemsetAsync(dl, 0, nn * sizeof(double2), s));
  }
  if (lv.q == NMODES_RF) {
    CKI(palloc(pr, &pr->rproj, nn));
    const size_t eb = fp32(pr) ? sizeof(float2) : sizeof(double2);
    unsigned char* df;
    CKI(palloc(pr, &df, nn * eb));
    pr->delta_rf = df;
    CKI(cudaMemsetAsync(df, 0, nn * eb, s));
  }
  {
    const size_t esz = fp32(pr) ? sizeof(float) : sizeof(double);
    const size_t ybytes = pr->cls ? (size_t)pr->cpd.nitems * pr->cpd.ystride * esz
                                  : (size_t)lv.M * relax_y_stride(lv) * esz;
    unsigned char* ys;
    CKI(palloc(pr, &ys, ybytes));
    pr->yscratch = ys;
  }
  const int n_c = pr->n_c, bw = pr->bw;
  const size_t nband = (size_t)n_c * (bw + 1);
  CKI(palloc(pr, &pr->a, n_c));
  CKI(palloc(pr, &pr->P, n_c));
  CKI(palloc(pr, &pr->slots_it, (size_t)lv.M * NSLOTS * slot_size(lv.q)));
  if (!pr->nd) {
    CKI(palloc(pr, &pr->band, nband));
    CKI(palloc(pr, &pr->sband, 2 * nband));
  }
  CKI(palloc(pr, &pr->scale, n_c));
  CKI(palloc(pr, &pr->b, n_c));
  CKI(palloc(pr, &pr->x, n_c));
  CKI(palloc(pr, &pr->res, n_c));
  if (pr->nd) {
    // the blocks of K_aa (the fronts' input), the plan and the fronts
    CKI(palloc(pr, &pr->blk, coarse_blocks_elems(lv)));
    const NDPlanHost& P = pr->ndp;
    NDPlanDev& D = pr->ndd;
    CKI(palloc(pr, &D.nodes, P.nodes.size()));
    CKI(palloc(pr, &D.sets, P.sets.size()));
    CKI(palloc(pr, &D.maps, std::max<size_t>(P.maps.size(), 1)));
    CKI(palloc(pr, &D.lvl_nodes, P.lvl_nodes.size()));
    CKI(cudaMemcpyAsync(D.nodes, P.nodes.data(), P.nodes.size() * sizeof(NDNode), cudaMemcpyHostToDevice, s));
    CKI(cudaMemcpyAsync(D.sets, P.sets.data(), P.sets.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    if (!P.maps.empty())
      CKI(cudaMemcpyAsync(D.maps, P.maps.data(), P.maps.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CKI(cudaMemcpyAsync(D.lvl_nodes, P.lvl_nodes.data(), P.lvl_nodes.size() * sizeof(int), cudaMemcpyHostToDevice,
                        s));
    CKI(palloc(pr, &D.bigs, std::max<size_t>(P.bigs.size(), 1)));
    CKI(palloc(pr, &D.inv, std::max<size_t>(P.inv.size(), 1)));
    CKI(palloc(pr, &D.dmask, 2 * std::max<size_t>(P.max_level_bigs, 1)));
    if (!P.bigs.empty())
      CKI(cudaMemcpyAsync(D.bigs, P.bigs.data(), P.bigs.size() * sizeof(NDBig), cudaMemcpyHostToDevice, s));
    if (!P.inv.empty())
      CKI(cudaMemcpyAsync(D.inv, P.inv.data(), P.inv.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CKI(palloc(pr, &D.F, P.f_elems));
    CKI(palloc(pr, &D.W, std::max<size_t>(P.w_elems, 1)));
    CKI(palloc(pr, &D.y, (size_t)n_c));
    CKI(palloc(pr, &D.xc, (size_t)n_c));
    CKI(cudaStreamSynchronize(s));  // the host vectors may change after return (clone copies)
  } else {
    // 8 bytes per entry (FP64 factor) plus the tail read by rounded-up bulk copies
    double *lc, *lr, *di;
    CKI(palloc(pr, &lc, nband + 16));
    CKI(palloc(pr, &lr, nband + 16));
    CKI(palloc(pr, &di, (size_t)coarse_dinv_size(n_c)));
    pr->lcol = lc;
    pr->lrow = lr;
    pr->dinv = di;
  }
  if (pr->big_stages > 0) CKI(palloc(pr, &pr->xinv, coarse_xinv_elems(n_c, pr->bw)));
  if (pr->two_sided) {
    for (int k = 0; k < 2; ++k) {
      const TwoSidedSizes z = coarse_two_sided_sizes(pr->ts.m[k], pr->ts.s);
      CKI(palloc(pr, &pr->ts.lin[k], z.lin));
      CKI(palloc(pr, &pr->ts.lcol[k], z.lcol));
      CKI(palloc(pr, &pr->ts.dinv[k], z.dinv));
      CKI(palloc(pr, &pr->ts.dropped[k], z.dropped));
      CKI(palloc(pr, &pr->ts.delta[k], z.delta));
      CKI(palloc(pr, &pr->ts.srow[k], z.srow));
      CKI(palloc(pr, &pr->ts.xinv[k], z.xinv));
    }
  }
  CKI(palloc(pr, &pr->dropped, n_c));
  CKI(palloc(pr, &pr->cstat, 4));
  CKI(cudaMemsetAsync(pr->cstat, 0, 4 * sizeof(unsigned long long), s));
  const size_t npart = (size_t)std::max(update_residual_blocks(lv), 1024) * 3;
  CKI(palloc(pr, &pr->partials, npart));
  CKI(palloc(pr, &pr->ticket, 1));
  CKI(cudaMemsetAsync(pr->ticket, 0, sizeof(unsigned), s));
  CKI(palloc(pr, &pr->ctl, 1));
  CKI(palloc(pr, &pr->err, 1));
  CKI(cudaMemsetAsync(pr->err, 0, sizeof(int), s));
  CKI(palloc(pr, &pr->norms, 4));
  if (pr->record_history) {
    pr->hist_cap = pr->max_iter + 1;
    CKI(palloc(pr, &pr->hist, 3 * (size_t)pr->hist_cap));
  } else {
    pr->hist_cap = 0;
    pr->hist = nullptr;
  }
  CKI(cudaMallocHost(&pr->ctl_host, sizeof(IterCtl)));
  CKI(cudaMemsetAsync(pr->a, 0, n_c * sizeof(double), s));

#undef CKI
  return cudaSuccess;
}

// The balanced relaxation schedule for this problem (relax.cu): the plan, its
// device copy and the per-set flags (per instance: clones run at the same
// time).  *ok = false where the schedule does not apply.
static cudaError_t setup_relax_sched(hms_problem* pr, bool* ok) {
  *ok = false;
  if (pr->cls) return cudaSuccess;
  int grid = 0;
  cudaError_t e = relax_sched_grid(pr->lv, fp32(pr), &grid);
  if (e != cudaSuccess || grid == 0) return e;
  std::vector<RelaxSeg> segs;
  std::vector<int> cta;
  if (!relax_sched_plan(pr->lv, grid, segs, cta)) return cudaSuccess;
  cudaStream_t s = pr->ctx->stream;
  if (!pr->sched_segs) {
    if ((e = palloc(pr, &pr->sched_segs, segs.size())) != cudaSuccess) return e;
    if ((e = palloc(pr, &pr->sched_cta, cta.size())) != cudaSuccess) return e;
    if ((e = palloc(pr, &pr->sched_flags, (size_t)pr->lv.M)) != cudaSuccess) return e;
  }
  if ((e = cudaMemcpyAsync(pr->sched_segs, segs.data(), segs.size() * sizeof(RelaxSeg), cudaMemcpyHostToDevice,
                           s)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(pr->sched_cta, cta.data(), cta.size() * sizeof(int), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(pr->sched_flags, 0, (size_t)pr->lv.M * sizeof(int), s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;  // the host vectors go out of scope
  pr->sched_grid = grid;
  *ok = true;
  return cudaSuccess;
}

// Relaxation launch shape by timing: the first problem of a (set width, set
// height, precision) on a context times one warm-up and three timed launches
// of each CTA size, copies per matrix and, where it applies, the balanced
// schedule on its own factors (r = 0; the kernel's time does not depend on the
// values) and the context keeps the fastest for that shape.  All candidates
// give bitwise the same results, so the choice only changes the time.
static cudaError_t autotune_relax(hms_problem* pr, int copies, bool try_sched) {
  hms_context* c = pr->ctx;
  const LatView& lv = pr->lv;
  bool sched_ok = false;
  if (try_sched && (copies == 0 || copies == 1)) {
    cudaError_t e = setup_relax_sched(pr, &sched_ok);
    if (e != cudaSuccess) return e;
  }
  // the relaxation region's overlap changes the factors' shapes and rules out
  // two copies per matrix, so it is part of the key; so is the set count
  // where the balanced schedule applies (its gain depends on it)
  const auto key = std::make_tuple(std::min(lv.sx, lv.nx), std::min(lv.sy, lv.ny), pr->precision * 10 + copies,
                                   lv.ov, sched_ok ? lv.M : 0);
  const auto it = c->relax_tuned.find(key);
  if (it != c->relax_tuned.end()) {
    pr->relax_threads = (it->second % 10000) / 10;
    pr->relax_chunks = it->second % 10;
    pr->relax_sched = it->second >= 10000;
    return cudaSuccess;
  }
  cudaStream_t s = c->stream;
  cudaError_t e = cudaMemsetAsync(pr->r, 0, nnodes(pr) * sizeof(double2), s);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  // candidates, each timed in two rounds (the smaller time counts) after a
  // warm-up, so that clocks ramping up from idle do not favour later ones
  // (threads, copies); copies 0 = the balanced schedule (256 threads, one copy)
  std::vector<std::pair<int, int>> cand;
  const int max_nc = copies != 0 ? copies : (relax_chunks_possible(lv, fp32(pr)) ? 2 : 1);
  for (int nc = copies != 0 ? copies : 1; nc <= max_nc; ++nc)
    for (int nt : {64, 128, 256}) cand.push_back({nt, nc});
  if (sched_ok) cand.push_back({256, 0});
  std::vector<float> tbest(cand.size(), 1e30f);
  auto run = [&](int nt, int nc) {
    if (nc == 0)
      return launch_relax_sched(s, lv, pr->set_off, pr->f64, pr->f32, pr->r, pr->delta, pr->P, pr->yscratch,
                                nullptr, pr->err, pr->sched_segs, pr->sched_cta, pr->sched_flags, pr->sched_grid);
    return launch_relax(s, lv, pr->set_off, pr->f64, pr->f32, pr->r, pr->delta, pr->P, pr->yscratch, nullptr,
                        pr->err, nt, nc);
  };
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = run(256, 1);
  for (int round = 0; round < 2 && e == cudaSuccess; ++round)
    for (size_t i = 0; i < cand.size() && e == cudaSuccess; ++i) {
      if ((e = run(cand[i].first, cand[i].second)) != cudaSuccess) break;
      if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
      for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = run(cand[i].first, cand[i].second);
      if (e != cudaSuccess || (e = cudaEventRecord(e1, s)) != cudaSuccess) break;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      tbest[i] = std::min(tbest[i], ms);
    }
  int best_nt = 256, best_nc = 1;
  float best = 1e30f;
  for (size_t i = 0; i < cand.size(); ++i)
    if (tbest[i] < best) best = tbest[i], best_nt = cand[i].first, best_nc = cand[i].second;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  pr->relax_threads = best_nt;
  pr->relax_chunks = best_nc == 0 ? 1 : best_nc;
  pr->relax_sched = best_nc == 0;
  c->relax_tuned[key] = (pr->relax_sched ? 10000 : 0) + best_nt * 10 + pr->relax_chunks;
  return cudaSuccess;
}

hms_status hms_problem_create(hms_context* c, const hms_lattice_desc* d, const hms_options* o,
                              hms_problem** out) {
  if (!c || !d || !o || !out) return HMS_ERR_ARG;
  *out = nullptr;
  if (d->nx < 2 || d->ny < 2) return fail(c, HMS_ERR_ARG, "nx, ny must be >= 2");
  if (!(d->bar_length > 0.0) || !std::isfinite(d->bar_length)) return fail(c, HMS_ERR_ARG, "bar_length must be > 0");
  if (d->set_sx < 1 || d->set_sx > MAX_SX || d->set_sy < 1)
    return fail(c, HMS_ERR_ARG, "set_sx must be in [1, 64] and set_sy >= 1");
  if (!d->ea && !(d->ea_uniform > 0.0)) return fail(c, HMS_ERR_ARG, "ea_uniform must be > 0");
  if (o->precision != HMS_FP64 && o->precision != HMS_MIXED) return fail(c, HMS_ERR_ARG, "bad precision");
  if (!(o->tol >= 0.0) || o->max_iter < 0) return fail(c, HMS_ERR_ARG, "bad tol / max_iter");
  if (o->coarse_solves < 0 || o->coarse_solves > 8) return fail(c, HMS_ERR_ARG, "coarse_solves must be in 0..8");
  if (o->coarse_factor < 0 || o->coarse_factor > 6) return fail(c, HMS_ERR_ARG, "coarse_factor must be in 0..6");
  if (o->relax_threads != 0 && o->relax_threads != 64 && o->relax_threads != 128 && o->relax_threads != 256)
    return fail(c, HMS_ERR_ARG, "relax_threads must be 0, 64, 128 or 256");
  if (o->relax_copies < 0 || o->relax_copies > 2) return fail(c, HMS_ERR_ARG, "relax_copies must be 0, 1 or 2");
  if (o->relax_balance < 0 || o->relax_balance > 2) return fail(c, HMS_ERR_ARG, "relax_balance must be 0, 1 or 2");
  if (o->relax_balance == 2 && ((o->relax_threads != 0 && o->relax_threads != 256) || o->relax_copies == 2 ||
                                o->relax_overlap != 0 || o->class_factors != 0))
    return fail(c, HMS_ERR_ARG, "relax_balance = 2 runs 256 threads, one copy per matrix, no overlap, per-set factors");
  // the region width in 64 bits: set_sx + 2 relax_overlap may exceed INT_MAX
  const long long rw = std::min((long long)d->nx, (long long)d->set_sx + 2LL * (long long)o->relax_overlap);
  if (o->relax_overlap < 0 || rw > MAX_RX)
    return fail(c, HMS_ERR_ARG, "relax_overlap must be >= 0 with min(nx, set_sx + 2 relax_overlap) <= 80");
  if (o->precision == HMS_FP64 && rw > MAX_SX)
    return fail(c, HMS_ERR_ARG, "the FP64 relaxation takes regions up to 64 nodes wide");
  if ((o->mode_mask >> NMODES_RF) != 0u) return fail(c, HMS_ERR_ARG, "mode_mask has bits above mode 12");
  if (o->record_history != 0 && o->record_history != 1) return fail(c, HMS_ERR_ARG, "record_history must be 0 or 1");
  if (o->class_factors != 0 && o->class_factors != 1) return fail(c, HMS_ERR_ARG, "class_factors must be 0 or 1");
  const bool force = (o->mode_mask >> NMODES) != 0u;  // modes 10-12: the force-controlled relaxation
  if (o->class_factors && (d->ea || o->relax_overlap != 0 || force))
    return fail(c, HMS_ERR_ARG, "class_factors needs a uniform EA (ea = NULL), relax_overlap = 0 and the nine "
                                "displacement-controlled modes");
  if (force) {
    const int wr = d->nx - ((d->nx + d->set_sx - 1) / d->set_sx - 1) * d->set_sx;
    const int hr = d->ny - ((d->ny + d->set_sy - 1) / d->set_sy - 1) * d->set_sy;
    if (std::min(std::min(d->set_sx, d->nx), wr) < 2 || std::min(std::min(d->set_sy, d->ny), hr) < 2)
      return fail(c, HMS_ERR_ARG, "the force-controlled modes need set tiles of at least 2 x 2 nodes (a cut-free "
                                  "one-row or one-column set is a mechanism)");
    if (o->relax_overlap != 0)
      return fail(c, HMS_ERR_ARG, "the force-controlled modes take no extended relaxation region");
  }
  CKC(c, cudaSetDevice(c->device));
  cudaStream_t s = c->stream;

  hms_problem* pr = new hms_problem();
  pr->ctx = c;
  pr->shared = new SharedSetup();
  LatView& lv = pr->lv;
  lv.nx = d->nx;
  lv.ny = d->ny;
  lv.sx = d->set_sx;
  lv.sy = d->set_sy;
  lv.Mx = (d->nx + d->set_sx - 1) / d->set_sx;
  lv.My = (d->ny + d->set_sy - 1) / d->set_sy;
  lv.M = lv.Mx * lv.My;
  lv.ov = o->relax_overlap;
  lv.q = force ? NMODES_RF : NMODES;
  lv.L = d->bar_length;
  lv.k_u = d->ea ? 0.0 : d->ea_uniform / d->bar_length;
  pr->precision = o->precision;
  pr->nsolve = o->coarse_solves > 0 ? o->coarse_solves : (o->precision == HMS_FP64 ? 5 : 2);
  pr->batch = o->batch > 0 ? (o->batch + 1) / 2 * 2 : 16;
  pr->profile = o->profile;
  pr->tol = o->tol;
  pr->max_iter = o->max_iter;
  pr->mode_mask = o->mode_mask ? o->mode_mask : 0x1FFu;
  pr->record_history = o->record_history != 0;
  pr->n_c = lv.q * lv.M;
  pr->bw = coarse_bw(lv);

  int maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  if (relax_smem_bytes(lv, fp32(pr)) + 2048 > (size_t)maxsm) {
    delete pr;
    return fail(c, HMS_ERR_ARG, "set tile too large for the relaxation kernel's shared memory");
  }
  if (!choose_coarse(pr, o, maxsm)) {
    delete pr;
    return fail(c, HMS_ERR_ARG, "set grid too wide for the upper-level factorisations");
  }
  if (coarse_slots_smem(lv) > (size_t)maxsm) {
    delete pr;
    return fail(c, HMS_ERR_ARG, "set tile too large for the upper-level assembly");
  }

  auto bail = [&](cudaError_t e, const char* what) {
    hms_status st = fail(c, e == cudaErrorMemoryAllocation ? HMS_ERR_OOM : HMS_ERR_CUDA,
                         std::string(what) + ": " + cudaGetErrorString(e));
    hms_problem_destroy(pr);
    return st;
  };
#define CKP(x)                          \
  do {                                  \
    cudaError_t e_ = (x);               \
    if (e_ != cudaSuccess) return bail(e_, #x); \
  } while (0)

  const size_t nn = (size_t)lv.nx * lv.ny;
  std::vector<uint8_t> fix_host;   // the supports (kept for the force-controlled setup)
  std::vector<double2> rep_host;   // the sets' representing points
  // ---- lattice description ----
  {
    std::vector<uint8_t> fm = fix_pattern(d);
    CKP(salloc(pr, &pr->fix, nn));
    CKP(cudaMemcpy(pr->fix, fm.data(), nn, cudaMemcpyHostToDevice));
    lv.fix = pr->fix;
    fix_host.swap(fm);
  }
  if (d->ea) {
    std::vector<double> kb(3 * nn, 0.0);
    for (int j = 0; j < lv.ny; ++j)
      for (int i = 0; i < lv.nx; ++i) {
        const size_t n = (size_t)j * lv.nx + i;
        const int off = j & 1;
        const bool e_ok = i + 1 < lv.nx;
        const bool ne_ok = j + 1 < lv.ny && i + off < lv.nx;
        const bool nw_ok = j + 1 < lv.ny && i - 1 + off >= 0;
        const bool ok[3] = {e_ok, ne_ok, nw_ok};
        for (int dd = 0; dd < 3; ++dd) {
          const double ea = d->ea[dd * nn + n];
          if (ok[dd]) {
            if (!(ea > 0.0) || !std::isfinite(ea)) {
              hms_problem_destroy(pr);
              return fail(c, HMS_ERR_ARG, "EA must be finite and > 0 on every bar");
            }
            kb[dd * nn + n] = ea / lv.L;
          }
        }
      }
    CKP(salloc(pr, &pr->kbar, 3 * nn));
    CKP(cudaMemcpy(pr->kbar, kb.data(), 3 * nn * sizeof(double), cudaMemcpyHostToDevice));
    lv.kbar = pr->kbar;
  }
  ClassPlanHost cph;  // with class factors
  {
    // representing node of each set: the centroid of its nodes (Eq. 10)
    std::vector<double2> rp(lv.M);
    std::vector<long long> so(lv.M + 1, 0);
    for (int I = 0; I < lv.M; ++I) {
      const int Ix = I % lv.Mx, Iy = I / lv.Mx;
      const int i0 = Ix * lv.sx, j0 = Iy * lv.sy;
      const int w = std::min(lv.sx, lv.nx - i0), h = std::min(lv.sy, lv.ny - j0);
      int nodd = 0;
      for (int j = j0; j < j0 + h; ++j) nodd += (j & 1);
      rp[I].x = lv.L * ((double)i0 + 0.5 * (double)(w - 1) + 0.5 * (double)nodd / (double)h);
      rp[I].y = lv.L * SQ3_2 * ((double)j0 + 0.5 * (double)(h - 1));
      const Region R = relax_region(lv, I);  // the factor is the relaxation region's
      so[I + 1] = so[I] + set_factor_stride(2 * R.w, R.h);
    }
    CKP(salloc(pr, &pr->rep, lv.M));
    CKP(cudaMemcpy(pr->rep, rp.data(), lv.M * sizeof(double2), cudaMemcpyHostToDevice));
    lv.rep = pr->rep;
    rep_host = rp;
    size_t fsz = (size_t)so[lv.M];
    if (o->class_factors) {
      pr->cls = true;
      class_plan_build(lv, fix_host, class_sets_per_cta(fp32(pr)), &cph);
      if (relax_class_smem(cph.slot_elems, cph.nb8max, fp32(pr)) + 1024 > (size_t)maxsm) {
        hms_problem_destroy(pr);
        return fail(c, HMS_ERR_ARG, "set tile too large for the class-factor relaxation's shared memory");
      }
      ClassPlanDev& cp = pr->cpd;
      ClassInfo* info;
      ClassItem* items;
      int* sets;
      CKP(salloc(pr, &info, cph.info.size()));
      CKP(salloc(pr, &items, cph.items.size()));
      CKP(salloc(pr, &sets, cph.sets.size()));
      CKP(cudaMemcpy(info, cph.info.data(), cph.info.size() * sizeof(ClassInfo), cudaMemcpyHostToDevice));
      CKP(cudaMemcpy(items, cph.items.data(), cph.items.size() * sizeof(ClassItem), cudaMemcpyHostToDevice));
      CKP(cudaMemcpy(sets, cph.sets.data(), cph.sets.size() * sizeof(int), cudaMemcpyHostToDevice));
      cp.info = info;
      cp.items = items;
      cp.sets = sets;
      cp.nitems = (int)cph.items.size();
      cp.nb8max = cph.nb8max;
      cp.slot_elems = cph.slot_elems;
      cp.ystride = (long long)cph.hmax * cph.nb8max * class_sets_per_cta(fp32(pr));
      fsz = (size_t)cph.fac_elems;
    } else {
      CKP(salloc(pr, &pr->set_off, lv.M + 1));
      CKP(cudaMemcpy(pr->set_off, so.data(), (lv.M + 1) * sizeof(long long), cudaMemcpyHostToDevice));
    }
    if (fp32(pr)) {
      CKP(salloc(pr, &pr->f32, fsz));
      CKP(cudaMemsetAsync(pr->f32, 0, fsz * sizeof(float), s));
    } else {
      CKP(salloc(pr, &pr->f64, fsz));
      CKP(cudaMemsetAsync(pr->f64, 0, fsz * sizeof(double), s));
    }
    if (force) {
      // the cut-free factors have the same shapes; supports | pins and the projections
      std::vector<double> Mh;
      std::vector<uint8_t> fixF;
      if (!force_set_data(lv, fix_host, rep_host, Mh, fixF)) {
        hms_problem_destroy(pr);
        return fail(c, HMS_ERR_ARG, "a set's free rigid motions cannot be pinned at its corner nodes");
      }
      if (fp32(pr)) {
        CKP(salloc(pr, &pr->f32F, fsz));
        CKP(cudaMemsetAsync(pr->f32F, 0, fsz * sizeof(float), s));
      } else {
        CKP(salloc(pr, &pr->f64F, fsz));
        CKP(cudaMemsetAsync(pr->f64F, 0, fsz * sizeof(double), s));
      }
      CKP(salloc(pr, &pr->fixF, nn));
      CKP(cudaMemcpy(pr->fixF, fixF.data(), nn, cudaMemcpyHostToDevice));
      CKP(salloc(pr, &pr->Mforce, 9 * (size_t)lv.M));
      CKP(cudaMemcpy(pr->Mforce, Mh.data(), 9 * (size_t)lv.M * sizeof(double), cudaMemcpyHostToDevice));
    }
  }
  // ---- iteration buffers ----
  CKP(salloc(pr, &pr->slots_base, (size_t)lv.M * NSLOTS * slot_size(lv.q)));
  CKP(alloc_instance(pr));

  // ---- setup kernels: local factors (K2f) and the constant part of K_aa ----
  cudaEvent_t e0, e1;
  CKP(cudaEventCreate(&e0));
  CKP(cudaEventCreate(&e1));
  CKP(cudaEventRecord(e0, s));
  {
    const int grid = std::max(1, std::min(lv.M, c->nsm));
    double* scratch = nullptr;
    CKP(cudaMalloc(&scratch, (size_t)grid * b_size(MAX_NB) * sizeof(double)));
    cudaError_t e = cudaSuccess;
    if (pr->cls) {
      // each class's first set in the standard layout (FP64), then its grouped copy
      const int nc = (int)cph.rep.size();
      std::vector<long long> ro(nc + 1, 0);
      for (int t = 0; t < nc; ++t) ro[t + 1] = ro[t] + set_factor_stride(2 * cph.info[t].w, cph.info[t].h);
      double* std64 = nullptr;
      long long* ro_d = nullptr;
      int* reps_d = nullptr;
      e = cudaMalloc(&std64, (size_t)ro[nc] * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&ro_d, (nc + 1) * sizeof(long long));
      if (e == cudaSuccess) e = cudaMalloc(&reps_d, nc * sizeof(int));
      if (e == cudaSuccess) e = cudaMemcpy(ro_d, ro.data(), (nc + 1) * sizeof(long long), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(reps_d, cph.rep.data(), nc * sizeof(int), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemsetAsync(std64, 0, (size_t)ro[nc] * sizeof(double), s);
      if (e == cudaSuccess)
        e = launch_set_factor(s, lv, ro_d, std64, nullptr, scratch, std::max(1, std::min(nc, c->nsm)), pr->err, false,
                              reps_d, nc);
      for (int t = 0; t < nc && e == cudaSuccess; ++t)
        e = launch_group_factor(s, std64 + ro[t], 2 * cph.info[t].w, cph.info[t].h,
                                pr->f64 ? pr->f64 + cph.info[t].off : nullptr,
                                pr->f32 ? pr->f32 + cph.info[t].off : nullptr);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      cudaFree(std64);
      cudaFree(ro_d);
      cudaFree(reps_d);
    } else {
      e = launch_set_factor(s, lv, pr->set_off, pr->f64, pr->f32, scratch, grid, pr->err);
    }
    if (e == cudaSuccess && force) {
      LatView lvF = lv;  // the cut-free sets with their pinned DOFs marked as constrained
      lvF.fix = pr->fixF;
      e = launch_set_factor(s, lvF, pr->set_off, pr->f64F, pr->f32F, scratch, grid, pr->err, true);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(scratch);
    CKP(e);
  }
  CKP(launch_coarse_slots(s, lv, pr->delta, fp32(pr), true, pr->slots_base, nullptr, pr->delta_rf));
  CKP(cudaEventRecord(e1, s));
  CKP(cudaEventSynchronize(e1));
  cudaEventElapsedTime(&pr->setup_ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    hms_status st = check_dev_err(pr);
    if (st != HMS_OK) {
      hms_problem_destroy(pr);
      return st;
    }
  }
  if (o->relax_copies == 2 && !relax_chunks_possible(lv, fp32(pr))) {
    hms_problem_destroy(pr);
    return fail(c, HMS_ERR_ARG, "relax_copies = 2 needs the FP64 path and even set widths >= 6");
  }
  if (pr->cls) {
    pr->relax_threads = 256;  // the class-factor kernel's fixed shape
    pr->relax_chunks = 1;
  } else if (o->relax_balance == 2) {
    bool ok = false;
    CKP(setup_relax_sched(pr, &ok));
    if (!ok) {
      hms_problem_destroy(pr);
      return fail(c, HMS_ERR_ARG, "relax_balance = 2: the balanced schedule does not apply (more sets than SMs, "
                                  "none costing more than an SM's share)");
    }
    pr->relax_sched = true;
    pr->relax_threads = 256;
    pr->relax_chunks = 1;
  } else if (o->relax_threads != 0 && o->relax_copies != 0) {
    pr->relax_threads = o->relax_threads;
    pr->relax_chunks = o->relax_copies;
  } else if (o->relax_threads != 0) {
    pr->relax_threads = o->relax_threads;
    pr->relax_chunks = 1;
  } else {
    CKP(autotune_relax(pr, o->relax_copies, o->relax_balance == 0));
  }
  if (!pr->profile) {
    hms_status st = build_graph(pr);
    if (st != HMS_OK && pr->relax_sched && o->relax_balance == 0) {
      // a cooperative launch the graph would not take: one CTA per set
      cudaGetLastError();
      pr->relax_sched = false;
      st = build_graph(pr);
    }
    if (st != HMS_OK) {
      hms_problem_destroy(pr);
      return st;
    }
  }
#undef CKP
  *out = pr;
  return HMS_OK;
}

hms_status hms_solve(hms_problem* pr, int32_t nrhs, const double* loads, const double* u0, double* u_out,
                     double* hist, int32_t hist_cap, int32_t* iters, int32_t mem_kind) {
  if (!pr || nrhs < 0 || !loads || !u_out) return HMS_ERR_ARG;
  if (mem_kind != HMS_MEM_HOST && mem_kind != HMS_MEM_DEVICE) return HMS_ERR_ARG;
  hms_context* c = pr->ctx;
  CKC(c, cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  const size_t nn = nnodes(pr);
  const size_t vb = nn * sizeof(double2);
  hms_status result = HMS_OK;
  for (int k = 0; k < KID_COUNT; ++k) {
    pr->ktime[k] = 0.0;
    pr->klaunch[k] = 0;
  }
  std::vector<cudaEvent_t> ev;
  if (pr->profile) {
    ev.resize(8 + 2 * pr->nsolve);
    for (auto& e : ev) CKC(c, cudaEventCreate(&e));
  }
  pr->refine_cap_hits = 0;
  CKC(c, cudaMemsetAsync(pr->cstat + 3, 0, sizeof(unsigned long long), s));
  for (int q = 0; q < nrhs; ++q) {
    CKC(c, cudaMemcpyAsync(pr->p, loads + 2 * nn * q, vb, kind_in(mem_kind), s));
    if (u0) {
      CKC(c, cudaMemcpyAsync(pr->u[0], u0 + 2 * nn * q, vb, kind_in(mem_kind), s));
      CKC(c, launch_mask_u(s, pr->lv, pr->u[0]));
    } else {
      CKC(c, cudaMemsetAsync(pr->u[0], 0, vb, s));
    }
    IterCtl hc{};
    hc.max_iter = pr->max_iter;
    hc.tol = pr->tol;
    *pr->ctl_host = hc;
    CKC(c, cudaMemcpyAsync(pr->ctl, pr->ctl_host, sizeof(IterCtl), cudaMemcpyHostToDevice, s));
    CKC(c, launch_load_norms(s, pr->lv, pr->p, pr->partials, pr->ticket, pr->ctl));
    const int max_launch = pr->max_iter / pr->batch + 3;
    if (!pr->profile) {
      for (int g = 0; g < max_launch; ++g) {
        CKC(c, cudaGraphLaunch(pr->graph, s));
        CKC(c, cudaMemcpyAsync(pr->ctl_host, pr->ctl, sizeof(IterCtl), cudaMemcpyDeviceToHost, s));
        CKC(c, cudaStreamSynchronize(s));
        if (pr->ctl_host->done) break;
      }
    } else {
      for (int it = 0; it <= pr->max_iter + 1; ++it) {
        CKC(c, launch_iteration(pr, s, it, ev.data()));
        CKC(c, cudaMemcpyAsync(pr->ctl_host, pr->ctl, sizeof(IterCtl), cudaMemcpyDeviceToHost, s));
        CKC(c, cudaStreamSynchronize(s));
        const int nev = 7 + 2 * (pr->nsolve - 1);  // marks recorded by launch_iteration
        const bool ran_all = !pr->ctl_host->done;
        for (int i = 0; i + 1 < nev; ++i) {
          if (i > 0 && !ran_all) break;  // after convergence only K1 did work
          float ms = 0.f;
          cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
          pr->ktime[interval_kid(i)] += ms;
          pr->klaunch[interval_kid(i)] += 1;
        }
        if (pr->ctl_host->done) break;
      }
    }
    IterCtl fin = *pr->ctl_host;
    const double2* ucur = pr->u[fin.t & 1];
    CKC(c, cudaMemcpyAsync(u_out + 2 * nn * q, ucur, vb, kind_out(mem_kind), s));
    if (hist && hist_cap > 0) {
      const int rows = std::min(hist_cap, std::min(fin.t, pr->hist_cap));
      std::vector<double> h(3 * (size_t)hist_cap, NAN);
      CKC(c, cudaMemcpyAsync(h.data(), pr->hist, 3 * rows * sizeof(double), cudaMemcpyDeviceToHost, s));
      CKC(c, cudaStreamSynchronize(s));
      if (mem_kind == HMS_MEM_DEVICE)
        CKC(c, cudaMemcpyAsync(hist + 3 * (size_t)hist_cap * q, h.data(), 3 * hist_cap * sizeof(double),
                               cudaMemcpyHostToDevice, s));
      else
        std::memcpy(hist + 3 * (size_t)hist_cap * q, h.data(), 3 * hist_cap * sizeof(double));
    }
    if (iters) {
      const int32_t nit = fin.t > 0 ? fin.t - 1 : 0;
      if (mem_kind == HMS_MEM_DEVICE)
        CKC(c, cudaMemcpyAsync(iters + q, &nit, sizeof(int32_t), cudaMemcpyHostToDevice, s));
      else
        iters[q] = nit;
    }
    CKC(c, cudaStreamSynchronize(s));
    {
      hms_status st = check_dev_err(pr);
      if (st != HMS_OK) return st;
    }
    if (fin.status == 3) result = fail(c, HMS_ERR_NONFINITE, "non-finite residual norm");
    else if (fin.status != 1 && result == HMS_OK)
      result = fail(c, HMS_ERR_NO_CONVERGENCE, "max_iter reached before tol");
  }
  for (auto& e : ev) cudaEventDestroy(e);
  {
    unsigned long long hits = 0;
    CKC(c, cudaMemcpyAsync(&hits, pr->cstat + 3, sizeof(hits), cudaMemcpyDeviceToHost, s));
    CKC(c, cudaStreamSynchronize(s));
    pr->refine_cap_hits = (long long)hits;
  }
  return result;
}

int64_t hms_problem_refine_cap_hits(const hms_problem* pr) { return pr ? (int64_t)pr->refine_cap_hits : 0; }

hms_status hms_problem_set_relax_wait_limit(hms_problem* pr, int32_t spins) {
  if (!pr) return HMS_ERR_ARG;
  hms_context* c = pr->ctx;
  CKC(c, cudaSetDevice(c->device));
  CKC(c, cudaStreamSynchronize(c->stream));
  pr->relax_wait0 = spins < 0 ? -1 : spins;
  if (pr->graph) {
    CKC(c, cudaGraphExecDestroy(pr->graph));
    pr->graph = nullptr;
  }
  if (!pr->profile) return build_graph(pr);
  return HMS_OK;
}

int32_t hms_kernel_times(const hms_problem* pr, double* ms_total, int64_t* launches, int32_t n) {
  if (!pr) return 0;
  const int m = std::min((int)KID_COUNT, (int)n);
  for (int k = 0; k < m; ++k) {
    if (ms_total) ms_total[k] = pr->ktime[k];
    if (launches) launches[k] = pr->klaunch[k];
  }
  return m;
}

static hms_status solve_batch_streams(hms_context* c, int32_t count, hms_problem* const* problems,
                                      const int32_t* nrhs, const double* const* loads, double* const* u_out,
                                      int32_t* iters, int32_t mem_kind);
static hms_status solve_batch_lockstep(hms_context* c, int32_t count, hms_problem* const* problems,
                                       const int32_t* nrhs, const double* const* loads, double* const* u_out,
                                       int32_t* iters, int32_t mem_kind);

hms_status hms_context_set_batch_mode(hms_context* c, int32_t mode) {
  if (!c || mode < HMS_BATCH_AUTO || mode > HMS_BATCH_LOCKSTEP) return HMS_ERR_ARG;
  c->batch_mode = mode;
  return HMS_OK;
}

// Whether the lockstep engine can run these problems together.
static bool lockstep_applies(int32_t count, hms_problem* const* problems) {
  for (int i = 0; i < count; ++i) {
    const hms_problem* pr = problems[i];
    if (!pr || pr->profile || pr->coarse_fp64 || pr->cluster_factor || pr->two_sided || pr->big_stages <= 0 ||
        pr->lv.q != NMODES || pr->cls)
      return false;
    if (pr->precision != problems[0]->precision || pr->nsolve != problems[0]->nsolve) return false;
  }
  return true;
}

hms_status hms_solve_batch(hms_context* c, int32_t count, hms_problem* const* problems, const int32_t* nrhs,
                           const double* const* loads, double* const* u_out, int32_t* iters, int32_t mem_kind) {
  if (!c) return HMS_ERR_ARG;
  if (count > 0 && problems && c->batch_mode != HMS_BATCH_STREAMS) {
    bool ok = true;
    for (int i = 0; i < count && ok; ++i) ok = problems[i] && problems[i]->ctx == c;
    if (ok && lockstep_applies(count, problems))
      return solve_batch_lockstep(c, count, problems, nrhs, loads, u_out, iters, mem_kind);
    if (c->batch_mode == HMS_BATCH_LOCKSTEP)
      return fail(c, HMS_ERR_ARG, "hms_solve_batch: lockstep needs one precision, one coarse_solves and the "
                                  "one-SM FP32 factor with the block solve for every problem");
  }
  return solve_batch_streams(c, count, problems, nrhs, loads, u_out, iters, mem_kind);
}

static hms_status solve_batch_streams(hms_context* c, int32_t count, hms_problem* const* problems,
                                      const int32_t* nrhs, const double* const* loads, double* const* u_out,
                                      int32_t* iters, int32_t mem_kind) {
  if (!c) return HMS_ERR_ARG;
  if (count < 0 || (count > 0 && (!problems || !nrhs || !loads || !u_out)))
    return fail(c, HMS_ERR_ARG, "hms_solve_batch: count < 0 or missing arrays");
  if (mem_kind != HMS_MEM_HOST && mem_kind != HMS_MEM_DEVICE) return fail(c, HMS_ERR_ARG, "bad mem_kind");
  {
    std::vector<const hms_problem*> seen(problems, problems + count);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
      return fail(c, HMS_ERR_ARG, "hms_solve_batch: a problem appears twice");
  }
  for (int i = 0; i < count; ++i) {
    const hms_problem* pr = problems[i];
    if (!pr || pr->ctx != c) return fail(c, HMS_ERR_ARG, "hms_solve_batch: problem of another context");
    if (nrhs[i] < 0 || (nrhs[i] > 0 && (!loads[i] || !u_out[i])))
      return fail(c, HMS_ERR_ARG, "hms_solve_batch: bad nrhs / loads / u_out");
    if (pr->profile) return fail(c, HMS_ERR_ARG, "hms_solve_batch: profile-mode problems run alone");
  }
  CKC(c, cudaSetDevice(c->device));
  const int nstreams = std::max(1, std::min(count, 64));
  while ((int)c->pool.size() < nstreams) {
    cudaStream_t s = nullptr;
    CKC(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    c->pool.push_back(s);
  }
  std::vector<long long> ioff(count + 1, 0);
  for (int i = 0; i < count; ++i) ioff[i + 1] = ioff[i] + nrhs[i];
  std::vector<int32_t> its((size_t)ioff[count], 0);
  std::vector<int> q(count, 0), launches(count, 0), status(count, 1);
  std::vector<char> active(count, 0);
  auto stream_of = [&](int i) { return c->pool[i % nstreams]; };
  // load vector q[i] of problem i: loads in, u = 0, iteration control reset, ||p|| (as hms_solve)
  auto start = [&](int i) -> cudaError_t {
    hms_problem* pr = problems[i];
    cudaStream_t s = stream_of(i);
    const size_t nn = nnodes(pr), vb = nn * sizeof(double2);
    cudaError_t e = cudaMemcpyAsync(pr->p, loads[i] + 2 * nn * q[i], vb, kind_in(mem_kind), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(pr->u[0], 0, vb, s);
    IterCtl hc{};
    hc.max_iter = pr->max_iter;
    hc.tol = pr->tol;
    *pr->ctl_host = hc;
    if (e == cudaSuccess) e = cudaMemcpyAsync(pr->ctl, pr->ctl_host, sizeof(IterCtl), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_load_norms(s, pr->lv, pr->p, pr->partials, pr->ticket, pr->ctl);
    launches[i] = 0;
    active[i] = 1;
    return e;
  };
  // every problem moves at its own pace: when its last round has ended (its
  // event), its load vector is taken out or its next round is queued; the host
  // blocks only when no problem can move
  std::vector<cudaEvent_t> ev(count, nullptr);
  std::vector<char> inflight(count, 0);
  struct EvGuard {
    std::vector<cudaEvent_t>& e;
    ~EvGuard() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
    }
  } guard{ev};
  int live = 0;
  for (int i = 0; i < count; ++i)
    if (nrhs[i] > 0) {
      CKC(c, cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
      CKC(c, start(i));
      ++live;
    }
  while (live > 0) {
    bool moved = false;
    for (int i = 0; i < count; ++i) {
      if (!active[i]) continue;
      hms_problem* pr = problems[i];
      cudaStream_t st = stream_of(i);
      if (inflight[i]) {
        const cudaError_t qe = cudaEventQuery(ev[i]);
        if (qe == cudaErrorNotReady) continue;
        CKC(c, qe);
        inflight[i] = 0;
        const IterCtl fin = *pr->ctl_host;
        if (fin.done || launches[i] >= pr->max_iter / pr->batch + 3) {
          const size_t nn = nnodes(pr), vb = nn * sizeof(double2);
          CKC(c, cudaMemcpyAsync(u_out[i] + 2 * nn * q[i], pr->u[fin.t & 1], vb, kind_out(mem_kind), st));
          its[(size_t)(ioff[i] + q[i])] = fin.t > 0 ? fin.t - 1 : 0;
          if (fin.status == 3) status[i] = 3;
          else if (fin.status != 1 && status[i] == 1) status[i] = 2;
          moved = true;
          if (++q[i] < nrhs[i]) {
            CKC(c, start(i));
          } else {
            active[i] = 0;
            --live;
            continue;
          }
        }
      }
      CKC(c, cudaGraphLaunch(pr->graph, st));
      CKC(c, cudaMemcpyAsync(pr->ctl_host, pr->ctl, sizeof(IterCtl), cudaMemcpyDeviceToHost, st));
      CKC(c, cudaEventRecord(ev[i], st));
      inflight[i] = 1;
      ++launches[i];
      moved = true;
    }
    if (!moved)
      for (int i = 0; i < count; ++i)
        if (inflight[i]) {
          CKC(c, cudaEventSynchronize(ev[i]));
          break;
        }
  }
  for (int k = 0; k < nstreams; ++k) CKC(c, cudaStreamSynchronize(c->pool[k]));
  if (iters && ioff[count] > 0) {
    if (mem_kind == HMS_MEM_DEVICE)
      CKC(c, cudaMemcpy(iters, its.data(), its.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    else
      std::memcpy(iters, its.data(), its.size() * sizeof(int32_t));
  }
  hms_status result = HMS_OK;
  for (int i = 0; i < count; ++i) {
    const hms_status st = check_dev_err(problems[i]);
    if (st != HMS_OK) return st;
    if (status[i] == 3 && result == HMS_OK) result = fail(c, HMS_ERR_NONFINITE, "non-finite residual norm");
    if (status[i] == 2 && result == HMS_OK) result = fail(c, HMS_ERR_NO_CONVERGENCE, "max_iter reached before tol");
  }
  return result;
}

// ---- lockstep batches ----

// The convergence state of the running problems of a lockstep batch, gathered
// into one array for one device-to-host copy per round.
__global__ void k_gather_ctl(const BatchProb* __restrict__ P, const int* __restrict__ which, int n,
                             IterCtl* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = *P[which[i]].ctl;
}

static BatchProb batch_prob_of(const hms_problem* pr) {
  BatchProb q{};
  q.lv = pr->lv;
  q.u[0] = pr->u[0];
  q.u[1] = pr->u[1];
  q.p = pr->p;
  q.r = pr->r;
  q.delta = pr->delta;
  q.a = pr->a;
  q.P = pr->P;
  q.partials = pr->partials;
  q.ticket = pr->ticket;
  q.ctl = pr->ctl;
  q.hist = pr->hist;
  q.hist_cap = pr->hist_cap;
  q.err = pr->err;
  q.set_off = pr->set_off;
  q.f64 = pr->f64;
  q.f32 = pr->f32;
  q.yscratch = pr->yscratch;
  q.slots_base = pr->slots_base;
  q.slots_it = pr->slots_it;
  q.band = pr->band;
  q.sband = pr->sband;
  q.scale = pr->scale;
  q.b = pr->b;
  q.x = pr->x;
  q.res = pr->res;
  q.lrow = (float*)pr->lrow;
  q.lcol = (float*)pr->lcol;
  q.dinv = (float*)pr->dinv;
  q.xinv = pr->xinv;
  q.dropped = pr->dropped;
  q.cstat = pr->cstat;
  q.n_c = pr->n_c;
  q.bw = pr->bw;
  q.mode_mask = pr->mode_mask;
  return q;
}

// Work lists of the batched launches for the running problems, one after
// another in one array; off[k] .. off[k + 1] is kernel k's list.
enum BatchList { BL_K1 = 0, BL_SETS, BL_BAND, BL_DIAG, BL_DROPS, BL_SCALE, BL_ONE, BL_BLOCKINV, BL_CRES, BL_COUNT };

static void build_lists(const std::vector<hms_problem*>& probs, const std::vector<int>& run,
                        std::vector<BatchItem>& items, int off[BL_COUNT + 1]) {
  items.clear();
  for (int k = 0; k < BL_COUNT; ++k) {
    off[k] = (int)items.size();
    for (int i : run) {
      const hms_problem* pr = probs[i];
      const LatView& lv = pr->lv;
      auto grid = [&](int g) {
        for (int b = 0; b < g; ++b) items.push_back(BatchItem{i, b, 0, g, 1});
      };
      switch (k) {
        case BL_K1: {
          const int gx = update_residual_grid_x(lv), gy = update_residual_grid_y(lv);
          for (int by = 0; by < gy; ++by)
            for (int bx = 0; bx < gx; ++bx) items.push_back(BatchItem{i, bx, by, gx, gy});
          break;
        }
        case BL_SETS: grid(lv.M); break;
        case BL_BAND: grid(coarse_grid_for((size_t)pr->n_c * (pr->bw + 1))); break;
        case BL_DIAG: grid(coarse_grid_for((size_t)pr->n_c)); break;
        case BL_DROPS: grid(set_drops_blocks(lv.M)); break;
        case BL_SCALE: grid(coarse_grid_for((size_t)pr->n_c * (pr->bw + 1))); break;
        case BL_ONE: items.push_back(BatchItem{i, 0, 0, 1, 1}); break;
        case BL_BLOCKINV: {
          const int nb = (pr->n_c + 63) / 64;
          for (int K = 0; K < nb; ++K)
            for (int part = 0; part < 4; ++part) items.push_back(BatchItem{i, K, part, nb, 4});
          break;
        }
        case BL_CRES: grid(coarse_residual_blocks(pr->n_c)); break;
      }
    }
  }
  off[BL_COUNT] = (int)items.size();
}

static hms_status solve_batch_lockstep(hms_context* c, int32_t count, hms_problem* const* problems,
                                       const int32_t* nrhs, const double* const* loads, double* const* u_out,
                                       int32_t* iters, int32_t mem_kind) {
  if (count < 0 || (count > 0 && (!problems || !nrhs || !loads || !u_out)))
    return fail(c, HMS_ERR_ARG, "hms_solve_batch: count < 0 or missing arrays");
  if (mem_kind != HMS_MEM_HOST && mem_kind != HMS_MEM_DEVICE) return fail(c, HMS_ERR_ARG, "bad mem_kind");
  {
    std::vector<const hms_problem*> seen(problems, problems + count);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
      return fail(c, HMS_ERR_ARG, "hms_solve_batch: a problem appears twice");
  }
  for (int i = 0; i < count; ++i)
    if (nrhs[i] < 0 || (nrhs[i] > 0 && (!loads[i] || !u_out[i])))
      return fail(c, HMS_ERR_ARG, "hms_solve_batch: bad nrhs / loads / u_out");
  CKC(c, cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  std::vector<hms_problem*> probs(problems, problems + count);
  const bool f32 = fp32(probs[0]);
  const int nsolve = probs[0]->nsolve;
  // one launch shape for all: the relaxation CTA size gives the same bits at
  // any size; the block solve's pipeline depth does not change its arithmetic
  const int rthreads = probs[0]->relax_threads;
  int rchunks = 2;
  for (hms_problem* pr : probs) rchunks = std::min(rchunks, pr->relax_chunks);
  int stages = 3;
  size_t sm_relax = 0, sm_slots = 0, sm_factor = 0, sm_solve = 0;
  for (hms_problem* pr : probs) stages = std::min(stages, pr->big_stages);
  for (hms_problem* pr : probs) {
    sm_relax = std::max(sm_relax, relax_smem_bytes(pr->lv, f32, rchunks));
    sm_slots = std::max(sm_slots, coarse_slots_smem(pr->lv));
    sm_factor = std::max(sm_factor, coarse_factor_smem_bytes(pr->n_c, pr->bw, false));
    sm_solve = std::max(sm_solve, big_solve_smem_bytes(pr->n_c, pr->bw, stages));
  }
  // device copies of the problems' buffers, the running set and the work lists
  struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
      if (p) cudaFree(p);
    }
  } dprob, dwhich, ditems, dctl;
  std::vector<BatchProb> hp(count);
  for (int i = 0; i < count; ++i) hp[i] = batch_prob_of(probs[i]);
  CKC(c, cudaMalloc(&dprob.p, std::max<size_t>(1, count) * sizeof(BatchProb)));
  CKC(c, cudaMalloc(&dwhich.p, std::max<size_t>(1, count) * sizeof(int)));
  CKC(c, cudaMalloc(&dctl.p, std::max<size_t>(1, count) * sizeof(IterCtl)));
  CKC(c, cudaMemcpyAsync(dprob.p, hp.data(), count * sizeof(BatchProb), cudaMemcpyHostToDevice, s));
  IterCtl* hctl = nullptr;
  CKC(c, cudaMallocHost(&hctl, std::max<size_t>(1, count) * sizeof(IterCtl)));
  struct HostFree {
    IterCtl* p;
    ~HostFree() { cudaFreeHost(p); }
  } hctl_guard{hctl};
  const BatchProb* P = (const BatchProb*)dprob.p;

  std::vector<long long> ioff(count + 1, 0);
  for (int i = 0; i < count; ++i) ioff[i + 1] = ioff[i] + nrhs[i];
  std::vector<int32_t> its((size_t)ioff[count], 0);
  std::vector<int> q(count, 0), launches(count, 0), status(count, 1);
  auto start = [&](int i) -> cudaError_t {
    hms_problem* pr = probs[i];
    const size_t nn = nnodes(pr), vb = nn * sizeof(double2);
    cudaError_t e = cudaMemcpyAsync(pr->p, loads[i] + 2 * nn * q[i], vb, kind_in(mem_kind), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(pr->u[0], 0, vb, s);
    IterCtl hc{};
    hc.max_iter = pr->max_iter;
    hc.tol = pr->tol;
    *pr->ctl_host = hc;
    if (e == cudaSuccess) e = cudaMemcpyAsync(pr->ctl, pr->ctl_host, sizeof(IterCtl), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_load_norms(s, pr->lv, pr->p, pr->partials, pr->ticket, pr->ctl);
    launches[i] = 0;
    return e;
  };
  std::vector<int> run;
  for (int i = 0; i < count; ++i)
    if (nrhs[i] > 0) {
      CKC(c, start(i));
      run.push_back(i);
    }
  std::vector<BatchItem> items;
  int off[BL_COUNT + 1];
  size_t items_cap = 0;
  cudaGraphExec_t exec = nullptr;
  struct ExecGuard {
    cudaGraphExec_t& e;
    ~ExecGuard() {
      if (e) cudaGraphExecDestroy(e);
    }
  } exec_guard{exec};
  bool rebuild = true;
  while (!run.empty()) {
    if (rebuild) {
      build_lists(probs, run, items, off);
      if (items.size() > items_cap) {
        if (ditems.p) cudaFree(ditems.p);
        ditems.p = nullptr;
        items_cap = items.size();
        CKC(c, cudaMalloc(&ditems.p, items_cap * sizeof(BatchItem)));
      }
      CKC(c, cudaMemcpyAsync(ditems.p, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, s));
      CKC(c, cudaMemcpyAsync(dwhich.p, run.data(), run.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      const BatchItem* I = (const BatchItem*)ditems.p;
      auto L = [&](int k) { return I + off[k]; };
      auto N = [&](int k) { return off[k + 1] - off[k]; };
      if (exec) {
        cudaGraphExecDestroy(exec);
        exec = nullptr;
      }
      cudaGraph_t g = nullptr;
      CKC(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = cudaSuccess;
      for (int k = 0; k < 16 && e == cudaSuccess; ++k) {
        e = launch_batch_update_residual(s, f32, P, L(BL_K1), N(BL_K1), k);
        if (e == cudaSuccess) e = launch_batch_relax(s, f32, rthreads, rchunks, sm_relax, P, L(BL_SETS), N(BL_SETS));
        if (e == cudaSuccess) e = launch_batch_slots(s, f32, sm_slots, P, L(BL_SETS), N(BL_SETS));
        if (e == cudaSuccess) e = launch_batch_band(s, P, L(BL_BAND), N(BL_BAND));
        if (e == cudaSuccess) e = launch_batch_diag(s, P, L(BL_DIAG), N(BL_DIAG));
        if (e == cudaSuccess) e = launch_batch_set_drops(s, P, L(BL_DROPS), N(BL_DROPS));
        if (e == cudaSuccess) e = launch_batch_scale_band(s, P, L(BL_SCALE), N(BL_SCALE));
        if (e == cudaSuccess) e = launch_batch_factor(s, sm_factor, P, L(BL_ONE), N(BL_ONE));
        if (e == cudaSuccess) e = launch_batch_blockinv(s, P, L(BL_BLOCKINV), N(BL_BLOCKINV));
        for (int qq = 0; qq < nsolve && e == cudaSuccess; ++qq) {
          if (qq > 0) e = launch_batch_coarse_residual(s, P, L(BL_CRES), N(BL_CRES));
          if (e == cudaSuccess) e = launch_batch_solve(s, stages, sm_solve, P, L(BL_ONE), N(BL_ONE), qq == 0);
        }
      }
      const cudaError_t ee = cudaStreamEndCapture(s, &g);
      if (e == cudaSuccess) e = ee;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
      if (g) cudaGraphDestroy(g);
      CKC(c, e);
      rebuild = false;
    }
    CKC(c, cudaGraphLaunch(exec, s));
    const int nr = (int)run.size();
    k_gather_ctl<<<(nr + 127) / 128, 128, 0, s>>>(P, (const int*)dwhich.p, nr, (IterCtl*)dctl.p);
    CKC(c, cudaGetLastError());
    CKC(c, cudaMemcpyAsync(hctl, dctl.p, nr * sizeof(IterCtl), cudaMemcpyDeviceToHost, s));
    CKC(c, cudaStreamSynchronize(s));
    std::vector<int> next;
    for (int r = 0; r < nr; ++r) {
      const int i = run[r];
      hms_problem* pr = probs[i];
      ++launches[i];
      const IterCtl fin = hctl[r];
      if (fin.done || launches[i] >= pr->max_iter / pr->batch + 3) {
        const size_t nn = nnodes(pr), vb = nn * sizeof(double2);
        CKC(c, cudaMemcpyAsync(u_out[i] + 2 * nn * q[i], pr->u[fin.t & 1], vb, kind_out(mem_kind), s));
        its[(size_t)(ioff[i] + q[i])] = fin.t > 0 ? fin.t - 1 : 0;
        if (fin.status == 3) status[i] = 3;
        else if (fin.status != 1 && status[i] == 1) status[i] = 2;
        if (++q[i] < nrhs[i]) {
          CKC(c, start(i));
          next.push_back(i);
        } else {
          rebuild = true;
        }
      } else {
        next.push_back(i);
      }
    }
    run.swap(next);
  }
  CKC(c, cudaStreamSynchronize(s));
  if (iters && ioff[count] > 0) {
    if (mem_kind == HMS_MEM_DEVICE)
      CKC(c, cudaMemcpy(iters, its.data(), its.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    else
      std::memcpy(iters, its.data(), its.size() * sizeof(int32_t));
  }
  hms_status result = HMS_OK;
  for (int i = 0; i < count; ++i) {
    const hms_status st = check_dev_err(probs[i]);
    if (st != HMS_OK) return st;
    if (status[i] == 3 && result == HMS_OK) result = fail(c, HMS_ERR_NONFINITE, "non-finite residual norm");
    if (status[i] == 2 && result == HMS_OK) result = fail(c, HMS_ERR_NO_CONVERGENCE, "max_iter reached before tol");
  }
  return result;
}

hms_status hms_residual(hms_problem* pr, const double* p, const double* u, double* r, double* norms,
                        int32_t mem_kind) {
  return hms_update_residual(pr, p, u, nullptr, nullptr, (double*)nullptr, r, norms, mem_kind);
}

hms_status hms_reactions(hms_problem* pr, const double* u, double* f_out, int32_t mem_kind) {
  if (!pr || !u || !f_out) return HMS_ERR_ARG;
  if (mem_kind != HMS_MEM_HOST && mem_kind != HMS_MEM_DEVICE) return HMS_ERR_ARG;
  hms_context* c = pr->ctx;
  const size_t nn = nnodes(pr), vb = nn * sizeof(double2);
  if (mem_kind == HMS_MEM_DEVICE && (const char*)f_out < (const char*)u + vb && (const char*)u < (const char*)f_out + vb)
    return fail(c, HMS_ERR_ARG, "hms_reactions: f_out may not overlap u");
  CKC(c, cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  CKC(c, cudaMemcpyAsync(pr->u[0], u, vb, kind_in(mem_kind), s));
  CKC(c, launch_reactions(s, pr->lv, pr->u[0], pr->r));
  CKC(c, cudaMemcpyAsync(f_out, pr->r, vb, kind_out(mem_kind), s));
  CKC(c, cudaStreamSynchronize(s));
  return HMS_OK;
}

// delta (and, with the force-controlled modes, delta^RF after it) from the
// caller into the problem's buffers, rounded to FP32 on the mixed path.
static cudaError_t stage_deltas(hms_problem* pr, const double* delta, int32_t mem_kind) {
  cudaStream_t s = pr->ctx->stream;
  const size_t nn = nnodes(pr), vb = nn * sizeof(double2);
  const int nf = pr->lv.q == NMODES_RF ? 2 : 1;
  for (int k = 0; k < nf; ++k) {
    void* dst = k == 0 ? pr->delta : pr->delta_rf;
    const double* src = delta + 2 * nn * k;
    cudaError_t e;
    if (fp32(pr)) {
      if ((e = cudaMemcpyAsync(pr->r, src, vb, kind_in(mem_kind), s)) != cudaSuccess) return e;  // staging
      if ((e = launch_d2f(s, (const double*)pr->r, (float*)dst, 2 * nn)) != cudaSuccess) return e;
    } else {
      if ((e = cudaMemcpyAsync(dst, src, vb, kind_in(mem_kind), s)) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// The relaxation increment d (FP64, or FP32 widened) out to the caller.
static cudaError_t copy_delta_out(hms_problem* pr, const void* d, double* out, int32_t mem_kind) {
  cudaStream_t s = pr->ctx->stream;
  const size_t nn = nnodes(pr), vb = nn * sizeof(double2);
  if (fp32(pr)) {
    cudaError_t e = launch_f2d(s, (const float*)d, (double*)pr->u[1], 2 * nn);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(out, pr->u[1], vb, kind_out(mem_kind), s);
  }
  return cudaMemcpyAsync(out, d, vb, kind_out(mem_kind), s);
}

hms_status hms_update_residual(hms_problem* pr, const double* p, const double* u, const double* delta,
                               const double* a, double* u_out, double* r, double* norms, int32_t mem_kind) {
  if (!pr || !p || !u || !r) return HMS_ERR_ARG;
  if ((delta == nullptr) != (a == nullptr)) return HMS_ERR_ARG;
  if (mem_kind != HMS_MEM_HOST && mem_kind != HMS_MEM_DEVICE) return HMS_ERR_ARG;
  hms_context* c = pr->ctx;
  CKC(c, cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  const size_t nn = nnodes(pr), vb = nn * sizeof(double2);
  CKC(c, cudaMemcpyAsync(pr->p, p, vb, kind_in(mem_kind), s));
  CKC(c, cudaMemcpyAsync(pr->u[0], u, vb, kind_in(mem_kind), s));
  CKC(c, launch_mask_u(s, pr->lv, pr->u[0]));
  if (delta) {
    CKC(c, stage_deltas(pr, delta, mem_kind));
    CKC(c, cudaMemcpyAsync(pr->a, a, pr->n_c * sizeof(double), kind_in(mem_kind), s));
  }
  CKC(c, launch_update_residual(s, pr->lv, pr->u[0], pr->u[1], pr->p, pr->delta, fp32(pr), delta ? pr->a : nullptr,
                                pr->r, pr->partials, pr->ticket, pr->norms, nullptr, nullptr, 0, pr->delta_rf));
  CKC(c, cudaMemcpyAsync(r, pr->r, vb, kind_out(mem_kind), s));
  if (u_out) CKC(c, cudaMemcpyAsync(u_out, pr->u[1], vb, kind_out(mem_kind), s));
  if (norms) CKC(c, cudaMemcpyAsync(norms, pr->norms, 3 * sizeof(double), kind_out(mem_kind), s));
  CKC(c, cudaStreamSynchronize(s));
  return HMS_OK;
}

hms_status hms_relax(hms_problem* pr, const double* r, double* delta, double* P, int32_t mem_kind) {
  if (!pr || !r || !delta || !P) return HMS_ERR_ARG;
  if (mem_kind != HMS_MEM_HOST && mem_kind != HMS_MEM_DEVICE) return HMS_ERR_ARG;
  hms_context* c = pr->ctx;
  CKC(c, cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  const size_t nn = nnodes(pr), vb = nn * sizeof(double2);
  CKC(c, cudaMemcpyAsync(pr->r, r, vb, kind_in(mem_kind), s));
  CKC(c, launch_mask_u(s, pr->lv, pr->r));
  CKC(c, launch_relax_main(pr, s, nullptr));
  if (pr->lv.q == NMODES_RF) CKC(c, launch_force_relax(pr, s, nullptr));
  CKC(c, copy_delta_out(pr, pr->delta, delta, mem_kind));
  CKC(c, cudaMemcpyAsync(P, pr->P, pr->n_c * sizeof(double), kind_out(mem_kind), s));
  CKC(c, cudaStreamSynchronize(s));
  return check_dev_err(pr);
}

hms_status hms_relax_force(hms_problem* pr, const double* r, double* delta_rf, int32_t mem_kind) {
  if (!pr || !r || !delta_rf) return HMS_ERR_ARG;
  if (mem_kind != HMS_MEM_HOST && mem_kind != HMS_MEM_DEVICE) return HMS_ERR_ARG;
  hms_context* c = pr->ctx;
  if (pr->lv.q != NMODES_RF) return fail(c, HMS_ERR_ARG, "hms_relax_force: the problem has no force-controlled modes");
  CKC(c, cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  const size_t nn = nnodes(pr), vb = nn * sizeof(double2);
  CKC(c, cudaMemcpyAsync(pr->r, r, vb, kind_in(mem_kind), s));
  CKC(c, launch_mask_u(s, pr->lv, pr->r));
  CKC(c, launch_force_relax(pr, s, nullptr));
  CKC(c, copy_delta_out(pr, pr->delta_rf, delta_rf, mem_kind));
  CKC(c, cudaStreamSynchronize(s));
  return check_dev_err(pr);
}

hms_status hms_coarse_matrix(hms_problem* pr, const double* delta, double* Kaa, int32_t mem_kind) {
  if (!pr || !delta || !Kaa) return HMS_ERR_ARG;
  if (pr->n_c > 4096) return fail(pr->ctx, HMS_ERR_ARG, "dense K_aa only for q M <= 4096");
  hms_context* c = pr->ctx;
  CKC(c, cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  CKC(c, stage_deltas(pr, delta, mem_kind));
  CKC(c, launch_coarse_slots(s, pr->lv, pr->delta, fp32(pr), false, pr->slots_it, nullptr, pr->delta_rf));
  if (pr->nd) CKC(c, launch_blocks_from_slots(s, pr->lv, pr->slots_base, pr->slots_it, pr->blk, nullptr));
  else CKC(c, launch_coarse_band_from_slots(s, pr->lv, pr->slots_base, pr->slots_it, pr->band, nullptr));
  double* dense = nullptr;
  const size_t nd = (size_t)pr->n_c * pr->n_c;
  CKC(c, cudaMallocAsync(&dense, nd * sizeof(double), s));
  cudaError_t e = pr->nd ? launch_dense_from_blocks(s, pr->lv, pr->blk, dense)
                         : launch_coarse_dense_from_band(s, pr->n_c, pr->bw, pr->band, dense);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Kaa, dense, nd * sizeof(double), kind_out(mem_kind), s);
  cudaFreeAsync(dense, s);
  CKC(c, e);
  CKC(c, cudaStreamSynchronize(s));
  return HMS_OK;
}

hms_status hms_coarse_solve(hms_problem* pr, const double* Kaa, const double* P, double* a, int32_t* dropped,
                            int32_t mem_kind) {
  if (!pr || !Kaa || !P || !a) return HMS_ERR_ARG;
  if (pr->n_c > 4096) return fail(pr->ctx, HMS_ERR_ARG, "dense K_aa only for q M <= 4096");
  hms_context* c = pr->ctx;
  CKC(c, cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  const int n = pr->n_c, bw = pr->bw;
  const size_t nd = (size_t)n * n;
  double* dense = nullptr;
  CKC(c, cudaMallocAsync(&dense, nd * sizeof(double), s));
  cudaError_t e = cudaMemcpyAsync(dense, Kaa, nd * sizeof(double), kind_in(mem_kind), s);
  if (e == cudaSuccess)
    e = pr->nd ? launch_blocks_from_dense(s, pr->lv, dense, pr->blk) : launch_coarse_band_from_dense(s, n, bw, dense,
                                                                                                      pr->band);
  cudaFreeAsync(dense, s);
  CKC(c, e);
  CKC(c, cudaMemcpyAsync(pr->P, P, n * sizeof(double), kind_in(mem_kind), s));
  if (pr->nd)
    CKC(c, launch_blk_diag(s, pr->lv, pr->blk, pr->P, pr->scale, pr->b, pr->x, pr->dropped, pr->mode_mask, nullptr));
  else
    CKC(c, launch_coarse_scale(s, n, bw, pr->coarse_fp64, pr->band, pr->P, pr->sband, pr->lrow, pr->scale, pr->b,
                               pr->x, pr->dropped, pr->mode_mask, pr->lv.q, nullptr));
  CKC(c, launch_factor_stage(pr, s, nullptr));
  for (int q = 0; q < pr->nsolve; ++q) {
    if (q > 0) CKC(c, launch_refine_residual(pr, s, nullptr));
    CKC(c, launch_solve_stage(pr, s, q, nullptr));
  }
  CKC(c, cudaMemcpyAsync(a, pr->a, n * sizeof(double), kind_out(mem_kind), s));
  if (dropped) CKC(c, cudaMemcpyAsync(dropped, pr->dropped, n * sizeof(int32_t), kind_out(mem_kind), s));
  CKC(c, cudaStreamSynchronize(s));
  return HMS_OK;
}

namespace {
// 1 if ptr is device or managed memory of `device`, with the given alignment
bool device_ptr_ok(const void* ptr, int device, size_t align) {
  if (!ptr || ((uintptr_t)ptr % align) != 0) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == device;
}
}  // namespace

hms_status hms_residual_noalloc(hms_problem* pr, const double* p, const double* u, double* r, double* norms) {
  if (!pr) return HMS_ERR_ARG;
  hms_context* c = pr->ctx;
  if (!p || !u || !r) return fail(c, HMS_ERR_ARG, "hms_residual_noalloc: p, u and r are required");
  {
    // r is written while other CTAs still read p and u (halos): no byte of r
    // may lie in either
    const size_t vb = nnodes(pr) * sizeof(double2);
    auto overlap = [vb](const void* a, const void* b) {
      const char *x = (const char*)a, *y = (const char*)b;
      return x < y + vb && y < x + vb;
    };
    if (overlap(r, p) || overlap(r, u)) return fail(c, HMS_ERR_ARG, "hms_residual_noalloc: r may not overlap p or u");
  }
  const int tiles = residual_noalloc_tiles(pr->lv);
  if (tiles > HMS_RESIDUAL_NOALLOC_MAX_TILES)
    return fail(c, HMS_ERR_ARG,
                "hms_residual_noalloc: the lattice needs " + std::to_string(tiles) +
                    " tiles of 32 x 8 nodes, the static scratch holds " +
                    std::to_string(HMS_RESIDUAL_NOALLOC_MAX_TILES) + "; use hms_residual");
  CKC(c, cudaSetDevice(c->device));
  if (!device_ptr_ok(p, c->device, 16) || !device_ptr_ok(u, c->device, 16) || !device_ptr_ok(r, c->device, 16))
    return fail(c, HMS_ERR_ARG, "hms_residual_noalloc: p, u, r must be 16-byte aligned device memory of the "
                                "context's device");
  if (norms && !device_ptr_ok(norms, c->device, 8))
    return fail(c, HMS_ERR_ARG, "hms_residual_noalloc: norms must be 8-byte aligned device memory or NULL");
  double* partials = nullptr;
  unsigned* ticket = nullptr;
  CKC(c, residual_noalloc_scratch(c->device, &partials, &ticket));
  CKC(c, launch_residual_noalloc(c->stream, pr->lv, (const double2*)u, (const double2*)p, (double2*)r, partials,
                                 ticket, norms));
  CKC(c, cudaStreamSynchronize(c->stream));
  return HMS_OK;
}

namespace {
// Device bytes of a problem for (d, o), following hms_problem_create's
// allocations one by one: the shared setup buffers, one instance's buffers
// and the scratch held while the set factors are computed.  False if the
// problem would be rejected.
bool estimate_parts(hms_context* c, const hms_lattice_desc* d, const hms_options* o, size_t* shared, size_t* inst,
                    size_t* scratch) {
  if (!c || !d || !o || d->nx < 2 || d->ny < 2 || d->set_sx < 1 || d->set_sx > MAX_SX || d->set_sy < 1) return false;
  if (o->precision != HMS_FP64 && o->precision != HMS_MIXED) return false;
  const long long rw = std::min((long long)d->nx, (long long)d->set_sx + 2LL * (long long)o->relax_overlap);
  if (o->relax_overlap < 0 || rw > MAX_RX) return false;
  if (o->precision == HMS_FP64 && rw > MAX_SX) return false;
  if ((o->mode_mask >> NMODES_RF) != 0u || (o->record_history != 0 && o->record_history != 1)) return false;
  if (o->class_factors != 0 && o->class_factors != 1) return false;
  if (o->relax_balance < 0 || o->relax_balance > 2) return false;
  const bool force = (o->mode_mask >> NMODES) != 0u;
  if (o->class_factors && (d->ea || o->relax_overlap != 0 || force)) return false;
  if (force) {
    const int wr = d->nx - ((d->nx + d->set_sx - 1) / d->set_sx - 1) * d->set_sx;
    const int hr = d->ny - ((d->ny + d->set_sy - 1) / d->set_sy - 1) * d->set_sy;
    if (std::min(std::min(d->set_sx, d->nx), wr) < 2 || std::min(std::min(d->set_sy, d->ny), hr) < 2 ||
        o->relax_overlap != 0)
      return false;
  }
  hms_problem pr;
  LatView& lv = pr.lv;
  lv.nx = d->nx;
  lv.ny = d->ny;
  lv.sx = d->set_sx;
  lv.sy = d->set_sy;
  lv.Mx = (d->nx + d->set_sx - 1) / d->set_sx;
  lv.My = (d->ny + d->set_sy - 1) / d->set_sy;
  lv.M = lv.Mx * lv.My;
  lv.ov = o->relax_overlap;
  lv.q = force ? NMODES_RF : NMODES;
  pr.precision = o->precision;
  pr.n_c = lv.q * lv.M;
  pr.bw = coarse_bw(lv);
  int maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  if (relax_smem_bytes(lv, fp32(&pr)) + 2048 > (size_t)maxsm || !choose_coarse(&pr, o, maxsm) ||
      coarse_slots_smem(lv) > (size_t)maxsm)
    return false;
  const size_t nn = (size_t)lv.nx * lv.ny, M = (size_t)lv.M, n_c = (size_t)pr.n_c;
  const size_t esz = fp32(&pr) ? 4 : 8;
  const size_t nband = n_c * (pr.bw + 1);
  size_t fac = 0, ybytes = 0, plan_bytes = 0, setup_bytes = 0;
  if (o->class_factors) {
    ClassPlanHost cph;
    class_plan_build(lv, fix_pattern(d), class_sets_per_cta(fp32(&pr)), &cph);
    if (relax_class_smem(cph.slot_elems, cph.nb8max, fp32(&pr)) + 1024 > (size_t)maxsm) return false;
    fac = (size_t)cph.fac_elems;
    plan_bytes = cph.info.size() * sizeof(ClassInfo) + cph.items.size() * sizeof(ClassItem) + cph.sets.size() * 4;
    ybytes = cph.items.size() * (size_t)cph.hmax * cph.nb8max * class_sets_per_cta(fp32(&pr)) * esz;
    const size_t nc = cph.rep.size();
    for (size_t t = 0; t < nc; ++t) setup_bytes += (size_t)set_factor_stride(2 * cph.info[t].w, cph.info[t].h) * 8;
    setup_bytes += (nc + 1) * 8 + nc * 4;
  } else {
    for (int I = 0; I < lv.M; ++I) {
      const Region R = relax_region(lv, I);
      fac += (size_t)set_factor_stride(2 * R.w, R.h);
    }
    plan_bytes = (M + 1) * 8;
    ybytes = M * (size_t)relax_y_stride(lv) * esz;
  }
  const size_t ss = (size_t)slot_size(lv.q);
  *shared = nn + (d->ea ? 3 * nn * 8 : 0) + M * 16 + plan_bytes + fac * esz + M * NSLOTS * ss * 8;
  if (force) *shared += fac * esz + nn + 9 * M * 8;  // cut-free factors, supports | pins, projections
  size_t b = 4 * nn * 16 + nn * 2 * esz + ybytes;
  if (force) b += nn * 16 + nn * 2 * esz;  // r projected, delta^RF
  b += 2 * n_c * 8 + M * NSLOTS * ss * 8 + (pr.nd ? 0 : 3 * nband * 8) + 4 * n_c * 8;
  if (pr.nd) {
    const NDPlanHost& P = pr.ndp;
    b += coarse_blocks_elems(lv) * 8 + P.nodes.size() * sizeof(NDNode) + P.sets.size() * 4 +
         std::max<size_t>(P.maps.size(), 1) * 4 + P.lvl_nodes.size() * 4 +
         std::max<size_t>(P.bigs.size(), 1) * sizeof(NDBig) + std::max<size_t>(P.inv.size(), 1) * 4 +
         2 * std::max<size_t>(P.max_level_bigs, 1) * 4 + P.f_elems * 4 + std::max<size_t>(P.w_elems, 1) * 4 + 2 * n_c * 4;
  } else {
    b += 2 * (nband + 16) * 8 + (size_t)coarse_dinv_size(pr.n_c) * 8;
  }
  if (pr.big_stages > 0) b += coarse_xinv_elems(pr.n_c, pr.bw) * 4;
  if (pr.two_sided)
    for (int k = 0; k < 2; ++k) {
      const TwoSidedSizes z = coarse_two_sided_sizes(pr.ts.m[k], pr.ts.s);
      b += (z.lin + z.lcol + z.dinv + z.dropped + z.delta + z.srow + z.xinv) * 4;
    }
  b += n_c * 4 + 32 + (size_t)std::max(update_residual_blocks(lv), 1024) * 3 * 8 + 4 + sizeof(IterCtl) + 4 + 32;
  if (o->record_history) b += 3 * ((size_t)o->max_iter + 1) * 8;
  if (!o->class_factors && o->relax_overlap == 0 && o->relax_balance != 1 && lv.M > c->nsm)
    b += ((size_t)lv.M + 2 * c->nsm) * sizeof(RelaxSeg) + ((size_t)c->nsm + 1) * 4 + (size_t)lv.M * 4;  // schedule
  *inst = b;
  *scratch = (size_t)std::max(1, std::min(lv.M, c->nsm)) * b_size(MAX_NB) * 8 + setup_bytes;
  return true;
}
}  // namespace

// Device bytes hms_problem_create would allocate for (d, o) (plus the
// set-factor scratch it holds during setup); 0 if it would be rejected.
size_t hms_problem_estimate_bytes(hms_context* c, const hms_lattice_desc* d, const hms_options* o) {
  size_t sh = 0, in = 0, sc = 0;
  if (!estimate_parts(c, d, o, &sh, &in, &sc)) return 0;
  return sh + in + sc;
}

// ---------------------------------------------------------------- serving
// Requests (a lattice, options and nrhs load vectors) are queued, admitted in
// arrival order while their estimated bytes fit the budget, and advanced
// together one CUDA-graph round per step.  A request runs one problem
// instance per load vector (the problem and nrhs - 1 clones sharing its set
// factors), each on a stream of the context's pool, so its load vectors are
// solved at the same time; its instances are destroyed, and the memory
// returned, when the last load vector is done.
struct hms_server {
  struct Req {
    int64_t id = 0;
    hms_lattice_desc d{};
    hms_options o{};
    std::vector<double> ea;
    std::vector<uint8_t> fixed;
    int nrhs = 0;
    double* loads = nullptr;  // pinned, [nrhs][2 nn]
    double* u = nullptr;      // pinned, [nrhs][2 nn]
    std::vector<int32_t> iters;
    std::vector<hms_problem*> inst;  // instance q solves load vector q
    std::vector<int> launches;
    std::vector<char> running;       // load vector q not finished yet
    std::vector<char> inflight;      // a round of instance q is queued (ev[q] marks its end)
    std::vector<cudaEvent_t> ev;
    uint64_t bytes = 0;
    int slot = 0;
    bool ran = false;  // admitted and solved (u holds results)
    hms_status status = HMS_OK;
  };
  hms_context* ctx = nullptr;
  uint64_t budget = 0, used = 0;
  int max_active = 0, next_slot = 0;
  int64_t next_id = 1;
  std::deque<Req*> queue;
  std::vector<Req*> active;
  std::unordered_map<int64_t, Req*> done;
};

namespace {
void free_instances(hms_server::Req* r) {
  for (size_t k = r->inst.size(); k-- > 0;)
    if (r->inst[k]) hms_problem_destroy(r->inst[k]);
  r->inst.clear();
  for (cudaEvent_t e : r->ev)
    if (e) cudaEventDestroy(e);
  r->ev.clear();
}
void free_req(hms_server::Req* r) {
  free_instances(r);
  if (r->loads) cudaFreeHost(r->loads);
  if (r->u) cudaFreeHost(r->u);
  delete r;
}
cudaStream_t inst_stream(hms_server* s, const hms_server::Req* r, int q) {
  return s->ctx->pool[(r->slot + q) % s->ctx->pool.size()];
}
// load vector q of a request on instance q: in, u = 0, iteration control reset, ||p||
cudaError_t inst_start(hms_server* s, hms_server::Req* r, int q) {
  hms_problem* pr = r->inst[q];
  cudaStream_t st = inst_stream(s, r, q);
  const size_t nn = nnodes(pr), vb = nn * sizeof(double2);
  cudaError_t e = cudaMemcpyAsync(pr->p, r->loads + 2 * nn * q, vb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(pr->u[0], 0, vb, st);
  IterCtl hc{};
  hc.max_iter = pr->max_iter;
  hc.tol = pr->tol;
  *pr->ctl_host = hc;
  if (e == cudaSuccess) e = cudaMemcpyAsync(pr->ctl, pr->ctl_host, sizeof(IterCtl), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_load_norms(st, pr->lv, pr->p, pr->partials, pr->ticket, pr->ctl);
  r->launches[q] = 0;
  r->running[q] = 1;
  return e;
}
}  // namespace

hms_status hms_server_create(hms_context* c, uint64_t hbm_budget_bytes, int32_t max_active, hms_server** out) {
  if (!c || !out || hbm_budget_bytes == 0 || max_active < 1) return HMS_ERR_ARG;
  CKC(c, cudaSetDevice(c->device));
  while ((int)c->pool.size() < 64) {
    cudaStream_t s = nullptr;
    CKC(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    c->pool.push_back(s);
  }
  hms_server* s = new hms_server();
  s->ctx = c;
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  *out = s;
  return HMS_OK;
}

void hms_server_destroy(hms_server* s) {
  if (!s) return;
  cudaSetDevice(s->ctx->device);
  for (auto& st : s->ctx->pool) cudaStreamSynchronize(st);
  for (auto* r : s->queue) free_req(r);
  for (auto* r : s->active) free_req(r);
  for (auto& kv : s->done) free_req(kv.second);
  delete s;
}

hms_status hms_server_submit(hms_server* s, const hms_lattice_desc* d, const hms_options* o, int32_t nrhs,
                             const double* loads, int64_t* id) {
  if (!s || !d || !o || nrhs < 1 || !loads || !id) return HMS_ERR_ARG;
  hms_context* c = s->ctx;
  if (o->profile) return fail(c, HMS_ERR_ARG, "hms_server_submit: profile mode is not served");
  size_t sh = 0, in = 0, sc = 0;
  if (!estimate_parts(c, d, o, &sh, &in, &sc))
    return fail(c, HMS_ERR_ARG, "hms_server_submit: the problem would be rejected (lattice / sets / options)");
  const uint64_t est = sh + (uint64_t)nrhs * in + sc;
  if (est > s->budget)
    return fail(c, HMS_ERR_OOM, "hms_server_submit: the request needs " + std::to_string(est) +
                                    " bytes, more than the whole budget of " + std::to_string(s->budget));
  auto* r = new hms_server::Req();
  r->d = *d;
  r->o = *o;
  const size_t nn = (size_t)d->nx * d->ny;
  if (d->ea) {
    r->ea.assign(d->ea, d->ea + 3 * nn);
    r->d.ea = r->ea.data();
  }
  if (d->fixed) {
    r->fixed.assign(d->fixed, d->fixed + 2 * nn);
    r->d.fixed = r->fixed.data();
  }
  r->nrhs = nrhs;
  r->bytes = est;
  r->iters.assign(nrhs, 0);
  r->launches.assign(nrhs, 0);
  r->running.assign(nrhs, 0);
  r->inflight.assign(nrhs, 0);
  const size_t vb = (size_t)nrhs * 2 * nn * sizeof(double);
  if (cudaMallocHost(&r->loads, vb) != cudaSuccess || cudaMallocHost(&r->u, vb) != cudaSuccess) {
    cudaGetLastError();
    free_req(r);
    return fail(c, HMS_ERR_OOM, "hms_server_submit: pinned host buffers");
  }
  std::memcpy(r->loads, loads, vb);
  r->id = s->next_id++;
  s->queue.push_back(r);
  *id = r->id;
  return HMS_OK;
}

hms_status hms_server_step(hms_server* s, int64_t* done_ids, int32_t cap, int32_t* n_done, int32_t* n_active,
                           int32_t* n_queued, uint64_t* bytes_in_use) {
  if (!s || (cap > 0 && !done_ids) || !n_done) return HMS_ERR_ARG;
  hms_context* c = s->ctx;
  CKC(c, cudaSetDevice(c->device));
  *n_done = 0;
  auto report = [&](int64_t id) {
    if (*n_done < cap) done_ids[*n_done] = id;
    ++*n_done;
  };
  auto retire = [&](hms_server::Req* r, hms_status st) {
    r->status = st;
    free_instances(r);
    s->done[r->id] = r;
    report(r->id);
  };
  // 1. admission in arrival order while the estimate fits the budget
  while (!s->queue.empty() && (int)s->active.size() < s->max_active) {
    hms_server::Req* r = s->queue.front();
    if (s->used + r->bytes > s->budget) break;
    s->queue.pop_front();
    hms_problem* base = nullptr;
    hms_status st = hms_problem_create(c, &r->d, &r->o, &base);
    if (st != HMS_OK) {
      retire(r, st);
      continue;
    }
    r->inst.push_back(base);
    for (int q = 1; q < r->nrhs && st == HMS_OK; ++q) {
      hms_problem* cl = nullptr;
      st = hms_problem_clone(base, &cl);
      if (st == HMS_OK) r->inst.push_back(cl);
    }
    if (st != HMS_OK) {
      retire(r, st);
      continue;
    }
    s->used += r->bytes;
    r->ran = true;
    r->slot = s->next_slot;
    s->next_slot = (s->next_slot + r->nrhs) % (int)c->pool.size();
    r->ev.assign(r->nrhs, nullptr);
    for (int q = 0; q < r->nrhs; ++q) {
      CKC(c, cudaEventCreateWithFlags(&r->ev[q], cudaEventDisableTiming));
      CKC(c, inst_start(s, r, q));
    }
    s->active.push_back(r);
  }
  // 2. every instance whose last round has ended: finished load vector out,
  // else the next round; instances run at their own pace, the host waits
  // only when none can move
  bool moved = false;
  for (int pass = 0; pass < 2 && !moved; ++pass) {
    for (auto* r : s->active)
      for (int q = 0; q < r->nrhs; ++q) {
        if (!r->running[q]) continue;
        hms_problem* pr = r->inst[q];
        cudaStream_t st = inst_stream(s, r, q);
        if (r->inflight[q]) {
          const cudaError_t qe = cudaEventQuery(r->ev[q]);
          if (qe == cudaErrorNotReady) continue;
          CKC(c, qe);
          r->inflight[q] = 0;
          const IterCtl fin = *pr->ctl_host;
          if (fin.done || r->launches[q] >= pr->max_iter / pr->batch + 3) {
            const size_t nn = nnodes(pr), vb = nn * sizeof(double2);
            CKC(c, cudaMemcpyAsync(r->u + 2 * nn * q, pr->u[fin.t & 1], vb, cudaMemcpyDeviceToHost, st));
            r->iters[q] = fin.t > 0 ? fin.t - 1 : 0;
            if (fin.status == 3 && r->status == HMS_OK) r->status = HMS_ERR_NONFINITE;
            else if (fin.status != 1 && r->status == HMS_OK) r->status = HMS_ERR_NO_CONVERGENCE;
            r->running[q] = 0;
            moved = true;
            continue;
          }
        }
        CKC(c, cudaGraphLaunch(pr->graph, st));
        CKC(c, cudaMemcpyAsync(pr->ctl_host, pr->ctl, sizeof(IterCtl), cudaMemcpyDeviceToHost, st));
        CKC(c, cudaEventRecord(r->ev[q], st));
        r->inflight[q] = 1;
        ++r->launches[q];
        moved = true;
      }
    if (!moved) {
      // nothing could move: wait for the oldest round still queued
      for (auto* r : s->active) {
        for (int q = 0; q < r->nrhs && !moved; ++q)
          if (r->inflight[q]) {
            CKC(c, cudaEventSynchronize(r->ev[q]));
            moved = true;
          }
        if (moved) break;
      }
      moved = false;
    }
  }
  // 3. retire the requests whose load vectors are all done
  std::vector<hms_server::Req*> keep;
  for (auto* r : s->active) {
    bool all = true;
    for (int q = 0; q < r->nrhs; ++q) all = all && !r->running[q];
    if (!all) {
      keep.push_back(r);
      continue;
    }
    for (int q = 0; q < r->nrhs; ++q) CKC(c, cudaStreamSynchronize(inst_stream(s, r, q)));
    for (auto* pr : r->inst) {
      const hms_status de = check_dev_err(pr);
      if (de != HMS_OK) r->status = de;
    }
    s->used -= r->bytes;
    retire(r, r->status);
  }
  s->active.swap(keep);
  if (n_active) *n_active = (int32_t)s->active.size();
  if (n_queued) *n_queued = (int32_t)s->queue.size();
  if (bytes_in_use) *bytes_in_use = s->used;
  return HMS_OK;
}

hms_status hms_server_take(hms_server* s, int64_t id, double* u_out, int32_t* iters) {
  if (!s) return HMS_ERR_ARG;
  auto it = s->done.find(id);
  if (it == s->done.end()) return fail(s->ctx, HMS_ERR_ARG, "hms_server_take: no finished request with this id");
  hms_server::Req* r = it->second;
  const size_t nn = (size_t)r->d.nx * r->d.ny;
  if (u_out && r->ran) std::memcpy(u_out, r->u, (size_t)r->nrhs * 2 * nn * sizeof(double));
  if (iters) std::memcpy(iters, r->iters.data(), r->nrhs * sizeof(int32_t));
  const hms_status st = r->status;
  s->done.erase(it);
  free_req(r);
  return st;
}

}  // extern "C"

namespace hms {
cudaError_t launch_d2f(cudaStream_t s, const double* in, float* out, size_t n) {
  k_d2f<<<grid1d(n), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}
cudaError_t launch_f2d(cudaStream_t s, const float* in, double* out, size_t n) {
  k_f2d<<<grid1d(n), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}
}  // namespace hms
