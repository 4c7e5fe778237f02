// Internal declarations of the HMS truss solver library (not part of the ABI).
//
// Data layout in HBM (all row-major over the node grid, node n = j*nx + i):
//   u, p, r            double2 [ny][nx]      displacement, load, residual
//   delta              double2 or float2     relaxation increment (Eq. 13)
//   kbar               double [3][ny][nx]    EA/L of the E, NE, NW bar owned by
//                                            node n (0 where the bar is absent);
//                                            null when EA is uniform
//   fix                uint8 [ny][nx]        bit 0: x constrained, bit 1: y
//   rep                double2 [M]           representing point of every set
//   a, P               double [M][9]         upper-level unknowns / forces
//   factor             per set, block-bidiagonal Cholesky factor of k^Inner
//                      (see setup.cu), FP64 or FP32
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace hms {

constexpr int NMODES = 9;     // incremental modes per set of the displacement-controlled form
constexpr int NMODES_RF = 12; // with the force-controlled modes 10-12 (Eqs. 15-18)
constexpr double SQ3_2 = 0.86602540378443864676;  // sqrt(3)/2
constexpr int MAX_SX = 64;                           // set width limit (nodes)
constexpr int MAX_RX = 80;                           // relaxation region width limit (nodes)
constexpr int MAX_NB = 2 * MAX_RX;                   // DOFs per region row

// slots of the per-set upper-level partial sums (Eq. 6), see coarse.cu
enum Slot { SLOT_SELF = 0, SLOT_E, SLOT_W, SLOT_N, SLOT_NE, SLOT_NW, NSLOTS };
constexpr int SLOT_DIM = 18;
constexpr int SLOT_SIZE = SLOT_DIM * SLOT_DIM;
// slot shape for q modes per set (q = 9: SLOT_DIM x SLOT_DIM)
__host__ __device__ inline int slot_dim(int q) { return 2 * q; }
__host__ __device__ inline int slot_size(int q) { return 4 * q * q; }

// blocks of K_aa kept per set (coarse_blocks.cu): the diagonal block and those
// of the four later neighbours J > I in row-major set order, K_aa[J][I]
enum Blk { BLK_SELF = 0, BLK_E, BLK_NW, BLK_N, BLK_NE, NBLK };
__host__ __device__ inline int blk_dx(int b) { return b == BLK_E || b == BLK_NE ? 1 : (b == BLK_NW ? -1 : 0); }
__host__ __device__ inline int blk_dy(int b) { return b >= BLK_NW ? 1 : 0; }
// block index of the later neighbour at offset (dx, dy); 0 if it is none
__host__ __device__ inline int blk_of(int dx, int dy) {
  if (dy == 0) return dx == 1 ? BLK_E : 0;
  if (dy != 1) return 0;
  return dx == -1 ? BLK_NW : (dx == 0 ? BLK_N : (dx == 1 ? BLK_NE : 0));
}

// device error flags (bit mask in a device int)
enum DevErr { DEVERR_NOT_SPD = 1, DEVERR_TIMEOUT = 2, DEVERR_NONFINITE = 4, DEVERR_COARSE = 8 };

// Read-only description of the lattice and its set partition, by value.
struct LatView {
  int nx, ny, sx, sy, Mx, My, M;
  int ov;          // relaxation region: the set's tile grown by ov nodes (Sec. 2.2)
  int q = 9;       // incremental modes per set: 9, or 12 with the force-controlled modes
  double L;        // bar length
  double k_u;      // EA/L when kbar == nullptr
  const double* kbar;
  const uint8_t* fix;
  const double2* rep;
};

// Iteration control block in device memory (one per load vector in flight).
struct IterCtl {
  int t;           // residual evaluations done (= upper-level updates + 1)
  int done;        // 1 once converged, out of iterations or failed
  int status;      // 0 running, 1 converged, 2 max_iter, 3 non-finite
  int err;         // DevErr bits raised by any kernel
  int max_iter;
  int pad;
  double tol;
  double p1, p2;   // ||p||_1, ||p||_2 of the current load vector
};

__host__ __device__ inline size_t nnodes_of(const LatView& lv) { return (size_t)lv.nx * lv.ny; }
__host__ __device__ inline int set_of(const LatView& lv, int i, int j) {
  return (j / lv.sy) * lv.Mx + (i / lv.sx);
}
// Relaxation region of set I: its tile grown by lv.ov nodes in i and j,
// clipped to the lattice (origin i0, j0; w x h nodes).  ov = 0: the set.
struct Region {
  int i0, j0, w, h;
};
__host__ __device__ inline Region relax_region(const LatView& lv, int I) {
  const int si0 = (I % lv.Mx) * lv.sx, sj0 = (I / lv.Mx) * lv.sy;
  const int si1 = si0 + lv.sx < lv.nx ? si0 + lv.sx : lv.nx, sj1 = sj0 + lv.sy < lv.ny ? sj0 + lv.sy : lv.ny;
  Region R;
  R.i0 = si0 - lv.ov > 0 ? si0 - lv.ov : 0;
  R.j0 = sj0 - lv.ov > 0 ? sj0 - lv.ov : 0;
  R.w = (si1 + lv.ov < lv.nx ? si1 + lv.ov : lv.nx) - R.i0;
  R.h = (sj1 + lv.ov < lv.ny ? sj1 + lv.ov : lv.ny) - R.j0;
  return R;
}
// bounds of every region's width and height (scratch and shared-memory sizes)
__host__ __device__ inline int region_w_max(const LatView& lv) {
  return lv.sx + 2 * lv.ov < lv.nx ? lv.sx + 2 * lv.ov : lv.nx;
}
__host__ __device__ inline int region_h_max(const LatView& lv) {
  return lv.sy + 2 * lv.ov < lv.ny ? lv.sy + 2 * lv.ov : lv.ny;
}
__host__ __device__ inline double node_x(const LatView& lv, int i, int j) {
  return lv.L * ((double)i + 0.5 * (double)(j & 1));
}
__host__ __device__ inline double node_y(const LatView& lv, int j) {
  return lv.L * SQ3_2 * (double)j;
}
// EA/L of the bar of direction d (0 E, 1 NE, 2 NW) owned by node (i, j);
// 0 if the bar or its owner does not exist.
__device__ inline double bar_k(const LatView& lv, int i, int j, int d) {
  if (i < 0 || i >= lv.nx || j < 0 || j >= lv.ny) return 0.0;
  if (lv.kbar) return __ldg(lv.kbar + (size_t)d * lv.nx * lv.ny + (size_t)j * lv.nx + i);
  // uniform stiffness: existence from the geometry
  if (d == 0) return (i + 1 < lv.nx) ? lv.k_u : 0.0;
  if (j + 1 >= lv.ny) return 0.0;
  int off = j & 1;
  int ie = (d == 1) ? i + off : i - 1 + off;
  return (ie >= 0 && ie < lv.nx) ? lv.k_u : 0.0;
}

// Timing of the kernels of one solve (profile mode).
enum KernelId {
  KID_UPDATE_RESIDUAL = 0, KID_RELAX, KID_COARSE_ASSEMBLE, KID_COARSE_BAND, KID_COARSE_FACTOR,
  KID_COARSE_RESIDUAL, KID_COARSE_SOLVE, KID_COUNT
};

// ---- per-set factor layout (setup.cu / relax.cu) ----
// Block row jj of a set of width w has nb = 2w DOFs.  Stored per set, in
// order: Linv_0, B_1, Linv_1, B_2, ..., Linv_{h-1}, where Linv_j is the
// inverse of the diagonal Cholesky block (lower triangular, row r holds
// columns 0..r) and B_j = L_{j,j-1} (row r holds columns lo(r)..nb-1,
// lo(r) = max(0, r-3)).  Each matrix is padded to a multiple of 4 elements.
__host__ __device__ inline int b_lo(int r) { return r > 3 ? r - 3 : 0; }
__host__ __device__ inline long long linv_row_off(int r) { return (long long)r * (r + 1) / 2; }
__host__ __device__ inline long long b_row_off(int nb, int r) {
  // sum_{r' < r} (nb - lo(r'))
  if (r <= 4) return (long long)r * nb;
  long long m = r - 4;  // rows 4..r-1 hold nb - (r' - 3) entries each
  return 4LL * nb + m * nb - m * (m + 1) / 2;
}
__host__ __device__ inline long long pad4(long long n) { return (n + 3) & ~3LL; }
__host__ __device__ inline long long linv_size(int nb) { return pad4(linv_row_off(nb)); }
__host__ __device__ inline long long b_size(int nb) { return pad4(b_row_off(nb, nb)); }
__host__ __device__ inline long long set_factor_size(int nb, int h) {
  return (long long)h * linv_size(nb) + (long long)(h - 1) * b_size(nb);
}
// element offset of matrix k (0 = Linv_0, 1 = B_1, 2 = Linv_1, ...) within a set
__host__ __device__ inline long long mat_off(int nb, int k) {
  return (long long)((k + 1) / 2) * linv_size(nb) + (long long)(k / 2) * b_size(nb);
}
// After these, a second copy of the same matrices stored by columns, read by
// the back substitution (offset set_factor_size + mat_off, same sizes):
//   Linv_j^T: row c holds Linv_j[r][c] for r = c..nb-1
//   B_j^T:    row c holds B_j[r][c] for r = 0..bt_hi(c), bt_hi(c) = min(nb-1, c+3)
__host__ __device__ inline long long lt_row_off(int nb, int c) {
  return (long long)c * nb - (long long)c * (c - 1) / 2;
}
__host__ __device__ inline int bt_hi(int nb, int c) { return c + 3 < nb - 1 ? c + 3 : nb - 1; }
__host__ __device__ inline long long bt_row_off(int nb, int c) {
  // sum_{c' < c} min(nb, c' + 4)
  const long long K = nb > 4 ? nb - 4 : 0;  // rows c' < K hold c' + 4 < nb entries
  if (c <= K) return (long long)c * (c - 1) / 2 + 4LL * c;
  return K * (K - 1) / 2 + 4 * K + (long long)(c - K) * nb;
}
__host__ __device__ inline long long set_factor_stride(int nb, int h) { return 2 * set_factor_size(nb, h); }

// ---- class factors (relax_class.cu): one factor per class of identical sets,
// stored "grouped" for the many-right-hand-side solves.  A matrix of kind K
// maps an input vector (columns) to an output vector (rows); its rows are
// taken in groups of 8, and group g stores, for each column its rows reach,
// the 8 values of that column (zero where a row does not reach it).  Kinds:
// Linv_j (row r: columns 0..r), B_j (row r: columns b_lo(r)..nb-1), Linv_j^T
// (row c: columns c..nb-1) and B_j^T (row c: columns 0..min(nb-1, c+3)).
enum GroupKind { GK_LINV = 0, GK_B, GK_LT, GK_BT };
__host__ __device__ inline void grp_range(int kind, int nb, int g, int& lo, int& hi) {
  const int r0 = 8 * g, r1 = 8 * g + 8 < nb ? 8 * g + 8 : nb;  // the group's rows [r0, r1)
  if (kind == GK_LINV) {
    lo = 0, hi = r1;
  } else if (kind == GK_B) {
    lo = b_lo(r0), hi = nb;
  } else if (kind == GK_LT) {
    lo = r0, hi = nb;
  } else {
    lo = 0, hi = r1 + 3 < nb ? r1 + 3 : nb;
  }
}
// element offset of group g within a grouped matrix
__host__ __device__ inline long long grp_off(int kind, int nb, int g) {
  long long o = 0;
  for (int q = 0; q < g; ++q) {
    int lo, hi;
    grp_range(kind, nb, q, lo, hi);
    o += 8LL * (hi - lo);
  }
  return o;
}
__host__ __device__ inline long long grp_size(int kind, int nb) { return pad4(grp_off(kind, nb, (nb + 7) / 8)); }
// a class's grouped factor: the forward ops' matrices (Linv_0, B_1, Linv_1, ...,
// Linv_{h-1}), then the backward ops' (Linv_{h-1}^T, B_{h-1}^T, ..., B_1^T,
// Linv_0^T), each in the order the solves use them
__host__ __device__ inline long long class_op_off(int nb, int h, int o) {
  const int nm = 2 * h - 1;
  if (o < nm) return (long long)((o + 1) / 2) * grp_size(GK_LINV, nb) + (long long)(o / 2) * grp_size(GK_B, nb);
  const int k = o - nm;
  const long long fwd = (long long)h * grp_size(GK_LINV, nb) + (long long)(h - 1) * grp_size(GK_B, nb);
  return fwd + (long long)((k + 1) / 2) * grp_size(GK_LT, nb) + (long long)(k / 2) * grp_size(GK_BT, nb);
}
__host__ __device__ inline long long class_factor_size(int nb, int h) { return class_op_off(nb, h, 2 * (2 * h - 1)); }
struct ClassInfo {
  long long off;  // element offset of the class's grouped factor
  int w, h;       // set width and height (nodes)
};
struct ClassItem {
  int cls, first, count, pad;  // the sets sets[first .. first + count) of class cls
};
struct ClassPlanDev {
  const ClassInfo* info = nullptr;
  const ClassItem* items = nullptr;
  const int* sets = nullptr;  // set indices, grouped by class
  int nitems = 0;
  int nb8max = 0;             // rows of a vector panel (largest nb rounded up to 8)
  size_t slot_elems = 0;      // largest grouped matrix (elements)
  long long ystride = 0;      // elements of one CTA's forward vectors
};

// ---- launchers (each returns the launch error) ----
// residual.cu
cudaError_t launch_update_residual(cudaStream_t s, const LatView& lv, const double2* u_in,
                                   double2* u_out, const double2* p, const void* delta,
                                   bool delta_fp32, const double* a, double2* r, double* partials,
                                   unsigned* ticket, double* norms_out, IterCtl* ctl, double* hist,
                                   int hist_cap, const void* delta_rf);
int update_residual_blocks(const LatView& lv);
cudaError_t launch_reactions(cudaStream_t s, const LatView& lv, const double2* u, double2* f);
cudaError_t launch_load_norms(cudaStream_t s, const LatView& lv, double2* p, double* partials,
                              unsigned* ticket, IterCtl* ctl);
// residual_noalloc.cu
int residual_noalloc_tiles(const LatView& lv);
cudaError_t residual_noalloc_scratch(int device, double** partials, unsigned** ticket);
cudaError_t launch_residual_noalloc(cudaStream_t s, const LatView& lv, const double2* u, const double2* p,
                                    double2* r, double* partials, unsigned* ticket, double* norms_out);
// setup.cu (cut = true: the set cut free, i.e. k^Inner + Delta k of Eq. 15, only the
// set's own bars; lv.fix then marks the constrained and the pinned DOFs)
cudaError_t launch_set_factor(cudaStream_t s, const LatView& lv, const long long* set_off,
                              double* f64, float* f32, double* scratch, int grid, int* err, bool cut = false,
                              const int* list = nullptr, int nlist = 0);
// force.cu: the force-controlled relaxation's projections (Eqs. 16-18).  M: per set the
// 3 x 3 matrix of the projection onto the rigid motions the set's supports leave free
// (zero for anchored sets); fixF: supports | pinned DOFs.
cudaError_t launch_force_in(cudaStream_t s, const LatView& lv, const double2* r, const double* M,
                            const uint8_t* fixF, double2* rproj, const IterCtl* ctl);
cudaError_t launch_force_out(cudaStream_t s, const LatView& lv, void* drf, bool fp32, const double* M,
                             const double2* r, double* P, const IterCtl* ctl);
bool force_set_data(const LatView& lv, const std::vector<uint8_t>& fix, const std::vector<double2>& rep,
                    std::vector<double>& M, std::vector<uint8_t>& fixF);
// relax.cu
cudaError_t launch_relax(cudaStream_t s, const LatView& lv, const long long* set_off,
                         const double* f64, const float* f32, const double2* r, void* delta,
                         double* P, void* yscratch, const IterCtl* ctl, int* err, int threads, int chunks,
                         int wait0 = -1);
size_t relax_smem_bytes(const LatView& lv, bool fp32, int chunks = 1);
// relax_class.cu: the relaxation with class factors (sets per CTA: 64 FP32, 32 FP64)
int class_sets_per_cta(bool fp32);
size_t relax_class_smem(size_t slot_elems, int nb8max, bool fp32);
cudaError_t launch_group_factor(cudaStream_t s, const double* src, int nb, int h, double* g64, float* g32);
cudaError_t launch_relax_class(cudaStream_t s, const LatView& lv, const ClassPlanDev& cp, const double* f64,
                               const float* f32, const double2* r, void* delta, double* P, void* yscratch,
                               const IterCtl* ctl, int* err, int wait0 = -1);
cudaError_t configure_relax_class(int max_smem);
bool relax_chunks_possible(const LatView& lv, bool fp32);
long long relax_y_stride(const LatView& lv);
// The relaxation on a balanced schedule (relax.cu): one persistent CTA per SM,
// each running an equal share of all sets' substitution steps.  Segment =
// ops [o0, o1) of set I (op o: matrix o of the forward pass, o < 2h - 1, then
// the backward pass's matrices in reverse).  cta[g] .. cta[g + 1] - 1 index
// CTA g's segments in the order it runs them.
struct RelaxSeg {
  int I, o0, o1, pad;
};
// Plans the schedule over `grid` CTAs; false where it does not apply (an
// extended relaxation region, no more sets than CTAs, or a set costing more
// than one CTA's share).  est_balance (optional): the busiest CTA's cost over
// the mean, and the same for one CTA per set in waves of `grid`.
bool relax_sched_plan(const LatView& lv, int grid, std::vector<RelaxSeg>& segs, std::vector<int>& cta,
                      double* est_sched = nullptr, double* est_waves = nullptr);
// CTAs of the balanced relaxation on this device (SMs x resident CTAs, 0 if none fits).
cudaError_t relax_sched_grid(const LatView& lv, bool fp32, int* grid);
cudaError_t launch_relax_sched(cudaStream_t s, const LatView& lv, const long long* set_off, const double* f64,
                               const float* f32, const double2* r, void* delta, double* P, void* yscratch,
                               const IterCtl* ctl, int* err, const RelaxSeg* segs, const int* cta, int* flags,
                               int grid, int wait0 = -1);
// coarse.cu
cudaError_t launch_coarse_slots(cudaStream_t s, const LatView& lv, const void* delta, bool delta_fp32,
                                bool full, double* slots, const IterCtl* ctl, const void* delta_rf = nullptr);
int coarse_bw(const LatView& lv);
cudaError_t launch_coarse_band_from_slots(cudaStream_t s, const LatView& lv, const double* base,
                                          const double* slots, double* band, const IterCtl* ctl);
cudaError_t launch_coarse_band_from_dense(cudaStream_t s, int n, int bw, const double* dense,
                                          double* band);
cudaError_t launch_coarse_dense_from_band(cudaStream_t s, int n, int bw, const double* band,
                                          double* dense);
cudaError_t launch_coarse_scale(cudaStream_t s, int n, int bw, bool fp64, const double* band, const double* P,
                                double* sband, void* frow, double* scale, double* b, double* x, int* dropped,
                                unsigned mode_mask, int nm, const IterCtl* ctl);
cudaError_t launch_coarse_factor(cudaStream_t s, int n, int bw, bool fp64, void* lrow, void* lcol, void* dinv,
                                 int* dropped, bool write_lrow, const IterCtl* ctl);
cudaError_t launch_coarse_solve(cudaStream_t s, int n, int bw, bool fp64, const void* lcol, const void* lrow,
                                const void* dinv, const int* dropped, const double* res, double* x,
                                const double* scale, double* a_out, unsigned long long* cstat, int flags,
                                const IterCtl* ctl, int* err);
size_t coarse_xinv_elems(int n, int bw);
int coarse_big_stages(int n, int bw, int max_smem);
cudaError_t launch_coarse_blockinv(cudaStream_t s, int n, int bw, const void* lcol, const void* lrow, float* xinv,
                                   const IterCtl* ctl);
cudaError_t launch_coarse_solve_big(cudaStream_t s, int stages, int n, int bw, const void* lcol, const void* lrow,
                                    const float* xinv, const int* dropped, const double* res, double* x,
                                    const double* scale, double* a_out, unsigned long long* cstat, int flags,
                                    const IterCtl* ctl, int* err);
cudaError_t launch_coarse_residual(cudaStream_t s, int n, int bw, const double* sband, const double* b,
                                   const double* x, const int* dropped, double* res, unsigned long long* cstat,
                                   const IterCtl* ctl);
// ---- lockstep batches (batch.cu drives them): one launch per step covers the
// work items of every problem of a batch.  A problem's per-iteration buffers:
struct BatchProb {
  LatView lv;
  double2* u[2];
  double2* p;
  double2* r;
  void* delta;
  double* a;
  double* P;
  double* partials;
  unsigned* ticket;
  IterCtl* ctl;
  double* hist;
  int hist_cap;
  int* err;
  const long long* set_off;
  const double* f64;
  const float* f32;
  void* yscratch;
  const double* slots_base;
  double* slots_it;
  double* band;
  double* sband;  // column layout, then row layout
  double* scale;
  double* b;
  double* x;
  double* res;
  float* lrow;
  float* lcol;
  float* dinv;
  float* xinv;
  int* dropped;
  unsigned long long* cstat;
  int n_c, bw;
  unsigned mode_mask;
};
// One CTA of a batched launch: the problem and the block index (bx, by) of the
// problem's own launch of that kernel, whose grid is gx x gy.
struct BatchItem {
  int prob, bx, by, gx, gy;
};
cudaError_t launch_batch_update_residual(cudaStream_t s, bool fp32, const BatchProb* P, const BatchItem* it, int n,
                                         int k);
cudaError_t launch_batch_relax(cudaStream_t s, bool fp32, int threads, int chunks, size_t smem, const BatchProb* P,
                               const BatchItem* it, int n);
cudaError_t launch_batch_slots(cudaStream_t s, bool fp32, size_t smem, const BatchProb* P, const BatchItem* it,
                               int n);
cudaError_t launch_batch_band(cudaStream_t s, const BatchProb* P, const BatchItem* it, int n);
cudaError_t launch_batch_diag(cudaStream_t s, const BatchProb* P, const BatchItem* it, int n);
cudaError_t launch_batch_set_drops(cudaStream_t s, const BatchProb* P, const BatchItem* it, int n);
cudaError_t launch_batch_scale_band(cudaStream_t s, const BatchProb* P, const BatchItem* it, int n);
cudaError_t launch_batch_factor(cudaStream_t s, size_t smem, const BatchProb* P, const BatchItem* it, int n);
cudaError_t launch_batch_blockinv(cudaStream_t s, const BatchProb* P, const BatchItem* it, int n);
cudaError_t launch_batch_solve(cudaStream_t s, int stages, size_t smem, const BatchProb* P, const BatchItem* it,
                               int n, bool first);
cudaError_t launch_batch_coarse_residual(cudaStream_t s, const BatchProb* P, const BatchItem* it, int n);
// grids of the per-problem launches the batched ones stand for
int update_residual_grid_x(const LatView& lv);
int update_residual_grid_y(const LatView& lv);
int coarse_grid_for(size_t n);   // 256-thread CTAs of a grid-stride kernel over n entries
int coarse_residual_blocks(int n);
int set_drops_blocks(int nsets);
size_t big_solve_smem_bytes(int n, int bw, int S);

// two-sided FP32 factor and solve (coarse_solve.cu): top [0, m[0]), separator
// [m[0], m[0] + s), bottom (m[1] rows, reversed frame); per side its row band,
// factor, drop flags, separator buffers and 64-row block matrices
struct TwoSided {
  int m[2] = {0, 0};
  int s = 0;
  int stages = 0;
  float* lin[2] = {nullptr, nullptr};
  float* lcol[2] = {nullptr, nullptr};
  float* dinv[2] = {nullptr, nullptr};
  int* dropped[2] = {nullptr, nullptr};
  float* delta[2] = {nullptr, nullptr};
  float* srow[2] = {nullptr, nullptr};
  float* xinv[2] = {nullptr, nullptr};
};
bool coarse_two_sided_split(int n, int bw, int* m0, int* m1, int* s);
// element counts of one side's buffers (float, except dropped: int)
struct TwoSidedSizes {
  size_t lin, lcol, dinv, dropped, delta, srow, xinv;
};
TwoSidedSizes coarse_two_sided_sizes(int m, int s);
size_t coarse_two_sided_factor_smem(int m0, int m1, int s);
int coarse_two_sided_stages(int m0, int m1, int s, int max_smem);
cudaError_t launch_coarse_factor_2s(cudaStream_t st, int n, int bw, const TwoSided& t, const double* sband,
                                    const int* dropped, const IterCtl* ctl);
cudaError_t launch_coarse_solve_2s(cudaStream_t st, int n, const TwoSided& t, const double* res, double* x,
                                   const double* scale, double* a_out, int* dropped_out, unsigned long long* cstat,
                                   int flags, const IterCtl* ctl, int* err);
size_t coarse_factor_smem_bytes(int n, int bw, bool fp64);
size_t coarse_solve_smem_bytes(int n, int bw, bool fp64);
int coarse_dinv_size(int n);
size_t coarse_slots_smem(const LatView& lv);
// one-time function attributes (max dynamic shared memory), per device
cudaError_t configure_setup(int max_smem);
cudaError_t configure_relax(int max_smem);
cudaError_t configure_coarse_assemble(int max_smem);
cudaError_t configure_coarse_solve(int max_smem);
// coarse_blocks.cu: K_aa by blocks of the set grid (the nested-dissection path)
size_t coarse_blocks_elems(const LatView& lv);
cudaError_t launch_blocks_from_slots(cudaStream_t s, const LatView& lv, const double* base, const double* slots,
                                     double* blk, const IterCtl* ctl);
cudaError_t launch_blk_diag(cudaStream_t s, const LatView& lv, const double* blk, const double* P, double* scale,
                            double* b, double* x, int* dropped, unsigned mode_mask, const IterCtl* ctl);
cudaError_t launch_blk_residual(cudaStream_t s, const LatView& lv, const double* blk, const double* scale,
                                const int* dropped, const double* b, const double* x, double* res,
                                unsigned long long* cstat, const IterCtl* ctl);
cudaError_t launch_blocks_from_dense(cudaStream_t s, const LatView& lv, const double* dense, double* blk);
cudaError_t launch_dense_from_blocks(cudaStream_t s, const LatView& lv, const double* blk, double* dense);
// coarse_nd.cu: nested-dissection factor and solve of Eq. 8 over the set grid.
// A tree node (front): its own sets S and boundary sets B (lists of set
// indices at s_off: S then B), up to two children whose boundary sets sit at
// the front positions maps[map_off[c] ...] (in sets, S first), its dense
// front F (9(ns+nb) squared floats at f_off) and its update vector W
// (9 nb floats at w_off).
struct NDNode {
  int ns, nb, s_off, nchild;
  int child[2];
  int map_off[2];
  int nm, pad;  // modes per set (9 or 12)
  long long f_off, w_off;
};
// A wide front (at least ND_BIG unknowns) is factored by many CTAs, panel by
// panel: its node, and per child the place of each of its sets (S then B) in
// the child's boundary list (-1 if absent), at inv_off[c].
constexpr int ND_BIG = 300;
struct NDBig {
  int node;
  int inv_off[2];
  int pad;
};
struct NDPlanHost {
  std::vector<NDNode> nodes;
  // nodes by height, leaves first; within a level the fronts factored by one
  // CTA each first, then the wide ones ([level_split[h], level_begin[h + 1]))
  std::vector<int> sets, maps, lvl_nodes, level_begin, level_split;
  std::vector<NDBig> bigs;          // the wide fronts, level by level (bigs[k] <-> lvl_nodes[level_split[h] + ...])
  std::vector<int> big_begin, inv;  // per level: first entry in bigs; inverse child maps
  std::vector<int> level_big_ns;    // per level: the largest pivot count of its wide fronts (unknowns)
  std::vector<int> level_big_nf;    // per level: the largest of its wide fronts (unknowns)
  std::vector<int> level_big_nb;    // per level: the largest boundary of its wide fronts (unknowns)
  std::vector<int> level_small_nf;  // per level: the largest of its one-CTA fronts (unknowns)
  std::vector<size_t> level_smem_factor, level_smem_solve;  // dynamic shared memory per level's launches
  int nlevels = 0, max_front = 0, max_level_nodes = 0, max_level_bigs = 0;
  size_t f_elems = 0, w_elems = 0;
};
struct NDPlanDev {
  NDNode* nodes = nullptr;
  int *sets = nullptr, *maps = nullptr, *lvl_nodes = nullptr;
  NDBig* bigs = nullptr;
  int *inv = nullptr, *dmask = nullptr;
  float *F = nullptr, *W = nullptr, *y = nullptr, *xc = nullptr;
};
bool nd_plan_build(const LatView& lv, NDPlanHost* P);
bool nd_plan_smem(NDPlanHost* P, int max_smem);  // false if a front is too large
cudaError_t configure_coarse_nd(int max_smem);
// the scaled matrix (Eq. 8 after Jacobi scaling) comes from the blocks of
// coarse_blocks.cu with the scale and drop flags of k_blk_diag
cudaError_t launch_nd_factor(cudaStream_t s, const LatView& lv, const NDPlanHost& P, const NDPlanDev& D,
                             const double* blk, const double* scale, int* dropped, const IterCtl* ctl);
cudaError_t launch_nd_solve(cudaStream_t s, int n, const NDPlanHost& P, const NDPlanDev& D, const double* rhs,
                            double* x, const double* scale, double* a_out, const int* dropped,
                            unsigned long long* cstat, int flags, const IterCtl* ctl);
// coarse_factor_cluster.cu
size_t coarse_factor_cl_smem_bytes(int n, int bw);
cudaError_t configure_coarse_factor_cl(int max_smem);
cudaError_t launch_coarse_factor_cl(cudaStream_t s, int n, int bw, const void* lrow, void* lcol, void* dinv,
                                    int* dropped, const IterCtl* ctl);
// small utility kernels (capi.cu)
cudaError_t launch_mask_u(cudaStream_t s, const LatView& lv, double2* u);
cudaError_t launch_d2f(cudaStream_t s, const double* in, float* out, size_t n);
cudaError_t launch_f2d(cudaStream_t s, const float* in, double* out, size_t n);

}  // namespace hms

namespace hms {
// Allows `func` the largest dynamic shared memory the device offers beside
// its static shared memory.
template <typename F>
inline cudaError_t set_max_dynamic_smem(F* func, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)func);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute((const void*)func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}
}  // namespace hms
