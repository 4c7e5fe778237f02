/*
 * hms.h -- C ABI of the GB300 hierarchical master-slave (HMS) truss solver.
 *
 * Solves K u = p (Eq. 1 of Xu, Liu, Dong, "Scalable hierarchical parallel
 * algorithm for the solution of super large-scale sparse linear equations")
 * for the 2-D triangle-lattice truss of its Sec. 3.1 by the paper's
 * iteration: matrix-free residual, displacement-controlled local relaxation
 * of every set (Eqs. 11-14; with hms_options.mode_mask bits 9-11 also the
 * force-controlled one, Eqs. 15-18), and the upper-level ("master")
 * correction over q = 9 (or 12) incremental modes per set (Eqs. 3-10),
 * stopped by the 1-norm relative residual of Eq. 19.  Every step runs in
 * CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice: nodes (i, j), 0 <= i < nx, 0 <= j < ny, node index n = j*nx + i,
 *   at x = L (i + (j mod 2)/2), y = L j sqrt(3)/2 (offset rows).  Node (i, j)
 *   owns up to three bars: E to (i+1, j), NE to (i + (j mod 2), j+1) and NW to
 *   (i - 1 + (j mod 2), j+1); a bar is a linear rod of axial stiffness EA/L.
 * Vectors (loads, displacements, residuals, relaxation increments) are
 *   float64 arrays of 2*nx*ny entries, DOF 2n = x and 2n+1 = y of node n.
 *   Loads on constrained DOFs are ignored; displacements and residuals are 0
 *   there.
 * Sets: rectangular node tiles of set_sx x set_sy nodes, the last tile of a
 *   row / column takes the remainder; set index I = Iy*Mx + Ix with
 *   Mx = ceil(nx/set_sx).  Mode m (0-based) of set I is the coarse unknown
 *   q*I + m: translations x, y (Eq. 9), gradients (xi,0), (eta,0), (0,xi),
 *   (0,eta) (Eq. 10), delta, xi*delta, eta*delta (Eqs. 13-14), and with
 *   q = 12 delta^RF, xi*delta^RF, eta*delta^RF (Eqs. 17-18), with
 *   xi = x - x^(I), eta = y - y^(I) and (x^(I), y^(I)) the centroid of the
 *   set's nodes.
 * Memory: functions taking `mem_kind` accept either host pointers
 *   (HMS_MEM_HOST: copied to and from the device inside the call) or device
 *   pointers on the context's device (HMS_MEM_DEVICE, e.g. torch tensors'
 *   data_ptr()).  The library copies every input it keeps; outputs go to
 *   caller-owned buffers.  Calls are ordered on the context's stream and
 *   return after the results are in the caller's buffers.  Device inputs are
 *   read on the context's stream: work that produces them on another stream
 *   must be complete (or ordered before the call by the caller) when the call
 *   starts; the Python binding waits for torch's current stream.
 * Errors: every function returns an hms_status (0 = HMS_OK, negative = error)
 *   and never throws; hms_last_error() gives a message.  Handles are opaque
 *   and not thread-safe: use one handle from one thread at a time.
 */
#ifndef HMS_H
#define HMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hms_status;
#define HMS_OK 0
#define HMS_ERR_ARG (-1)             /* invalid argument or size */
#define HMS_ERR_NOT_SPD (-2)         /* non-positive pivot in a local factorisation */
#define HMS_ERR_NO_CONVERGENCE (-3)  /* max_iter reached; the last iterate is returned */
#define HMS_ERR_NONFINITE (-4)       /* NaN or Inf in inputs or in a residual norm */
#define HMS_ERR_OOM (-5)             /* device allocation failed or over budget */
#define HMS_ERR_TIMEOUT (-6)         /* a bounded device wait gave up */
#define HMS_ERR_CUDA (-7)            /* any other CUDA runtime error */

#define HMS_MEM_HOST 0
#define HMS_MEM_DEVICE 1

#define HMS_FP64 0   /* every step in FP64 (the plain form) */
#define HMS_MIXED 1  /* FP32 local relaxation, K_aa bar products and increment V a;
                        FP64 residual, u, master correction, norms */

typedef struct hms_context hms_context;
typedef struct hms_problem hms_problem;

/* Problem statement (Sec. 3.1): lattice, bar stiffnesses, supports, sets. */
typedef struct {
  int32_t nx, ny;            /* nodes per row, rows (>= 2 each) */
  double bar_length;         /* L > 0 */
  const double* ea;          /* host [3][ny][nx]: EA of the E, NE, NW bar owned by
                                node (i, j) (entries of absent bars ignored), or
                                NULL for ea_uniform everywhere */
  double ea_uniform;         /* EA when ea == NULL (> 0) */
  const uint8_t* fixed;      /* host [ny][nx][2], 1 = constrained DOF (u = 0), or NULL */
  int32_t fix_bottom_edge;   /* used when fixed == NULL: 1 = clamp row j = 0 */
  int32_t set_sx, set_sy;    /* set tile in nodes: 1 <= set_sx <= 64, set_sy >= 1 */
} hms_lattice_desc;

typedef struct {
  int32_t precision;         /* HMS_FP64 or HMS_MIXED */
  double tol;                /* stop when R1 = ||K u - p||_1 / ||p||_1 < tol (Eq. 19) */
  int32_t max_iter;          /* upper-level updates per load vector (>= 0) */
  int32_t coarse_solves;     /* most solves of Eq. 8 per update with the FP32 factor,
                                incl. FP64 refinement steps (1..8; refinement stops early
                                once max|res| <= 1e-14 max|b|); 0 = default (FP64: 5,
                                mixed: 2) */
  int32_t batch;             /* iterations per CUDA-graph launch; 0 = default (16) */
  int32_t profile;           /* 1 = time every kernel with CUDA events */
  int32_t coarse_factor;     /* factor of Eq. 8: 0 = auto (FP64 for one- or two-node-wide
                                set tiles, else FP32 with FP64 refinement: two-sided on two
                                SMs when the system is at least three bands long, else on
                                one SM, or on a cluster of 4 SMs when the band is too wide
                                for one; solved by 64-row blocks with inverted diagonal
                                blocks where they fit), 1 = FP32 on a cluster of 4 SMs,
                                2 = FP64, 3 = FP32 on one SM solved in 16-row steps,
                                4 = FP32 on one SM, 5 = FP32 two-sided: top and bottom
                                segments eliminated at once on two SMs, then the
                                separator between them, 6 = FP32 nested dissection of
                                the set grid over K_aa kept as 9 x 9 blocks per set
                                pair (no band): boxes of sets cut by a middle column or
                                row of sets, the fronts of one level of the tree
                                factored at once, one CTA each, fronts of 300 or more
                                unknowns by many CTAs (set grids of any width, up to
                                the 350 x 350 sets of a 1e9-DOF lattice; auto takes it
                                where no band factor fits, e.g. more than about 22
                                sets across) */
  int32_t relax_threads;     /* compute threads per CTA of the relaxation (Eqs. 11-13; one more
                                warp issues its copies): 64, 128 or 256, or
                                0 = autotuned: the first problem of a set-tile shape and
                                precision on a context times each size on its own factors
                                and the context keeps the fastest for that shape.  Results
                                are bitwise the same for every size */
  int32_t relax_copies;      /* bulk copies per factor matrix in the FP64 relaxation: 1, or
                                2 (the rows of the outer and of the inner row pairs apart,
                                half the shared memory per CTA, so two CTAs share an SM;
                                even set widths >= 6 only), or 0 = with relax_threads = 0
                                timed together with it, else 1.  Same results either way */
  int32_t relax_overlap;     /* extended relaxation region (Sec. 2.2, the region around a
                                set in Fig. 1): each set relaxes together with the nodes
                                within relax_overlap nodes of its tile (clipped to the
                                lattice), all other DOFs held, and keeps its own nodes' part
                                of the increment as its mode of Eq. 13.  0 = the set itself.
                                The grown tile must be at most 80 nodes wide
                                (min(nx, set_sx + 2 relax_overlap) <= 80), and at most 64 on
                                the FP64 path (the relaxation kernel's shared memory); with
                                overlap the FP64 relaxation uses one copy per matrix */
  uint32_t mode_mask;        /* incremental modes of every set taking part in the upper-level
                                correction (Eqs. 3 and 8): bit m keeps mode m+1 (bit 0, 1:
                                translations of Eq. 9; bits 2-5: gradients of Eq. 10; bit 6:
                                delta of Eq. 13; bits 7, 8: its gradient-weighted copies of
                                Eq. 14; bits 9-11: the force-controlled modes of Eqs. 17-18,
                                delta^RF and its gradient-weighted copies).  A cleared mode
                                gets a = 0, as a mode the coarse solve drops.  0 = the nine
                                displacement-controlled modes (0x1FF).  Any of bits 9-11 set
                                makes q = 12 modes per set: every set also relaxes with the
                                forces from outside held (the set cut free, Eqs. 15-17; a
                                floating set's increment is the minimum-norm one), the
                                coefficient vector a and P hold 12 entries per set, and set
                                tiles must be at least 2 x 2 nodes with relax_overlap = 0.
                                Bits above 11 must be 0 */
  int32_t record_history;    /* 1 = keep the (R1, R2, Pi) row of every residual evaluation on
                                the device for hms_solve's hist output; 0 = record nothing
                                (no history buffer; hist rows come back as NaN) */
  int32_t class_factors;     /* 0 = one factor of k^Inner per set (end of Sec. 2.2);
                                1 = one factor per class of identical sets, for lattices whose
                                per-set factors would not fit in device memory: with a uniform
                                EA, sets of the same width and height, parity of the first
                                row, lattice edges touched and constrained DOFs have the same
                                k^Inner, so each class is factored once and its sets are
                                relaxed together, 64 (FP32) or 32 (FP64) right-hand sides per
                                CTA.  Needs ea = NULL, relax_overlap = 0 and mode_mask bits
                                9-11 clear.  The increments equal the per-set ones up to
                                rounding (another order of the sums) */
  int32_t relax_balance;     /* schedule of the relaxation with per-set factors:
                                1 = one CTA per set (sets in waves of the SM count);
                                2 = balanced: one persistent CTA per SM (cooperative
                                launch), each running an equal share of all sets'
                                substitution steps, a set cut between two CTAs at a step
                                whose state is in device memory (McNaughton's wrap-around
                                rule: the first CTA runs the set's head first, the second
                                its tail last, after a bounded wait on a per-set flag).
                                Needs more sets than SMs, none costing more than an SM's
                                share, relax_threads 0 or 256, relax_copies 0 or 1,
                                relax_overlap = 0 and class_factors = 0 (else
                                HMS_ERR_ARG);
                                0 = with relax_threads = 0 timed together with the CTA
                                sizes where it applies, else 1.  Results are bitwise the
                                same either way */
} hms_options;

/* Context: one device, one CUDA stream.  device = CUDA ordinal. */
hms_status hms_context_create(int32_t device, hms_context** out);
void hms_context_destroy(hms_context* ctx);
/* The context's cudaStream_t (as void*), for callers that time or order work. */
void* hms_context_stream(hms_context* ctx);
/* Message of the last error on ctx; with ctx == NULL, of the last failed
 * hms_context_create.  Valid until the next call on the same handle. */
const char* hms_last_error(hms_context* ctx);

/* Setup (end of Sec. 2.2: the local matrices of Eq. 12 are constant, so each
 * set's k^Inner is factored once).  Copies the description, uploads it,
 * factors every set's k^Inner (block Cholesky, FP64, plus an FP32 copy for
 * HMS_MIXED) and precomputes the constant translation/gradient part of the
 * upper-level matrix (Eq. 6).  Returns HMS_ERR_NOT_SPD if a local pivot is
 * <= 0, HMS_ERR_OOM if device memory runs out. */
hms_status hms_problem_create(hms_context* ctx, const hms_lattice_desc* d,
                              const hms_options* o, hms_problem** out);
void hms_problem_destroy(hms_problem* pr);
/* A problem that shares src's read-only setup -- lattice description, set
 * factors, constant part of K_aa -- and has its own iteration state, so that
 * it can solve other load vectors at the same time as src (e.g. in one
 * hms_solve_batch call).  The shared buffers are freed with the last of src
 * and its clones; hms_problem_device_bytes of a clone counts its own buffers
 * only.  Results equal those of src on the same loads. */
hms_status hms_problem_clone(hms_problem* src, hms_problem** out);
/* Bytes of device memory the problem holds. */
size_t hms_problem_device_bytes(const hms_problem* pr);
/* Milliseconds the setup kernels took (CUDA events). */
double hms_problem_setup_ms(const hms_problem* pr);
/* CTA size and copies per matrix the relaxation of pr runs with (the options,
 * or the autotuned choice). */
int32_t hms_problem_relax_threads(const hms_problem* pr);
int32_t hms_problem_relax_copies(const hms_problem* pr);
/* 1 if the relaxation of pr runs on the balanced schedule (relax_balance). */
int32_t hms_problem_relax_balanced(const hms_problem* pr);
/* No counterpart in the paper (a launch plan of the relaxation of Eqs. 12-13):
 * the balanced relaxation schedule (relax_balance) of a lattice's sets over
 * `ctas` persistent CTAs (one per SM), computed on the host; no device is
 * needed.  It is the plan hms_problem_create makes on a device with that many
 * SMs for set tiles of set_sx x set_sy nodes (no overlap).  A set of h rows
 * has 2(2h - 1) ops: op o < 2h - 1 applies matrix o of the forward
 * substitution (Linv_0, B_1, Linv_1, ...), the rest the back substitution's
 * matrices in reverse order.  Output, host memory: segs_out[3 k .. 3 k + 2] =
 * (set index, first op, end op) of segment k; CTA g runs segments
 * cta_out[g] .. cta_out[g + 1] - 1 in that order (cta_out: ctas + 1 int32).
 * Returns the segment count, 0 if the schedule does not apply (no more sets
 * than CTAs, or a set costing more than one CTA's share), -1 for bad
 * arguments or cap (segments segs_out holds) too small. */
int32_t hms_relax_schedule(int32_t nx, int32_t ny, int32_t set_sx, int32_t set_sy, int32_t ctas,
                           int32_t* segs_out, int32_t cap, int32_t* cta_out);
/* The classes of identical sets that class_factors = 1 factors once each,
 * computed on the host; no device is needed.  With a uniform EA two sets have
 * the same k^Inner (Eq. 12) when they agree in width, height, parity of the
 * first row, the lattice edges they touch and their constrained DOFs.
 * class_out (host, cap >= set count int32) receives each set's class in set
 * order (row-major over the set grid), the classes numbered by first
 * appearance.  Returns the class count; -1 for bad arguments, cap too small,
 * or a per-bar EA (d->ea != NULL: no two sets need share a matrix). */
int32_t hms_set_classes(const hms_lattice_desc* d, int32_t* class_out, int32_t cap);
/* The nested-dissection plan of the upper level (Eq. 8; coarse_factor = 6)
 * for a grid of mx x my sets, computed on the host; no device is needed.
 * Node k eliminates the unknowns of its sets S_k and couples to its boundary
 * sets B_k, which lie on its ancestors' separators; children come before
 * their parents, the root last.  nodes_out[6 k .. 6 k + 5] = (|S_k|, |B_k|,
 * first entry in sets_out, child count, child 0, child 1; -1 for no child);
 * sets_out holds S_k then B_k (set indices, row-major over the set grid)
 * node by node.  Returns the node count; -1 for bad arguments or caps
 * (nodes_out holds 6 node_cap int32, sets_out sets_cap) too small. */
int32_t hms_nd_plan(int32_t mx, int32_t my, int32_t* nodes_out, int32_t node_cap, int32_t* sets_out,
                    int32_t sets_cap);

/* The whole iteration (Fig. 3) for nrhs load vectors, each from u0 (NULL =
 * zero): loads [nrhs][2*nx*ny], u0 and u_out likewise.  hist (nullable)
 * receives per load vector hist_cap rows of (R1, R2, Pi) -- the 1- and
 * 2-norm relative residuals and the energy of Eq. 2 -- one row per residual
 * evaluation, iteration 0 first; iters (nullable) receives the number of
 * upper-level updates per load vector.  Returns HMS_ERR_NO_CONVERGENCE
 * (with u_out and hist written) if some load vector did not reach tol within
 * max_iter. */
hms_status hms_solve(hms_problem* pr, int32_t nrhs, const double* loads, const double* u0,
                     double* u_out, double* hist, int32_t hist_cap, int32_t* iters,
                     int32_t mem_kind);

/* Many independent problems of one context solved together (batched uneven
 * lattices; the paper solves one lattice at a time).  Problem i solves its
 * nrhs[i] load vectors loads[i] ([nrhs[i]][2*nx_i*ny_i]) from u0 = 0 into
 * u_out[i] (same shape), one after another, exactly as hms_solve would
 * (bitwise the same results).  Two engines (hms_context_set_batch_mode):
 *  - lockstep (default where it applies): every step of an update is one
 *    launch over a work list of (problem, tile) items of all running
 *    problems; 16 updates of all of them are one CUDA graph launch; after
 *    each, the host reads every problem's convergence flag (one gathered
 *    copy), takes finished load vectors out and starts the next ones, and
 *    rebuilds the work lists when the set of running problems has changed.
 *    It applies when all problems share precision and coarse_solves and use
 *    the FP32 one-SM factor with the 64-row block solve (coarse_factor = 4,
 *    or auto where that is its choice);
 *  - streams: each problem runs its own graph rounds on one of up to 64
 *    streams of the context at its own pace.
 * Clones (hms_problem_clone) let one lattice's load vectors run at the same
 * time.  iters (nullable) receives the update counts, problem by problem and
 * load vector by load vector.  The problems must belong to c, appear once,
 * and not use options.profile.  Returns the first device error, else
 * HMS_ERR_NONFINITE / HMS_ERR_NO_CONVERGENCE if a load vector ended that way
 * (all results still written), else HMS_OK. */
hms_status hms_solve_batch(hms_context* c, int32_t count, hms_problem* const* problems,
                           const int32_t* nrhs, const double* const* loads, double* const* u_out,
                           int32_t* iters, int32_t mem_kind);
/* Engine of hms_solve_batch on c: HMS_BATCH_AUTO (lockstep where it applies,
 * else streams; the default), HMS_BATCH_STREAMS, HMS_BATCH_LOCKSTEP (fails
 * with HMS_ERR_ARG where it does not apply). */
#define HMS_BATCH_AUTO 0
#define HMS_BATCH_STREAMS 1
#define HMS_BATCH_LOCKSTEP 2
hms_status hms_context_set_batch_mode(hms_context* c, int32_t mode);

/* Upper-level updates of the last hms_solve call (all its load vectors)
 * whose FP64 refinement of the Eq. 8 solve used every solve
 * options.coarse_solves allows while the residual before the last one was
 * still above 1e-14 max|b|: the update then went on with the refined
 * solution as it stood.  0 when every update's refinement met the criterion
 * before its last solve, and always with coarse_solves = 1 (no
 * refinement). */
int64_t hms_problem_refine_cap_hits(const hms_problem* pr);

/* Per-kernel CUDA-event time of the last hms_solve with options.profile = 1:
 * names "update_residual", "relax", "coarse_assemble", "coarse_band",
 * "coarse_factor", "coarse_residual", "coarse_solve", in that order;
 * ms_total[k] and launches[k] for k < n (n <= 7).  Returns the count. */
int32_t hms_kernel_times(const hms_problem* pr, double* ms_total, int64_t* launches, int32_t n);

/* Measured FP64 rate of `device` in GFLOP/s (a DFMA counting two flops): an
 * FMA-loop kernel over every SM, timed with CUDA events after a warm-up.  The
 * roofline denominator measured beside the nominal one (SMs x DFMA lanes x
 * clock) for the kernels bound by the FP64 units; no counterpart in the
 * paper.  Allocates and frees a small buffer; runs on its own stream. */
hms_status hms_measure_fp64_rate(int32_t device, double* gflops);

/* ---- single steps of one iteration (for parity tests and custom drivers) ---- */

/* Step a1 (Eqs. 1, 19, 2): r = p - K u on the free DOFs and the sums
 * norms[0] = ||r||_1, norms[1] = ||r||_2^2, norms[2] = u.(p + r) (so that
 * Pi = -norms[2]/2).  p, u, r: [2*nx*ny]. */
hms_status hms_residual(hms_problem* pr, const double* p, const double* u, double* r,
                        double* norms, int32_t mem_kind);

/* K u at every DOF, the constrained ones included (Eq. 1 read as the nodal
 * forces the bars exert: (K u)_a = sum over the bars ab at node a of
 * (EA/L)_ab e_ab e_ab^T (u_a - u_b)).  On a free DOF this is the internal
 * force that balances the load; on a constrained DOF it is the support
 * reaction (Sec. 3.1's clamped supports), so that at a converged solution the
 * reactions and the loads are in equilibrium.  u: [2*nx*ny], read with its
 * constrained DOFs taken as 0 (u itself is not modified); f_out: [2*nx*ny]
 * (may not alias u).  HMS_ERR_ARG for NULL pointers or a bad mem_kind. */
hms_status hms_reactions(hms_problem* pr, const double* u, double* f_out, int32_t mem_kind);

/* Steps a2 + a1 (Eq. 3 then Eq. 1): u_out = u + V a with modes built from
 * delta [2*nx*ny] (q = 12: [2][2*nx*ny], delta then delta^RF) and
 * coefficients a [q*M] (set-major, q per set), then r = p - K u_out and the
 * sums of hms_residual.  u_out may not alias u.  For HMS_MIXED problems with
 * q = 9 delta is rounded to FP32 and the increment V a is formed in FP32
 * (coefficients and the node's offsets from its set's representative point
 * rounded to FP32), then added to the FP64 u, wherever a 34 x 10-node block
 * (a 32 x 8 tile and its halo) touches at most 32 sets (set tiles of 8 x 8
 * nodes and larger; smaller ones keep the FP64 increment); r is exact for
 * the u_out written. */
hms_status hms_update_residual(hms_problem* pr, const double* p, const double* u,
                               const double* delta, const double* a, double* u_out,
                               double* r, double* norms, int32_t mem_kind);

/* Steps a3 + a4 (Eqs. 12-13 and Eq. 7): delta_I = (k^Inner_I)^-1 r_I on every
 * set from the setup factors (FP64, or FP32 for HMS_MIXED), and P = V^T r
 * [q*M] with the modes built from that delta (with q = 12, also from the
 * force-controlled delta^RF of hms_relax_force). */
hms_status hms_relax(hms_problem* pr, const double* r, double* delta, double* P,
                     int32_t mem_kind);

/* The force-controlled relaxation (Eqs. 15-17) of a problem with q = 12:
 * delta^RF_I solves (k^Inner_I + Delta k_I) delta = r_I, the set cut free
 * (Delta k of Eq. 15 removes the stiffness of the bars to the outer region);
 * where that matrix is singular (the rigid motions the set's supports leave
 * free), the minimum-norm solution of the system with r_I projected onto its
 * range.  r, delta_rf: [2*nx*ny]; delta_rf is 0 on constrained DOFs.
 * HMS_ERR_ARG for a problem without the force-controlled modes. */
hms_status hms_relax_force(hms_problem* pr, const double* r, double* delta_rf, int32_t mem_kind);

/* Step a5 (Eq. 6): the upper-level matrix K_aa = V^T K V for the modes built
 * from delta (q = 12: [2][2*nx*ny], delta then delta^RF), written dense
 * [qM][qM] row-major (only for qM <= 4096).  For
 * HMS_MIXED problems delta is rounded to FP32 (as the relaxation leaves it)
 * and the per-iteration bar products are formed in FP32, summed in FP64. */
hms_status hms_coarse_matrix(hms_problem* pr, const double* delta, double* Kaa,
                             int32_t mem_kind);

/* Step a6 (Eq. 8): a = K_aa^-1 P for a dense symmetric Kaa [9M][9M] whose
 * entries outside the set-grid band are zero, by the Jacobi-scaled Cholesky
 * that drops a mode (a = 0) whose diagonal is <= 1e-300 or <= 1e-28 times the
 * largest diagonal of its set's nine modes, or which depends on earlier modes
 * of its set (FP64 test per set); FP32 factor with FP64 refinement (at most
 * options.coarse_solves solves, fewer once converged) unless the problem uses
 * the FP64 factor.  dropped (nullable) receives 1 per dropped mode. */
hms_status hms_coarse_solve(hms_problem* pr, const double* Kaa, const double* P, double* a,
                            int32_t* dropped, int32_t mem_kind);

/* For tests of the timeout path: the relaxation kernel's first wait for its
 * factor copies (of every set) gives up after `spins` tries instead of the
 * usual bound, so that hms_relax and hms_solve return HMS_ERR_TIMEOUT (0
 * tries: always).  The kernel then waits, with the usual bound, for the
 * copies it has in flight, raises the error flag and returns; the context
 * stays usable.  spins < 0 restores the usual bound.  The problem's CUDA
 * graph is rebuilt. */
hms_status hms_problem_set_relax_wait_limit(hms_problem* pr, int32_t spins);

/* ---- allocation-free residual (no counterpart in the paper) ---- */

/* Node tiles of 32 x 8 per CTA; the static scratch of
 * hms_residual_noalloc holds the per-CTA sums of at most this many tiles,
 * ceil(nx/32) * ceil(ny/8) (3 doubles each: 384 KiB of device memory). */
#define HMS_RESIDUAL_NOALLOC_MAX_TILES 16384

/* No counterpart in the paper: a library service.  It gives what
 * hms_residual gives -- r = p - K u on the free DOFs (0 on constrained
 * ones), and norms[0] = the sum of |r|, norms[1] = the sum of r^2, norms[2] =
 * u.(p + r) -- for vectors the caller already holds on the device, without
 * allocating device memory and without touching the problem's own buffers.
 *
 * Who needs it: callers that must not allocate while the device is busy --
 * cudaFree (and, with a full pool, cudaMalloc) synchronises the whole device,
 * which stalls work the caller has in flight on other streams; callers whose
 * device memory is fully committed (e.g. the factors of many problems
 * filling HBM), where an allocation could fail with out-of-memory at an
 * arbitrary point; and callers checking a solution between other solves of
 * the same problem, whose buffers hms_residual would overwrite.
 *
 * p, u, r: DEVICE pointers on the context's device (device or managed memory),
 * 2*nx*ny doubles each, 16-byte aligned; r may not overlap p or u anywhere.
 * Constrained DOFs of u are read as 0 (u itself is not modified).  norms:
 * device pointer to 3 doubles, 8-byte aligned, or NULL.  The kernel runs on
 * the context's stream; the call returns after it completed (a stream
 * synchronisation, which allocates nothing).
 *
 * Scratch: a static device array of HMS_RESIDUAL_NOALLOC_MAX_TILES * 3
 * doubles plus a completion counter, part of the library's device image; it
 * stays allocated on every device that loads the library until the process
 * exits.  The first call on each device looks up their addresses
 * (cudaGetSymbolAddress, with the device made current) and caches them; make
 * that first call before any stream capture begins on the device.  The
 * counter must be 0 when a kernel starts; it is 0 at load and every kernel
 * resets it when it completes.  Calls that run at the same time on one
 * device -- from two threads, two contexts or two problems -- share the
 * scratch and race: serialise them.
 *
 * Errors: HMS_ERR_ARG for a NULL problem/vector, host or foreign-device
 * pointers, misalignment, r overlapping p or u, or a lattice of more than
 * HMS_RESIDUAL_NOALLOC_MAX_TILES tiles (use hms_residual there);
 * HMS_ERR_CUDA if the scratch lookup or the launch fails. */
hms_status hms_residual_noalloc(hms_problem* pr, const double* p, const double* u, double* r,
                                double* norms);

/* ---- serving (no counterpart in the paper) ---- */

/* Device bytes hms_problem_create would allocate for (d, o), counted
 * allocation by allocation as the library makes them, including the scratch
 * held while the set factors are computed; 0 if the problem would be
 * rejected (bad arguments, set tile or set grid too large). */
size_t hms_problem_estimate_bytes(hms_context* c, const hms_lattice_desc* d, const hms_options* o);

/* A request server on one context: requests (lattice, options, nrhs load
 * vectors) are queued and admitted in arrival order while the sum of the
 * admitted requests' device bytes stays within hbm_budget_bytes (and at most
 * max_active run at once); every hms_server_step advances all admitted
 * requests together by one CUDA-graph round (options.batch updates), each on
 * its own stream, so requests that arrive while others run join them at the
 * next step (continuous batching).  A request runs one problem instance per
 * load vector (the problem and nrhs - 1 clones sharing its set factors,
 * see hms_problem_clone), so its load vectors are solved at the same time,
 * each exactly as hms_solve would; the instances are destroyed, and the
 * memory returned to the budget, when the last load vector is done.  A
 * request is admitted with shared + nrhs x instance + setup-scratch bytes.
 * A server is not thread-safe; other work on the same context must not run
 * while requests are active. */
typedef struct hms_server hms_server;
hms_status hms_server_create(hms_context* c, uint64_t hbm_budget_bytes, int32_t max_active,
                             hms_server** out);
void hms_server_destroy(hms_server* s);
/* Queue a request; d, its ea / fixed arrays (host) and the nrhs load vectors
 * loads [nrhs][2*nx*ny] (host) are copied.  *id receives its id.  A request
 * whose problem would be rejected gives HMS_ERR_ARG, one larger than the
 * whole budget HMS_ERR_OOM. */
hms_status hms_server_submit(hms_server* s, const hms_lattice_desc* d, const hms_options* o,
                             int32_t nrhs, const double* loads, int64_t* id);
/* One scheduling pass, asynchronous: admit what fits; for every instance
 * whose previous round has ended, take its finished load vector out or queue
 * its next round (instances run at their own pace); retire the requests whose
 * load vectors are all done.  Blocks only when no instance could move, until
 * the oldest queued round ends.  done_ids [cap] receives the ids finished in
 * this pass (*n_done of them; only the first cap are written); n_active,
 * n_queued, bytes_in_use (nullable) the state after the pass. */
hms_status hms_server_step(hms_server* s, int64_t* done_ids, int32_t cap, int32_t* n_done,
                           int32_t* n_active, int32_t* n_queued, uint64_t* bytes_in_use);
/* Results of a finished request, then forgotten: u_out [nrhs][2*nx*ny] (host,
 * nullable), iters [nrhs] (host, nullable).  Returns the request's status
 * (HMS_OK, HMS_ERR_NO_CONVERGENCE, HMS_ERR_NONFINITE, or the error that kept
 * it from being set up, in which case nothing is written to u_out). */
hms_status hms_server_take(hms_server* s, int64_t id, double* u_out, int32_t* iters);

#ifdef __cplusplus
}
#endif
#endif /* HMS_H */
