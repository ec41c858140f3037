/*
 * ll_mg.h -- C ABI of the B300 (sm_103a) aggregation-multigrid solver for the
 * semi-implicit BDF1 Landau-Lifshitz system.
 *
 * The problem (Sec. 2.1, Sec. 2.2 of the paper): one time step of the damped
 * scheme with first-order extrapolation m~ = m^n solves
 *
 *     (I + dt m~ x Delta_h + alpha dt m~ x (m~ x Delta_h)) m^{n+1} = m^n,
 *
 * one 3x3 block per cell coupled through the discrete Laplacian.  The library
 * solves it divided by dt:  (A x)_k = x_k/dt + C(m~_k) (Delta_h x)_k with
 * C(m) = [m]_x + alpha (m m^T - |m|^2 I), right-hand side m^n/dt (the relative
 * residual is the same for both scalings).  Delta_h is the cell-centred
 * 7-point (3-D), 5-point (2-D) or 3-point (1-D) Laplacian with spacing h and
 * homogeneous Neumann boundaries (missing neighbours are left out).
 *
 * Solver (Sec. 3): aggregation algebraic multigrid -- two passes of pairwise
 * matching per level, Boolean prolongation (Eq. Pagg), Galerkin coarse
 * operators A_c = P^T A P (Eq. galerkin), block Gauss-Seidel smoothing, dense
 * LU at the coarsest level -- as a V-cycle preconditioner of GCR
 * (Algorithm 1), everything in hand-written CUDA kernels on one GPU.
 *
 * Layout of every field argument: structure of arrays, component-major,
 * float64, 3*N values: m1 of all cells, then m2, then m3; within a component
 * the cell (x, y, z) sits at x + nx*(y + ny*z).  N = nx*ny*nz.
 *
 * Ownership: the caller owns every field buffer; the library never keeps a
 * pointer to one after a call returns.  The hierarchy (aggregates, coarse
 * operators, workspaces) is owned by the library and freed by
 * ll_mg_destroy.  Unless stated otherwise, pointers are DEVICE pointers on
 * the current CUDA device, and all work is enqueued on `cuda_stream` (a
 * cudaStream_t, NULL for the legacy default stream); calls return after the
 * work they launched has completed.
 *
 * Errors: a return value of 0 (LL_OK) means success.  Positive values are
 * numerical outcomes with the outputs written (best iterate, true residual).
 * Negative values mean failure with the outputs untouched.
 *
 * Threads: one hierarchy, batch or adjoint is used by one host thread at a
 * time.  Different ones may be used concurrently from different threads (a
 * batch with per-instance parameters does so itself, one thread per group):
 * the library's process-wide state is a launch counter (atomic), kernel
 * attributes that every call sets to the same values, and the error text of
 * ll_last_cuda_error (per thread).  Graph captures are thread-local.
 */
#ifndef LL_MG_H
#define LL_MG_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define LL_OK 0
#define LL_NOT_CONVERGED 1    /* maxit reached, or the stagnation stop of
                                 ll_mg_params; x = last iterate */
#define LL_BREAKDOWN 2        /* non-finite residual or gamma_jj = 0 in GCR */
#define LL_EINVAL (-1)        /* bad argument (null pointer, dt <= 0, ...) */
#define LL_ECUDA (-2)         /* a CUDA runtime call failed */
#define LL_ENOMEM (-3)        /* device allocation failed */
#define LL_SINGULAR_COARSE (-4) /* zero pivot in the coarsest LU */
#define LL_ELIMIT (-5)        /* a structural limit was exceeded (see below) */

/* ---- precision of the V-cycle preconditioner ----------------------------- */
#define LL_FP64 0        /* everything in float64 */
#define LL_MIXED_FP32 1  /* V-cycle vectors and operators in float32, GCR float64 */
#define LL_MIXED_BF16 2  /* as LL_MIXED_FP32, coarse-level operators stored in bfloat16
                            (widened to float32 for the arithmetic) */

typedef struct ll_grid {
  int nx, ny, nz; /* cells per direction; ny = nz = 1 for 1-D, nz = 1 for 2-D */
} ll_grid;

/* Solver parameters.  Fill with ll_mg_default_params(). */
typedef struct ll_mg_params {
  double rtol;         /* stop when ||b - A x||_2 < rtol ||b||_2      (1e-8) */
  int maxit;           /* GCR iterations in total, over restarts      (1000) */
  int restart;         /* GCR restart length, 1..64                   (10)   */
  int nu_pre;          /* forward block-GS sweeps before restriction  (1)    */
  int nu_post;         /* backward block-GS sweeps after prolongation (1)    */
  int coarsest_cells;  /* stop coarsening at or below this many cells (64)   */
  int max_levels;      /* at most this many levels, 1..32             (20)   */
  int rounds;          /* handshake rounds per matching pass          (32)   */
  unsigned int seed;   /* tie-break hash seed of matching, colouring  (0)    */
  int precision;       /* LL_FP64, LL_MIXED_FP32 or LL_MIXED_BF16     (LL_FP64) */
  int kcycle;          /* coarse levels 1..kcycle are solved by two inner
                          GCR steps (K-cycle, Sec. 3.1); 0: V-cycle   (0)    */
  int coarse_lanes;    /* launch shape of the per-class coarse-level
                          kernels: lanes per block row, 4 or 8; 0: by
                          the level's size                            (0)    */
  int coarse_block;    /* their threads per block, 32/64/128/256; 0: 64 (0)  */
  /* stagnation stop (no counterpart in the paper: a safeguard for instances
   * whose preconditioned GCR makes no progress): at a restart, stop with
   * LL_NOT_CONVERGED when the true residual norm exceeds stall_ratio times
   * its value at the latest restart at least stall_window iterations
   * earlier.  Restarted GCR that cannot reduce the residual in a cycle
   * rebuilds nearly the same Krylov space in the next, so such an instance
   * would spend its remaining iterations up to maxit without progress. */
  int stall_window;    /* iterations; 0: off                         (0)    */
  double stall_ratio;  /* > 0 when stall_window > 0                  (0.99) */
} ll_mg_params;

typedef struct ll_mg_hierarchy ll_mg_hierarchy; /* opaque, library-owned */

/* Fill *p with the defaults listed above. */
void ll_mg_default_params(ll_mg_params* p);

/* Build the hierarchy for one time step (Sec. 3.1.1: aggregation, Galerkin
 * coarse operators; Sec. 3: smoother and coarsest factorisation).
 *   m_tilde  device, SoA 3*N float64: the frozen field m~ = m^n (any length;
 *            the operator uses |m~|^2 as written).  Read during the call only.
 *   alpha >= 0, dt > 0, h > 0; grid with nx >= 1, ny >= 1, nz >= 1, N >= 2.
 *   p        parameters (NULL: defaults).
 *   out      receives the new hierarchy.
 * Aggregates depend on the grid only (integer graph weights), so they are
 * computed here once; ll_mg_update reuses them.
 * Errors: LL_EINVAL, LL_ENOMEM, LL_ECUDA, LL_SINGULAR_COARSE, LL_ELIMIT (a
 * coarse graph needs more than 128 colours, or N >= 2^30). */
int ll_mg_setup(const double* m_tilde, double alpha, double dt, double h, ll_grid grid,
                const ll_mg_params* p, void* cuda_stream, ll_mg_hierarchy** out);

/* Recompute the numeric part (operators, smoother blocks, coarsest LU) for
 * a new m~, alpha, dt on the same grid (the system changes every step,
 * Sec. 2.2).  Errors as ll_mg_setup. */
int ll_mg_update(ll_mg_hierarchy* H, const double* m_tilde, double alpha, double dt);

/* Solve A x = rhs by V-cycle-preconditioned GCR (Algorithm 1, restarted).
 *   rhs        device, SoA 3*N float64 (read only).
 *   x          device, SoA 3*N float64: initial guess in, solution out.
 *   rtol       relative tolerance on the true residual (<= 0: the
 *              hierarchy's parameter).
 *   iterations host, optional: preconditioner applications, summed over
 *              restarts.
 *   rel_residual host, optional: ||rhs - A x||_2 / ||rhs||_2 of the returned
 *              x, recomputed in float64 from the true residual.
 * Returns LL_OK, LL_NOT_CONVERGED or LL_BREAKDOWN (x written), or an error. */
int ll_mg_solve(ll_mg_hierarchy* H, const double* rhs, double* x, double rtol, int* iterations,
                double* rel_residual);

/* n_steps time steps of the semi-implicit scheme with projection (Sec. 4):
 * per step m~ = m, rhs = m/dt, solve (Algorithm 1) from the initial
 * approximation u_0, then m <- x/|x| per cell.  u_0 = m for the first step;
 * for step k, m^n and the d = min(k, 6) states before it extrapolated one
 * step ahead with the terms of Newton's backward-difference series
 * m^n + D m^n + D^2 m^n + ... that keep shrinking: D m^n, then D^j m^n while
 * ||D^j m^n|| < ||D^{j-1} m^n|| (j <= d); up to D^k the sum is the degree-k
 * extrapolation sum_l (-1)^l C(k+1, l+1) m^{n-l} (k = 1: 2 m^n - m^{n-1}).
 * The stopping test ||r|| < rtol ||rhs|| is the same for any u_0.
 * Aggregates are computed once; each step redoes the numeric setup.
 *   m               device SoA 3*N float64, in/out (cells must be nonzero).
 *   iters_per_step  host, optional, n_steps ints.
 *   relres_per_step host, optional, n_steps doubles.
 * Returns the worst status over the steps (errors stop early). */
int ll_step(double* m, int n_steps, double alpha, double dt, double h, ll_grid grid,
            const ll_mg_params* p, void* cuda_stream, int* iters_per_step, double* relres_per_step);

/* n_steps time steps on an existing hierarchy (same grid and parameters;
 * alpha and dt are the hierarchy's): per step the numeric setup is redone for
 * m~ = m, then solve and project as ll_step does.  Reuses the aggregates.
 * The hierarchy keeps up to six states before its last output and that
 * output: when m is bit for bit that output (a continued integration), the
 * call's first step also starts from the extrapolation.  ll_mg_update with
 * another alpha or dt drops them.
 *   m device SoA 3*N float64, in/out; iters/relres host, optional, n_steps.
 * Returns the worst status over the steps (errors stop early). */
int ll_mg_step(ll_mg_hierarchy* H, double* m, int n_steps, int* iters_per_step, double* relres_per_step);

/* n_steps time steps of the full model with explicit source terms (the LLG
 * scheme at the end of Sec. 2.1, without the stray field):
 *   (m^{n+1} - m^n)/dt = -m^n x (eps Delta_h m^{n+1} + f^n)
 *                        - alpha m^n x (m^n x (eps Delta_h m^{n+1} + f^n)),
 *   f^n = -q (m2^n e2 + m3^n e3) + h_e   (anisotropy along e1, external field),
 * i.e. the same operator with Delta_h scaled by eps and the right-hand side
 * m^n/dt - C(m^n) f^n.  The exchange factor eps enters through the
 * hierarchy's spacing: set it up with h/sqrt(eps).  Then as ll_mg_step
 * (numeric setup per step, solve from the same initial approximations,
 * projection).
 *   m  device SoA 3*N float64, in/out;  he  host, 3 doubles (NULL: zero). */
int ll_mg_step_llg(ll_mg_hierarchy* H, double* m, int n_steps, double q, const double* he,
                   int* iters_per_step, double* relres_per_step);

/* As ll_mg_step, for a field held in HOST memory: m_host (3*N float64, SoA,
 * pinned or pageable) is copied to a device buffer of the hierarchy (allocated
 * on the first call, 24 N bytes, freed by ll_mg_destroy), n_steps steps run
 * there, and the new field is copied back into m_host.  Both copies are
 * queued on the hierarchy's stream after the work already queued on the
 * caller's; the call returns when m_host holds the result.  Returns as
 * ll_mg_step; on an error (negative status) m_host is left unchanged. */
int ll_mg_step_host(ll_mg_hierarchy* H, double* m_host, int n_steps, int* iters_per_step,
                    double* relres_per_step);

/* Release the hierarchy and all its device memory (NULL is ignored). */
void ll_mg_destroy(ll_mg_hierarchy* H);

/* Human-readable text of a status code (static storage). */
const char* ll_status_string(int status);

/* The CUDA runtime call behind the calling thread's last LL_ECUDA or
 * LL_ENOMEM: error name, its text and the library source line, e.g.
 * "cudaErrorInvalidConfiguration (invalid configuration argument) at
 * ll_solver.cu:812"; "" if no call of this thread has failed.  Thread-local
 * storage, valid until the thread's next failing call; no counterpart in the
 * paper (a diagnostic). */
const char* ll_last_cuda_error(void);

/* ---- introspection (for tests and benchmarks) ------------------------------ */

/* Number of levels (level 0 = the grid). */
int ll_mg_levels(const ll_mg_hierarchy* H);
/* Cells on level l, or -1. */
int ll_mg_level_cells(const ll_mg_hierarchy* H, int l);
/* Copy the aggregate map of level l (cells of l -> cells of l+1, natural
 * cell order on level 0) to the HOST buffer agg (ll_mg_level_cells(l) ints). */
int ll_mg_level_aggregates(const ll_mg_hierarchy* H, int l, int* agg);
/* Copy the colour of each cell of level l to the HOST buffer colour. */
int ll_mg_level_colours(const ll_mg_hierarchy* H, int l, int* colour);
/* Number of 3x3 blocks of the operator of level l >= 1 (BSR), or -1. */
int ll_mg_level_blocks(const ll_mg_hierarchy* H, int l);
/* Copy the BSR operator of level l >= 1 to HOST buffers: rowptr (n+1),
 * col (nnzb), val (9*nnzb, each block row-major, component (r, c) at
 * 3r + c, cell-major unknowns).  Values are float64: a mixed-precision
 * hierarchy's float32 Galerkin values (its V-cycle's operators) widened. */
int ll_mg_level_operator(const ll_mg_hierarchy* H, int l, int* rowptr, int* col, double* val);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all hierarchies, all threads). */
long long ll_launch_count(void);

/* Measurement helper (no counterpart in the paper): one launch of a kernel
 * that only issues float64 fused multiply-adds (8 independent chains per
 * thread, 256 threads per block, `blocks` blocks, `iters` multiply-adds per
 * chain) on cuda_stream, for timing the GPU's float64 throughput with CUDA
 * events around the call.  *flops (host, optional) receives the launch's
 * floating-point operations, 2 per multiply-add.  sink: device, 1 double,
 * written only in a case that does not occur.  Returns without waiting.
 * Errors: LL_EINVAL, LL_ECUDA. */
int ll_fp64_fma_probe(double* sink, long long iters, int blocks, void* cuda_stream, double* flops);

/* Kernel timing by kind, for benchmarks.  While enabled, every kernel of a
 * kind whose bit is set in `kinds` is bracketed by two CUDA events on the
 * hierarchy's stream (no synchronisation is added).  Kinds: */
#define LL_KIND_L0_SMOOTH 0   /* level-0 block Gauss-Seidel half-sweeps */
#define LL_KIND_L0_RESTRICT 1 /* level-0 residual + restriction */
#define LL_KIND_OUTER_APPLY 2 /* float64 operator of the GCR (A z) and true residual */
#define LL_KIND_BSR_SMOOTH 3  /* coarse-level block Gauss-Seidel */
#define LL_KIND_BSR_OTHER 4   /* coarse-level residual, restriction, prolongation, zeroing */
#define LL_KIND_GCR_VECTOR 5  /* GCR dots, updates, reductions, scalar kernels */
#define LL_KIND_COARSEST 6    /* coarsest-level LU solve */
#define LL_KIND_NUMERIC 7     /* numeric setup: coefficients, Galerkin, LU factor */
#define LL_KIND_COARSE_TAIL 8 /* the small coarse levels, one thread-block-cluster kernel */
#define LL_NUM_KINDS 9
/* Start (kinds != 0) or stop (kinds == 0) timing; starting clears totals. */
int ll_mg_profile(ll_mg_hierarchy* H, unsigned int kinds);
/* Totals for one kind since timing started (synchronises the stream):
 * milliseconds, launches, and the algorithmic floating-point operations and
 * DRAM bytes of those launches (any output may be NULL).  "Algorithmic"
 * counts what the arithmetic needs, each array touched once per launch, from
 * per-unit models: with w the word size of the V-cycle (8 or 4 bytes),
 *   level-0 half-sweep, per updated cell: 48 flop (15 from zero, 66 with the
 *     prolongation), 24 + 24w bytes (24 + 12w from zero);
 *   level-0 residual+restriction, per colour-0 cell: 48 flop, 24 + 15w bytes;
 *   float64 operator / true residual, per cell: 42 flop, 120 / 144 bytes;
 *   coarse sweep or residual, per 3x3 block read: 18 flop, 12w + 4 bytes,
 *     plus per row 15 flop and 15w + 8 bytes;
 *   GCR vector kernels, per element and basis vector: 2 flop, 8 bytes;
 *   coarsest solve: 2 N^2 flop, 8 N^2 bytes. */
int ll_mg_profile_read(ll_mg_hierarchy* H, int kind, double* total_ms, long long* launches, double* flops,
                       double* bytes);

/* y = A_0 x on level 0 (device SoA buffers), float64. */
int ll_mg_apply(ll_mg_hierarchy* H, const double* x, double* y);
/* One V-cycle z = B r from level 0 (device SoA buffers), in the
 * hierarchy's precision. */
int ll_mg_vcycle(ll_mg_hierarchy* H, const double* r, double* z);
/* One block Gauss-Seidel sweep on level l: x <- GS(b, x), forward (colours
 * ascending) if forward != 0 else backward.  Device buffers; on level 0 SoA
 * 3*N, on coarse levels cell-major 3*n_l.  float64 hierarchies only. */
int ll_mg_smooth(ll_mg_hierarchy* H, int l, const double* b, double* x, int forward);

/* ---- allocation-free residual ---------------------------------------------
 * The paper has no counterpart of this call; it exists for callers that
 * cannot call cudaMalloc (or anything that allocates device memory) at the
 * point where they need a residual -- for example code running inside a
 * memory pool or arena that forbids further allocations, or a host that has
 * reserved all device memory for itself.  It computes the same residual as
 * the hierarchy-based calls without needing a hierarchy:
 *     r = rhs - A x,   norms2[0] = ||r||_2^2,   norms2[1] = ||rhs||_2^2,
 * with A the operator of ll_mg_setup for (m_tilde, alpha, dt, h, grid), its
 * coefficients formed on the fly.  relres = sqrt(norms2[0] / norms2[1]).
 *   m_tilde, rhs, x  device, SoA 3*N float64 (read only)
 *   r                device, SoA 3*N float64 output, or NULL to skip it
 *   norms2           device, 2 float64 outputs
 * The call allocates nothing: its reduction scratch is a fixed 32 KB array
 * in device memory that every GPU loading the library keeps until the
 * process exits.  That bounds the grid: N <= 8,388,608 cells (e.g. 256^2 x
 * 128); larger grids return LL_ELIMIT without touching the device.  The
 * first call on each device looks up the array's device address (the only
 * set-up); make that first call before any CUDA stream capture.  All calls
 * share the array: calls whose kernels overlap on the GPU (different streams
 * or devices sharing a context) race and give wrong norms -- serialise them.
 * Work is enqueued on cuda_stream and the call returns without waiting;
 * outputs are valid once the stream reaches that point.
 * Errors: LL_EINVAL (null input, dt <= 0, h <= 0, alpha < 0, empty grid),
 * LL_ELIMIT (grid too large, or device index >= 64), LL_ECUDA. */
int ll_residual_noalloc(const double* m_tilde, double alpha, double dt, double h, ll_grid grid,
                        const double* rhs, const double* x, double* r, double* norms2, void* cuda_stream);

/* ---- batches of independent instances -------------------------------------
 * Many independent problems (each its own grid, alpha, dt and h; the
 * parameter-study and ensemble setting) solved together.  Each instance gets
 * the hierarchy ll_mg_setup would build for it (same aggregates, colours and
 * Galerkin operators, Sec. 3); the batch concatenates them level by level so
 * that each smoothing step, residual, transfer and coarsest solve of the
 * V-cycle is one launch for all instances, and runs GCR (Algorithm 1) in
 * lockstep with separate scalars, stopping tests and restarts per instance.
 * The paper solves one problem at a time; its results per instance are
 * unchanged up to rounding.
 *   count     number of instances, >= 1
 *   m_tilde   host array of count device pointers, each SoA 3*N_i float64
 *   alpha, dt, h, grids   host arrays of count values (as ll_mg_setup)
 *   p         parameters shared by all instances, or NULL for the defaults;
 *             precision LL_FP64 or LL_MIXED_FP32 (LL_EINVAL otherwise);
 *             kcycle > 0 runs the K-cycle on those coarse levels of every
 *             instance, with each instance's own inner-step scalars
 * Every instance must coarsen at least once (more cells than
 * p->coarsest_cells), else LL_EINVAL.  The batch owns all its memory;
 * m_tilde is not retained.  Errors as ll_mg_setup. */
typedef struct ll_mg_batch ll_mg_batch;
int ll_mg_batch_setup(int count, const double* const* m_tilde, const double* alpha, const double* dt,
                      const double* h, const ll_grid* grids, const ll_mg_params* p, void* cuda_stream,
                      ll_mg_batch** out);
/* Numeric setup of every instance for new (m_tilde, alpha, dt); the grids
 * and the aggregation stay.  Arrays as in ll_mg_batch_setup. */
int ll_mg_batch_update(ll_mg_batch* B, const double* const* m_tilde, const double* alpha, const double* dt);
/* Solve A_i x_i = rhs_i for every instance from the guesses in x_i.
 *   rhs, x        host arrays of count device pointers (SoA 3*N_i float64)
 *   rtol          stopping tolerance of every instance, or <= 0: p->rtol
 *   iterations    host, count ints, or NULL: GCR iterations per instance
 *   rel_residual  host, count doubles, or NULL: true relative residuals
 *   status        host, count ints, or NULL: LL_OK / LL_NOT_CONVERGED /
 *                 LL_BREAKDOWN per instance
 * Returns LL_OK when every instance converged, else LL_BREAKDOWN if any
 * instance broke down, else LL_NOT_CONVERGED; x holds every instance's
 * final iterate in all three cases.  Blocks until done. */
int ll_mg_batch_solve(ll_mg_batch* B, const double* const* rhs, double* const* x, double rtol, int* iterations,
                      double* rel_residual, int* status);
int ll_mg_batch_count(const ll_mg_batch* B);
/* levels of the concatenated hierarchy (the deepest instance's count) */
int ll_mg_batch_levels(const ll_mg_batch* B);
/* rows (cells of all instances) and colour classes of a concatenated level */
long long ll_mg_batch_level_rows(const ll_mg_batch* B, int level);
int ll_mg_batch_level_colours(const ll_mg_batch* B, int level);
/* levels of instance i's own hierarchy */
int ll_mg_batch_instance_levels(const ll_mg_batch* B, int i);
/* Compaction: when, at a restart boundary, the instances still iterating
 * hold under half of the concatenated rows, they continue (from their
 * current iterates, as after any restart) in a sub-batch of their own, so
 * that the converged instances cost nothing more.  Each instance's
 * arithmetic is the same either way.  Sub-batches are built on first use and
 * kept (ll_mg_batch_update refreshes them); this returns how many exist.
 * Setting the environment variable LLMG_BATCH_NO_COMPACT=1 turns compaction
 * off. */
int ll_mg_batch_subbatches(const ll_mg_batch* B);
void ll_mg_batch_destroy(ll_mg_batch* B);

/* ---- batches with per-instance parameters, and their autotuner -------------
 * The paper tunes nothing; these calls exist because the instances of a
 * ragged batch differ widely in how hard they are (dt/h^2 from 0.01 to
 * several hundred, alpha from 0.005 to 1): a cycle that suits most of them
 * stagnates on some, and a stronger one costs the rest time.
 *
 * ll_mg_batch_setup_groups: as ll_mg_batch_setup, with one parameter set per
 * instance (p: host array of count ll_mg_params).  Instances with equal
 * parameters form a group, one batch each; update and solve run the groups
 * concurrently (one host thread and one CUDA stream per group) and give
 * per-instance results as ll_mg_batch_solve.  With a single distinct
 * parameter set this is ll_mg_batch_setup.  The introspection calls above
 * return -1 for the levels of a batch of several groups. */
int ll_mg_batch_setup_groups(int count, const double* const* m_tilde, const double* alpha, const double* dt,
                             const double* h, const ll_grid* grids, const ll_mg_params* p, void* cuda_stream,
                             ll_mg_batch** out);
/* number of groups (1 for a batch made by ll_mg_batch_setup) and the group
 * of instance i */
int ll_mg_batch_groups(const ll_mg_batch* B);
int ll_mg_batch_instance_group(const ll_mg_batch* B, int i);

/* Autotuner.  Instances are classed by (precision, grid nx ny nz, octave of
 * dt/h^2 = floor(log2(dt/h^2))).  For every class not yet in the cache, the
 * class's (up to) 3 instances with the smallest alpha are solved as one
 * batch (rhs = m/dt from the guess m, base's rtol, at most 300 iterations)
 * with each candidate cycle -- V(1,1), V(2,2), and each with the K-cycle on
 * level 1 -- then, for the best cycle, with the coarse kernels' launch shapes
 * (lanes 8 and/or 128 threads per block); the best converges the most
 * instances, then takes the least time (the second of two solves).
 *   m_tilde, alpha, dt, h, grids  as ll_mg_batch_setup (device fields)
 *   base        parameters of everything not tuned (NULL: defaults);
 *               precision LL_FP64 or LL_MIXED_FP32
 *   cache_path  text file of earlier choices, read first and rewritten with
 *               the new ones (NULL: no cache)
 *   chosen      host output, count ll_mg_params: base with the choice of the
 *               instance's class (pass it to ll_mg_batch_setup_groups)
 *   keys_tuned  host output (optional): classes timed by this call
 * Errors: LL_EINVAL (bad argument, or the cache cannot be written),
 * LL_ENOMEM, LL_ECUDA. */
int ll_mg_batch_autotune(int count, const double* const* m_tilde, const double* alpha, const double* dt,
                         const double* h, const ll_grid* grids, const ll_mg_params* base, const char* cache_path,
                         void* cuda_stream, ll_mg_params* chosen, int* keys_tuned);
/* Host-only helpers of the autotuner's cache (no device work): the octave
 * floor(log2(dt/h^2)) of a class (INT_MIN for bad input), and the cached
 * choice for one instance: p is read (its precision selects the class) and,
 * when the cache holds the class, overwritten with base p plus the choice;
 * returns 1 (found), 0 (not found) or LL_EINVAL. */
int ll_mg_tune_octave(double dt, double h);
int ll_mg_tune_lookup(const char* cache_path, ll_grid grid, double dt, double h, ll_mg_params* p);

/* ---- differentiation of the time step (adjoint) ----------------------------
 * A loss L on a later state depends on m^n through every step
 *     m^{n+1}_k = x_k / |x_k|,   A(m^n) x = m^n / dt   (m~ = m^n, Sec. 2.1).
 * The paper derives no adjoint; these calls give the exact discrete gradient
 * of that map (up to the solver tolerances), for gradient-based fitting of
 * initial states and damping.
 *
 * ll_mg_step_save: n_steps steps as ll_mg_step, also storing each step's
 * solution before the projection: x_save (device) receives n_steps vectors
 * of 3*N float64 (SoA), step k at offset 3*N*k.  Every solve starts from
 * u_0 = m (the map whose gradient the calls below give).  Blocks until done. */
int ll_mg_step_save(ll_mg_hierarchy* H, double* m, int n_steps, double* x_save, int* iters_per_step,
                    double* relres_per_step);
/* A one-instance batch (see above) that solves with the transposed operator
 * A^T: the same aggregation and colouring as A's hierarchy, every level
 * operator transposed ((P^T A P)^T = P^T A^T P), the transposed smoother and
 * coarsest solve.  ll_mg_batch_update / ll_mg_batch_solve then solve
 * A(m~)^T lambda = rhs.  Arguments and errors as ll_mg_setup; precision
 * LL_FP64 or LL_MIXED_FP32, kcycle 0. */
int ll_mg_adjoint_setup(const double* m_tilde, double alpha, double dt, double h, ll_grid grid,
                        const ll_mg_params* p, void* cuda_stream, ll_mg_batch** out);
/* Vector-Jacobian product of one step, on an adjoint context T:
 *   m, x      device SoA 3*N: the step's input state m^n and its solution x
 *             (ll_mg_step_save)
 *   g         device SoA 3*N: dL/dm^{n+1}
 *   m_bar     device SoA 3*N output: dL/dm^n
 *   alpha_bar host output (or NULL): this step's part of dL/dalpha
 *   rtol      tolerance of the adjoint solve (<= 0: the context's)
 * With u = x/|x|:  xbar = (g - (u.g) u)/|x|,  A^T lambda = xbar,
 *   m_bar = lambda/dt - [y x lambda + alpha((m.y) lambda + (lambda.m) y
 *           - 2 (lambda.y) m)],   alpha_bar = -sum lambda.(m (m.y) - |m|^2 y),
 * y = Delta_h x per cell.  Returns the adjoint solve's status (LL_OK,
 * LL_NOT_CONVERGED, LL_BREAKDOWN; outputs written in all three) or an
 * error.  Blocks until done. */
int ll_mg_step_vjp(ll_mg_batch* T, const double* m, double alpha, double dt, const double* x, const double* g,
                   double* m_bar, double* alpha_bar, double rtol, int* iterations, double* rel_residual);

#ifdef __cplusplus
}
#endif
#endif /* LL_MG_H */
