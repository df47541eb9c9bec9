/*
 * bmg.h -- C ABI of a GB300 (sm_103a) black-box multigrid (BoxMG) solver for
 * 2D 5- and 9-point variable-coefficient stencils with zero Dirichlet
 * boundaries (Nytko, Reisner, Moulton, Olson, West, "Teaching an old dog new
 * tricks", arXiv 2502.05279: the problem A x = b of Sec. 2 and the V-cycle of
 * Fig. 1; the method itself is Dendy's black-box multigrid, which Sec. 2 cites).
 *
 * Conventions shared by every call
 * ---------------------------------
 * Grid.  A level with n = 2^m - 1 interior points per side (n >= 3) is stored
 * as an (n+2) x (n+2) row-major array of doubles indexed [j][i] (i = x is the
 * fastest index), interior i, j in 1..n; the ghost ring i, j in {0, n+1}
 * carries the Dirichlet value 0.  Coarse point (ic, jc) lies on fine point
 * (2ic, 2jc); n_c = (n - 1) / 2.
 *
 * Stencil.  Five planes O, W, S, SW, NW, each (n+2)^2, back to back: the
 * matrix entries a(p,p), a(p,p-x), a(p,p-y), a(p,p-x-y), a(p,p-x+y).  A is
 * symmetric, so E(p) = W(p+x), N(p) = S(p+y), NE(p) = SW(p+x+y),
 * SE(p) = NW(p+x-y).  A 5-point stencil (kind 5) passes three planes O, W, S.
 * Couplings from an interior point to a ghost point are not entries of A; the
 * library ignores (zeroes) them and the ghost ring of every plane.
 * Natural (Neumann) sides need no option: a stencil whose couplings across a
 * side vanish (for -div(k grad u), zero k in the cells beyond it) has rows
 * with no Dirichlet term there, and the solver treats it like any other
 * stencil.  The all-Neumann (singular) operator is not supported.
 *
 * General sizes.  bmg_setup also takes any nx x ny grid (1 <= nx, ny <= 65535):
 * the caller's arrays are then (ny+2) x (nx+2), row-major with row length nx+2,
 * and the hierarchy embeds the problem in the n x n level 0 with
 * n = the smallest 2^m - 1 >= max(nx, ny, 3): the caller's points keep their
 * (i, j) and equations, and every other interior point of level 0 gets the
 * identity row a_O = 1 with no couplings (its unknown is zero in the solution).
 * bmg_solve, bmg_time_cycles and bmg_profile take rhs and x in the caller's
 * layout; every other call on the hierarchy speaks of its levels (level 0 of
 * size n, bmg_level_size).  Batched solves take 2^m - 1 squares only.
 *
 * Periodic sides (bmg_opts.periodic; the paper states Dirichlet grids only, and
 * periodic axes are the black-box method's capability that Sec. 2 defers to).
 * A periodic axis has N = 2^m points (point N + 1 is point 1 and point 0 is
 * point N), a Dirichlet axis 2^m - 1, both axes the same m >= 2, so
 * nx = ny + 1 (periodic in x), ny = nx + 1 (in y) or nx = ny = 2^m (both).
 * Arrays keep the (ny+2) x (nx+2) layout; a coupling across a periodic side is
 * an entry of A (W at i = 1 couples point 1 to point N, S at j = 1 point 1 to
 * point N, SW and NW likewise), and the ghost lines are ignored.  Coarse point
 * c still sits on fine point 2c, so a periodic axis of N points coarsens to a
 * periodic axis of N / 2, down to 4 points (3 on a Dirichlet axis).  The
 * interpolation planes of such a hierarchy have N_c cells along a periodic
 * axis (ic = 1..N_c) and N_c + 1 along a Dirichlet one.  With both axes
 * periodic a diffusion operator annihilates constants: the caller makes it
 * non-singular (for instance with a positive term on the diagonal), else the
 * coarsest factorisation may fail with BMG_ESINGULAR.
 *
 * Interpolation weights.  Eight planes of (n_c+2)^2 doubles in the order
 * LSW, LSE, LNW, LNE, LL, LR, LB, LA (the labels of Fig. 2), indexed by the
 * coarse cell (ic, jc) whose north-east corner is coarse point (ic, jc):
 *   fine (2ic-1, 2jc-1): LSW, LSE, LNW, LNE = weights toward coarse
 *                        (ic-1,jc-1), (ic,jc-1), (ic-1,jc), (ic,jc);
 *   fine (2ic-1, 2jc):   LL, LR = toward (ic-1,jc), (ic,jc);
 *   fine (2ic, 2jc-1):   LB, LA = toward (ic,jc-1), (ic,jc).
 *
 * Arithmetic.  By default (BMG_ARITH_ROUNDED) the cycle rounds every multiply,
 * add and subtract separately (no fused multiply-add) and sums each row of A
 * in the order O, W, E, S, N, SW, NE, NW, SE, so its iterates are reproducible
 * bit for bit; BMG_ARITH_FUSED (bmg_opts.arith) keeps the order and fuses
 * each multiply-add.
 *
 * Pointers.  "device" = memory the calling process allocated on the current
 * CUDA device; "host" = ordinary host memory.  `stream` is a cudaStream_t
 * (NULL = legacy default stream); all device work is enqueued on it and a call
 * returns once its results are ready, unless stated otherwise.  No call takes
 * ownership of a caller pointer.
 *
 * Environment.  BMG_TUNE_CACHE=<file>: the autotuner appends each decision it
 * times (Gauss-Seidel kernel and shape per level or batched stage, the fused
 * two-sweep pass) to the file, keyed by the device model, and reuses the
 * decisions it finds there instead of timing again; every candidate computes
 * the same bits, and records with out-of-range values are ignored.
 * BMG_FAIL_ALLOC=k (testing): the k-th device or pinned allocation of the setup
 * calls, counted from when the value last changed, fails as BMG_ENOMEM.
 *
 * Errors.  Every int-returning call returns BMG_OK (0) or a negative code;
 * bmg_strerror() names it and bmg_last_error() gives the detail of the most
 * recent failure on the calling thread.  No exception crosses the ABI.  A
 * hierarchy is not thread-safe.
 */
#ifndef BMG_H
#define BMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  BMG_OK = 0,
  BMG_EINVAL = -1,      /* bad size, kind, option or pointer */
  BMG_ENOMEM = -2,      /* device allocation failed */
  BMG_ECUDA = -3,       /* a CUDA runtime call failed (detail in bmg_last_error) */
  BMG_ESINGULAR = -4,   /* non-positive pivot in the coarsest Cholesky, a non-positive
                           diagonal, or a zero / non-finite interpolation denominator */
  BMG_ENAN = -5,        /* the residual norm became NaN or Inf */
  BMG_ENOTCONV = -6,    /* maxit cycles ran without reaching tol; x holds the last iterate */
  BMG_ETIMEOUT = -7,    /* a bounded device-side wait gave up */
  BMG_EBOUNDS = -8      /* debug builds only: a device bounds check failed (bmg_debug_take) */
};

enum { BMG_FP64 = 0, BMG_FP32_IR = 1, BMG_BF16_IR = 2 };
enum { BMG_INTERP_DENDY = 0, BMG_INTERP_LEARNED = 1 };
enum { BMG_KRYLOV_NONE = 0, BMG_KRYLOV_FCG = 1 };

typedef struct bmg_hierarchy bmg_hierarchy;   /* opaque, library-owned */

typedef struct {
  int kind;             /* 5 or 9 */
  const double* coef;   /* device; kind 9: 5 planes O,W,S,SW,NW; kind 5: 3 planes O,W,S;
                           each (n+2)^2 doubles (see Stencil above) */
} bmg_stencil;

typedef struct {
  int precision;        /* BMG_FP64 (default), BMG_FP32_IR or BMG_BF16_IR */
  int interp;           /* BMG_INTERP_DENDY (default), or BMG_INTERP_LEARNED: level 0 uses the
                           network `mlp`; setup also builds the Dendy hierarchy, measures the
                           V-cycle factor of both and keeps the better (Dendy is the fallback) */
  int coarsest;         /* coarsest level size, 2^m - 1 >= 3 (0 = 3) */
  int nu1, nu2;         /* pre- and post-smoothing sweeps (0,0 = 2,1) */
  int inner_cycles;     /* FP32 V-cycles per refinement step (0 = 1) */
  int bf16_levels;      /* levels with BF16 stencils under BMG_BF16_IR (0 = 2) */
  int use_graph;        /* 1 (default): replay one captured CUDA graph per cycle, autotune the
                           row-kernel tiles and run the coarse levels (n <= 63 FP32, n <= 15 FP64)
                           as one level-fused launch; 0: plain launches, one per step */
  int krylov;           /* BMG_KRYLOV_NONE (default): stationary V-cycle iteration;
                           BMG_KRYLOV_FCG: flexible CG with one cycle as preconditioner */
  const void* mlp;      /* bmg_mlp* for interp = BMG_INTERP_LEARNED, else NULL */
  void* stream;         /* cudaStream_t for setup and every later call on the hierarchy */
  int smoother;         /* Gauss-Seidel kernel of the cycle's 9-point levels (all choices compute
                           the same bits): BMG_SMOOTHER_AUTO (0, default; the autotuner picks per
                           level when use_graph = 1, else the row kernel), BMG_SMOOTHER_ROWS (row
                           kernel, in place), BMG_SMOOTHER_TILE + s (one-pass kernel with shape s
                           on every level outside the level-fused tail and the coarsest: FP32
                           cycles s = 0 .. 5, FP64 cycles s = 0 .. 3), or BMG_SMOOTHER_PAIR + s
                           (FP32 cycles only: the same levels, pairs of sweeps as one two-sweep
                           pass); EINVAL for a choice the precision has no kernel for */
  int arith;            /* BMG_ARITH_ROUNDED (0, default): one rounding per operation, the oracle's
                           default arithmetic; BMG_ARITH_FUSED: every product that is added to or
                           subtracted from a running sum in the cycle (stencil row sums of the
                           residual, Gauss-Seidel and A p; the weighted restriction and
                           interpolation terms; squared-norm and inner-product accumulation; the
                           flexible-CG updates) is one fused multiply-add, in FP64 and FP32 alike.
                           Same expressions, same order, fewer roundings; setup, line relaxation
                           and the coarsest solve are unchanged */
  int fuse_restrict;    /* FP32 / BF16 levels whose two pre-smoothing sweeps run as one two-sweep
                           pass (nu1 = 2): BMG_FUSE_AUTO (0, default; the autotuner weighs one pass
                           that also forms the residual and restricts it -- temporal blocking --
                           against the two-sweep pass plus the separate residual + restriction),
                           BMG_FUSE_OFF, or BMG_FUSE_ON (always the fused pass).  Same bits. */
  int rhs_block;        /* batches of right-hand sides of one operator (bmg_batch_rhs), FP32 / BF16
                           levels swept by the one-pass kernel: BMG_RHS_BLOCK_AUTO (0, default; the
                           autotuner weighs sweeping 2 or 4 members per warp, each stencil value read
                           once for them, against one member per warp), BMG_RHS_BLOCK_OFF, or 2 / 4
                           (always that many per warp).  Same bits. */
  int periodic;         /* 0 (default): Dirichlet sides; BMG_PERIODIC_X | BMG_PERIODIC_Y: those axes
                           wrap around (see Periodic sides above).  Periodic hierarchies run FP64
                           V(nu1, nu2) cycles, stationary or as the preconditioner of flexible CG
                           (krylov), with point Gauss-Seidel, Dendy interpolation and the default
                           coarsest level, in either arithmetic mode, with or without graphs; other
                           options give EINVAL.  Their 9-point levels
                           are swept (the same bits either way) by two row-parity launches in place
                           (smoother ROWS), by the one-pass strip kernel into a second iterate
                           (smoother TILE), or, by default (AUTO), per level by whichever of the
                           two setup timed as faster */
} bmg_opts;

#define BMG_PERIODIC_X 1
#define BMG_PERIODIC_Y 2

#define BMG_RHS_BLOCK_AUTO 0
#define BMG_RHS_BLOCK_OFF 1

#define BMG_FUSE_AUTO 0
#define BMG_FUSE_OFF 1
#define BMG_FUSE_ON 2

#define BMG_ARITH_ROUNDED 0
#define BMG_ARITH_FUSED 1

#define BMG_SMOOTHER_AUTO 0
#define BMG_SMOOTHER_ROWS 1
#define BMG_SMOOTHER_TILE 2
#define BMG_SMOOTHER_PAIR 8   /* + s (s = 0 .. 3): pairs of sweeps as one two-sweep pass of shape s,
                                 single sweeps with one-pass shape 3 */
#define BMG_SMOOTHER_LINE 12  /* zebra x-line Gauss-Seidel on every level (FP64 and FP32 cycles, single
                                 problems): odd rows, then even rows, each solved exactly along x */
#define BMG_SMOOTHER_LINE_Y 13   /* zebra y-lines likewise: odd columns, then even columns, each solved
                                    exactly along y (for operators coupled strongly along y) */
#define BMG_SMOOTHER_LINE_XY 14  /* alternating lines: every sweep an x-line sweep, then a y-line sweep
                                    (anisotropy along x in some regions and along y in others) */

/* ---- whole solver ------------------------------------------------------ */

/* Build the hierarchy (Sec. 2: "construction of coarse programs through local
 * stencil operations"): Dendy interpolation and the Galerkin operator
 * A_c = P^T A P level by level down to `coarsest`, then the Cholesky factor of
 * the coarsest operator (Fig. 1 "Cholesky").  The stencil is copied; the caller
 * may free it on return.  nx x ny interior points: nx == ny == 2^m - 1 >= 3
 * natively, any 1 <= nx, ny <= 65535 by embedding (see "General sizes"; not
 * with learned interpolation).  Stencil planes are (ny+2) x (nx+2).  opts may
 * be NULL.  Returns BMG_EINVAL (sizes, kind, options), BMG_ENOMEM, BMG_ECUDA
 * or BMG_ESINGULAR; *out is NULL on failure. */
int bmg_setup(const bmg_stencil* A, int nx, int ny, const bmg_opts* opts, bmg_hierarchy** out);

/* Solve A x = rhs by V(nu1,nu2) cycles (Fig. 1) until ||r_k||/||r_0|| <= tol
 * (r_0 = rhs - A x_in, Euclidean norm over the interior) or `maxit` cycles.
 * With krylov = BMG_KRYLOV_FCG each iteration is one step of flexible CG
 * (one-term recurrence) preconditioned by one cycle from a zero guess, and the
 * test uses the recursively updated residual.  Norms and inner products sum in
 * one fixed order (rows b, b+G, ... per block b < G = min(n,1024), columns
 * t, t+256, ... per thread t < 256, then halving trees), so histories repeat
 * bit for bit.
 * rhs: device, (ny+2) x (nx+2) (the grid given to bmg_setup), read only.
 * x: device, same layout, in: initial guess, out: solution (its ghost ring is
 * not written).  iters, relres: host, may be
 * NULL.  Under BMG_FP32_IR / BMG_BF16_IR one "cycle" is one FP64 refinement
 * step around `inner_cycles` FP32 V-cycles.  Returns BMG_OK, BMG_ENOTCONV,
 * BMG_ENAN, BMG_EINVAL or BMG_ECUDA. */
int bmg_solve(bmg_hierarchy* h, const double* rhs, double* x, double tol, int maxit,
              int* iters, double* relres);

/* Residual norms [||r_0||, ||r_1||, ...] of the last solve, copied to the host
 * array out (capacity cap): the l2 norms the convergence test of the solve
 * loop takes after every cycle (Fig. 1's V-cycle repeated until the norm test
 * of Sec. 4 passes; ||r_k|| = ||f - A x_k|| over the interior points).  out is
 * caller-owned host memory (NULL: nothing is written); the hierarchy keeps
 * the history until the next solve or bmg_free.  Returns the number of entries
 * available (which may exceed cap; min(cap, that number) are written) or
 * BMG_EINVAL for a NULL hierarchy. */
int bmg_history(const bmg_hierarchy* h, double* out, int cap);

/* Measurement: enqueue `cycles` solve iterations (one V-cycle, or one
 * refinement step, plus the residual norm each) with no convergence test,
 * bracketed by CUDA events recorded on the hierarchy's own stream, and return
 * their elapsed device time in *ms.  The iterations replay the same CUDA graph
 * bmg_solve uses (when use_graph is set).  x: in/out iterate (device).  Waits
 * for completion. */
int bmg_time_cycles(bmg_hierarchy* h, const double* rhs, double* x, int cycles, double* ms);

/* Per-level, per-kernel device time of `cycles` iterations launched one step
 * at a time without the graph, each step bracketed by CUDA events on the
 * hierarchy's stream (the Fig. 10 breakdown).  Fills up to `cap` rows of the
 * host array `rows` and returns the number of rows. */
enum { BMG_K_RELAX = 0, BMG_K_RESID_RESTRICT = 1, BMG_K_INTERP = 2, BMG_K_COARSE = 3, BMG_K_NORM = 4,
       BMG_K_FINALIZE = 5, BMG_K_IR_UPDATE = 6, BMG_K_IR_RESIDUAL = 7, BMG_K_FCG = 8,
       BMG_K_TAIL = 9 /* the level-fused coarse levels, counted at their top level */,
       BMG_K_RELAX_PAIR = 10 /* two-sweep passes (each launch = two sweeps) */,
       BMG_K_PAIR_RESTRICT = 11 /* two sweeps + residual + restriction in one pass */ };
typedef struct {
  int level;            /* 0 = finest */
  int kernel;           /* BMG_K_* */
  int fp32;             /* 1 = a kernel of the FP32 inner cycle */
  int launches;         /* kernel launches summed into this row */
  double ms;            /* total device time */
} bmg_prof_row;
int bmg_profile(bmg_hierarchy* h, const double* rhs, double* x, int cycles, bmg_prof_row* rows, int cap);

/* Gauss-Seidel kernel the setup autotuner chose for level `level` of the cycle
 * the hierarchy runs (FP64 or FP32): the row kernel's cluster size (1, 2, 4,
 * 8), BMG_TILE_SWEEP + s when the one-pass tile kernel with tile shape s won
 * (warp strips of 56 x TY points; FP32 cycles: shapes 0 .. 3 stream rows by
 * bulk copies into 4 row slots, TY = W, 8, 16, 32 (W: the smallest even
 * height whose strips fit into one wave of resident warps), shapes 4, 5 load
 * rows into registers, TY = 32, 16; FP64 cycles: rows copied per lane into RING
 * slots, (TY, RING) = (W, 4), (16, 4), (W, 6), (8, 4), W the smallest even
 * height whose strips fit into one wave of resident warps), or 0 (default;
 * not tuned).  With periodic sides: BMG_TILE_SWEEP for a level swept by the
 * one-pass strip kernel, 1 for the row-parity pair (or, on a 5-point level 0,
 * one launch per colour), 0 for the coarsest level.  Every choice computes the
 * same bits. */
#define BMG_TILE_SWEEP 16
int bmg_tuned_cluster(const bmg_hierarchy* h, int level);

/* Shape (0 .. 3) of the two-sweep pass (temporal blocking: two Gauss-Seidel
 * sweeps for one read of the level's arrays, 48 x TY warp strips with
 * TY = W (one wave), 16, 32, 26 and 4, 4, 6, 4 row slots) that runs each pair of sweeps
 * on level `level` of an FP32 cycle, or -1 (sweeps one at a time).  Same bits
 * either way. */
int bmg_tuned_pair(const bmg_hierarchy* h, int level);

/* Number of levels, and the size n of level l (0 = finest; EINVAL for a
 * hierarchy with periodic sides, whose levels are not square). */
int bmg_num_levels(const bmg_hierarchy* h);
int bmg_level_size(const bmg_hierarchy* h, int level);

/* Interior points of level l along x and y (host outputs, either may be NULL):
 * n and n for a Dirichlet hierarchy, the two axes' counts with periodic sides.
 * EINVAL for a bad level. */
int bmg_level_shape(const bmg_hierarchy* h, int level, int* nx, int* ny);

/* Copy level `level`'s stencil (5 planes O,W,S,SW,NW, FP64, ghost couplings
 * zero) or its interpolation weights (8 planes, FP64; not for the coarsest
 * level) into device memory `out` of the matching size: planes of
 * (ny+2) x (nx+2) for level l's or level l+1's bmg_level_shape. */
int bmg_get_stencil(const bmg_hierarchy* h, int level, double* out);
int bmg_get_interp(const bmg_hierarchy* h, int level, double* out);

/* Kernel launches issued on the hierarchy's stream since setup (a counter kept
 * by the host side of the library). */
long long bmg_launch_count(const bmg_hierarchy* h);

/* Release everything the hierarchy owns: the level arrays of the setup
 * (stencils, the Fig. 2 interpolation weights, the coarsest Cholesky factor),
 * the solve loop's vectors, CUDA graphs, events and its stream, after waiting
 * for the hierarchy's queued work.  The caller's arrays (stencil, rhs, x) are
 * not touched.  NULL is a no-op; h must not be used afterwards. */
void bmg_free(bmg_hierarchy* h);

const char* bmg_strerror(int code);
const char* bmg_last_error(void);

/* ---- batched solver ---------------------------------------------------------
 * Many independent problems solved together: every stage of the cycle (a
 * level counted from the coarsest, so all problems in it share one size) is
 * one kernel launch over all problems, and one iteration of the whole batch is
 * one CUDA graph.  Each problem keeps its own hierarchy, convergence test and
 * history, and its arithmetic is that of a solo solve, so its iterates and
 * history equal those of bmg_solve on that problem bit for bit.  Stationary
 * cycles only (krylov must be BMG_KRYLOV_NONE); all problems share `kind`. */
typedef struct bmg_batch bmg_batch;   /* opaque, library-owned */

/* nprob problems; A[p] and n[p] as in bmg_setup (n[p] = 2^m - 1 >= coarsest).
 * opts (may be NULL) apply to every problem.  With opts->use_graph the row
 * tile of the Gauss-Seidel kernels of every stage with n >= 127 is chosen by
 * timing the candidates on scratch copies of that stage (autotuner); stages
 * with n >= 255 also time the one-pass kernel (FP64 and FP32/BF16) and the
 * two-sweep pass (FP32/BF16).  opts->smoother may force BMG_SMOOTHER_ROWS,
 * BMG_SMOOTHER_TILE + s (s = 0 .. 3, every precision) or BMG_SMOOTHER_PAIR + s
 * (FP32/BF16 only) on every stage outside the level-fused tails; line
 * relaxation and the other shapes are EINVAL. */
int bmg_setup_batched(int nprob, const bmg_stencil* A, const int* n, const bmg_opts* opts, bmg_batch** out);

/* A batch of k right-hand sides for the operator of hierarchy h (built by
 * bmg_setup, any options): the k members share h's stencils, interpolation
 * weights and Cholesky factor (read-only; h must outlive the batch and is not
 * modified) and own their iterates, right-hand sides and norm partials, so k
 * solves of one operator need one setup and run as one batch
 * (bmg_solve_batched: one launch per cycle stage for all k, one CUDA graph per
 * iteration; every member's iterates and history equal h's solve of that
 * right-hand side bit for bit).  opts as for bmg_setup_batched (stationary
 * cycles only; precision, if given, must equal h's; coarsest and bf16 levels
 * come from h).  Returns BMG_EINVAL, BMG_ENOMEM or BMG_ECUDA. */
int bmg_batch_rhs(const bmg_hierarchy* h, int k, const bmg_opts* opts, bmg_batch** out);

/* rhs[p], x[p]: host arrays of nprob device pointers, layouts as in bmg_solve.
 * iters, relres: host arrays of nprob entries (may be NULL).  Problems stop
 * individually at ||r_k||/||r_0|| <= tol.  Returns BMG_OK when all converged,
 * else BMG_ENOTCONV / BMG_ENAN (per-problem detail in iters, relres). */
int bmg_solve_batched(bmg_batch* b, const double* const* rhs, double* const* x, double tol, int maxit,
                      int* iters, double* relres);

/* History of problem p in the last batched solve (as bmg_history). */
int bmg_batched_history(const bmg_batch* b, int p, double* out, int cap);

/* `cycles` batch iterations with no convergence test, timed with CUDA events
 * on the batch's stream (as bmg_time_cycles). */
int bmg_time_cycles_batched(bmg_batch* b, const double* const* rhs, double* const* x, int cycles, double* ms);

/* Kernel launches issued for the batch since setup; the Gauss-Seidel kernel
 * the autotuner chose for stage `stage` (0 = coarsest): the row kernel's
 * cluster size, BMG_TILE_SWEEP + s for the one-pass kernel of shape s (stages
 * with n >= 255, FP64 or FP32/BF16; in FP32/BF16 stages pairs of sweeps may then
 * run as two-sweep passes), or 0 (not tuned). */
long long bmg_batched_launch_count(const bmg_batch* b);
int bmg_batched_tuned_cluster(const bmg_batch* b, int stage);

void bmg_free_batched(bmg_batch* b);   /* NULL is a no-op */

/* ---- learned interpolation ----------------------------------------------------
 * An extension, not in the paper: an 18-64-64-4 GELU network maps the 3x3
 * fine-stencil neighbourhood of each coarse point (features (a_W + a_E)/a_O and
 * (a_S + a_N)/a_O at each of the 9 points) to four logits, one per edge fine
 * neighbour.  An edge point between coarse points c1, c2 keeps Dendy's total
 * weight S_D = -(col_1 + col_2)/D and splits it as w_k = S_D u_k/(u_1 + u_2),
 * u_k = -col_k exp(logit of c_k); centre points use Dendy's centre formula.
 * Zero logits give Dendy's weights.  Parameters: MLP_PARAMS = 5636 floats,
 * W1 (18x64), b1, W2 (64x64), b2, W3 (64x4), b3, row-major (input index first).
 * Training loss over K test vectors v_k: L = (1/K) sum_k E_k / Eref_k,
 * E_k = ||v_k - P R v_k||_A^2 (R: values at coarse points). */
typedef struct bmg_mlp bmg_mlp;
int bmg_mlp_create(bmg_mlp** out);
int bmg_mlp_set_params(bmg_mlp* m, const float* host, int count);
int bmg_mlp_get_params(const bmg_mlp* m, float* host, int count);

/* The optimizer state of bmg_mlp_adam, for checkpoints: the first and second
 * moment estimates (count = MLP_PARAMS floats each, host) and the step
 * count.  get copies them out; set restores them (bmg_mlp_set_params resets
 * them to zero and the step to 0, so a resumed run sets the parameters first,
 * then the state).  EINVAL for NULL pointers, a wrong count or a negative step. */
int bmg_mlp_get_adam(const bmg_mlp* m, float* moment1, float* moment2, int* step, int count);
int bmg_mlp_set_adam(bmg_mlp* m, const float* moment1, const float* moment2, int step, int count);
/* One loss and gradient evaluation on one problem (FP32 network, FP64 weights
 * and loss): coef 5 planes (n+2)^2 (ghost couplings zero), vecs K planes
 * (n+2)^2 (device), eref K host values (NULL: loss normalised by the weights of
 * zero logits, which then also come back in eref_out if given).  loss: host.
 * grad: host array of MLP_PARAMS floats or NULL; the gradient also stays on the
 * device for bmg_mlp_adam. */
int bmg_mlp_loss_grad(bmg_mlp* m, int n, const double* coef, int K, const double* vecs, const double* eref,
                      double* loss, float* grad, double* eref_out, void* stream);
/* The two-grid training loss and its gradient on a batch of crops (the
 * training objective of the learned interpolation; not in the paper).  For
 * each crop c (an n x n Dirichlet problem, n = 7, 15 or 31) and error vector
 * e_ck, with the crop's learned P (network outputs on its features), A_c =
 * P^T A P and the two-grid error propagation of V(2,1) with an exact coarse
 * solve, E = S (I - P A_c^{-1} P^T A) S^2 (S: one four-colour Gauss-Seidel
 * sweep of A e = 0), the energy E_ck = ||E e_ck||_A^2 and
 *     loss = 1/(ncrop K) sum_ck E_ck / eref_ck.
 * The gradient with respect to P is (A P v - g) u^T - (A e2) v^T with
 * u = A_c^{-1} P^T A S^2 e, e2 = S^2 e - P u, g = S^T dloss/d(E e) and the
 * adjoint solve v = A_c^{-1} P^T g; it is chained to the logits and through
 * the network.  FP64 throughout except the FP32 network.
 *   coefs: device, ncrop x 5 planes (n+2)^2 (O, W, S, SW, NW; ghost ring and
 *          couplings to it ignored).  vecs: device, ncrop x K vectors
 *          (n+2)^2 (ghost ring ignored).  Caller-owned, read only.
 *   eref:  device, ncrop x K normalisers; NULL: only the energies of Dendy's
 *          weights (zero logits) are computed, into `energies` (loss and grad
 *          untouched) -- the normalisers of later calls.
 *   energies: device, ncrop x K, out.  loss: host, out (with eref).
 *   grad: host array of MLP_PARAMS floats or NULL; the gradient also stays on
 *          the device for bmg_mlp_adam.
 * Returns BMG_EINVAL (sizes, NULLs), BMG_ESINGULAR (a non-positive pivot of a
 * crop's A_c), BMG_ENAN (a non-finite loss) or BMG_ECUDA.  Synchronizes the
 * stream. */
int bmg_mlp_twogrid(bmg_mlp* m, int ncrop, int n, const double* coefs, int K, const double* vecs,
                    const double* eref, double* energies, double* loss, float* grad, void* stream);
/* Adam step (beta 0.9, 0.999, eps 1e-8) with the last gradient. */
int bmg_mlp_adam(bmg_mlp* m, float lr, void* stream);
/* Logits of every interior coarse point, row-major (jc outer), 4 per point,
 * from the BF16 tensor-core inference kernel: delta device floats (n_c^2 * 4). */
int bmg_mlp_infer(const bmg_mlp* m, int n, const double* coef, float* delta, void* stream);
/* The network's inputs: for every interior coarse point (rows jc outer), the
 * 18 features (a_W + a_E)/a_O and (a_S + a_N)/a_O at the 9 fine points of its
 * 3x3 block (dy outer, dx inner), formed in FP64 and rounded to FP32.
 * coef: device, 5 planes (n+2)^2, ghost couplings zero; X: device floats
 * (n_c^2 x 18). */
int bmg_mlp_features(int n, const double* coef, float* X, void* stream);
/* Interpolation weights (8 planes (n_c+2)^2, FP64) from logits delta. */
int bmg_learned_interp(int n, const double* coef, const float* delta, double* ci, void* stream);
/* Which interpolation the hierarchy kept at level 0 (BMG_INTERP_*), and the
 * measured V-cycle factors of the learned and the Dendy hierarchy: 15
 * stationary V(2,1) cycles on A x = 0 from a SplitMix64 start (stream
 * 0x5EED), factor (||r_15|| / ||r_5||)^(1/10); 0 if not measured. */
int bmg_interp_info(const bmg_hierarchy* h, int* used, double* factor_learned, double* factor_dendy);
/* SplitMix64 uniform[-1,1) values on the interior of an (n+2)^2 device array
 * (counter form, stream `seed`, interior point k = (j-1) n + (i-1)). */
int bmg_fill_uniform(int n, unsigned long long seed, double* x, void* stream);
void bmg_mlp_free(bmg_mlp* m);

/* Self-test of the bounded device-side wait that the bulk-copy form of the
 * one-pass sweep uses (no counterpart in the paper): one warp waits on an
 * mbarrier phase that nothing completes.  The wait must give up after its
 * poll limit (about a second), record the timeout and return, leaving the
 * context usable.  Returns BMG_OK when that happened, BMG_ECUDA otherwise. */
int bmg_wait_selftest(void);

/* ---- single steps, for testing and composition -------------------------
 * Stateless: every pointer is caller-owned device memory in the layouts above;
 * `kind` is 5 or 9 and `coef` holds 5 planes either way (kind 5 ignores SW, NW).
 * The caller zeroes ghost couplings (bmg_setup does it for the hierarchy). */

/* Dendy operator-dependent interpolation weights of one level (setup of
 * Fig. 1's "Interpolate" and of the Fig. 2 restriction).  coef: 5 planes
 * (n+2)^2; ci: out, 8 planes (n_c+2)^2 (entries outside the defined ranges
 * are set to 0). */
int bmg_dendy_interp(int n, const double* coef, double* ci, void* stream);

/* Galerkin coarse operator A_c = P^T A P as a coarse 9-point stencil.
 * coef: 5 planes (n+2)^2; ci: 8 planes (n_c+2)^2; coarse: out, 5 planes
 * (n_c+2)^2 with zero ghost ring and ghost couplings. */
int bmg_rap(int n, const double* coef, const double* ci, double* coarse, void* stream);

/* `sweeps` Gauss-Seidel sweeps in place on x (Fig. 1 "Gauss Seidel"):
 * red-black for kind 5, four colours (i,j parities (odd,odd), (even,odd),
 * (odd,even), (even,even)) for kind 9; x_p = (f_p - sum_{q!=p} a_pq x_q) * (1/a_pp). */
int bmg_relax(int n, int kind, const double* coef, const double* f, double* x, int sweeps, void* stream);

/* Zebra x-line Gauss-Seidel (Fig. 1 "Line" relaxation; the smoother for
 * operators coupled much more strongly along x than along y), `sweeps`
 * sweeps in place on x: the odd rows, then the even rows, each solved
 * exactly along x (Thomas algorithm) with the other rows held fixed; the
 * couplings to rows j - 1, j + 1 move to the right-hand side in the order
 * S, N, SW, NE, NW, SE.  coef, f, x as bmg_relax; work: device scratch of
 * (n+2)^2 doubles (the elimination multipliers).  Returns BMG_EINVAL or
 * BMG_ECUDA. */
int bmg_relax_line(int n, int kind, const double* coef, const double* f, double* x, double* work, int sweeps,
                   void* stream);

/* ---- debug build ------------------------------------------------------- */
/* libbmg_debug.so (the same sources compiled with -DBMG_DEBUG) checks, in its
 * cycle and setup kernels, the index of each global store and the source range
 * of each asynchronous row copy against the logical extent of the level array it
 * addresses (the (n+2)^2 points of a level, the guard bands of FP32 arrays
 * included for copies).  A failed check does not trap: the store is skipped
 * (a copy is zero-filled, or reads the array's first element so that its
 * transaction completes) and the first failure of each source file is
 * recorded.  bmg_solve, bmg_solve_batched, bmg_time_cycles, bmg_profile,
 * bmg_inner_cycle and the single-kernel entry points then return BMG_EBOUNDS
 * until the record is taken.  compute-sanitizer is not needed for it; the
 * release library compiles every check to the constant true. */
int bmg_debug_build(void);   /* 1 for libbmg_debug.so, 0 for libbmg.so */
/* The first failure recorded since the last call (the device is synchronized
 * first): returns 1 and fills site (a kernel family, bmg_debug_site_name),
 * index and extent, or returns 0 when there is none; then clears the records.
 * Release builds return 0. */
int bmg_debug_take(int* site, long long* index, long long* extent);
const char* bmg_debug_site_name(int site);
/* Test hook (debug builds; BMG_EINVAL in release builds): every later check
 * uses extent - k, so that accesses to the last k elements of each array
 * count as outside and are skipped; none of them leaves its array.  k = 0
 * restores the exact extents. */
int bmg_debug_shrink(long long k);

/* Zebra y-line Gauss-Seidel (the same relaxation with the axes exchanged),
 * `sweeps` sweeps in place on x: the odd columns, then the even columns, each
 * solved exactly along y (Thomas algorithm from j = 1 upward, sub-diagonal
 * a_S, super-diagonal a_N) with the other columns held fixed; the couplings
 * to columns i - 1, i + 1 move to the right-hand side in the order W, E, SW,
 * NE, SE, NW.  Arguments, scratch and errors as bmg_relax_line. */
int bmg_relax_line_y(int n, int kind, const double* coef, const double* f, double* x, double* work, int sweeps,
                     void* stream);

/* f_c = P^T (f - A x) with the Fig. 2 restriction (Fig. 1 "Residual",
 * "Restrict"); fc: out, (n_c+2)^2, interior written, ghost ring zeroed. */
int bmg_resid_restrict(int n, int kind, const double* coef, const double* ci, const double* x,
                       const double* f, double* fc, void* stream);

/* x += P e_c (Fig. 1 "Interpolate"); ec: (n_c+2)^2 with zero ghost ring. */
int bmg_interp_correct(int n, const double* ci, const double* ec, double* x, void* stream);

/* r = f - A x over the interior (ghost ring of r zeroed) and, if norm != NULL,
 * its Euclidean norm to host *norm. */
int bmg_residual(int n, int kind, const double* coef, const double* x, const double* f,
                 double* r, double* norm, void* stream);

/* bmg_residual without any device allocation.  The paper has no counterpart:
 * this entry point serves callers that cannot let the library allocate device
 * memory (a host framework that owns the device memory pool, allocation-free
 * real-time or callback paths, checks that forbid allocator calls in a region
 * of work).  Arguments, layouts and results are those of bmg_residual; r and
 * norm may each be NULL.  The partial sums of the norm live in one fixed
 * device array of the library (1024 partial sums + the result, 8 KiB, held by
 * every GPU that loads the library until the process exits); the kernel uses
 * min(n, 1024) of them, so every valid n fits, and a partial count beyond the
 * array is rejected with BMG_EINVAL.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and keeps it for the process;
 * make that first call before any stream capture, and do not call the entry
 * point again after a cudaDeviceReset of that device.  The call synchronizes
 * its stream before it returns.  All calls share the array: calls whose GPU
 * work overlaps (other streams or host threads) race on it, so serialise them.
 * Calls no cudaMalloc/cudaFree or allocating routine. */
int bmg_residual_noalloc(int n, int kind, const double* coef, const double* x, const double* f,
                         double* r, double* norm, void* stream);

/* Lower-triangular Cholesky factor L (row-major m x m, m = n^2, lexicographic
 * unknowns j outer, i inner) of a level's operator (Fig. 1 "Cholesky");
 * BMG_ESINGULAR on a non-positive pivot.  n <= 15. */
int bmg_coarse_factor(int n, const double* coef, double* L, void* stream);

/* x = (L L^T)^{-1} f on one level, FP64 forward and back substitution. */
int bmg_coarse_solve(int n, const double* L, const double* f, double* x, void* stream);

/* One FP32 inner V(nu1,nu2) cycle of a BMG_FP32_IR / BMG_BF16_IR hierarchy on a
 * caller-supplied FP32 right-hand side: e = V32(r32) from a zero guess.
 * r32, e32: device floats, (n+2)^2 (ghost ring of e32 not written). */
int bmg_inner_cycle(bmg_hierarchy* h, const float* r32, float* e32);

/* Measured FP64 instruction throughput of this GPU (giga-instructions per
 * second, dependent multiply-add chains on every SM), for roofline reports. */
int bmg_measure_fp64_rate(double* ginstr_per_s, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BMG_H */
