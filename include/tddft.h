/*
 * tddft.h -- C boundary of the GB300 library for the iterative
 * polarizability solve of Koval, Foerster and Coulaud (arXiv:1005.5340).
 *
 * At every frequency omega the library solves eq. sle,
 *     (1 - chi0(omega) K) X_k = chi0(omega) d_k ,
 * by restarted GMRES (Sec. 4.1) and returns P_ik(omega) = d_i . X_k
 * (eq. eqpolarizability).  chi0(omega) is never formed: chi0 . z is applied
 * in the five steps of Sec. 4.2 (Fig. f:flops, Table t:flops) with the
 * vertex contraction re-associated (W(z) = sum_nu z^nu V_nu, then W X_occ),
 * and K . z is a dense product (Sec. 4.1).  Everything runs on one GPU.
 *
 * Conventions for every entry point:
 *  - Complex vectors cross the boundary interleaved (re, im) in float64;
 *    a block of n_rhs vectors of length n_prod is n_rhs x n_prod complex,
 *    vector-major (vector r occupies entries [r*n_prod, (r+1)*n_prod)).
 *  - flags bit 0 (TDDFT_DEVICE_PTRS): the z/out/omega pointers of that call
 *    are device pointers; otherwise they are host pointers and the call copies
 *    through a device staging buffer on the context's stream and returns after
 *    the result is on the host.  Device-pointer calls are asynchronous on the
 *    context's stream.
 *  - Every call returns a status and never aborts or traps.  On failure,
 *    tddft_last_error() describes the cause.  A context is not thread-safe.
 *  - Inputs are deep-copied by tddft_create; the caller keeps ownership of
 *    its buffers and may free them on return.  Outputs are caller-allocated.
 */
#ifndef TDDFT_H_
#define TDDFT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tddft_ctx tddft_ctx;

typedef enum {
  TDDFT_OK = 0,
  TDDFT_ERR_INVALID_ARG = 1,   /* null pointer, eps <= 0, NaN/Inf input, bad option */
  TDDFT_ERR_SHAPE = 2,         /* inconsistent sizes or offsets */
  TDDFT_ERR_NOMEM = 3,         /* device or pinned host allocation failed */
  TDDFT_ERR_CUDA = 4,          /* a CUDA runtime call or kernel launch failed */
  TDDFT_ERR_NOT_CONVERGED = 5, /* some (omega, direction) did not reach tol */
  TDDFT_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
  TDDFT_ERR_UNSUPPORTED = 7    /* input outside what the GPU path implements */
} tddft_status;

#define TDDFT_DEVICE_PTRS 1

typedef enum {
  TDDFT_PREC_FP64 = 0,      /* every step in float64 */
  TDDFT_PREC_FP64_EMU = 1,  /* as TDDFT_PREC_FP64, but the three dense products of every
                               operator application (K z, X_virt^T beta, X_virt a) are
                               float64 products emulated on the bf16 tensor cores
                               (tddft_gemm_f64_emulated with 6 slices: error about
                               2^-42 |A|_row |B|_col K); vertex contractions, block dots,
                               Arnoldi and Givens stay native float64 */
  TDDFT_PREC_BF16X3_IR = 2, /* inner GMRES cycles whose products all run in split bf16
                               on the tensor cores (hi*hi + hi*lo + lo*hi, float32
                               accumulation): K z, steps 2 and 5 on the stored transition
                               vertex, both transforms; their Krylov basis in float32
                               with the Arnoldi coefficients, Givens rotations and
                               reductions in float64; right-hand sides and the residual
                               that ends each cycle in float64 (iterative refinement) */
  TDDFT_PREC_BF16X3_IR_EMU = 3, /* TDDFT_PREC_BF16X3_IR whose float64 right-hand sides and
                                   cycle-end residuals use emulated float64 products as in
                                   TDDFT_PREC_FP64_EMU, with the slice count chosen from tol
                                   so that their error stays well below it: 5 slices (about
                                   2^-35 |A|_row |B|_col K) for tol >= 1e-8, 6 for tol >=
                                   1e-12, 7 below */
  TDDFT_PREC_TF32_IR = 4,     /* as TDDFT_PREC_BF16X3_IR, but every product of the inner
                                 cycles is one TF32 product on the tensor cores
                                 (tcgen05 kind::tf32: operands rounded to 10 mantissa bits,
                                 float32 accumulation; relative error ~1e-3) */
  TDDFT_PREC_TF32_IR_EMU = 5  /* TDDFT_PREC_TF32_IR with the float64 right-hand sides and
                                 residuals of TDDFT_PREC_BF16X3_IR_EMU */
} tddft_precision;

/* Initial guesses of tddft_polarizability (Sec. 4.1 starts from zero; the
 * other two are warm starts from neighbouring solved frequencies). */
typedef enum {
  TDDFT_GUESS_ZERO = 0,    /* every right-hand side from x0 = 0 */
  TDDFT_GUESS_INTERP = 1,  /* frequency sweep in three passes (every 4th frequency and the
                              last from zero; then index 2 mod 4 from the solved neighbours
                              at distance 2; then the rest from distance 1), each guess the
                              linear interpolation of the two neighbours' solutions */
  TDDFT_GUESS_LEARNED = 2, /* the same sweep, each guess interpolation + the learned
                              correction of the network loaded by tddft_guess_load */
  TDDFT_GUESS_INTERP_SUBSPACE = 3,  /* the sweep with an augmentation subspace per frequency:
                                       the six neighbour solutions X_k(omega-), X_k(omega+)
                                       (k = 0, 1, 2) and the three interpolated guesses; each
                                       direction starts from the minimum-residual point of
                                       that span, ||chi0 d_k - A x|| minimised with A applied
                                       in the context's precision (9 products per frequency,
                                       3 per right-hand side) */
  TDDFT_GUESS_LEARNED_SUBSPACE = 4  /* the same with the learned guesses in the subspace */
} tddft_guess;

/*
 * One molecule (inputs of Sec. 2-3: eqs. lcao, vertex-ansatz,
 * matrix_self_energy; dipoles of eq. eqpolarizability).  Host pointers.
 *
 *  atom_orb_offset [n_atoms+1]: orbitals of atom A are
 *      [atom_orb_offset[A], atom_orb_offset[A+1]), at most 16 per atom.
 *  eigenvalues [n_orb]: Kohn-Sham energies (Hartree), non-decreasing.
 *  occupations [n_orb]: a step profile: the first n_occ entries equal and
 *      > 0, the rest 0 (closed-shell filling).  Other profiles are
 *      TDDFT_ERR_UNSUPPORTED.
 *  X [n_orb*n_orb]: LCAO coefficients, column-major: X[a + E*n_orb] = X_a^E
 *      (column E = state E).
 *  prod_atoms [2*n_prod]: (A, B) per product, A <= B; A == B is a local
 *      product, A < B a bilocal one.
 *  vertex_offset [n_prod+1], vertex[vertex_offset[n_prod]]: product mu owns
 *      the n_A x n_B row-major block V_mu^{ab} (a in A, b in B) at
 *      vertex[vertex_offset[mu]].  Local blocks must be symmetric; for a
 *      bilocal product the B x A entries are the transpose (implied).
 *  K [n_prod*n_prod]: f_Hxc^{mu nu}, row-major, symmetric
 *      (|K - K^T| <= 1e-12 |K| elementwise in max norm).
 *  dipole [3*n_prod]: d_i^mu, direction-major.
 */
typedef struct {
  int32_t n_atoms;
  const int32_t *atom_orb_offset;
  int32_t n_orb;
  const double *eigenvalues;
  const double *occupations;
  const double *X;
  int32_t n_prod;
  const int32_t *prod_atoms;
  const int64_t *vertex_offset;
  const double *vertex;
  const double *K;
  const double *dipole;
} tddft_system;

/* GMRES stopping rules (Sec. 4.1).  The error estimates use |A^-1| ~ the
 * Frobenius norm of the inverse of the square Krylov representation of A at
 * the cycle's latest step, and d = the dipole of the right-hand side's field
 * direction (P = <d|X>):
 *   eps_P = |A^-1| |<d|r>| / |<d|X>|,   eps_X = |A^-1| ||r|| / ||X||. */
typedef enum {
  TDDFT_STOP_RESIDUAL = 0, /* ||b - A x||_2 / ||b||_2 <= tol */
  TDDFT_STOP_EPS_P = 1,    /* eps_P <= tol (the paper's quick rule) */
  TDDFT_STOP_EPS_PX = 2    /* eps_P <= tol and eps_X <= tol (the paper's combined rule) */
} tddft_stop_rule;

/*
 * Solver and resource options.
 *  prec: a tddft_precision.  With BF16X3_IR(_EMU), tddft_chi0_apply and
 *      tddft_apply_A use the reduced-precision operator (relative error
 *      ~1e-5) and tddft_kernel_apply stays float64 (emulated with _EMU).
 *  restart: GMRES restart length m (1..256).
 *  max_restarts: cycles before an (omega, direction) is declared not
 *      converged (>= 1).
 *  tol: the tolerance of the stopping rule (> 0).  With TDDFT_STOP_RESIDUAL
 *      the solve stops when ||b - A x||_2 / ||b||_2 <= tol, the residual
 *      recomputed in float64 at the end of each cycle.
 *  batch: maximum number of right-hand sides solved together (>= 1); sizes
 *      every device workspace allocated by tddft_create.
 *  stream: cudaStream_t for all work (NULL = legacy default stream).
 *  inner_tol: refinement forms only: a GMRES cycle (whose products are in
 *      reduced precision) also ends once its residual estimate has dropped
 *      by this factor; the float64 residual then starts the next cycle.
 *      In (0, 1); ignored for TDDFT_PREC_FP64 and TDDFT_PREC_FP64_EMU.
 *  graph: how tddft_polarizability drives the GMRES iterations of a group.
 *      0 = one launch sequence per iteration, sized on the host from the
 *      live count (an 8-byte read-back per iteration).
 *      1 = one iteration (selection, gathers, operators, Arnoldi/Givens/
 *      residual updates) captured in a CUDA graph and replayed, every kernel
 *      reading the live count on the device; the host checks for completion
 *      every few replays.
 *      2 = the whole loop on the device: one graph launch per group, whose
 *      conditional WHILE node repeats the captured iteration until no
 *      right-hand side of the group is live; the host waits once per group.
 *      The loop is bounded by (max_restarts + 1)(restart + 1) + 4
 *      iterations (beyond it: TDDFT_ERR_TIMEOUT).
 *      Per-kernel timing (tddft_timing_*) forces 0.
 *  stop: a tddft_stop_rule.  With the error estimates a cycle ends at the
 *      first Arnoldi step whose estimates (from the Givens/Hessenberg data
 *      and the cycle's <d|v_i>, <x0|v_i>, <d|A v_i>) meet the rule, and the
 *      solve ends when the rule holds for the float64 residual recomputed at
 *      the end of the cycle, with |A^-1| of the cycle's last step.
 *  emu_slices: slices of the emulated float64 products (TDDFT_PREC_FP64_EMU,
 *      TDDFT_PREC_BF16X3_IR_EMU, TDDFT_PREC_TF32_IR_EMU): 0 chooses them (6
 *      for FP64_EMU; from tol for the refinement forms), else 3..8.  Fewer
 *      slices are faster and coarser: s slices keep about 7 s + 1 bits of
 *      each row or column.
 *  n_tile: tensor-core forms: 0 lets the autotuner pick the N tile of each
 *      product at create; 64, 128 or 256 uses that tile for all of them.
 *  guess: a tddft_guess for tddft_polarizability (TDDFT_GUESS_LEARNED needs
 *      tddft_guess_load before the first solve).
 *  wait_timeout_ns: the limit of every wait inside the tensor-core kernels
 *      (mbarrier waits on copies, MMAs and the epilogue); 0 means 2 s.  On
 *      expiry the kernel records the failure, stops issuing work, lets its
 *      own copies and MMAs in flight finish (bounded by 2 s), frees its
 *      tensor memory and returns; the call then returns TDDFT_ERR_TIMEOUT
 *      and the context stays usable.  tddft_set_wait_timeout changes it.
 */
typedef struct {
  int32_t prec;
  int32_t restart;
  int32_t max_restarts;
  double tol;
  int32_t batch;
  void *stream;
  double inner_tol;
  int32_t graph;
  int32_t stop;
  int32_t emu_slices;
  int32_t n_tile;
  int32_t guess;
  int64_t wait_timeout_ns;
} tddft_options;

/* Change the wait limit of a context's tensor-core kernels (see
 * tddft_options.wait_timeout_ns; 0 = 2 s) for its later calls.
 * Synchronises the context's stream. */
tddft_status tddft_set_wait_timeout(tddft_ctx *ctx, int64_t wait_timeout_ns);

/* Per-(omega, direction) solver report. */
typedef struct {
  int32_t matvecs;   /* applications of A, residual checks included */
  int32_t cycles;    /* GMRES cycles started */
  double resid;      /* final ||b - A x|| / ||b|| (float64) */
  int32_t converged; /* 1 if the stopping rule was met */
  int32_t flags;     /* bit 0: a supplied initial guess was worse than zero and dropped */
  double eps_p;      /* final eps_P and eps_X (TDDFT_STOP_EPS_*; NaN with the residual rule) */
  double eps_x;
} tddft_solve_stats;

/*
 * Validate and upload one molecule; allocate every device workspace for up
 * to opts->batch right-hand sides.  *out receives the context.
 * Errors: INVALID_ARG (null, NaN/Inf, bad option), SHAPE, UNSUPPORTED
 * (occupations not a step profile, > 16 orbitals on an atom, K not
 * symmetric), NOMEM, CUDA.
 */
tddft_status tddft_create(const tddft_system *sys, const tddft_options *opts, tddft_ctx **out);

/*
 * out_r = chi0(omega_r) . z_r for r < n_rhs (eq. response-mat applied by the
 * steps of Table t:flops; Sec. 4.2).  omega [n_rhs] real frequencies
 * (Hartree), eps > 0 the broadening of eq. response-eig.  z, out:
 * n_rhs x n_prod complex interleaved.  1 <= n_rhs <= batch.
 */
tddft_status tddft_chi0_apply(tddft_ctx *ctx, int32_t n_rhs, const double *omega, double eps,
                              const double *z, double *out, int32_t flags);

/*
 * The float64 product of tddft_chi0_apply, for callers that cannot allocate
 * device memory when they need it -- for example code whose device memory is
 * entirely owned by another allocator, or that runs where a cudaMalloc would
 * be refused.  The paper has no counterpart: this is a deployment variant.
 *
 * It allocates nothing and does not use the context's workspace: every
 * intermediate lives in a 16 MiB block that the library reserves as a static
 * device array on each GPU that loads it (held until the process exits).
 * The context supplies only the molecule uploaded by tddft_create.
 *  - z, omega, out: DEVICE pointers (flags must include TDDFT_DEVICE_PTRS),
 *    same layouts as tddft_chi0_apply; float64 whatever the context's prec.
 *  - Scratch needed, in doubles, each term rounded up to a multiple of 32:
 *    4 n_rhs n_prod + 2 n_rhs n_blocks 256 + 2 n_rhs n_occ (2 n_orb + n_virt)
 *    + n_rhs; beyond 16 MiB the call returns TDDFT_ERR_SHAPE.
 *  - The first call on a device looks up the device address of the block
 *    (cudaGetSymbolAddress, no allocation); make that first call before any
 *    stream capture.
 *  - All calls share the one block: calls that overlap on the GPU (other
 *    streams, other threads, other contexts) race and corrupt each other.
 *    Nothing in the block needs clearing between calls.
 *  - Asynchronous on the context's stream.
 */
tddft_status tddft_chi0_apply_noalloc(tddft_ctx *ctx, int32_t n_rhs, const double *omega,
                                      double eps, const double *z, double *out, int32_t flags);

/* out_r = K . z_r (the precomputed kernel of Sec. 4.1); same layout rules. */
tddft_status tddft_kernel_apply(tddft_ctx *ctx, int32_t n_rhs, const double *z, double *out,
                                int32_t flags);

/*
 * Matrix-free K z from the product centres: a labelled variant of the
 * matrix-free Hartree product the paper names as future work (Sec. 8), in
 * the multipole form of Sec. 5 restricted to its monopole term, for kernels
 *     K_{mu nu} = g(|C_{c(mu)} - C_{c(nu)}|) + diag delta_{mu nu},
 *     g(r) = 1 / sqrt(r^2 + softening^2),
 * i.e. every product a point charge at its centre (the synthetic inputs'
 * kernel; extended product functions would add l > 0 moments, not built).
 * Products sharing a centre act through the centre's total charge, so
 *     (K z)_mu = diag z_mu + sum_c g(|C_{c(mu)} - C_c|) sum_{nu at c} z_nu
 * is exact up to rounding with n_centres^2 kernel evaluations per vector and
 * no stored K.  Float64, deterministic.
 *  centres [n_centres][3] (bohr) and prod_centre [n_prod] (centre index of
 *  each product, 0 <= c < n_centres): HOST pointers.  z, out: DEVICE
 *  pointers, n_rhs x n_prod complex interleaved.  stream: cudaStream_t
 *  (NULL = legacy default), synchronised before returning.  Allocates and
 *  frees its scratch (about 32 n_rhs n_centres bytes).
 * Errors: INVALID_ARG (NULL, sizes < 1, softening < 0 or NaN), SHAPE (a
 * centre index out of range), NOMEM, CUDA.
 */
tddft_status tddft_kernel_apply_centres(int32_t n_prod, int32_t n_centres, const double *centres,
                                        const int32_t *prod_centre, double softening, double diag,
                                        int32_t n_rhs, const double *z, double *out, void *stream);

/* out_r = A(omega_r) z_r = z_r - chi0(omega_r) (K z_r)  (Sec. 4.1). */
tddft_status tddft_apply_A(tddft_ctx *ctx, int32_t n_rhs, const double *omega, double eps,
                           const double *z, double *out, int32_t flags);

/*
 * The polarizability spectrum (eq. eqpolarizability via eq. sle).
 * For each omega[w] (w < n_omega) and field direction k < 3, GMRES solves
 * A(omega) X_k = chi0(omega) d_k from a zero initial guess; then
 * P[w][i][k] = d_i . X_k.  P: n_omega x 3 x 3 complex interleaved
 * (row i, column k).  stats (may be NULL): n_omega x 3 entries, index w*3+k.
 * Right-hand sides are solved in groups of at most opts->batch.  Returns
 * NOT_CONVERGED (with P filled from the last iterate) if any entry missed tol.
 */
tddft_status tddft_polarizability(tddft_ctx *ctx, int32_t n_omega, const double *omega,
                                  double eps, double *P, tddft_solve_stats *stats,
                                  int32_t flags);

/*
 * tddft_polarizability with checkpoint and resume.  Every (omega, direction)
 * is independent (Sec. 6.2.3), so a spectrum can be computed in pieces: the
 * frequencies of omega[] without a record in the file at `path` (created if
 * missing) are solved, in groups of the context's batch / 3 frequencies, and
 * each group's records are appended and synced to the file before the next
 * group starts; P and stats are then filled for every requested frequency,
 * solved now or read back.  A record holds omega, eps, P and the three
 * directions' statistics; frequencies are matched by the exact bits of omega
 * and eps.  The file's header fingerprints the problem (n_prod, n_orb, n_occ,
 * precision, stopping rule, restart, tol): a file of another problem is
 * refused (INVALID_ARG).  A record cut short by an interruption is dropped
 * and its frequency solved again.  Host pointers.  *n_solved (may be NULL)
 * receives the number of frequencies solved by this call.  Errors: as
 * tddft_polarizability, and INVALID_ARG for an unreadable or unwritable file.
 */
tddft_status tddft_polarizability_resume(tddft_ctx *ctx, int32_t n_omega, const double *omega,
                                         double eps, double *P, tddft_solve_stats *stats,
                                         const char *path, int32_t *n_solved);

/*
 * Adaptive frequency grid and pole extraction: the step the paper names as
 * its next one (Sec. 8, conclusions), for a spectrum resolved only where it
 * has structure.  The absorption is S(omega) = Im alpha_tr(omega) with
 * alpha_tr = -(P_xx + P_yy + P_zz) / 3 (alpha = -P, eq. eqpolarizability).
 *
 * Grid: n_initial uniform points on [w_lo, w_hi] (both included), then
 * rounds.  The first round takes every interval.  A round solves the
 * midpoints of its intervals longer than 2 min_step (whose midpoint is not
 * already a grid point), in ascending order and as many as the grid has room
 * for, with one tddft_polarizability call
 * (batched on the GPU).  Both halves of an interval go to the next round when
 * |S(mid) - (S(left) + S(right)) / 2| > rel_tol * max |S| over the grid so
 * far.  It stops when no interval is left or the grid holds max_points.
 *
 * Poles: each local maximum i of S on the final grid (S_i > S_{i-1},
 * S_i >= S_{i+1}, S_i > peak_floor * max S) is fitted on its five nearest
 * grid points (a window of five indices clamped to the grid) with one pole
 * and a constant background,
 *     alpha_tr(z) = g / (Omega^2 - z^2) + b,   z = omega + i eps,
 * by linear least squares in (p = Omega^2, b, q = g + b p):
 * alpha p + z^2 b - q = alpha z^2.  For an isolated transition this is the
 * exact form of the response of this model (its poles are the eigenvalues
 * Omega_n^2 of Delta^2 + W^1/2 M^T K M W^1/2, W = 2 (n_o - n_u) Delta).
 */
typedef struct {
  int32_t n_initial;   /* >= 2 */
  int32_t max_points;  /* >= n_initial; capacity of omega and P */
  double rel_tol;      /* > 0 */
  double min_step;     /* >= 0 (Hartree) */
  double peak_floor;   /* in [0, 1) */
} tddft_adaptive_options;

typedef struct {
  double omega;        /* Omega = sqrt(max(Re p, 0)) (Hartree) */
  double g_re, g_im;   /* the fitted residue g */
  double peak;         /* S at the grid maximum */
  double omega_peak;   /* the grid frequency of that maximum */
} tddft_pole;

/*
 * Run the adaptive grid on ctx (its precision, tol, stopping rule and batch)
 * and extract the poles.  Host buffers: omega [max_points] (ascending on
 * return), P [max_points][3][3] complex interleaved, poles [max_poles].
 * *n_points receives the grid size; *n_poles the number of peaks found (the
 * first max_poles of them, in ascending frequency, are written).
 * Errors: INVALID_ARG (null pointers, w_hi <= w_lo, eps <= 0, bad options),
 * and whatever tddft_polarizability returns (NOT_CONVERGED included), in
 * which case the outputs hold the grid solved so far.
 */
tddft_status tddft_spectrum_adaptive(tddft_ctx *ctx, double w_lo, double w_hi, double eps,
                                     const tddft_adaptive_options *opts, double *omega,
                                     double *P, int32_t *n_points, tddft_pole *poles,
                                     int32_t max_poles, int32_t *n_poles);

/*
 * tddft_polarizability with warm starts and the solutions returned.
 *  x0 (may be NULL): n_omega x 3 x n_prod complex interleaved, row w*3+k the
 *      initial guess of (omega[w], direction k).  Each guess first costs one
 *      float64 product A x0; if ||b - A x0|| > ||b||, zero is used instead
 *      (stats flags bit 0), so plain zero-guess GMRES is both the fallback
 *      and the arbiter of a guess.
 *  X (may be NULL): receives the solutions X_k(omega) in the same layout.
 *  x0 and X are device pointers: flags must include TDDFT_DEVICE_PTRS when
 *  either is given.  Everything else as tddft_polarizability.
 */
tddft_status tddft_polarizability_guess(tddft_ctx *ctx, int32_t n_omega, const double *omega,
                                        double eps, const double *x0, double *X, double *P,
                                        tddft_solve_stats *stats, int32_t flags);

/*
 * Tile shapes chosen by the autotuner of a refinement-form context: at
 * create, each tensor-core product (K z, X_virt^T beta, X_virt a) is timed
 * with 64-, 128- and 256-wide N tiles on the context's full batch (K z also
 * at half of it), best of four runs, and the fastest is kept.  n_tiles[0..2]
 * receive the widths (0 for a float64 context).
 */
tddft_status tddft_tuning(const tddft_ctx *ctx, int32_t *n_tiles);

/*
 * Launch plan of the split-bf16 K product (tensor-core forms) for n_rhs
 * right-hand sides (2 n_rhs real columns) with the context's N tile: *ncl
 * receives the cluster size (1: no clusters; 2..4: one CTA per N tile of an
 * M row block, in one cluster), *ksplit the number of K slices (1 or 2, the
 * slices added into a zeroed output).  Host-side query, no device work.
 */
tddft_status tddft_kproduct_plan(const tddft_ctx *ctx, int32_t n_rhs, int32_t *ncl,
                                 int32_t *ksplit);

/* Sizes of a context (any pointer may be NULL). */
tddft_status tddft_sizes(const tddft_ctx *ctx, int32_t *n_orb, int32_t *n_occ, int32_t *n_prod,
                         int32_t *n_blocks);

/*
 * Per-kernel timing.  While enabled, every kernel launch of the context is
 * bracketed by CUDA events on the context's stream; the totals are per kernel
 * class (the K product, vertex contraction, beta, the two transform GEMMs, the
 * D(omega) scaling, the block dot, the GMRES kernels).  Enabling resets the
 * totals.  tddft_timing_get synchronises the stream and returns, for class
 * i < tddft_timing_count(), its name (static string), the number of timed
 * launches, their summed device time in ms and the algorithmic float64
 * flops those launches performed (2 M N K for a GEMM; 0 where not counted).
 */
tddft_status tddft_timing_enable(tddft_ctx *ctx, int32_t on);
int32_t tddft_timing_count(const tddft_ctx *ctx);
tddft_status tddft_timing_get(tddft_ctx *ctx, int32_t i, const char **name, int32_t *launches,
                              double *total_ms, double *flops);
/*
 * Algorithmic bytes moved by the timed launches of class i, where counted
 * (0 otherwise).  The GMRES step counts on the device, per right-hand side
 * and step, the vectors it must read or write at least, a basis vector being
 * 2 n_prod elements of the basis type (float64, or float32 in the refinement
 * forms) and a float64 vector 16 n_prod bytes: for Arnoldi step j, 2 (j + 1)
 * + 3 basis vectors (v_0..v_j read for the inner products and again for the
 * update, v_{j+1} written and normalised) and A v_j; at a cycle end, j + 1
 * more basis vectors and x read and written; for a residual check, b and A x
 * read and v_0 written and normalised.  Synchronises the stream.
 */
tddft_status tddft_timing_bytes(tddft_ctx *ctx, int32_t i, double *bytes);

/*
 * Self-test of the split-bf16 tensor-core GEMM used by TDDFT_PREC_BF16X3_IR:
 * C^T = A B^T for deterministic pseudo-random A [M x K], B [N x K] (entries
 * uniform in [-1, 1) from a hash of (index, seed)), compared with a float64
 * product of the same operands, for both N-tile widths (128 and 64).
 * *max_rel_err = max |C - C_ref| / max |C_ref| over both.
 * Allocates and frees its own device buffers; synchronises the device.
 * Returns TIMEOUT if a bounded wait inside the GEMM gave up.
 */
tddft_status tddft_selftest_gemm(int32_t M, int32_t N, int32_t K, uint64_t seed,
                                 double *max_rel_err);

/*
 * The same self-test for the TF32 GEMM of TDDFT_PREC_TF32_IR (tcgen05
 * kind::tf32, Sec. 4.2 transforms in tf32): both operands rounded to tf32
 * (10 explicit mantissa bits), float32 accumulation; expected error
 * about 2^-11 relative per entry.  Same arguments, allocation and errors.
 */
tddft_status tddft_selftest_gemm_tf32(int32_t M, int32_t N, int32_t K, uint64_t seed,
                                      double *max_rel_err);

/*
 * Float64 matrix product emulated on the bf16 tensor cores (the dense
 * products of eqs. chi0-transform-1/-2 and of K z, Sec. 3, in float64
 * accuracy; used by TDDFT_PREC_FP64_EMU and TDDFT_PREC_BF16X3_IR_EMU):
 *     C[m*ldc + n] = sum_k A[m*lda + k] B[k*ldb + n],  m < M, n < N, k < K.
 * Device pointers (row-major, unaligned strides allowed); the stream
 * (cudaStream_t, NULL = legacy default) orders the work and is synchronised
 * before returning.  Each row of A and each column of B is scaled by a power
 * of two and cut into `slices` (3..8) integer slices of 7 bits; the slice
 * products are summed exactly in float32 on the tensor cores over chunks of
 * K and in 64-bit integers across chunks.  Error:
 *     |C - AB|_mn <= about (1 + (slices+1)/4) 2^(-7 slices) max_k|A_mk| max_k|B_kn| K
 * (2.3e-13 relative to that scale for 6 slices); an exact result whenever
 * the operands' entries are integers of at most 7*slices - 1 bits scaled
 * alike.  Allocates and frees its own slice buffers (about
 * (M+N) * slices * 2 bytes per K entry).  Errors: INVALID_ARG (NULL, sizes
 * < 1, slices outside 3..8), SHAPE (lda < K, ldb < N or ldc < N), NOMEM,
 * CUDA, TIMEOUT (a bounded wait inside the kernel gave up).
 */
tddft_status tddft_gemm_f64_emulated(int32_t M, int32_t N, int32_t K, const double *A,
                                     int64_t lda, const double *B, int64_t ldb, double *C,
                                     int64_t ldc, int32_t slices, void *stream);

/*
 * Learned initial guess (the frequency sweep solves a coarse grid from zero,
 * then each remaining frequency from its two solved neighbours omega- and
 * omega+).  A small network, the same for every product mu, maps per-product
 * features to a complex correction y_mu of the linear interpolation:
 *     x0_mu = (1 - t) X_mu(omega-) + t X_mu(omega+) + s y_mu ,
 * with t = (omega - omega-) / (omega+ - omega-) and s the rms of the two
 * neighbours.  Features (10 per product): Re/Im X(omega-)/s, Re/Im
 * X(omega+)/s, t, omega, (omega+ - omega-)/eps, bilocal flag, d_k^mu / rms(d_k),
 * ||V_mu|| / mean ||V||.  The guess enters tddft_polarizability_guess, where
 * zero-guess GMRES remains the fallback and the arbiter.
 *
 * Network: n_in -> width -> width -> n_out, tanh on the hidden layers,
 * float32 parameters packed [W1 (width x n_in, row-major), b1, W2, b2,
 * W3 (n_out x width), b3]; W3 and b3 start at zero, W1 and W2 uniform in
 * +-1/sqrt(fan_in) from a hash of (index, seed).  Training (float32) and
 * inference (bf16 weights, float32 activations) run in the library's kernels.
 * All row arrays are device pointers; a network is not thread-safe.
 */
typedef struct tddft_mlp tddft_mlp;

/* Allocate a network and scratch for up to max_rows rows on `stream`. */
tddft_status tddft_mlp_create(int32_t n_in, int32_t width, int32_t n_out, int64_t max_rows,
                              uint64_t seed, void *stream, tddft_mlp **out);
void tddft_mlp_destroy(tddft_mlp *mlp);
const char *tddft_mlp_last_error(const tddft_mlp *mlp);
int64_t tddft_mlp_num_params(const tddft_mlp *mlp);
/* Copy the packed parameters to (set = 0) or from (set = 1) a host buffer of
 * n = tddft_mlp_num_params floats; setting also resets the Adam state. */
tddft_status tddft_mlp_params(tddft_mlp *mlp, float *host, int64_t n, int32_t set);
/* Write the packed parameters to a file, or read them back into a network of
 * the same shape (this also resets the Adam state).  Format (little endian):
 * the 8 bytes "TDDFTMLP", int32 version 1, int32 n_in, width, n_out, int64
 * n_params, then n_params float32.  Errors: INVALID_ARG (null, unopenable or
 * truncated file, bad magic or version), SHAPE (another network's shape). */
tddft_status tddft_mlp_save(tddft_mlp *mlp, const char *path);
tddft_status tddft_mlp_load(tddft_mlp *mlp, const char *path);
/* Y [rows][n_out] = network(F [rows][n_in]); bf16 != 0 uses bf16 weights. */
tddft_status tddft_mlp_forward(tddft_mlp *mlp, int64_t rows, const float *F, float *Y,
                               int32_t bf16);
/* Gradient of sum_rows dY . Y with respect to the parameters (float32
 * forward then backward); copied to grad_host (n floats) when not NULL. */
tddft_status tddft_mlp_backward(tddft_mlp *mlp, int64_t rows, const float *F, const float *dY,
                                float *grad_host);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on the mean
 * over n_target targets of |x0 - x*|^2 / |x*|^2, where x0 = lin + s y and
 * the rows are n_target blocks of n_prod products.  lin, xstar: complex
 * interleaved [n_target][n_prod]; scale [n_target]; loss[n_target] receives
 * each target's relative squared error before the step. */
tddft_status tddft_mlp_train_step(tddft_mlp *mlp, int32_t n_target, int32_t n_prod, const float *F,
                                  const double *lin, const double *xstar, const double *scale,
                                  double *loss, float lr);
/* Features, interpolation and scale of n_target right-hand sides from the
 * solved rows X (complex interleaved, n_prod per row): target r takes rows
 * nb[2r] (omega-) and nb[2r+1] (omega+), weight t[r], frequency omega[r],
 * direction dir[r].  F [n_target*n_prod][10] float, lin [n_target][n_prod]
 * complex, scale [n_target].  On the context's stream. */
tddft_status tddft_guess_features(tddft_ctx *ctx, int32_t n_target, const int32_t *nb,
                                  const double *t, const double *omega, const int32_t *dir,
                                  double h_over_eps, const double *X, float *F, double *lin,
                                  double *scale);
/* x0 [n_target][n_prod] complex = lin + scale * Y (Y [rows][2]). */
tddft_status tddft_guess_combine(int64_t n_target, int32_t n_prod, const float *Y,
                                 const double *lin, const double *scale, double *x0,
                                 void *stream);

/*
 * Warm-started frequency sweep inside tddft_polarizability (and inside
 * tddft_polarizability_guess when x0 is NULL) for a context whose guess
 * mode (tddft_options.guess, tddft_set_guess) is not TDDFT_GUESS_ZERO.  The
 * paper solves each frequency from zero (Sec. 4.1) and names warm starts
 * from neighbouring frequencies as future work (Sec. 8).  The frequencies
 * must increase.  Passes (tddft_sweep_plan): every 4th frequency and the
 * last from zero; then the rest of index 2 mod 4; then the others, each
 * guessed from its two nearest solved neighbours omega- < omega < omega+ as
 * the interpolation (1 - t) X(omega-) + t X(omega+), plus s y with the
 * network's correction y for TDDFT_GUESS_LEARNED (features: the spacing
 * term is the pass's mean (omega+ - omega-) over eps).  Each guess is
 * arbitrated as in tddft_polarizability_guess, so every frequency meets the
 * same float64 tolerance whatever the mode.  Allocates its device buffers
 * per call (the solutions of all frequencies and one chunk's guesses).
 */
/* pass[i] (0, 1, 2) and the neighbours left[i], right[i] (-1 in pass 0) of
 * frequency i of an n_omega-point sweep.  Host only. */
tddft_status tddft_sweep_plan(int32_t n_omega, int32_t *pass, int32_t *left, int32_t *right);
/* Set the context's guess mode (a tddft_guess) for its later solves. */
tddft_status tddft_set_guess(tddft_ctx *ctx, int32_t guess);
/* Load the learned guess's network (a tddft_mlp_save file of a 10 -> width
 * -> width -> 2 network) into the context, replacing any earlier one; its
 * inference scratch is sized for the context's batch.  Errors: INVALID_ARG
 * (unreadable file), SHAPE (not 10 inputs and 2 outputs), NOMEM. */
tddft_status tddft_guess_load(tddft_ctx *ctx, const char *weights_path);

/*
 * Several molecules of uneven size solved together (every (molecule, omega,
 * direction) is an independent right-hand side).  tddft_batch_create makes
 * one context per molecule, each on a private stream, with the same options
 * (options.stream and options.graph are ignored).  tddft_batch_polarizability
 * solves the same omega grid (host pointer) for every molecule: in each
 * round, every molecule forms its next group of at most options.batch
 * right-hand sides, then one CUDA graph is launched once: it holds, for
 * every molecule, a conditional WHILE node (independent of the others, so
 * they run side by side) that repeats that molecule's device-driven GMRES
 * iteration until its group is done (the bound of options.graph = 2).  P (host): n_mol x n_omega x 3 x 3 complex interleaved;
 * stats (host, may be NULL): n_mol x n_omega x 3.  Returns NOT_CONVERGED if
 * any entry missed tol (P still filled).
 */
typedef struct tddft_batch tddft_batch;
tddft_status tddft_batch_create(int32_t n_mol, const tddft_system *systems,
                                const tddft_options *opts, tddft_batch **out);
tddft_status tddft_batch_polarizability(tddft_batch *batch, int32_t n_omega, const double *omega,
                                        double eps, double *P, tddft_solve_stats *stats);
/* The context of molecule i (owned by the batch; NULL if out of range). */
tddft_ctx *tddft_batch_context(tddft_batch *batch, int32_t i);
const char *tddft_batch_last_error(const tddft_batch *batch);
void tddft_batch_destroy(tddft_batch *batch);

/* Text of the last error on this context (never NULL; "" if none).  With
 * ctx == NULL: the last error of a failed tddft_create on this thread. */
const char *tddft_last_error(const tddft_ctx *ctx);

/* Release the context and every device buffer it owns.  NULL is a no-op. */
void tddft_destroy(tddft_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* TDDFT_H_ */
