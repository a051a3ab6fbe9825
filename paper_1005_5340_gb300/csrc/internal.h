// Internal declarations shared by the CUDA translation units of libtddft.
// Nothing here crosses the C boundary (include/tddft.h).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tddft.h"

namespace tddft {

// Orbitals of one atom are padded to this many rows/columns in every
// per-block layout (vertex blocks, contracted blocks W).
constexpr int kMaxOrb = 16;
constexpr int kBlk = kMaxOrb * kMaxOrb;

// Algorithmic flops per real column of the block-sparse kernels (set at create).
struct SparseFlops {
  double beta = 0.0;   // 2 n_occ sum over adjacency entries of n_A n_B
  double dot = 0.0;    // G on the block pattern (twice for bilocal) + <V_mu, G>
};

// Device copy of one molecule in the layouts the kernels read.
struct DevSystem {
  int n_atoms = 0, n_orb = 0, n_occ = 0, n_virt = 0, n_prod = 0, n_blocks = 0;
  int n_adj = 0;
  SparseFlops sf;
  double occ_value = 0.0;      // n_o of every occupied state (n_u = 0)
  int *aoff = nullptr;         // [n_atoms+1]
  double *energy = nullptr;    // [n_orb]
  double *Xo = nullptr;        // [n_orb][n_occ]   Xo[a][E]  = X_a^E, E occupied
  double *XvT = nullptr;       // [n_virt][n_orb]  XvT[F][a] = X_a^{n_occ+F}
  double *Xv = nullptr;        // [n_orb][n_virt]  Xv[a][F]  = X_a^{n_occ+F}
  double *K = nullptr;         // [n_prod][n_prod] symmetric
  double *dip = nullptr;       // [3][n_prod]
  int2 *blk_atoms = nullptr;   // [n_blocks] (A, B), A <= B
  int *blk_ptr = nullptr;      // [n_blocks+1] into blk_prod
  int *blk_prod = nullptr;     // [n_prod] product index, grouped by block
  double *Vpad = nullptr;      // [n_prod][kBlk] vertex blocks in blk_prod order, zero padded
  int *adj_ptr = nullptr;      // [n_atoms+1]
  int4 *adj = nullptr;         // [n_adj] (block, other atom, transposed, 0)
  float *pfeat = nullptr;      // [n_prod][2] (bilocal flag, ||V_mu|| / mean ||V||)
};

// Optional per-kernel timing: CUDA events recorded on the launching stream
// around every launch of a kernel class; resolved when the host next waits.
enum KernelClass {
  // float64 operator
  kcGemmK = 0, kcVertex, kcBeta, kcGemmT1, kcDscale, kcGemmT2, kcSddmm,
  // reduced-precision operator (tensor-core GEMMs, float32 sparse kernels)
  kcTcK, kcLpVertex, kcLpBeta, kcTcT1, kcTcT2, kcLpSddmm, kcLpSplit,
  // solver
  kcGmresStep, kcGmresGather, kcGmresSelect, kcRhs, kcMisc,
  // float64 products emulated on the tensor cores (integer slices)
  kcOzSlice, kcOzK, kcOzT1, kcOzT2, kcCount
};
const char *kernel_class_name(int k);

struct Timer {
  bool on = false;
  struct Rec { int cls; cudaEvent_t a, b; double flops; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  int launches[kcCount] = {};
  double ms[kcCount] = {};
  double flops[kcCount] = {};
  cudaEvent_t get();
  void begin(cudaStream_t st, int cls, cudaEvent_t *a);
  void end(cudaStream_t st, int cls, cudaEvent_t a, double fl);
  void resolve();   // host-side; call after the stream has been synchronised
  void reset();
  void destroy();
};

struct OzWork;

// Workspace of the chi0 / A operator for up to `slots` right-hand sides.
// Real columns: c = 2*s + p, p = 0 real plane, 1 imaginary plane.
struct OpWork {
  int slots = 0;
  double *Y = nullptr;        // [2S][n_prod]   K z
  double *W = nullptr;        // [2S][n_blocks][kBlk]  sum_nu y^nu V_nu per block
  double *beta = nullptr;     // [n_orb][2S][n_occ]
  double *abuf = nullptr;     // [n_virt][2S][n_occ]
  double *gamma = nullptr;    // [n_orb][2S][n_occ]
  double *omega = nullptr;    // [S] frequency of each slot
  Timer *timer = nullptr;
  const int *dcnt = nullptr;  // graph replays: device count of live slots (NULL: all S)
  double *splitws = nullptr;  // split-K slices of the K product
  int64_t splitws_elems = 0;
  OzWork *oz = nullptr;       // non-NULL: the three GEMMs are emulated float64 products
};

enum OpMode { kChi0 = 0, kKernel = 1, kA = 2 };

// Launchers (stream-ordered, no synchronisation).  Return cudaGetLastError().
// dcnt (may be NULL): device count of live right-hand sides; rows beyond
// mul_m * count and columns beyond mul_n * count are skipped (0 = no limit).
// ws (may be NULL): workspace of ws_elems doubles for a deterministic split-K
// when the tile grid is too small to fill the GPU.
cudaError_t launch_gemm_f64(cudaStream_t st, int M, int N, int K, const double *A, int64_t lda,
                            const double *B, int64_t ldb, double *C, int64_t ldc,
                            const int *dcnt = nullptr, int mul_m = 0, int mul_n = 0,
                            double *ws = nullptr, int64_t ws_elems = 0);
cudaError_t launch_apply_operator(cudaStream_t st, const DevSystem &sys, OpWork &wk, int S,
                                  OpMode mode, double eps, const double *Zin, double *Out);
// Right-hand sides b = chi0(omega) d_k of a spectrum group (rows g0..g0+S-1,
// g -> omega_all[g/3], direction g%3).  W(d_k), beta and X_virt^T beta do not
// depend on omega, so they are formed once for the three directions (Z3, a3)
// and only the D(omega) scaling, the second transform and the block dot run
// per right-hand side.
cudaError_t launch_rhs_formation(cudaStream_t st, const DevSystem &sys, OpWork &wk, int S, int g0,
                                 const double *omega_all, double eps, double *Z3, double *a3,
                                 double *Out);
// Step 5 (block dots) for ncols real columns: float64 (gamma [n_orb][ncols][n_occ],
// Vpad/Xo double) or float32 (gamma^T [(s n_occ+E) 2+p][n_orb], Vpad/Xo float).
cudaError_t launch_block_dot(cudaStream_t st, bool f64, int ncols, const DevSystem &sys,
                             const void *Vpad, const void *Xo, const void *gamma,
                             const double *Zin, int subtract, double *Out, const int *dcnt);
cudaError_t launch_interleaved_to_planar(cudaStream_t st, int n_rhs, int n, const double *in,
                                         double *out);
cudaError_t launch_planar_to_interleaved(cudaStream_t st, int n_rhs, int n, const double *in,
                                         double *out);

// ---------------------------------------------------------------------------
// Reduced-precision operator (split bf16 on tcgen05, float32 elsewhere)
// ---------------------------------------------------------------------------
enum TcEpi { kStoreF32 = 0, kDscaleSplit = 1 };

// A bf16 operand [rows][2*Kp] ([hi | lo] planes) with its TMA descriptor.
struct TcOperand {
  CUtensorMap map;     // boxes of 64 x 128 rows
  CUtensorMap map64;   // boxes of 64 x 64 rows (the B operand of the 64-wide tile)
  bool has64 = false;
  int64_t rows = 0;
  int Kp = 0;
};

struct TcEpilogue {
  float *outF = nullptr;           // kStoreF32: C^T[n][m] at n*ldo + m
  __nv_bfloat16 *outB = nullptr;   // kDscaleSplit: hi at n*ldo + m, lo at n*ldo + lo_off + m
  int64_t ldo = 0;
  int64_t lo_off = 0;
  int rows_out = 0;                // kDscaleSplit: rows m < rows_out written (zeros past M)
  const double *energy = nullptr;  // [n_orb]
  const double *omega = nullptr;   // [S]
  double eps = 0.0;
  double occ_value = 0.0;
  int n_occ = 0;
};

cudaError_t make_operand_map(TcOperand &op, const void *base, int64_t rows, int Kp, int box_rows);
// Row-major bf16 [rows][cols] (cols a multiple of 64) with 128-byte swizzled
// boxes of 64 columns x box_rows rows.
cudaError_t encode_bf16_map(CUtensorMap *map, const void *base, int64_t rows, int64_t cols,
                            int box_rows);
// dcnt (may be NULL): columns beyond mul_n * (*dcnt) are skipped.
// bn: N tile of the kernel, 128 or 64.
cudaError_t launch_gemm_tc(cudaStream_t st, const TcOperand &A, const TcOperand &B, int M, int N,
                           int epi, const TcEpilogue &ep, int *err, const int *dcnt = nullptr,
                           int mul_n = 0, int bn = 128);
void tc_init_attributes();

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct LpWork {
  int slots = 0;
  int KpK = 0, Kp1 = 0, Kp2 = 0;   // padded K of the K product, transform 1, transform 2
  __nv_bfloat16 *Ks = nullptr;     // [n_prod][2 KpK]   K split
  __nv_bfloat16 *XvTs = nullptr;   // [n_virt][2 Kp1]   X_virt^T split
  __nv_bfloat16 *Xvs = nullptr;    // [n_orb][2 Kp2]    X_virt split
  float *Xo32 = nullptr;           // [n_orb][n_occ]
  float *Vpad32 = nullptr;         // [n_prod][kBlk]
  __nv_bfloat16 *Zb = nullptr;     // [2S][2 KpK]       operator input, split
  float *Yt = nullptr;             // [2S][n_prod]      K z
  float *W = nullptr;              // [2S][n_blocks][kBlk]
  __nv_bfloat16 *betaT = nullptr;  // [2 S n_occ][2 Kp1], row (s*n_occ+E)*2+p
  __nv_bfloat16 *aT = nullptr;     // [2 S n_occ][2 Kp2]
  float *gammaT = nullptr;         // [2 S n_occ][n_orb]
  double *omega = nullptr;         // [S]
  int *err = nullptr;              // [1] device-side error code of the GEMM waits
  TcOperand opK, opXvT, opXv, opZ, opBeta, opA;
  int bnK = 128, bn1 = 128, bn2 = 128;   // N tiles chosen by the autotuner
  Timer *timer = nullptr;
  const int *dcnt = nullptr;  // graph replays: device count of live slots (NULL: all S)
};

cudaError_t lp_prepare_constants(cudaStream_t st, const DevSystem &sys, LpWork &lp);
// Time both N tiles on this context's three products (full batch) and keep the faster.
cudaError_t lp_autotune(cudaStream_t st, const DevSystem &sys, LpWork &lp);
// Out[c][mu] (float64) = Zin - chi0 K Zin (kA) or chi0 Zin (kChi0), reduced precision.
cudaError_t launch_apply_operator_lp(cudaStream_t st, const DevSystem &sys, LpWork &lp, int S,
                                     OpMode mode, double eps, const double *Zin, double *Out);

// ---------------------------------------------------------------------------
// Float64 products emulated on the tensor cores (ozaki.cu)
// ---------------------------------------------------------------------------
// A float64 operand cut into s integer slices per row: row r is
//   x[r][k] = 2^e[r] * sum_i q_i[r][k] 2^(-7 i),   |q_1| <= 128, |q_i| <= 64,
// stored as exact bf16 integers [rows][s*Kp] (slice i at column i*Kp).
struct OzOperand {
  CUtensorMap map;
  __nv_bfloat16 *q = nullptr;
  int *e = nullptr;
  int64_t rows = 0;
  int Kp = 0;
  int s = 0;
};
constexpr int kOzMinSlices = 3, kOzMaxSlices = 8;
constexpr int kOzDefaultSlices = 6;

// Allocation-free set-up of an operand over caller-owned storage
// (q: rows * s * Kp bf16, 16-byte aligned; e: rows ints).  box_rows 128 for
// the A role, 64 for the B role.
cudaError_t oz_operand(OzOperand &op, __nv_bfloat16 *q, int *e, int64_t rows, int Kdim, int s,
                       int box_rows);
// Slices of rows r < rows (live rows mul*dcnt) of X [rows][ldx] (first Kdim entries).
cudaError_t launch_oz_slice_rows(cudaStream_t st, const double *X, int64_t ldx, int rows, int Kdim,
                                 OzOperand &op, const int *dcnt = nullptr, int mul = 0);
// Slices of the columns n < N (live mul*dcnt) of X [Kdim][ldx]: operand row n
// holds column n of X.
cudaError_t launch_oz_slice_cols(cudaStream_t st, const double *X, int64_t ldx, int Kdim, int N,
                                 OzOperand &op, const int *dcnt = nullptr, int mul = 0);
// C = A B^T over the sliced operands (A rows m < M, B rows n < N, shared K):
// C[m*ldc + n] (trans = 0) or C[n*ldc + m] (trans = 1), float64.
cudaError_t launch_gemm_oz(cudaStream_t st, const OzOperand &A, const OzOperand &B, int M, int N,
                           double *C, int64_t ldc, int trans, int *err, const int *dcnt = nullptr,
                           int mul_n = 0);

struct OzWork {
  int s = kOzDefaultSlices;
  OzOperand K, XvT, Xv;   // constants, A role
  OzOperand Z;            // [2S][s KpK] operator input, B role
  OzOperand Bt1, Bt2;     // [2S n_occ] rows: beta^T (K = n_orb), a^T (K = n_virt); one buffer
  int *err = nullptr;
};
cudaError_t oz_setup(cudaStream_t st, const DevSystem &sys, OzWork &oz, int slots,
                     std::vector<void *> &allocs);

// GMRES state of a group of right-hand sides (one per (omega, direction)).
struct GmresState {
  int cap = 0;          // right-hand sides allocated
  int m = 0;            // restart length
  int max_restarts = 0;
  double tol = 0.0;
  int *state = nullptr;     // [cap] 0 Arnoldi, 1 awaiting A x, 2 done
  int *jcur = nullptr;      // [cap]
  int *cycles = nullptr;    // [cap]
  int *matvecs = nullptr;   // [cap]
  int *conv = nullptr;      // [cap]
  int *flags = nullptr;     // [cap] bit 0: the supplied initial guess was rejected
  double *bnorm = nullptr;  // [cap]
  double *resid = nullptr;  // [cap]
  double *omega = nullptr;  // [cap]
  double *rho0 = nullptr;   // [cap] residual norm at the start of the current cycle
  double inner_tol = 0.0;   // cycle stops once |g| <= inner_tol * rho0 (refinement forms)
  double2 *H = nullptr;     // [cap][(m+1)*m] column-major
  double *cs = nullptr;     // [cap][m]
  double2 *sn = nullptr;    // [cap][m]
  double2 *g = nullptr;     // [cap][m+1]
  double *V = nullptr;      // [cap][m+1][2][n_prod]
  double *x = nullptr;      // [cap][2][n_prod]
  double *b = nullptr;      // [cap][2][n_prod]
  int *act = nullptr;       // [cap] active right-hand sides, in order
  int *act2 = nullptr;      // [cap] second list (right-hand sides awaiting A x) when split
  int *count = nullptr;     // [2]
};

cudaError_t launch_gmres_start(cudaStream_t st, const DevSystem &sys, GmresState &gs, int n,
                               const double *Bplanar /*[2n][n_prod]*/);
// split = 0: every live right-hand side in act (count[0]); split = 1: those in
// an Arnoldi step in act (count[0]), those awaiting A x in act2 (count[1]).
// min_b: with split, the float64 group runs only once min_b right-hand sides
// await it or no Arnoldi work is left (otherwise count[1] is reported as 0).
cudaError_t launch_gmres_select(cudaStream_t st, GmresState &gs, int n, int split, int min_b = 1);
cudaError_t launch_gmres_gather(cudaStream_t st, const DevSystem &sys, GmresState &gs,
                                const int *list, int S, double *Zc, double *slot_omega,
                                const int *dcnt = nullptr);
cudaError_t launch_gmres_step(cudaStream_t st, const DevSystem &sys, GmresState &gs,
                              const int *list, int S, const double *Wout,
                              const int *dcnt = nullptr);
// Right-hand sides g0..g0+n-1 of a spectrum (g -> omega g/3, direction g%3):
// Zc rows 2r, 2r+1 = (d_{g%3}, 0), slot and solver frequencies set.
cudaError_t launch_rhs_init(cudaStream_t st, const DevSystem &sys, int n, int g0,
                            const double *omega_all, double *Zc, double *slot_omega,
                            double *gs_omega);
// x of right-hand sides g0..g0+n-1 = rows of x0 (interleaved); their first
// product is then the residual of the guess.
cudaError_t launch_gmres_guess(cudaStream_t st, const DevSystem &sys, GmresState &gs, int n, int g0,
                               const double *x0);
// rows g0..g0+n-1 of X (interleaved) = x of each right-hand side
cudaError_t launch_gmres_export(cudaStream_t st, const DevSystem &sys, GmresState &gs, int n, int g0,
                                double *X);
// P[w][i][k] (complex) = d_i . x_g for g = w*3 + k in g0..g0+n-1.
cudaError_t launch_polarization(cudaStream_t st, const DevSystem &sys, GmresState &gs, int n,
                                int g0, double2 *P);

}  // namespace tddft
