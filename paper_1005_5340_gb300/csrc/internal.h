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
  // reduced-precision operator (split-bf16 tensor-core GEMMs)
  kcTcK, kcTcT1, kcTcT2, kcLpSplit,
  // solver
  kcGmresStep, kcGmresGather, kcGmresSelect, kcRhs, kcMisc,
  // float64 products emulated on the tensor cores (integer slices)
  kcOzSlice, kcOzK, kcOzT1, kcOzT2,
  // steps 2 and 5 on the stored transition vertex
  kcAlphaGather, kcTcStep2, kcTcStep5, kcOzStep2, kcOzStep5,
  // small kernels of the tensor-core forms: D(omega) terms, sum of the step-5 partials
  kcDterm, kcCombine, kcCount
};
const char *kernel_class_name(int k);
// Record msg as the context's last error (tddft_last_error) and return s.
tddft_status set_ctx_error(tddft_ctx *c, tddft_status s, const std::string &msg);

struct Timer {
  bool on = false;
  struct Rec { int cls; cudaEvent_t a, b; double flops; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  int launches[kcCount] = {};
  double ms[kcCount] = {};
  double flops[kcCount] = {};
  double bytes[kcCount] = {};
  // a device counter of algorithmic bytes (kernels whose traffic depends on
  // device state), added to class dev_bytes_cls at every resolve
  unsigned long long *dev_bytes = nullptr;
  int dev_bytes_cls = -1;
  cudaEvent_t get();
  void begin(cudaStream_t st, int cls, cudaEvent_t *a);
  void end(cudaStream_t st, int cls, cudaEvent_t a, double fl);
  void resolve();   // host-side; call after the stream has been synchronised
  void reset();
  void destroy();
};

struct OzWork;
struct AlphaRoute;

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
  AlphaRoute *ar = nullptr;   // with oz: steps 2 and 5 on the stored transition vertex
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
// Step 5 (block dots) for ncols real columns in float64, gamma [n_orb][ncols][n_occ].
cudaError_t launch_block_dot(cudaStream_t st, int ncols, const DevSystem &sys,
                             const double *Vpad, const double *Xo, const double *gamma,
                             const double *Zin, int subtract, double *Out, const int *dcnt);
cudaError_t launch_interleaved_to_planar(cudaStream_t st, int n_rhs, int n, const double *in,
                                         double *out);
cudaError_t launch_planar_to_interleaved(cudaStream_t st, int n_rhs, int n, const double *in,
                                         double *out);

// ---------------------------------------------------------------------------
// Reduced-precision operator (split bf16 on tcgen05, float32 elsewhere)
// ---------------------------------------------------------------------------
// One M tile of a grouped product (per-atom operands of steps 2 and 5 of
// Table t:flops): A rows row0 .. row0 + rows - 1 (rows <= 128), B columns
// from xoff (within each slice / split plane) over nkb 64-deep K blocks.
struct GTile {
  int row0, xoff, nkb, rows, atom, pad0, pad1, pad2;
};

enum TcEpi { kStoreF32 = 0, kDscaleSplit = 1, kBetaPartSplit = 2, kGammaCatSplit = 3, kPartialF32 = 4 };

// A bf16 operand [rows][2*Kp] ([hi | lo] planes) with its TMA descriptor.
struct TcOperand {
  CUtensorMap map;     // boxes of 64 x 128 rows
  CUtensorMap map64;   // boxes of 64 x 64 rows (the B operand of the 64-wide tile)
  CUtensorMap map256;  // boxes of 64 x 256 rows (the B operand of the 256-wide tile)
  bool has64 = false;
  bool tf32 = false;   // float32 rows of Kp tf32 values instead of split bf16
  int64_t rows = 0;
  int Kp = 0;
};

struct TcEpilogue {
  float *outF = nullptr;           // kStoreF32: C^T[n][m] at n*ldo + m
  void *outB = nullptr;            // kDscaleSplit: hi at n*ldo + m, lo at n*ldo + lo_off + m
                                   // (bf16; a tf32 float at n*ldo + m for tf32 operands)
  int64_t ldo = 0;
  int64_t lo_off = 0;
  int rows_out = 0;                // kDscaleSplit: rows m < rows_out written (zeros past M)
  const double *energy = nullptr;  // [n_orb]
  const float2 *eocc2 = nullptr;   // [n_occ] occupied energies as float (hi, lo)
  const float4 *dterm = nullptr;   // [S][M] omega_s -+ e_F as float (hi, lo, hi, lo)
  const double *omega = nullptr;   // [S]
  double eps = 0.0;
  double occ_value = 0.0;
  int n_occ = 0;
  int split_ok = 0;                // kStoreF32: the launch may split K in two (adds into outF)
  int ksplit = 1;                  // set by the launcher
  int ncl = 1;                     // set by the launcher: > 1, clusters of ncl CTAs, one per N tile
  const int *aoff = nullptr;       // kGammaCatSplit
  const int *orb_atom = nullptr;   // kGammaCatSplit
  const int *xoff5 = nullptr;      // kGammaCatSplit
  const int4 *parts = nullptr;     // kBetaPartSplit: the chunks' parts
};

cudaError_t make_operand_map(TcOperand &op, const void *base, int64_t rows, int Kp, int box_rows,
                             bool tf32 = false);
// Row-major bf16 [rows][cols] (cols a multiple of 64) with 128-byte swizzled
// boxes of 64 columns x box_rows rows.
cudaError_t encode_bf16_map(CUtensorMap *map, const void *base, int64_t rows, int64_t cols,
                            int box_rows);
// dcnt (may be NULL): columns beyond mul_n * (*dcnt) are skipped.
// bn: N tile of the kernel, 64, 128 or 256.
cudaError_t launch_gemm_tc(cudaStream_t st, const TcOperand &A, const TcOperand &B, int M, int N,
                           int epi, const TcEpilogue &ep, int *err, const int *dcnt = nullptr,
                           int mul_n = 0, int bn = 128);
// Grouped product over a tile table (see GTile):
//   kBetaPartSplit  (N tile 256) the table runs over (chunk k, E block b)
//                   entries (atom = k, row0 = B row base, xoff / nkb = the
//                   first part and the part count, rows = valid E); A =
//                   Ycat, its rows (the M axis, N columns of the launch,
//                   128-row tiles fastest) are the columns m = 2 s + p.  Each
//                   part (an atom's run of the chunk's orbitals) is a K loop
//                   of its own into its own columns c16 16 + e; the tile
//                   writes beta^T row E M + m, columns 16 k .. 16 k + 15 (hi at
//                   outB[row*ldo + col], lo at + lo_off), 16-byte stores
//   kPartialF32     one table entry per tile (A rows, up to 256: two M
//                   blocks sharing the B tile; B K offset and length);
//                   outF[m*ldo + n] for the valid rows
// (the plain launch_gemm_tc also takes kGammaCatSplit: row m = orbital (B, b),
// column n = (s n_occ + E) 2 + p -> Gcat split at row 2 s + p, column
// xoff5_B + b n_occ + E.)
cudaError_t launch_gemm_tc_grouped(cudaStream_t st, const TcOperand &A, const TcOperand &B,
                                   const GTile *tiles, int n_tiles, int N, int epi,
                                   const TcEpilogue &ep, int *err, const int *dcnt = nullptr,
                                   int mul_n = 0, int bn = 128);
void tc_init_attributes();
// Split K (ksplit 1 or 2) and cluster size (ncl 1..4) of a kStoreF32 product
// with split_ok (the K product): A of M rows and padded K Kp, N columns, N tile bn.
void tc_split_plan(int Kp, int M, int N, int bn, int *ksplit, int *ncl);

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Warm-started sweep (sweep.cu): frequencies solved per chunk, one solver
// group at most, and the learned network's rows (3 x frequencies x n_prod)
// at most kSweepMaxRows (its float32 activations: 2 x rows x width).
constexpr int64_t kSweepMaxRows = (int64_t)1 << 22;
inline int sweep_chunk_freqs(int slots, int n_prod) {
  const int64_t cw = slots / 3 > 1 ? slots / 3 : 1;
  const int64_t cap = kSweepMaxRows / (3 * (int64_t)n_prod);
  return (int)(cw < cap ? cw : (cap > 1 ? cap : 1));
}
tddft_status sweep_polarizability(tddft_ctx *c, int32_t n_omega, const double *omega, double eps,
                                  double *Xout, double *P, tddft_solve_stats *stats,
                                  int32_t flags);

struct LpWork {
  int slots = 0;
  bool tf32 = false;               // operands are float32 rows of tf32 values (same bytes)
  int KpK = 0, Kp1 = 0, Kp2 = 0;   // padded K of the K product, transform 1, transform 2
  __nv_bfloat16 *Ks = nullptr;     // [n_prod][2 KpK]   K split
  __nv_bfloat16 *XvTs = nullptr;   // [n_virt][2 Kp1]   X_virt^T split
  __nv_bfloat16 *Xvs = nullptr;    // [n_orb][2 Kp2]    X_virt split
  __nv_bfloat16 *Zb = nullptr;     // [2S][2 KpK]       operator input, split
  float *Yt = nullptr;             // [2S][n_prod]      K z
  __nv_bfloat16 *betaT = nullptr;  // [2 S n_occ][2 Kp1], row E*nc + 2s+p (nc live columns)
  __nv_bfloat16 *aT = nullptr;     // [2 S n_occ][2 Kp2]
  double *omega = nullptr;         // [S]
  int *err = nullptr;              // [1] device-side error code of the GEMM waits
  float2 *eocc2 = nullptr;         // [n_occ] occupied energies as float (hi, lo)
  float4 *dterm = nullptr;         // [S][n_virt] omega_s -+ e_F as float (hi, lo) pairs
  TcOperand opK, opXvT, opXv, opZ, opBeta, opA;
  AlphaRoute *ar = nullptr;        // steps 2 and 5 on the stored transition vertex
  int bnK = 128, bn1 = 128, bn2 = 128;   // N tiles chosen by the autotuner
  Timer *timer = nullptr;
  const int *dcnt = nullptr;  // graph replays: device count of live slots (NULL: all S)
};

cudaError_t lp_prepare_constants(cudaStream_t st, const DevSystem &sys, LpWork &lp);
// Time the N tiles (64, 128, 256) on this context's three products (the full batch; the
// K product also at half of it) and keep the fastest, best of four runs each.
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
  CUtensorMap map;     // boxes of 64 columns x box_rows rows
  CUtensorMap map96;   // B role only: boxes of 96 rows (has96)
  bool has96 = false;
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
// Slices of rows r < rows (live rows mul*dcnt) of X [rows][ldx] (first Kdim
// entries; with cols, entry k of row r is X[r][cols[k]], zero where cols[k] < 0).
cudaError_t launch_oz_slice_rows(cudaStream_t st, const double *X, int64_t ldx, int rows, int Kdim,
                                 OzOperand &op, const int *dcnt = nullptr, int mul = 0,
                                 const int *cols = nullptr);
// Slices of the columns n < N (live mul*dcnt) of X [Kdim][ldx]: operand row n
// holds column n of X.
cudaError_t launch_oz_slice_cols(cudaStream_t st, const double *X, int64_t ldx, int Kdim, int N,
                                 OzOperand &op, const int *dcnt = nullptr, int mul = 0);
enum OzEpiMode { kOzC = 0, kOzCT = 1, kOzBetaT = 2, kOzGammaCat = 3 };
struct OzEpilogue {
  int mode = kOzC;
  double *C = nullptr;
  int64_t ldc = 0;
  const int *aoff = nullptr;      // kOzBetaT, kOzGammaCat: atom orbital offsets
  const int *orb_atom = nullptr;  // kOzGammaCat: atom of each orbital
  const int *xoff5 = nullptr;     // kOzGammaCat: Gcat segment of each atom
  int n_occ = 0;
};
// Grouped or plain product with a chosen epilogue:
//   kOzC      C[m*ldc + n]                 kOzCT  C[n*ldc + m]
//   kOzBetaT  A row m = (atom A, E, c) of the step-2 operand:
//             beta^T[(n n_occ + E) ldc + ao_A + c]
//   kOzGammaCat  A row m = orbital (B, b), column n = j n_occ + E:
//             Gcat[j ldc + xoff5_B + b n_occ + E]
// tiles (device, n_tiles entries; max_nkb = largest nkb) or NULL for plain
// 128-row tiles of M rows.
cudaError_t launch_gemm_oz_ex(cudaStream_t st, const OzOperand &A, const OzOperand &B, int M,
                              int N, const OzEpilogue &ep, const GTile *tiles, int n_tiles,
                              int max_nkb, int *err, const int *dcnt = nullptr, int mul_n = 0);
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

// ---------------------------------------------------------------------------
// The stored transition vertex (alpha.cu): step 1 of Table t:flops,
//   alpha_nu^{cE} = sum_d V_nu^{cd} X_d^E ,
// kept for steps 2 (beta^{cE} = sum_nu alpha_nu^{cE} v^nu) and 5
// (n_mu = sum_{bE} alpha_mu^{bE} gamma_b^E) as per-atom dense operands:
//   step 2, atom A: rows (E, c) (c in A, row ao_A n_occ + E n_A + c), one
//           column per product of L_A (the products whose block holds A, in
//           increasing order), row length K2max; the right-hand side rows are
//           gathered into Ycat = [v^nu, nu in L_A] per atom (segments of
//           round_up(|L_A|, 64))
//   step 5, atom B: one row per product of L_B (rows rowoff5_B + index),
//           columns b n_occ + E (b in B), row length K5max; gamma is written
//           by the second transform into Gcat = [gamma_b^E] per atom (segments
//           of round_up(n_B n_occ, 64)); the per-atom partial sums of n_mu
//           (P2, one row per (atom, product)) are added per product.
// ---------------------------------------------------------------------------
struct AlphaRoute {
  int K2max = 0, K5max = 0;
  int64_t rows2 = 0;          // n_orb n_occ
  int rows5 = 0;              // sum_B |L_B|
  int kcat2 = 0, kcat5 = 0;   // Ycat, Gcat row lengths
  int n_tiles2 = 0, n_tiles5 = 0, max_nkb2 = 0, max_nkb5 = 0;
  double flops2 = 0.0, flops5 = 0.0;   // per real column
  GTile *tiles2 = nullptr, *tiles5 = nullptr;
  int *lcat = nullptr;        // [kcat2] product at each Ycat position (-1: padding)
  int2 *pos5 = nullptr;       // [n_prod] P2 rows of each product (y = -1: local product)
  int *xoff5 = nullptr;       // [n_atoms] Gcat segment of each atom
  int *orb_atom = nullptr;    // [n_orb]
  int ldp = 0;                // P2 row stride (2 S)
  // split bf16 (reduced-precision operator), or tf32 rows of the same bytes;
  // its step 2 runs over the parts of 16-orbital chunks: a2 [rows2p][K2max]
  // with row ((k nEB + b) 16 + c16) 16 + e, Ycat [2S][kcat2] per atom
  bool lp = false;
  bool tf32 = false;
  int n_tiles2p = 0;
  int64_t rows2p = 0;          // 256 ceil(n_orb / 16) ceil(n_occ / 16)
  GTile *tiles2p = nullptr;    // per (chunk, E block): row0, parts index (xoff) and
                               // count (nkb), valid E (rows), chunk (atom)
  int4 *parts = nullptr;       // {c16 start | n << 8, atom, Ycat K offset, K blocks}
  GTile *tiles5lp = nullptr;   // step 5 of the reduced-precision operator: 256-row entries
  int n_tiles5lp = 0;
  TcOperand a2, a5, ycat, gcat;
  __nv_bfloat16 *ycat_q = nullptr, *gcat_q = nullptr;   // [2S][2 kcat2c], [2S][2 kcat5]
  float *P2f = nullptr;
  // emulated float64
  bool emu = false;
  OzOperand oa2, oa5, oycat, ogcat;
  double *gcat64 = nullptr;   // [2S][kcat5]
  double *P2d = nullptr;      // [rows5][2S]
};
// Lists, tiles and both operand forms (lp: split bf16; emu: s slices);
// device buffers recorded in allocs.
cudaError_t alpha_setup(cudaStream_t st, const tddft_system *host, const DevSystem &sys,
                        AlphaRoute &ar, int slots, bool lp, bool emu, int slices,
                        std::vector<void *> &allocs);
// Ycat split bf16 from rows of Y (float32 or float64, row stride ld)
cudaError_t launch_alpha_gather_lp(cudaStream_t st, const AlphaRoute &ar, int ncols, const void *Y,
                                   bool y_f64, int64_t ld, const int *dcnt);
// Out[c][mu] = Zin - n (subtract) or n, n_mu summed from the per-atom partials
cudaError_t launch_alpha_combine(cudaStream_t st, const AlphaRoute &ar, int ncols, int n_prod,
                                 bool p_f64, const double *Zin, int subtract, double *Out,
                                 const int *dcnt);

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
  double2 *Gm = nullptr;    // [cap][(m+1)*(m+1)] basis Gram matrix, column k holds <v_i, v_k>, i <= k
  double *cs = nullptr;     // [cap][m]
  double2 *sn = nullptr;    // [cap][m]
  double2 *g = nullptr;     // [cap][m+1]
  double *V = nullptr;      // [cap][m+1][2][n_prod]
  float *Vf = nullptr;      // the same basis in float32 (refinement forms; then V is NULL)
  double *x = nullptr;      // [cap][2][n_prod]
  double *b = nullptr;      // [cap][2][n_prod]
  int *act = nullptr;       // [cap] active right-hand sides, in order
  int *act2 = nullptr;      // [cap] second list (right-hand sides awaiting A x) when split
  int *count = nullptr;     // [2]
  int *loopctl = nullptr;   // [2] device-driven loop: iterations run, 1 if the bound was hit
  unsigned long long *bytes = nullptr;   // [1] algorithmic bytes of the GMRES steps
  // stopping rule: 0 relative residual, 1 eps_P <= tol, 2 eps_P and eps_X <= tol
  // (Sec. 4.1 error estimates; the buffers below exist only for 1 and 2)
  int stop = 0;
  int *dir = nullptr;       // [cap] field direction of each right-hand side
  double *crit = nullptr;   // [cap][10] scalars of the estimates (gmres.cu)
  double2 *cvec = nullptr;  // [cap][3 m + 2] <d|v_i>, <x0|v_i>, <d|A v_i> of the cycle
  float *dipf = nullptr;    // [3][n_prod] dipoles in float32 (float32 basis with estimates)
  float *xf = nullptr;      // [cap][2][n_prod] x in float32 (float32 basis, rule 2)
};

cudaError_t launch_gmres_start(cudaStream_t st, const DevSystem &sys, GmresState &gs, int n,
                               const double *Bplanar /*[2n][n_prod]*/);
// split = 0: every live right-hand side in act (count[0]); split = 1: those in
// an Arnoldi step in act (count[0]), those awaiting A x in act2 (count[1]).
// min_b: with split, the float64 group runs only once min_b right-hand sides
// await it or no Arnoldi work is left (otherwise count[1] is reported as 0).
// Create-time constants of the GMRES state (the float32 dipoles).
cudaError_t launch_gmres_prepare(cudaStream_t st, const DevSystem &sys, GmresState &gs);
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
                            double *gs_omega, int *gs_dir);
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
