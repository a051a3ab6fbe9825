// Float64 kernels of the matrix-free operator A(omega) z = z - chi0(omega) (K z)
// (Sec. 4.1) with chi0 . y applied by the steps of Sec. 4.2 (Fig. f:flops,
// Table t:flops), re-associated so that the vertex is read instead of the
// stored alpha object:
//   W_k(y)  = sum_{nu in block k} y^nu V_nu              (steps 1+2, per block)
//   beta    = W(y) X_occ                                 (steps 1+2)
//   a       = X_virt^T beta,  a^{FE} *= D_EF(omega)      (step 3 + denominator)
//   gamma   = X_virt a                                   (step 4)
//   n_mu    = sum_ab V_mu^{ab} (X_occ gamma^T)^{ab}      (step 5, blockdot.cu)
// Complex vectors are kept as two real planes; X, V and K are real, so only
// the D(omega) scaling mixes the planes.
#include <algorithm>

#include "internal.h"

namespace tddft {

// ---------------------------------------------------------------------------
// C[M x N] = A[M x K] . B[K x N], all row-major float64 (DFMA).
// BM x BN tile per CTA (64 x 64, or 32 x 128 when M is small so that few rows
// of the tile are wasted), 16-deep K slices staged in shared memory through
// registers (double buffered), (BM/16) x (BN/16) outputs per thread on a
// 16 x 16 thread grid.  Every edge is bounds-checked (ragged M, N, K).
// ---------------------------------------------------------------------------
namespace {
constexpr int GB_K = 16;

template <int BM, int BN>
__global__ void __launch_bounds__(256, (BM == 32 ? 2 : 3)) gemm_f64_nn(int M, int N, int K, const double *__restrict__ A,
                                                   int64_t lda, const double *__restrict__ B,
                                                   int64_t ldb, double *__restrict__ C,
                                                   int64_t ldc, const int *__restrict__ dcnt,
                                                   int mul_m, int mul_n, int kchunk,
                                                   int64_t zstride) {
  constexpr int TM = BM / 16, TN = BN / 16;     // outputs per thread
  constexpr int LA = BM * GB_K / 256, LB = BN * GB_K / 256;   // loads per thread
  __shared__ double As[2][GB_K][BM + 2];
  __shared__ double Bs[2][GB_K][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * BM;
  const int64_t n0 = (int64_t)blockIdx.x * BN;
  if (dcnt) {
    // graph replays: the live extent is read on the device
    const int c = *dcnt;
    if (mul_m) M = min(M, mul_m * c);
    if (mul_n) N = (int)min((int64_t)N, (int64_t)mul_n * c);
  }
  if (m0 >= M || n0 >= N) return;
  // split K: CTA z sums k in [z kchunk, (z+1) kchunk) into its own slice of C
  const int kb = blockIdx.z * kchunk;
  K = min(K, kb + kchunk) - kb;
  A += kb;
  B += (int64_t)kb * ldb;
  C += (int64_t)blockIdx.z * zstride;
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  double ra[LA], rb[LB];
  auto load_regs = [&](int k0) {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int idx = tid + 256 * l;
      const int i = idx >> 4, kk = idx & 15;                  // A: BM rows x 16 k
      const int64_t gm = m0 + i;
      const int gk = k0 + kk;
      ra[l] = (gm < M && gk < K) ? A[gm * lda + gk] : 0.0;
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int idx = tid + 256 * l;
      const int kb = idx / BN, j = idx % BN;                  // B: 16 k x BN cols
      const int64_t gn = n0 + j;
      const int gkb = k0 + kb;
      rb[l] = (gn < N && gkb < K) ? B[(int64_t)gkb * ldb + gn] : 0.0;
    }
  };
  auto store_smem = [&](int buf) {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int idx = tid + 256 * l;
      As[buf][idx & 15][idx >> 4] = ra[l];
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int idx = tid + 256 * l;
      Bs[buf][idx / BN][idx % BN] = rb[l];
    }
  };

  const int nk = (K + GB_K - 1) / GB_K;
  if (nk > 0) {
    load_regs(0);
    store_smem(0);
  }
  __syncthreads();
  for (int t = 0; t < nk; ++t) {
    const int buf = t & 1;
    if (t + 1 < nk) load_regs((t + 1) * GB_K);
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      double a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (t + 1 < nk) store_smem(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn < N) C[gm * ldc + gn] = acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------
// W[c][k][ab] = sum_{nu in block k} Y[c][nu] * V_nu[ab]  (per block k, column c)
// One CTA per (block, group of 8 columns); thread t owns entry ab = t.
// ---------------------------------------------------------------------------
constexpr int VW_COLS = 8;

__global__ void __launch_bounds__(256) vertex_contract(int nb, int ncols, int n_prod,
                                                       const int *__restrict__ blk_ptr,
                                                       const int *__restrict__ blk_prod,
                                                       const double *__restrict__ Vpad,
                                                       const double *__restrict__ Y,
                                                       double *__restrict__ W,
                                                       const int *__restrict__ dcnt) {
  __shared__ double ys[32][VW_COLS];
  const int k = blockIdx.x;
  const int c0 = blockIdx.y * VW_COLS;
  if (dcnt) ncols = min(ncols, 2 * *dcnt);
  if (c0 >= ncols) return;
  const int t = threadIdx.x;
  const int p0 = blk_ptr[k], p1 = blk_ptr[k + 1];
  double acc[VW_COLS];
#pragma unroll
  for (int c = 0; c < VW_COLS; ++c) acc[c] = 0.0;
  for (int q0 = p0; q0 < p1; q0 += 32) {
    __syncthreads();
    {
      int pp = t / VW_COLS, c = t % VW_COLS;
      int q = q0 + pp;
      ys[pp][c] = (q < p1 && c0 + c < ncols) ? Y[(int64_t)(c0 + c) * n_prod + blk_prod[q]] : 0.0;
    }
    __syncthreads();
    const int qn = min(32, p1 - q0);
    for (int pp = 0; pp < qn; ++pp) {
      double v = Vpad[(int64_t)(q0 + pp) * kBlk + t];
#pragma unroll
      for (int c = 0; c < VW_COLS; ++c) acc[c] = fma(ys[pp][c], v, acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < VW_COLS; ++c)
    if (c0 + c < ncols) W[((int64_t)(c0 + c) * nb + k) * kBlk + t] = acc[c];
}

// ---------------------------------------------------------------------------
// beta[aoff[A]+a][c][E] = sum over blocks touching atom A of
//   (W_k or W_k^T)[a][b] * Xo[aoff[B]+b][E]
// One CTA per (atom A, group of 4 columns); thread = occupied state E.
// ---------------------------------------------------------------------------
constexpr int BT_COLS = 4;
constexpr int BT_THREADS = 128;

__global__ void __launch_bounds__(BT_THREADS) beta_kernel(
    int ncols, int nb, int n_occ, const int *__restrict__ aoff, const int *__restrict__ adj_ptr,
    const int4 *__restrict__ adj, const double *__restrict__ W, const double *__restrict__ Xo,
    double *__restrict__ beta, const int *__restrict__ dcnt) {
  __shared__ double Ws[BT_COLS][kMaxOrb][kMaxOrb + 1];
  __shared__ double Xs[kMaxOrb][BT_THREADS];
  const int A = blockIdx.x;
  const int c0 = blockIdx.y * BT_COLS;
  // ncols is the column stride of beta; nact the live columns
  const int nact = dcnt ? min(ncols, 2 * *dcnt) : ncols;
  if (c0 >= nact) return;
  const int nA = aoff[A + 1] - aoff[A];
  const int e0 = adj_ptr[A], e1 = adj_ptr[A + 1];
  for (int E0 = 0; E0 < n_occ; E0 += BT_THREADS) {
    const int E = E0 + threadIdx.x;
    double acc[BT_COLS][kMaxOrb];
#pragma unroll
    for (int c = 0; c < BT_COLS; ++c)
#pragma unroll
      for (int a = 0; a < kMaxOrb; ++a) acc[c][a] = 0.0;
    for (int e = e0; e < e1; ++e) {
      const int4 ent = adj[e];
      const int k = ent.x, B = ent.y, tr = ent.z;
      const int bo = aoff[B], nB = aoff[B + 1] - bo;
      // this entry's X_occ column: all loads issued together, parked in shared memory
      {
        double xr[kMaxOrb];
#pragma unroll
        for (int b = 0; b < kMaxOrb; ++b)
          xr[b] = (b < nB && E < n_occ) ? Xo[(int64_t)(bo + b) * n_occ + E] : 0.0;
        __syncthreads();
#pragma unroll
        for (int b = 0; b < kMaxOrb; ++b) Xs[b][threadIdx.x] = xr[b];
      }
      for (int i = threadIdx.x; i < BT_COLS * kBlk; i += BT_THREADS) {
        int c = i / kBlk, ab = i % kBlk, a = ab / kMaxOrb, b = ab % kMaxOrb;
        double v = 0.0;
        if (c0 + c < nact)
          v = tr ? W[((int64_t)(c0 + c) * nb + k) * kBlk + b * kMaxOrb + a]
                 : W[((int64_t)(c0 + c) * nb + k) * kBlk + a * kMaxOrb + b];
        Ws[c][a][b] = v;
      }
      __syncthreads();
      for (int b = 0; b < nB; ++b) {
        const double xv = Xs[b][threadIdx.x];
#pragma unroll
        for (int c = 0; c < BT_COLS; ++c)
#pragma unroll
          for (int a = 0; a < kMaxOrb; ++a) acc[c][a] = fma(Ws[c][a][b], xv, acc[c][a]);
      }
    }
    if (E < n_occ) {
#pragma unroll
      for (int c = 0; c < BT_COLS; ++c) {
        if (c0 + c >= nact) continue;
#pragma unroll
        for (int a = 0; a < kMaxOrb; ++a)
          if (a < nA) beta[((int64_t)(aoff[A] + a) * ncols + c0 + c) * n_occ + E] = acc[c][a];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// a[F][(2s, 2s+1)][E] *= D_EF(omega_s),
// D = n_E [1/(omega - Delta + i eps) - 1/(omega + Delta + i eps)],
// Delta = e_F - e_E  (eq. response-mat, both orderings of the pair merged).
// ---------------------------------------------------------------------------
// 1 / x for x > 0 of normal range (here x is a product of two sums of
// squares, between ~1e-10 and ~1e4): a float32 seed refined by two
// Newton-Raphson steps y <- y + y (1 - x y), each squaring the relative
// error (2^-23 -> 2^-46 -> below the float64 rounding).
__device__ __forceinline__ double recip_nr(double x) {
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"((float)x));
  double y = (double)yf;
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// D(omega) of one (occupied E, virtual F) pair, Delta = e_F - e_E:
// occ [1/(omega - Delta + i eps) - 1/(omega + Delta + i eps)] from
// xm = omega - Delta and xp = omega + Delta; the two denominators share one
// reciprocal: 1/Am = Ap / (Am Ap), 1/Ap = Am / (Am Ap).
__device__ __forceinline__ double2 d_factor(double xm, double xp, double eps, double occ) {
  const double e2 = eps * eps;
  const double Am = fma(xm, xm, e2), Ap = fma(xp, xp, e2);
  const double q = occ * recip_nr(Am * Ap);
  const double im2 = Ap * q, ip2 = Am * q;   // occ / Am, occ / Ap
  return make_double2(xm * im2 - xp * ip2, eps * (ip2 - im2));
}

// a[F][(2s, 2s+1)][E] *= D_EF(omega_s): one block per (F, s) row pair, the
// threads over E
__global__ void dscale_kernel(int n_virt, int S, int n_occ, double occ_value,
                              const double *__restrict__ energy, const double *__restrict__ omega,
                              double eps, double *__restrict__ a, const int *__restrict__ dcnt) {
  const int64_t row = blockIdx.x;   // F * S + s
  const int F = (int)(row / S), s = (int)(row - (int64_t)F * S);
  const int S_act = dcnt ? min(S, *dcnt) : S;
  if (F >= n_virt || s >= S_act) return;
  const double eF = energy[n_occ + F], w = omega[s];
  double *re_row = a + ((int64_t)F * 2 * S + 2 * s) * n_occ, *im_row = re_row + n_occ;
  for (int E = threadIdx.x; E < n_occ; E += blockDim.x) {
    const double delta = eF - energy[E];
    const double2 d = d_factor(w - delta, w + delta, eps, occ_value);
    const double re = re_row[E], im = im_row[E];
    re_row[E] = d.x * re - d.y * im;
    im_row[E] = d.x * im + d.y * re;
  }
}

__global__ void i2p_kernel(int n_rhs, int n, const double *__restrict__ in, double *__restrict__ out) {
  const int64_t total = (int64_t)n_rhs * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / n, mu = i % n;
    out[(2 * r) * n + mu] = in[2 * i];
    out[(2 * r + 1) * n + mu] = in[2 * i + 1];
  }
}

__global__ void p2i_kernel(int n_rhs, int n, const double *__restrict__ in, double *__restrict__ out) {
  const int64_t total = (int64_t)n_rhs * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / n, mu = i % n;
    out[2 * i] = in[(2 * r) * n + mu];
    out[2 * i + 1] = in[(2 * r + 1) * n + mu];
  }
}

// a[F][(2s, 2s+1)][E] = D_EF(omega_{(g0+s)/3}) * a3[F][(2k, 2k+1)][E], k = (g0+s) % 3:
// one block per (F, s) row pair, the threads over E
__global__ void rhs_expand_kernel(int n_virt, int S, int n_occ, int g0, double occ_value,
                                  const double *__restrict__ energy,
                                  const double *__restrict__ omega_all, double eps,
                                  const double *__restrict__ a3, double *__restrict__ a) {
  const int64_t row = blockIdx.x;   // F * S + s
  const int F = (int)(row / S), s = (int)(row - (int64_t)F * S);
  if (F >= n_virt) return;
  const int g = g0 + s, k = g % 3;
  const double eF = energy[n_occ + F], w = omega_all[g / 3];
  const double *src = a3 + ((int64_t)F * 6 + 2 * k) * n_occ;
  double *dst = a + ((int64_t)F * 2 * S + 2 * s) * n_occ;
  for (int E = threadIdx.x; E < n_occ; E += blockDim.x) {
    const double delta = eF - energy[E];
    const double2 d = d_factor(w - delta, w + delta, eps, occ_value);
    const double re = src[E], im = src[E + n_occ];
    dst[E] = d.x * re - d.y * im;
    dst[E + n_occ] = d.x * im + d.y * re;
  }
}

// Z3 rows (d_0, 0, d_1, 0, d_2, 0)
__global__ void dipole_rows_kernel(int n_prod, const double *__restrict__ dip, double *__restrict__ Z3) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n_prod; i += gridDim.x * blockDim.x) {
    const int k = i / n_prod, mu = i % n_prod;
    Z3[(2 * k) * n_prod + mu] = dip[(int64_t)k * n_prod + mu];
    Z3[(2 * k + 1) * n_prod + mu] = 0.0;
  }
}

int grid_for(int64_t total, int threads) {
  int64_t g = (total + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (int)(g < 1 ? 1 : g);
}
}  // namespace

// C[m][n] = sum over the split slices ws[z][m][n], in slice order (deterministic)
// (slices of zstride elements, rows of ldw; only the live M x N part is summed)
__global__ void splitk_reduce_kernel(int M, int N, int splits, const double *__restrict__ ws,
                                     int64_t zstride, int64_t ldw, double *__restrict__ C,
                                     int64_t ldc, const int *__restrict__ dcnt, int mul_m,
                                     int mul_n) {
  if (dcnt) {
    const int c = *dcnt;
    if (mul_m) M = min(M, mul_m * c);
    if (mul_n) N = (int)min((int64_t)N, (int64_t)mul_n * c);
  }
  const int64_t total = (int64_t)M * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = i / N, n = i % N;
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += ws[z * zstride + m * ldw + n];
    C[m * ldc + n] = s;
  }
}

cudaError_t launch_gemm_f64(cudaStream_t st, int M, int N, int K, const double *A, int64_t lda,
                            const double *B, int64_t ldb, double *C, int64_t ldc,
                            const int *dcnt, int mul_m, int mul_n, double *ws, int64_t ws_elems) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const bool small = M < 256;
  // Long reductions (the K product: K = n_prod) with few output tiles leave SMs
  // idle, so K is cut into slices of 2048 summed afterwards in a fixed order.
  // The slicing depends on K alone: every launch shape (host-driven or graph
  // replay, any batch) sums each output in the same order.
  constexpr int kSlice = 2048, kMaxSlices = 8;
  int kchunk = K, splits = 1;
  if (ws && K >= 2 * kSlice) {
    kchunk = std::max(kSlice, ((K + kMaxSlices - 1) / kMaxSlices + 15) / 16 * 16);
    splits = (K + kchunk - 1) / kchunk;
    if ((int64_t)splits * M * N > ws_elems) return cudaErrorInvalidValue;
  }
  double *out = splits > 1 ? ws : C;
  const int64_t ldo = splits > 1 ? N : ldc;
  const int64_t zstride = (int64_t)M * N;
  if (small) {
    dim3 grid((N + 127) / 128, (M + 31) / 32, splits);
    if (grid.y > 65535) return cudaErrorInvalidConfiguration;
    gemm_f64_nn<32, 128><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, out, ldo, dcnt, mul_m,
                                               mul_n, kchunk, zstride);
  } else {
    dim3 grid((N + 63) / 64, (M + 63) / 64, splits);
    if (grid.y > 65535) return cudaErrorInvalidConfiguration;
    gemm_f64_nn<64, 64><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, out, ldo, dcnt, mul_m,
                                              mul_n, kchunk, zstride);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  splitk_reduce_kernel<<<grid_for((int64_t)M * N, 256), 256, 0, st>>>(
      M, N, splits, ws, zstride, N, C, ldc, dcnt, mul_m, mul_n);
  return cudaGetLastError();
}

cudaError_t launch_interleaved_to_planar(cudaStream_t st, int n_rhs, int n, const double *in,
                                         double *out) {
  i2p_kernel<<<grid_for((int64_t)n_rhs * n, 256), 256, 0, st>>>(n_rhs, n, in, out);
  return cudaGetLastError();
}

cudaError_t launch_planar_to_interleaved(cudaStream_t st, int n_rhs, int n, const double *in,
                                         double *out) {
  p2i_kernel<<<grid_for((int64_t)n_rhs * n, 256), 256, 0, st>>>(n_rhs, n, in, out);
  return cudaGetLastError();
}

namespace {
struct Scope {
  Timer *t;
  cudaStream_t st;
  int cls;
  double flops;
  cudaEvent_t a = nullptr;
  Scope(Timer *t_, cudaStream_t st_, int cls_, double fl) : t(t_), st(st_), cls(cls_), flops(fl) {
    if (t && t->on) t->begin(st, cls, &a);
  }
  ~Scope() {
    if (t && t->on) t->end(st, cls, a, flops);
  }
};
}  // namespace

namespace {
// Step 2 on the stored transition vertex, emulated float64: rows of Ysrc
// (n_rows columns y, row stride n_prod) gathered per atom and sliced, then
// beta^T[(c n_occ + E)][a] (into wk.beta) per atom on the tensor cores.
cudaError_t alpha_beta_emulated(cudaStream_t st, const DevSystem &sys, OpWork &wk, int n_rows,
                                const double *Ysrc, const int *dcnt) {
  AlphaRoute &ar = *wk.ar;
  cudaError_t err;
  {
    Scope sc(wk.timer, st, kcOzSlice, 0.0);
    err = launch_oz_slice_rows(st, Ysrc, sys.n_prod, n_rows, ar.kcat2, ar.oycat, dcnt, 2, ar.lcat);
    if (err != cudaSuccess) return err;
  }
  Scope sc(wk.timer, st, kcOzStep2, n_rows * ar.flops2);
  OzEpilogue eb;
  eb.mode = kOzBetaT;
  eb.C = wk.beta;
  eb.ldc = sys.n_orb;
  eb.aoff = sys.aoff;
  eb.n_occ = sys.n_occ;
  return launch_gemm_oz_ex(st, ar.oa2, ar.oycat, 0, n_rows, eb, ar.tiles2, ar.n_tiles2,
                           ar.max_nkb2, wk.oz->err, dcnt, 2);
}

// Transform 2 (X_virt a, a = wk.abuf [n_virt][ncols n_occ]) written per atom
// into Gcat, step 5 per atom, and Out = Zin - n (subtract) or n.
cudaError_t alpha_dot_emulated(cudaStream_t st, const DevSystem &sys, OpWork &wk, int ncols,
                               const double *Zin, int subtract, double *Out, const int *dcnt,
                               int timer_class) {
  AlphaRoute &ar = *wk.ar;
  OzWork &oz = *wk.oz;
  const int64_t ncolE = (int64_t)ncols * sys.n_occ;
  cudaError_t err;
  {
    Scope sc(wk.timer, st, kcOzSlice, 0.0);
    err = launch_oz_slice_cols(st, wk.abuf, ncolE, sys.n_virt, (int)ncolE, oz.Bt2, dcnt,
                               2 * sys.n_occ);
    if (err != cudaSuccess) return err;
  }
  {
    Scope sc(wk.timer, st, timer_class,
             timer_class == kcOzT2 ? 2.0 * sys.n_virt * (double)sys.n_orb * ncolE : 0.0);
    OzEpilogue eg;
    eg.mode = kOzGammaCat;
    eg.C = ar.gcat64;
    eg.ldc = ar.kcat5;
    eg.aoff = sys.aoff;
    eg.orb_atom = ar.orb_atom;
    eg.xoff5 = ar.xoff5;
    eg.n_occ = sys.n_occ;
    err = launch_gemm_oz_ex(st, oz.Xv, oz.Bt2, sys.n_orb, (int)ncolE, eg, nullptr, 0, 0, oz.err,
                            dcnt, 2 * sys.n_occ);
    if (err != cudaSuccess) return err;
  }
  {
    Scope sc(wk.timer, st, kcOzSlice, 0.0);
    err = launch_oz_slice_rows(st, ar.gcat64, ar.kcat5, ncols, ar.kcat5, ar.ogcat, dcnt, 2);
    if (err != cudaSuccess) return err;
  }
  {
    Scope sc(wk.timer, st, kcOzStep5, ncols * ar.flops5);
    OzEpilogue ep;
    ep.mode = kOzC;
    ep.C = ar.P2d;
    ep.ldc = ar.ldp;
    err = launch_gemm_oz_ex(st, ar.oa5, ar.ogcat, 0, ncols, ep, ar.tiles5, ar.n_tiles5,
                            ar.max_nkb5, oz.err, dcnt, 2);
    if (err != cudaSuccess) return err;
  }
  Scope sc(wk.timer, st, kcCombine, 0.0);
  return launch_alpha_combine(st, ar, ncols, sys.n_prod, true, Zin, subtract, Out, dcnt);
}

// chi0 (or A) with every dense product emulated in float64 and steps 2 and
// 5 on the stored transition vertex; Y = K z (kA) or z (kChi0).
cudaError_t apply_alpha_emulated(cudaStream_t st, const DevSystem &sys, OpWork &wk, int S,
                                 OpMode mode, double eps, const double *Y, const double *Zin,
                                 double *Out) {
  const int ncols = 2 * S;
  const int64_t ncolE = (int64_t)ncols * sys.n_occ;
  OzWork &oz = *wk.oz;
  cudaError_t err = alpha_beta_emulated(st, sys, wk, ncols, Y, wk.dcnt);
  if (err != cudaSuccess) return err;
  {
    Scope sc(wk.timer, st, kcOzSlice, 0.0);
    err = launch_oz_slice_rows(st, wk.beta, sys.n_orb, (int)ncolE, sys.n_orb, oz.Bt1, wk.dcnt,
                               2 * sys.n_occ);
    if (err != cudaSuccess) return err;
  }
  {
    Scope sc(wk.timer, st, kcOzT1, 2.0 * sys.n_virt * (double)sys.n_orb * ncolE);
    err = launch_gemm_oz(st, oz.XvT, oz.Bt1, sys.n_virt, (int)ncolE, wk.abuf, ncolE, 0, oz.err,
                         wk.dcnt, 2 * sys.n_occ);
    if (err != cudaSuccess) return err;
  }
  {
    Scope sc(wk.timer, st, kcDscale, 0.0);
    dscale_kernel<<<(unsigned)std::max<int64_t>(1, (int64_t)sys.n_virt * S), 128, 0, st>>>(
        sys.n_virt, S, sys.n_occ, sys.occ_value, sys.energy, wk.omega, eps, wk.abuf, wk.dcnt);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  return alpha_dot_emulated(st, sys, wk, ncols, Zin, mode == kA ? 1 : 0, Out, wk.dcnt, kcOzT2);
}
}  // namespace

cudaError_t launch_rhs_formation(cudaStream_t st, const DevSystem &sys, OpWork &wk, int S, int g0,
                                 const double *omega_all, double eps, double *Z3, double *a3,
                                 double *Out) {
  if (S <= 0) return cudaSuccess;
  if (S > wk.slots) return cudaErrorInvalidValue;
  const int np = sys.n_prod;
  cudaError_t err;
  Scope sc(wk.timer, st, kcRhs, 0.0);
  dipole_rows_kernel<<<grid_for(3 * (int64_t)np, 256), 256, 0, st>>>(np, sys.dip, Z3);
  if (wk.oz && wk.ar) {
    // emulated float64 on the stored transition vertex: beta(d_k) and
    // X_virt^T beta once, then per right-hand side D(omega), X_virt a, step 5
    Timer *saved = wk.timer;
    wk.timer = nullptr;
    const int n6 = 6 * sys.n_occ;
    err = alpha_beta_emulated(st, sys, wk, 6, Z3, nullptr);
    if (err == cudaSuccess)
      err = launch_oz_slice_rows(st, wk.beta, sys.n_orb, n6, sys.n_orb, wk.oz->Bt1);
    if (err == cudaSuccess)
      err = launch_gemm_oz(st, wk.oz->XvT, wk.oz->Bt1, sys.n_virt, n6, a3, n6, 0, wk.oz->err);
    if (err == cudaSuccess) {
      rhs_expand_kernel<<<(unsigned)std::max<int64_t>(1, (int64_t)sys.n_virt * S), 128, 0, st>>>(
          sys.n_virt, S, sys.n_occ, g0, sys.occ_value, sys.energy, omega_all, eps, a3, wk.abuf);
      err = cudaGetLastError();
    }
    if (err == cudaSuccess)
      err = alpha_dot_emulated(st, sys, wk, 2 * S, nullptr, 0, Out, nullptr, kcRhs);
    wk.timer = saved;
    return err;
  }
  // omega-independent part for the three directions (6 real columns)
  {
    dim3 grid(sys.n_blocks, 1);
    vertex_contract<<<grid, 256, 0, st>>>(sys.n_blocks, 6, np, sys.blk_ptr, sys.blk_prod, sys.Vpad,
                                          Z3, wk.W, nullptr);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    dim3 gb(sys.n_atoms, 2);
    beta_kernel<<<gb, BT_THREADS, 0, st>>>(6, sys.n_blocks, sys.n_occ, sys.aoff, sys.adj_ptr,
                                           sys.adj, wk.W, sys.Xo, wk.beta, nullptr);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  const int n6 = 6 * sys.n_occ;
  if (wk.oz) {
    err = launch_oz_slice_cols(st, wk.beta, n6, sys.n_orb, n6, wk.oz->Bt1);
    if (err == cudaSuccess)
      err = launch_gemm_oz(st, wk.oz->XvT, wk.oz->Bt1, sys.n_virt, n6, a3, n6, 0, wk.oz->err);
  } else {
    err = launch_gemm_f64(st, sys.n_virt, n6, sys.n_orb, sys.XvT, sys.n_orb, wk.beta, n6, a3, n6);
  }
  if (err != cudaSuccess) return err;
  // per right-hand side: D(omega) a_k, X_virt a, block dot
  const int64_t ncolE = (int64_t)2 * S * sys.n_occ;
  rhs_expand_kernel<<<(unsigned)std::max<int64_t>(1, (int64_t)sys.n_virt * S), 128, 0, st>>>(
      sys.n_virt, S, sys.n_occ, g0, sys.occ_value, sys.energy, omega_all, eps, a3, wk.abuf);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (wk.oz) {
    err = launch_oz_slice_cols(st, wk.abuf, ncolE, sys.n_virt, (int)ncolE, wk.oz->Bt2);
    if (err == cudaSuccess)
      err = launch_gemm_oz(st, wk.oz->Xv, wk.oz->Bt2, sys.n_orb, (int)ncolE, wk.gamma, ncolE, 0,
                           wk.oz->err);
  } else {
    err = launch_gemm_f64(st, sys.n_orb, (int)ncolE, sys.n_virt, sys.Xv, sys.n_virt, wk.abuf,
                          ncolE, wk.gamma, ncolE);
  }
  if (err != cudaSuccess) return err;
  return launch_block_dot(st, 2 * S, sys, sys.Vpad, sys.Xo, wk.gamma, nullptr, 0, Out,
                          nullptr);
}

cudaError_t launch_apply_operator(cudaStream_t st, const DevSystem &sys, OpWork &wk, int S,
                                  OpMode mode, double eps, const double *Zin, double *Out) {
  if (S <= 0) return cudaSuccess;
  if (S > wk.slots) return cudaErrorInvalidValue;
  const int ncols = 2 * S;
  const int np = sys.n_prod;
  cudaError_t err;
  const double *Y = Zin;
  if (mode == kKernel || mode == kA) {
    // Y = Z K  (K symmetric, so row c of Y is K z_c)
    double *Yout = (mode == kKernel) ? Out : wk.Y;
    if (wk.oz) {
      // emulated: (K z_c)_mu = sum_nu K[mu][nu] z_c[nu], stored transposed
      {
        Scope sc(wk.timer, st, kcOzSlice, 0.0);
        err = launch_oz_slice_rows(st, Zin, np, ncols, np, wk.oz->Z, wk.dcnt, 2);
      }
      Scope sc(wk.timer, st, kcOzK, 2.0 * ncols * (double)np * np);
      if (err == cudaSuccess)
        err = launch_gemm_oz(st, wk.oz->K, wk.oz->Z, np, ncols, Yout, np, 1, wk.oz->err, wk.dcnt,
                             2);
    } else {
      Scope sc(wk.timer, st, kcGemmK, 2.0 * ncols * (double)np * np);
      err = launch_gemm_f64(st, ncols, np, np, Zin, np, sys.K, np, Yout, np, wk.dcnt, 2, 0,
                            wk.splitws, wk.splitws_elems);
    }
    if (err != cudaSuccess || mode == kKernel) return err;
    Y = wk.Y;
  }
  if (wk.oz && wk.ar) return apply_alpha_emulated(st, sys, wk, S, mode, eps, Y, Zin, Out);
  {
    Scope sc(wk.timer, st, kcVertex, 2.0 * ncols * (double)kBlk * np);
    dim3 grid(sys.n_blocks, (ncols + VW_COLS - 1) / VW_COLS);
    vertex_contract<<<grid, 256, 0, st>>>(sys.n_blocks, ncols, np, sys.blk_ptr, sys.blk_prod,
                                          sys.Vpad, Y, wk.W, wk.dcnt);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  {
    Scope sc(wk.timer, st, kcBeta, ncols * sys.sf.beta);
    dim3 grid(sys.n_atoms, (ncols + BT_COLS - 1) / BT_COLS);
    beta_kernel<<<grid, BT_THREADS, 0, st>>>(ncols, sys.n_blocks, sys.n_occ, sys.aoff, sys.adj_ptr,
                                             sys.adj, wk.W, sys.Xo, wk.beta, wk.dcnt);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  const int64_t ncolE = (int64_t)ncols * sys.n_occ;
  if (ncolE > INT32_MAX) return cudaErrorInvalidValue;
  const double tflops = 2.0 * sys.n_virt * (double)sys.n_orb * (double)ncolE;
  if (wk.oz) {
    // emulated: slices of the columns of beta (rows of beta^T), then X_virt^T beta
    {
      Scope sc(wk.timer, st, kcOzSlice, 0.0);
      err = launch_oz_slice_cols(st, wk.beta, ncolE, sys.n_orb, (int)ncolE, wk.oz->Bt1, wk.dcnt,
                                 2 * sys.n_occ);
    }
    Scope sc(wk.timer, st, kcOzT1, tflops);
    if (err == cudaSuccess)
      err = launch_gemm_oz(st, wk.oz->XvT, wk.oz->Bt1, sys.n_virt, (int)ncolE, wk.abuf, ncolE, 0,
                           wk.oz->err, wk.dcnt, 2 * sys.n_occ);
    if (err != cudaSuccess) return err;
  } else {
    Scope sc(wk.timer, st, kcGemmT1, tflops);
    err = launch_gemm_f64(st, sys.n_virt, (int)ncolE, sys.n_orb, sys.XvT, sys.n_orb, wk.beta,
                          ncolE, wk.abuf, ncolE, wk.dcnt, 0, 2 * sys.n_occ);
    if (err != cudaSuccess) return err;
  }
  {
    Scope sc(wk.timer, st, kcDscale, 0.0);
    dscale_kernel<<<(unsigned)std::max<int64_t>(1, (int64_t)sys.n_virt * S), 128, 0, st>>>(
        sys.n_virt, S, sys.n_occ, sys.occ_value, sys.energy, wk.omega, eps, wk.abuf, wk.dcnt);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  if (wk.oz) {
    {
      Scope sc(wk.timer, st, kcOzSlice, 0.0);
      err = launch_oz_slice_cols(st, wk.abuf, ncolE, sys.n_virt, (int)ncolE, wk.oz->Bt2, wk.dcnt,
                                 2 * sys.n_occ);
    }
    Scope sc(wk.timer, st, kcOzT2, tflops);
    if (err == cudaSuccess)
      err = launch_gemm_oz(st, wk.oz->Xv, wk.oz->Bt2, sys.n_orb, (int)ncolE, wk.gamma, ncolE, 0,
                           wk.oz->err, wk.dcnt, 2 * sys.n_occ);
    if (err != cudaSuccess) return err;
  } else {
    Scope sc(wk.timer, st, kcGemmT2, tflops);
    err = launch_gemm_f64(st, sys.n_orb, (int)ncolE, sys.n_virt, sys.Xv, sys.n_virt, wk.abuf,
                          ncolE, wk.gamma, ncolE, wk.dcnt, 0, 2 * sys.n_occ);
    if (err != cudaSuccess) return err;
  }
  {
    Scope sc(wk.timer, st, kcSddmm, ncols * sys.sf.dot);
    err = launch_block_dot(st, ncols, sys, sys.Vpad, sys.Xo, wk.gamma, Zin,
                           mode == kA ? 1 : 0, Out, wk.dcnt);
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

}  // namespace tddft
