// Frequency sweep with warm starts (interpolated or learned initial guesses).
//
// The paper solves every frequency from the zero guess (Sec. 4.1) and names
// the use of neighbouring frequencies as future work (Sec. 8).  The sweep
// solves the grid in three passes so that every guessed frequency has two
// solved neighbours:
//   pass 0: every 4th frequency and the last one, from zero;
//   pass 1: the other frequencies of index 2 mod 4, each from its nearest
//           solved neighbours (at distance 2);
//   pass 2: the rest, from their nearest solved neighbours (distance 1).
// The guess of (omega, direction k) is the linear interpolation of the two
// neighbours' solutions X_k, or that interpolation plus the learned
// per-product correction of the context's network (tddft_guess_load).  Each
// guess costs one float64 product and is dropped for zero when it is worse
// (tddft_polarizability_guess), so zero-guess GMRES stays the fallback.
// Host code only: every step runs in the library's kernels through its own
// entry points.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace tddft {
const DevSystem *ctx_system(const tddft_ctx *c);
cudaStream_t ctx_stream(const tddft_ctx *c);
void ctx_set_error(tddft_ctx *c, const char *msg);
int ctx_slots(const tddft_ctx *c);
int ctx_guess_mode(const tddft_ctx *c);
tddft_mlp *ctx_guess_net(const tddft_ctx *c);
tddft_status ctx_polarizability_groups(tddft_ctx *c, int32_t n_omega, const double *omega,
                                       double eps, const double *x0, double *X, double *P,
                                       tddft_solve_stats *stats, int32_t flags);
}  // namespace tddft

namespace {
using namespace tddft;

// Augmentation subspace of one frequency: the six neighbour solutions
// X_k(omega-), X_k(omega+) (k = 0, 1, 2) and the three guesses x0_k.
constexpr int kSub = 9;

// Gram data of frequency w (one CTA per frequency): G[w][i][j] = <W_i, W_j>
// and h[w][k][i] = <W_i, b_k> (complex, conjugate-linear in the first
// argument) over n_prod entries, with W = A U (kSub vectors) and b the three
// right-hand sides, all complex interleaved, vectors of one frequency
// adjacent.  Each thread accumulates, for one i at a time, the 12 products
// of W_i with W_0..8 and b_0..2 over its share of the entries; a block
// reduction in a fixed order finishes each (deterministic).
__global__ void __launch_bounds__(256) sub_gram_kernel(int n_prod, const double2 *__restrict__ W,
                                                       const double2 *__restrict__ B,
                                                       double2 *__restrict__ G,
                                                       double2 *__restrict__ h) {
  const int w = blockIdx.x;
  const double2 *Ww = W + (int64_t)w * kSub * n_prod;
  const double2 *Bw = B + (int64_t)w * 3 * n_prod;
  __shared__ double2 red[256];
  for (int i = 0; i < kSub; ++i) {
    double2 acc[kSub + 3];
#pragma unroll
    for (int j = 0; j < kSub + 3; ++j) acc[j] = make_double2(0.0, 0.0);
    for (int mu = threadIdx.x; mu < n_prod; mu += blockDim.x) {
      const double2 a = Ww[(int64_t)i * n_prod + mu];
#pragma unroll
      for (int j = 0; j < kSub + 3; ++j) {
        const double2 b = j < kSub ? Ww[(int64_t)j * n_prod + mu] : Bw[(int64_t)(j - kSub) * n_prod + mu];
        acc[j].x = fma(a.x, b.x, fma(a.y, b.y, acc[j].x));   // conj(a) b
        acc[j].y = fma(a.x, b.y, fma(-a.y, b.x, acc[j].y));
      }
    }
    for (int j = 0; j < kSub + 3; ++j) {
      red[threadIdx.x] = acc[j];
      __syncthreads();
      for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
          red[threadIdx.x].x += red[threadIdx.x + s].x;
          red[threadIdx.x].y += red[threadIdx.x + s].y;
        }
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        if (j < kSub)
          G[((int64_t)w * kSub + i) * kSub + j] = red[0];
        else
          h[((int64_t)w * 3 + (j - kSub)) * kSub + i] = red[0];
      }
      __syncthreads();
    }
  }
}

// x[w][k] = sum_i c[w][k][i] U[w][i] (complex, interleaved)
__global__ void sub_combine_kernel(int n_freq, int n_prod, const double2 *__restrict__ U,
                                   const double2 *__restrict__ c, double2 *__restrict__ x) {
  const int64_t total = (int64_t)n_freq * 3 * n_prod;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / n_prod;   // w * 3 + k
    const int mu = (int)(t - r * n_prod);
    const int64_t w = r / 3;
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int i = 0; i < kSub; ++i) {
      const double2 ci = c[r * kSub + i], u = U[(w * kSub + i) * n_prod + mu];
      re = fma(ci.x, u.x, fma(-ci.y, u.y, re));
      im = fma(ci.x, u.y, fma(ci.y, u.x, im));
    }
    x[t] = make_double2(re, im);
  }
}

// rows 3 w + k of D = (d_k, 0): the dipoles as complex vectors for n_freq frequencies
__global__ void sub_dipoles_kernel(int n_freq, int n_prod, const double *__restrict__ dip,
                                   double2 *__restrict__ D) {
  const int64_t total = (int64_t)n_freq * 3 * n_prod;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / n_prod;
    const int mu = (int)(t - r * n_prod);
    D[t] = make_double2(dip[(r % 3) * n_prod + mu], 0.0);
  }
}

// Solve the kSub x kSub Hermitian system (G + delta I) c = h by Cholesky
// (complex, in place on a copy); delta = 1e-12 max_i G_ii keeps a subspace
// with dependent vectors (interpolation lies in the span of the neighbours)
// solvable.  Returns false if a pivot is not positive.
bool solve_hermitian(const double2 *G, const double2 *h, double2 *c) {
  double L[kSub][kSub][2] = {};
  double dmax = 0.0;
  for (int i = 0; i < kSub; ++i) dmax = std::max(dmax, G[i * kSub + i].x);
  if (!(dmax > 0.0)) return false;
  const double delta = 1e-12 * dmax;
  for (int j = 0; j < kSub; ++j) {
    double d = G[j * kSub + j].x + delta;
    for (int k = 0; k < j; ++k) d -= L[j][k][0] * L[j][k][0] + L[j][k][1] * L[j][k][1];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[j][j][0] = ljj;
    for (int i = j + 1; i < kSub; ++i) {
      // G = L L^H with G[i][j] = <W_i, W_j>:  L_ij = (G_ij - sum_k L_ik conj(L_jk)) / L_jj
      double re = G[i * kSub + j].x, im = G[i * kSub + j].y;
      for (int k = 0; k < j; ++k) {
        // L_ik conj(L_jk)
        re -= L[i][k][0] * L[j][k][0] + L[i][k][1] * L[j][k][1];
        im -= L[i][k][1] * L[j][k][0] - L[i][k][0] * L[j][k][1];
      }
      L[i][j][0] = re / ljj;
      L[i][j][1] = im / ljj;
    }
  }
  // forward: L y = h ; backward: L^H c = y
  double y[kSub][2];
  for (int i = 0; i < kSub; ++i) {
    double re = h[i].x, im = h[i].y;
    for (int k = 0; k < i; ++k) {
      re -= L[i][k][0] * y[k][0] - L[i][k][1] * y[k][1];
      im -= L[i][k][0] * y[k][1] + L[i][k][1] * y[k][0];
    }
    y[i][0] = re / L[i][i][0];
    y[i][1] = im / L[i][i][0];
  }
  for (int i = kSub - 1; i >= 0; --i) {
    double re = y[i][0], im = y[i][1];
    for (int k = i + 1; k < kSub; ++k) {
      // conj(L_ki) c_k
      re -= L[k][i][0] * c[k].x + L[k][i][1] * c[k].y;
      im -= L[k][i][0] * c[k].y - L[k][i][1] * c[k].x;
    }
    c[i] = make_double2(re / L[i][i][0], im / L[i][i][0]);
  }
  return true;
}

struct DeviceBuffers {
  std::vector<void *> p;
  ~DeviceBuffers() {
    for (void *q : p) cudaFree(q);
  }
  template <class T>
  cudaError_t get(T **out, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) {
      p.push_back(q);
      *out = static_cast<T *>(q);
    }
    return e;
  }
};
}  // namespace

extern "C" tddft_status tddft_sweep_plan(int32_t n_omega, int32_t *pass, int32_t *left,
                                         int32_t *right) {
  if (n_omega < 1 || !pass || !left || !right) return TDDFT_ERR_INVALID_ARG;
  const int n = n_omega;
  std::vector<char> solved(n, 0);
  for (int i = 0; i < n; ++i) {
    pass[i] = -1;
    left[i] = right[i] = -1;
  }
  for (int i = 0; i < n; i += 4) pass[i] = 0;
  pass[n - 1] = 0;
  for (int i = 0; i < n; ++i) solved[i] = pass[i] == 0;
  for (int p = 1; p <= 2; ++p) {
    std::vector<int> idx;
    for (int i = 0; i < n; ++i)
      if (!solved[i] && (p == 2 || i % 4 == 2)) idx.push_back(i);
    for (int i : idx) {
      int l = i - 1, r = i + 1;
      while (l >= 0 && !solved[l]) --l;
      while (r < n && !solved[r]) ++r;
      pass[i] = p;
      left[i] = l;
      right[i] = r;
    }
    for (int i : idx) solved[i] = 1;
  }
  return TDDFT_OK;
}

namespace tddft {

// Minimum-residual projection of the guesses of m frequencies: for
// frequency w the subspace U_w holds the six neighbour solutions X_k(omega-),
// X_k(omega+) and the three guesses; W = A(omega_w) U_w and b_k = chi0 d_k in
// the context's operator (an initial guess needs no more accuracy), then
// each direction's guess is U_w c with c minimising ||b_k - W c|| (normal
// equations, Cholesky, on the host: 9 x 9 per right-hand side).
static tddft_status project_guesses(tddft_ctx *c, int m, const int *idx, const int32_t *left,
                                    const int32_t *right, const double *omc, double eps,
                                    int slots, int np, const double *Xall, const double *guess,
                                    double *U, double *Wv, double *Dv, double *Bv, double *Gd,
                                    double *hd, double *cd, double *om9, double *om3,
                                    double *xp) {
  cudaStream_t st = ctx_stream(c);
  const size_t vec = (size_t)np * 2, vb = vec * sizeof(double);
  cudaError_t e = cudaSuccess;
  std::vector<double> h9(kSub * m), h3(3 * m);
  for (int w = 0; w < m; ++w) {
    const int i = idx[w];
    for (int k = 0; k < 3; ++k) {
      const double *src[3] = {Xall + (size_t)(3 * left[i] + k) * vec,
                              Xall + (size_t)(3 * right[i] + k) * vec,
                              guess + (size_t)(3 * w + k) * vec};
      for (int q = 0; q < 3 && e == cudaSuccess; ++q)
        e = cudaMemcpyAsync(U + (size_t)(kSub * w + 3 * q + k) * vec, src[q], vb,
                            cudaMemcpyDeviceToDevice, st);
      h3[3 * w + k] = omc[w];
    }
    for (int q = 0; q < kSub; ++q) h9[kSub * w + q] = omc[w];
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(om9, h9.data(), h9.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(om3, h3.data(), h3.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    const int64_t total = (int64_t)m * 3 * np;
    sub_dipoles_kernel<<<(int)std::min<int64_t>((total + 255) / 256, 152 * 32), 256, 0, st>>>(
        m, np, ctx_system(c)->dip, (double2 *)Dv);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // h9 and h3 leave scope after the calls
  if (e != cudaSuccess) {
    ctx_set_error(c, cudaGetErrorString(e));
    return TDDFT_ERR_CUDA;
  }
  // W = A U and B = chi0 D, in batches of at most `slots` vectors
  for (int v0 = 0; v0 < kSub * m; v0 += slots) {
    const int nv = std::min(slots, kSub * m - v0);
    tddft_status s = tddft_apply_A(c, nv, om9 + v0, eps, U + (size_t)v0 * vec,
                                   Wv + (size_t)v0 * vec, TDDFT_DEVICE_PTRS);
    if (s != TDDFT_OK) return s;
  }
  for (int v0 = 0; v0 < 3 * m; v0 += slots) {
    const int nv = std::min(slots, 3 * m - v0);
    tddft_status s = tddft_chi0_apply(c, nv, om3 + v0, eps, Dv + (size_t)v0 * vec,
                                      Bv + (size_t)v0 * vec, TDDFT_DEVICE_PTRS);
    if (s != TDDFT_OK) return s;
  }
  sub_gram_kernel<<<m, 256, 0, st>>>(np, (const double2 *)Wv, (const double2 *)Bv,
                                     (double2 *)Gd, (double2 *)hd);
  std::vector<double2> G((size_t)m * kSub * kSub), h((size_t)3 * m * kSub), cc((size_t)3 * m * kSub);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G.data(), Gd, G.size() * sizeof(double2), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), hd, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    ctx_set_error(c, cudaGetErrorString(e));
    return TDDFT_ERR_CUDA;
  }
  for (int w = 0; w < m; ++w)
    for (int k = 0; k < 3; ++k) {
      double2 *ck = cc.data() + (size_t)(3 * w + k) * kSub;
      if (!solve_hermitian(G.data() + (size_t)w * kSub * kSub, h.data() + (size_t)(3 * w + k) * kSub,
                           ck)) {
        // a degenerate subspace: keep the guess itself (the last three vectors)
        for (int q = 0; q < kSub; ++q) ck[q] = make_double2(q == 6 + k ? 1.0 : 0.0, 0.0);
      }
    }
  e = cudaMemcpyAsync(cd, cc.data(), cc.size() * sizeof(double2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    const int64_t total = (int64_t)m * 3 * np;
    sub_combine_kernel<<<(int)std::min<int64_t>((total + 255) / 256, 152 * 32), 256, 0, st>>>(
        m, np, (const double2 *)U, (const double2 *)cd, (double2 *)xp);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    ctx_set_error(c, cudaGetErrorString(e));
    return TDDFT_ERR_CUDA;
  }
  return TDDFT_OK;
}

// The sweep behind tddft_polarizability (and tddft_polarizability_guess
// without x0) when the context's guess mode is not zero.  omega, P and X
// follow flags (X: device, may be NULL).
tddft_status sweep_polarizability(tddft_ctx *c, int32_t n_omega, const double *omega, double eps,
                                  double *Xout, double *P, tddft_solve_stats *stats,
                                  int32_t flags) {
  const bool dev = (flags & TDDFT_DEVICE_PTRS) != 0;
  const int mode0 = ctx_guess_mode(c);
  // the subspace modes use the interpolated or learned guesses as three of
  // the nine vectors of each frequency's projection
  const bool subspace = mode0 == TDDFT_GUESS_INTERP_SUBSPACE || mode0 == TDDFT_GUESS_LEARNED_SUBSPACE;
  const int mode = mode0 == TDDFT_GUESS_LEARNED_SUBSPACE ? (int)TDDFT_GUESS_LEARNED
                   : mode0 == TDDFT_GUESS_INTERP_SUBSPACE ? (int)TDDFT_GUESS_INTERP
                                                          : mode0;
  tddft_mlp *net = ctx_guess_net(c);
  if (mode == TDDFT_GUESS_LEARNED && !net) {
    ctx_set_error(c, "the learned guess needs a network: call tddft_guess_load first");
    return TDDFT_ERR_INVALID_ARG;
  }
  const DevSystem &sys = *ctx_system(c);
  const int np = sys.n_prod, n = n_omega;
  cudaStream_t st = ctx_stream(c);
  auto cuda_fail = [&](cudaError_t e) {
    ctx_set_error(c, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? TDDFT_ERR_NOMEM : TDDFT_ERR_CUDA;
  };
  std::vector<double> om(n);
  cudaError_t e = cudaMemcpyAsync(om.data(), omega, n * sizeof(double),
                                  dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  for (int i = 1; i < n; ++i)
    if (!(om[i] > om[i - 1])) {
      ctx_set_error(c, "a warm-started sweep needs increasing frequencies");
      return TDDFT_ERR_INVALID_ARG;
    }
  std::vector<int32_t> pass(n), left(n), right(n);
  tddft_sweep_plan(n, pass.data(), left.data(), right.data());

  // frequencies per chunk: one solver group, and the network's row budget
  const int cw = sweep_chunk_freqs(ctx_slots(c), np);
  const size_t vec = (size_t)np * 2;   // doubles per complex vector
  DeviceBuffers buf;
  double *Xall = nullptr, *dP = nullptr, *d_om = nullptr, *x0 = nullptr, *Xp = nullptr,
         *Pp = nullptr, *d_t = nullptr, *d_omt = nullptr, *lin = nullptr, *scale = nullptr;
  int32_t *d_nb = nullptr, *d_dir = nullptr;
  float *F = nullptr, *Y = nullptr;
  const int T = 3 * cw;
  if (e == cudaSuccess) e = buf.get(&Xall, (size_t)3 * n * vec);
  if (e == cudaSuccess) e = buf.get(&dP, (size_t)n * 18);
  if (e == cudaSuccess) e = buf.get(&d_om, (size_t)cw);
  if (e == cudaSuccess) e = buf.get(&x0, (size_t)T * vec);
  if (e == cudaSuccess) e = buf.get(&Xp, (size_t)T * vec);
  if (e == cudaSuccess) e = buf.get(&Pp, (size_t)cw * 18);
  if (e == cudaSuccess) e = buf.get(&d_t, (size_t)T);
  if (e == cudaSuccess) e = buf.get(&d_omt, (size_t)T);
  if (e == cudaSuccess) e = buf.get(&lin, (size_t)T * vec);
  if (e == cudaSuccess) e = buf.get(&scale, (size_t)T);
  if (e == cudaSuccess) e = buf.get(&d_nb, (size_t)2 * T);
  if (e == cudaSuccess) e = buf.get(&d_dir, (size_t)T);
  if (e == cudaSuccess) e = buf.get(&F, (size_t)T * np * 10);
  if (e == cudaSuccess && mode == TDDFT_GUESS_LEARNED) e = buf.get(&Y, (size_t)T * np * 2);
  // projection: U and W = A U (kSub vectors per frequency), D and B = chi0 D
  // (3 per frequency), Gram data, coefficients, per-vector frequencies
  double *U = nullptr, *Wv = nullptr, *Dv = nullptr, *Bv = nullptr, *xp = nullptr;
  double *Gd = nullptr, *hd = nullptr, *cd = nullptr, *om9 = nullptr, *om3 = nullptr;
  if (subspace) {
    if (e == cudaSuccess) e = buf.get(&U, (size_t)kSub * cw * vec);
    if (e == cudaSuccess) e = buf.get(&Wv, (size_t)kSub * cw * vec);
    if (e == cudaSuccess) e = buf.get(&Dv, (size_t)T * vec);
    if (e == cudaSuccess) e = buf.get(&Bv, (size_t)T * vec);
    if (e == cudaSuccess) e = buf.get(&xp, (size_t)T * vec);
    if (e == cudaSuccess) e = buf.get(&Gd, (size_t)cw * kSub * kSub * 2);
    if (e == cudaSuccess) e = buf.get(&hd, (size_t)T * kSub * 2);
    if (e == cudaSuccess) e = buf.get(&cd, (size_t)T * kSub * 2);
    if (e == cudaSuccess) e = buf.get(&om9, (size_t)kSub * cw);
    if (e == cudaSuccess) e = buf.get(&om3, (size_t)T);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  const int slots = ctx_slots(c);

  bool all_conv = true;
  std::vector<tddft_solve_stats> cst(T);
  for (int p = 0; p <= 2; ++p) {
    std::vector<int> idx;
    for (int i = 0; i < n; ++i)
      if (pass[i] == p) idx.push_back(i);
    if (idx.empty()) continue;
    // the spacing feature: mean neighbour distance of the pass over eps
    double h = 0.0;
    if (p > 0) {
      for (int i : idx) h += om[right[i]] - om[left[i]];
      h /= (double)idx.size() * eps;
    }
    for (size_t c0 = 0; c0 < idx.size(); c0 += cw) {
      const int m = (int)std::min<size_t>(cw, idx.size() - c0);
      std::vector<double> omc(m);
      for (int w = 0; w < m; ++w) omc[w] = om[idx[c0 + w]];
      e = cudaMemcpyAsync(d_om, omc.data(), m * sizeof(double), cudaMemcpyHostToDevice, st);
      const double *guess = nullptr;
      if (e == cudaSuccess && p > 0) {
        // targets (frequency w, direction k) -> neighbour rows of Xall, weight t
        std::vector<int32_t> nb(2 * 3 * m), dir(3 * m);
        std::vector<double> t(3 * m), omt(3 * m);
        for (int w = 0; w < m; ++w) {
          const int i = idx[c0 + w];
          for (int k = 0; k < 3; ++k) {
            const int r = 3 * w + k;
            nb[2 * r] = 3 * left[i] + k;
            nb[2 * r + 1] = 3 * right[i] + k;
            dir[r] = k;
            t[r] = (om[i] - om[left[i]]) / (om[right[i]] - om[left[i]]);
            omt[r] = om[i];
          }
        }
        e = cudaMemcpyAsync(d_nb, nb.data(), nb.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(d_dir, dir.data(), dir.size() * sizeof(int32_t),
                              cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(d_t, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(d_omt, omt.data(), omt.size() * sizeof(double),
                              cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // host vectors go out of scope
        if (e != cudaSuccess) return cuda_fail(e);
        tddft_status s1 = tddft_guess_features(c, 3 * m, d_nb, d_t, d_omt, d_dir, h, Xall, F,
                                               lin, scale);
        if (s1 != TDDFT_OK) return s1;
        guess = lin;
        if (mode == TDDFT_GUESS_LEARNED) {
          s1 = tddft_mlp_forward(net, (int64_t)3 * m * np, F, Y, 1);
          if (s1 == TDDFT_OK) s1 = tddft_guess_combine(3 * m, np, Y, lin, scale, x0, st);
          if (s1 != TDDFT_OK) {
            ctx_set_error(c, "learned guess: network inference failed");
            return s1;
          }
          guess = x0;
        }
        if (subspace) {
          tddft_status s3 = project_guesses(c, m, idx.data() + c0, left.data(), right.data(),
                                            omc.data(), eps, slots, np, Xall, guess, U, Wv, Dv,
                                            Bv, Gd, hd, cd, om9, om3, xp);
          if (s3 != TDDFT_OK) return s3;
          guess = xp;
        }
      }
      if (e != cudaSuccess) return cuda_fail(e);
      const tddft_status s2 = ctx_polarizability_groups(c, m, d_om, eps, guess, Xp, Pp, cst.data(),
                                                        TDDFT_DEVICE_PTRS);
      if (s2 != TDDFT_OK && s2 != TDDFT_ERR_NOT_CONVERGED) return s2;
      if (s2 == TDDFT_ERR_NOT_CONVERGED) all_conv = false;
      // scatter the chunk's solutions, P and statistics to their frequencies
      for (int w = 0; w < m && e == cudaSuccess; ++w) {
        const int i = idx[c0 + w];
        e = cudaMemcpyAsync(Xall + (size_t)3 * i * vec, Xp + (size_t)3 * w * vec,
                            3 * vec * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(dP + (size_t)18 * i, Pp + (size_t)18 * w, 18 * sizeof(double),
                              cudaMemcpyDeviceToDevice, st);
        if (stats)
          for (int k = 0; k < 3; ++k) stats[3 * i + k] = cst[3 * w + k];
      }
      if (e != cudaSuccess) return cuda_fail(e);
    }
  }
  e = cudaMemcpyAsync(P, dP, (size_t)n * 18 * sizeof(double),
                      dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && Xout)
    e = cudaMemcpyAsync(Xout, Xall, (size_t)3 * n * vec * sizeof(double), cudaMemcpyDeviceToDevice,
                        st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (!all_conv) {
    ctx_set_error(c, "some (omega, direction) missed tol");
    return TDDFT_ERR_NOT_CONVERGED;
  }
  return TDDFT_OK;
}

}  // namespace tddft
