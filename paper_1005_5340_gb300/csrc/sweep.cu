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

// The sweep behind tddft_polarizability (and tddft_polarizability_guess
// without x0) when the context's guess mode is not zero.  omega, P and X
// follow flags (X: device, may be NULL).
tddft_status sweep_polarizability(tddft_ctx *c, int32_t n_omega, const double *omega, double eps,
                                  double *Xout, double *P, tddft_solve_stats *stats,
                                  int32_t flags) {
  const bool dev = (flags & TDDFT_DEVICE_PTRS) != 0;
  const int mode = ctx_guess_mode(c);
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
  if (e != cudaSuccess) return cuda_fail(e);

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
