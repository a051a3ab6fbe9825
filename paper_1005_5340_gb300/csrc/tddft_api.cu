// C boundary of libtddft (include/tddft.h): validation, device layouts,
// workspace ownership and the host side of the batched GMRES driver.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

using namespace tddft;

struct tddft_ctx {
  DevSystem sys;
  OpWork wk;
  LpWork lp;
  bool lowprec = false;
  OzWork oz;
  bool emu = false;
  AlphaRoute ar;
  GmresState gs;
  Timer timer;
  tddft_options opts{};
  cudaStream_t st = nullptr;
  cudaStream_t gst = nullptr;  // private stream for graph capture and replay
  double *Zc = nullptr;     // [2S][n_prod] operator input (planar)
  double *Wout = nullptr;   // [2S][n_prod] operator output (planar)
  double *stage = nullptr;  // [2S][n_prod] interleaved staging for boundary calls
  double *Z3 = nullptr;     // [6][n_prod] the three dipole vectors (planar)
  double *a3 = nullptr;     // [n_virt][6][n_occ] X_virt^T beta(d_k)
  int *h_count = nullptr;   // pinned
  tddft_mlp *guess_net = nullptr;   // network of the learned guess (tddft_guess_load)
  std::vector<void *> dev_allocs;
  std::string err;
};

namespace {
thread_local std::string g_create_error;

tddft_status fail(tddft_ctx *c, tddft_status s, const std::string &msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return s;
}

#define CUDA_TRY(ctx, expr)                                                              \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, TDDFT_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
cudaError_t dev_alloc(tddft_ctx *c, T **p, size_t count) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
  if (e != cudaSuccess) return e;
  c->dev_allocs.push_back(q);
  *p = static_cast<T *>(q);
  return cudaSuccess;
}

template <class T>
cudaError_t upload(tddft_ctx *c, T **p, const std::vector<T> &h) {
  cudaError_t e = dev_alloc(c, p, h.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

bool all_finite(const double *p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

void release(tddft_ctx *c) {
  if (c->guess_net) tddft_mlp_destroy(c->guess_net);
  c->guess_net = nullptr;
  c->timer.destroy();
  if (c->gst) cudaStreamDestroy(c->gst);
  c->gst = nullptr;
  for (void *p : c->dev_allocs) cudaFree(p);
  c->dev_allocs.clear();
  if (c->h_count) cudaFreeHost(c->h_count);
  c->h_count = nullptr;
}

tddft_status check_omega(tddft_ctx *c, int n, const double *omega, bool device) {
  if (!omega) return fail(c, TDDFT_ERR_INVALID_ARG, "omega is NULL");
  if (!device && !all_finite(omega, (size_t)n))
    return fail(c, TDDFT_ERR_INVALID_ARG, "omega holds NaN or Inf");
  return TDDFT_OK;
}
}  // namespace

namespace tddft {
tddft_status set_ctx_error(tddft_ctx *c, tddft_status s, const std::string &msg) {
  return fail(c, s, msg);
}

const char *kernel_class_name(int k) {
  static const char *names[kcCount] = {
      "f64_gemm_K",  "f64_vertex",   "f64_beta",      "f64_gemm_T1",  "f64_dscale",
      "f64_gemm_T2", "f64_block_dot", "tc_gemm_K",    "tc_gemm_T1_dscale", "tc_gemm_T2",
      "lp_split_z", "gmres_step",
      "gmres_gather", "gmres_select", "rhs_formation", "misc", "emu_slice", "emu_gemm_K",
      "emu_gemm_T1", "emu_gemm_T2", "alpha_gather", "tc_alpha_beta", "tc_alpha_dot",
      "emu_alpha_beta", "emu_alpha_dot", "lp_dterm", "alpha_combine"};
  return (k >= 0 && k < kcCount) ? names[k] : "?";
}

cudaEvent_t Timer::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
void Timer::begin(cudaStream_t st, int, cudaEvent_t *a) {
  *a = get();
  cudaEventRecord(*a, st);
}
void Timer::end(cudaStream_t st, int cls, cudaEvent_t a, double fl) {
  cudaEvent_t b = get();
  cudaEventRecord(b, st);
  pending.push_back({cls, a, b, fl});
}
void Timer::resolve() {
  for (auto &r : pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      ms[r.cls] += t;
      launches[r.cls] += 1;
      flops[r.cls] += r.flops;
    }
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  pending.clear();
  if (dev_bytes && dev_bytes_cls >= 0) {
    unsigned long long h = 0;
    if (cudaMemcpy(&h, dev_bytes, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess) {
      if (on) bytes[dev_bytes_cls] += (double)h;
      cudaMemset(dev_bytes, 0, sizeof(h));
    }
  }
}
void Timer::reset() {
  resolve();
  for (int i = 0; i < kcCount; ++i) { ms[i] = 0; launches[i] = 0; flops[i] = 0; bytes[i] = 0; }
}
void Timer::destroy() {
  for (auto &r : pending) { pool.push_back(r.a); pool.push_back(r.b); }
  pending.clear();
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
}
}  // namespace tddft

namespace {
struct TimedLaunch {
  Timer &t; cudaStream_t st; int cls; cudaEvent_t a = nullptr;
  TimedLaunch(Timer &t_, cudaStream_t s, int c) : t(t_), st(s), cls(c) { if (t.on) t.begin(st, cls, &a); }
  ~TimedLaunch() { if (t.on) t.end(st, cls, a, 0.0); }
};

tddft_status validate_system(const tddft_system *s, std::string &msg, tddft_status &code,
                             int &n_occ, double &occ_value) {
  code = TDDFT_ERR_INVALID_ARG;
  if (!s) { msg = "system is NULL"; return code; }
  if (s->n_atoms < 1 || s->n_orb < 2 || s->n_prod < 1) {
    code = TDDFT_ERR_SHAPE; msg = "need n_atoms >= 1, n_orb >= 2, n_prod >= 1"; return code;
  }
  if (!s->atom_orb_offset || !s->eigenvalues || !s->occupations || !s->X || !s->prod_atoms ||
      !s->vertex_offset || !s->vertex || !s->K || !s->dipole) {
    msg = "a system pointer is NULL"; return code;
  }
  const int32_t *ao = s->atom_orb_offset;
  if (ao[0] != 0 || ao[s->n_atoms] != s->n_orb) {
    code = TDDFT_ERR_SHAPE; msg = "atom_orb_offset must start at 0 and end at n_orb"; return code;
  }
  for (int A = 0; A < s->n_atoms; ++A) {
    int n = ao[A + 1] - ao[A];
    if (n < 1) { code = TDDFT_ERR_SHAPE; msg = "every atom needs at least one orbital"; return code; }
    if (n > kMaxOrb) {
      code = TDDFT_ERR_UNSUPPORTED; msg = "more than 16 orbitals on one atom"; return code;
    }
  }
  const size_t no = (size_t)s->n_orb, np = (size_t)s->n_prod;
  if (!all_finite(s->eigenvalues, no) || !all_finite(s->occupations, no) ||
      !all_finite(s->X, no * no) || !all_finite(s->dipole, 3 * np) || !all_finite(s->K, np * np)) {
    msg = "NaN or Inf in the system"; return code;
  }
  for (size_t i = 1; i < no; ++i)
    if (s->eigenvalues[i] < s->eigenvalues[i - 1]) { msg = "eigenvalues not ascending"; return code; }
  // step profile: n_occ equal positive values, then zeros
  n_occ = 0;
  occ_value = s->occupations[0];
  while (n_occ < s->n_orb && s->occupations[n_occ] > 0.0) ++n_occ;
  bool step = n_occ >= 1 && n_occ < s->n_orb;
  for (int i = 0; step && i < s->n_orb; ++i) {
    if (i < n_occ && s->occupations[i] != occ_value) step = false;
    if (i >= n_occ && s->occupations[i] != 0.0) step = false;
  }
  if (!step) {
    code = TDDFT_ERR_UNSUPPORTED;
    msg = "occupations must be equal positive values on the lowest states, then zeros";
    return code;
  }
  if (s->vertex_offset[0] != 0) { code = TDDFT_ERR_SHAPE; msg = "vertex_offset[0] != 0"; return code; }
  double vmax = 0.0;
  for (int mu = 0; mu < s->n_prod; ++mu) {
    int A = s->prod_atoms[2 * mu], B = s->prod_atoms[2 * mu + 1];
    if (A < 0 || B < A || B >= s->n_atoms) {
      code = TDDFT_ERR_SHAPE; msg = "prod_atoms must satisfy 0 <= A <= B < n_atoms"; return code;
    }
    int64_t sz = (int64_t)(ao[A + 1] - ao[A]) * (ao[B + 1] - ao[B]);
    if (s->vertex_offset[mu + 1] - s->vertex_offset[mu] != sz) {
      code = TDDFT_ERR_SHAPE; msg = "vertex_offset does not match the block sizes"; return code;
    }
  }
  const size_t nv = (size_t)s->vertex_offset[s->n_prod];
  if (!all_finite(s->vertex, nv)) { msg = "NaN or Inf in the vertex"; return code; }
  for (size_t i = 0; i < nv; ++i) vmax = std::fmax(vmax, std::fabs(s->vertex[i]));
  for (int mu = 0; mu < s->n_prod; ++mu) {
    int A = s->prod_atoms[2 * mu], B = s->prod_atoms[2 * mu + 1];
    if (A != B) continue;
    int n = ao[A + 1] - ao[A];
    const double *v = s->vertex + s->vertex_offset[mu];
    for (int a = 0; a < n; ++a)
      for (int b = a + 1; b < n; ++b)
        if (std::fabs(v[a * n + b] - v[b * n + a]) > 1e-12 * vmax) {
          msg = "a local vertex block is not symmetric"; return code;
        }
  }
  double kmax = 0.0;
  for (size_t i = 0; i < np * np; ++i) kmax = std::fmax(kmax, std::fabs(s->K[i]));
  const size_t T = 64;
  for (size_t i0 = 0; i0 < np; i0 += T)
    for (size_t j0 = i0; j0 < np; j0 += T)
      for (size_t i = i0; i < std::min(np, i0 + T); ++i)
        for (size_t j = std::max(j0, i + 1); j < std::min(np, j0 + T); ++j)
          if (std::fabs(s->K[i * np + j] - s->K[j * np + i]) > 1e-12 * kmax) {
            code = TDDFT_ERR_UNSUPPORTED; msg = "K is not symmetric"; return code;
          }
  code = TDDFT_OK;
  return TDDFT_OK;
}
int ptx_err_ints() { return 4; }   // the tensor-core kernels' error buffer (tc_ptx.h)

// The wait limit of the context's tensor-core kernels, in their error
// buffers (int[4]: code, reserved, 64-bit limit in ns; 0 = 2 s).
cudaError_t set_wait_limit(tddft_ctx *c, int64_t ns) {
  const unsigned long long v = (unsigned long long)ns;
  cudaError_t e = cudaSuccess;
  for (int *flag : {c->lowprec ? c->lp.err : nullptr, c->emu ? c->oz.err : nullptr}) {
    if (!flag || e != cudaSuccess) continue;
    e = cudaMemcpyAsync(flag + 2, &v, sizeof(v), cudaMemcpyHostToDevice, c->st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  return e;
}
}  // namespace

extern "C" {

tddft_status tddft_create(const tddft_system *s, const tddft_options *o, tddft_ctx **out) {
  g_create_error.clear();
  if (!out) return fail(nullptr, TDDFT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!o) return fail(nullptr, TDDFT_ERR_INVALID_ARG, "options are NULL");
  if (o->prec < TDDFT_PREC_FP64 || o->prec > TDDFT_PREC_TF32_IR_EMU)
    return fail(nullptr, TDDFT_ERR_UNSUPPORTED, "unknown precision");
  if (o->n_tile != 0 && o->n_tile != 64 && o->n_tile != 128 && o->n_tile != 256)
    return fail(nullptr, TDDFT_ERR_INVALID_ARG, "n_tile must be 0, 64, 128 or 256");
  if (o->guess < TDDFT_GUESS_ZERO || o->guess > TDDFT_GUESS_LEARNED_SUBSPACE)
    return fail(nullptr, TDDFT_ERR_INVALID_ARG, "unknown initial guess");
  if (o->wait_timeout_ns < 0)
    return fail(nullptr, TDDFT_ERR_INVALID_ARG, "wait_timeout_ns must be >= 0");
  const bool tf32 = o->prec == TDDFT_PREC_TF32_IR || o->prec == TDDFT_PREC_TF32_IR_EMU;
  const bool refine = o->prec == TDDFT_PREC_BF16X3_IR || o->prec == TDDFT_PREC_BF16X3_IR_EMU || tf32;
  if (refine && !(o->inner_tol > 0.0 && o->inner_tol < 1.0))
    return fail(nullptr, TDDFT_ERR_INVALID_ARG, "inner_tol must be in (0, 1)");
  if (o->restart < 1 || o->restart > 256 || o->max_restarts < 1 || !(o->tol > 0.0) ||
      !std::isfinite(o->tol) || o->batch < 1)
    return fail(nullptr, TDDFT_ERR_INVALID_ARG, "bad options (restart 1..256, max_restarts >= 1, tol > 0, batch >= 1)");
  if (o->graph < 0 || o->graph > 2)
    return fail(nullptr, TDDFT_ERR_INVALID_ARG, "graph must be 0, 1 or 2");
  if (o->stop < TDDFT_STOP_RESIDUAL || o->stop > TDDFT_STOP_EPS_PX)
    return fail(nullptr, TDDFT_ERR_INVALID_ARG, "unknown stopping rule");
  if (o->emu_slices != 0 && (o->emu_slices < kOzMinSlices || o->emu_slices > kOzMaxSlices))
    return fail(nullptr, TDDFT_ERR_INVALID_ARG, "emu_slices must be 0 or 3..8");
  std::string msg;
  tddft_status code;
  int n_occ = 0;
  double occ_value = 0.0;
  if (validate_system(s, msg, code, n_occ, occ_value) != TDDFT_OK) return fail(nullptr, code, msg);

  tddft_ctx *c = new tddft_ctx();
  c->opts = *o;
  c->st = static_cast<cudaStream_t>(o->stream);
  DevSystem &d = c->sys;
  d.n_atoms = s->n_atoms;
  d.n_orb = s->n_orb;
  d.n_occ = n_occ;
  d.n_virt = s->n_orb - n_occ;
  d.n_prod = s->n_prod;
  d.occ_value = occ_value;
  const int no = d.n_orb, nocc = d.n_occ, nv = d.n_virt, np = d.n_prod;

  // blocks: distinct (A, B) pairs in (A, B) order; products grouped per block
  std::map<std::pair<int, int>, std::vector<int>> groups;
  for (int mu = 0; mu < np; ++mu)
    groups[{s->prod_atoms[2 * mu], s->prod_atoms[2 * mu + 1]}].push_back(mu);
  std::vector<int2> blk_atoms;
  std::vector<int> blk_ptr{0}, blk_prod;
  std::vector<double> Vpad;
  Vpad.reserve((size_t)np * kBlk);
  std::vector<std::vector<int4>> adj_of(d.n_atoms);
  const int32_t *ao = s->atom_orb_offset;
  for (auto &kv : groups) {
    const int A = kv.first.first, B = kv.first.second;
    const int k = (int)blk_atoms.size();
    blk_atoms.push_back(make_int2(A, B));
    const int nA = ao[A + 1] - ao[A], nB = ao[B + 1] - ao[B];
    for (int mu : kv.second) {
      blk_prod.push_back(mu);
      const double *v = s->vertex + s->vertex_offset[mu];
      for (int a = 0; a < kMaxOrb; ++a)
        for (int b = 0; b < kMaxOrb; ++b)
          Vpad.push_back((a < nA && b < nB) ? v[a * nB + b] : 0.0);
    }
    blk_ptr.push_back((int)blk_prod.size());
    adj_of[A].push_back(make_int4(k, B, 0, 0));
    if (A != B) adj_of[B].push_back(make_int4(k, A, 1, 0));
  }
  d.n_blocks = (int)blk_atoms.size();
  std::vector<int> adj_ptr{0};
  std::vector<int4> adj;
  for (int A = 0; A < d.n_atoms; ++A) {
    for (auto &e : adj_of[A]) adj.push_back(e);
    adj_ptr.push_back((int)adj.size());
  }
  d.n_adj = (int)adj.size();
  {
    double fb = 0.0, fd = 0.0;
    for (int A = 0; A < d.n_atoms; ++A)
      for (auto &en : adj_of[A])
        fb += 2.0 * nocc * (ao[A + 1] - ao[A]) * (ao[en.y + 1] - ao[en.y]);
    for (size_t k = 0; k < blk_atoms.size(); ++k) {
      const int A = blk_atoms[k].x, B = blk_atoms[k].y;
      const double nab = (double)(ao[A + 1] - ao[A]) * (ao[B + 1] - ao[B]);
      fd += (A == B ? 1.0 : 2.0) * 2.0 * nocc * nab + 2.0 * nab * (blk_ptr[k + 1] - blk_ptr[k]);
    }
    d.sf.beta = fb;
    d.sf.dot = fd;
  }

  std::vector<double> Xo((size_t)no * nocc), XvT((size_t)nv * no), Xv((size_t)no * nv);
  for (int a = 0; a < no; ++a) {
    for (int E = 0; E < nocc; ++E) Xo[(size_t)a * nocc + E] = s->X[a + (size_t)E * no];
    for (int F = 0; F < nv; ++F) {
      const double x = s->X[a + (size_t)(nocc + F) * no];
      XvT[(size_t)F * no + a] = x;
      Xv[(size_t)a * nv + F] = x;
    }
  }
  std::vector<float> pfeat(2 * (size_t)np);
  {
    double mean = 0.0;
    std::vector<double> nrm(np);
    for (int mu = 0; mu < np; ++mu) {
      const int64_t a0 = s->vertex_offset[mu], a1 = s->vertex_offset[mu + 1];
      double q = 0.0;
      for (int64_t i = a0; i < a1; ++i) q += s->vertex[i] * s->vertex[i];
      nrm[mu] = std::sqrt(q);
      mean += nrm[mu] / np;
    }
    for (int mu = 0; mu < np; ++mu) {
      pfeat[2 * mu] = s->prod_atoms[2 * mu] != s->prod_atoms[2 * mu + 1] ? 1.f : 0.f;
      pfeat[2 * mu + 1] = mean > 0.0 ? (float)(nrm[mu] / mean) : 0.f;
    }
  }
  std::vector<int> aoffv(ao, ao + d.n_atoms + 1);
  std::vector<double> energy(s->eigenvalues, s->eigenvalues + no);
  std::vector<double> dip(s->dipole, s->dipole + 3 * (size_t)np);

  cudaError_t e = cudaSuccess;
#define UP(ptr, vec)                             \
  do {                                           \
    if (e == cudaSuccess) e = upload(c, &(ptr), vec); \
  } while (0)
  UP(d.aoff, aoffv);
  UP(d.energy, energy);
  UP(d.Xo, Xo);
  UP(d.XvT, XvT);
  UP(d.Xv, Xv);
  UP(d.dip, dip);
  UP(d.blk_atoms, blk_atoms);
  UP(d.blk_ptr, blk_ptr);
  UP(d.blk_prod, blk_prod);
  UP(d.Vpad, Vpad);
  UP(d.adj_ptr, adj_ptr);
  UP(d.adj, adj);
  UP(d.pfeat, pfeat);
#undef UP
  if (e == cudaSuccess) e = dev_alloc(c, &d.K, (size_t)np * np);
  if (e == cudaSuccess)
    e = cudaMemcpy(d.K, s->K, (size_t)np * np * sizeof(double), cudaMemcpyHostToDevice);

  const size_t S = (size_t)o->batch, m = (size_t)o->restart;
  const size_t S3 = S < 3 ? 3 : S;   // W and beta also hold the three dipole columns
  OpWork &w = c->wk;
  w.slots = (int)S;
  w.timer = &c->timer;
#define AL(ptr, n)                                   \
  do {                                               \
    if (e == cudaSuccess) e = dev_alloc(c, &(ptr), (n)); \
  } while (0)
  AL(w.Y, 2 * S * np);
  AL(w.W, 2 * S3 * (size_t)d.n_blocks * kBlk);
  AL(w.beta, (size_t)no * 2 * S3 * nocc);
  w.splitws_elems = (int64_t)8 * 2 * S * np;
  AL(w.splitws, (size_t)w.splitws_elems);
  AL(c->Z3, 6 * (size_t)np);
  AL(c->a3, (size_t)nv * 6 * nocc);
  AL(w.abuf, (size_t)nv * 2 * S * nocc);
  AL(w.gamma, (size_t)no * 2 * S * nocc);
  AL(w.omega, S);
  AL(c->Zc, 2 * S * np);
  AL(c->Wout, 2 * S * np);
  AL(c->stage, 2 * S * np);
  GmresState &g = c->gs;
  g.cap = (int)S;
  g.m = o->restart;
  g.max_restarts = o->max_restarts;
  g.tol = o->tol;
  AL(g.state, S); AL(g.jcur, S); AL(g.cycles, S); AL(g.matvecs, S); AL(g.conv, S);
  AL(g.flags, S);
  AL(g.bnorm, S); AL(g.resid, S); AL(g.omega, S);
  AL(g.H, S * (m + 1) * m); AL(g.Gm, S * (m + 1) * (m + 1)); AL(g.cs, S * m); AL(g.sn, S * m); AL(g.g, S * (m + 1));
  // the refinement forms keep their inner Krylov basis in float32: each cycle
  // is closed by a float64 residual, so its rounding only enters the correction
  if (refine) {
    AL(g.Vf, S * (m + 1) * 2 * np);
  } else {
    AL(g.V, S * (m + 1) * 2 * np);
  }
  AL(g.x, S * 2 * np); AL(g.b, S * 2 * np);
  AL(g.act, S); AL(g.act2, S); AL(g.count, 2); AL(g.rho0, S); AL(g.bytes, 1); AL(g.loopctl, 2);
  g.stop = o->stop;
  if (g.stop) {
    AL(g.dir, S); AL(g.crit, S * 10); AL(g.cvec, S * (3 * m + 2));
    if (refine) AL(g.dipf, 3 * (size_t)np);
    if (refine && g.stop == TDDFT_STOP_EPS_PX) AL(g.xf, S * 2 * np);
  }
  if (e == cudaSuccess) e = launch_gmres_prepare(c->st, d, g);
  if (e == cudaSuccess) e = cudaMemset(g.bytes, 0, sizeof(unsigned long long));
  c->timer.dev_bytes = g.bytes;
  c->timer.dev_bytes_cls = kcGmresStep;
  g.inner_tol = 0.0;
  c->lowprec = refine;
  c->emu = o->prec == TDDFT_PREC_FP64_EMU || o->prec == TDDFT_PREC_BF16X3_IR_EMU ||
           o->prec == TDDFT_PREC_TF32_IR_EMU;
  // the refinement form's float64 products need only resolve residuals well
  // below its tolerance: 5 slices (2^-35 of the operand scales) down to 1e-8,
  // 6 (2^-42) down to 1e-12, 7 below; 6 for the emulated float64 form
  if (o->prec == TDDFT_PREC_BF16X3_IR_EMU || o->prec == TDDFT_PREC_TF32_IR_EMU)
    c->oz.s = o->tol >= 1e-8 ? 5 : (o->tol >= 1e-12 ? 6 : 7);
  else
    c->oz.s = kOzDefaultSlices;
  if (o->emu_slices) c->oz.s = o->emu_slices;
  if (e == cudaSuccess && c->emu) {
    e = oz_setup(c->st, d, c->oz, (int)S, c->dev_allocs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    w.oz = &c->oz;
    w.ar = &c->ar;
    // beta^T columns of atoms without products are never written
    if (e == cudaSuccess)
      e = cudaMemset(w.beta, 0, (size_t)no * 2 * S3 * nocc * sizeof(double));
  }
  c->ar.tf32 = tf32;
  if (e == cudaSuccess && (c->emu || refine))
    e = alpha_setup(c->st, s, d, c->ar, (int)S, refine, c->emu, c->oz.s, c->dev_allocs);
  if (c->lowprec) {
    g.inner_tol = o->inner_tol;
    LpWork &L = c->lp;
    L.slots = (int)S;
    L.tf32 = tf32;
    L.KpK = round_up(np, 64);
    L.Kp1 = round_up(no, 64);
    L.Kp2 = round_up(nv, 64);
    L.timer = &c->timer;
    L.ar = &c->ar;
    const size_t rows1 = 2 * S * (size_t)nocc;
    AL(L.Ks, (size_t)np * 2 * L.KpK);
    AL(L.XvTs, (size_t)nv * 2 * L.Kp1);
    AL(L.Xvs, (size_t)no * 2 * L.Kp2);
    AL(L.Zb, 2 * S * 2 * (size_t)L.KpK);
    AL(L.Yt, 2 * S * (size_t)np);
    AL(L.betaT, rows1 * 2 * L.Kp1);
    AL(L.aT, rows1 * 2 * L.Kp2);
    AL(L.omega, S);
    AL(L.err, ptx_err_ints());
    AL(L.eocc2, (size_t)nocc);
    AL(L.dterm, S * (size_t)nv);
    if (e == cudaSuccess) e = make_operand_map(L.opK, L.Ks, np, L.KpK, 128, tf32);
    if (e == cudaSuccess) e = make_operand_map(L.opXvT, L.XvTs, nv, L.Kp1, 128, tf32);
    if (e == cudaSuccess) e = make_operand_map(L.opXv, L.Xvs, no, L.Kp2, 128, tf32);
    if (e == cudaSuccess) e = make_operand_map(L.opZ, L.Zb, 2 * (int64_t)S, L.KpK, 128, tf32);
    if (e == cudaSuccess) e = make_operand_map(L.opBeta, L.betaT, (int64_t)rows1, L.Kp1, 128, tf32);
    if (e == cudaSuccess) e = make_operand_map(L.opA, L.aT, (int64_t)rows1, L.Kp2, 128, tf32);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(L.err, 0, ptx_err_ints() * sizeof(int), c->st);
    if (e == cudaSuccess) e = lp_prepare_constants(c->st, d, L);
    if (e == cudaSuccess) tc_init_attributes();
    if (o->n_tile) {
      L.bnK = L.bn1 = L.bn2 = o->n_tile;
    } else if (e == cudaSuccess) {
      e = lp_autotune(c->st, d, L);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  }
#undef AL
  if (e == cudaSuccess) e = set_wait_limit(c, o->wait_timeout_ns);
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_count, 2 * sizeof(int));
  if (e == cudaSuccess && o->graph) e = cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking);
  if (e == cudaSuccess) tc_init_attributes();
  if (e != cudaSuccess) {
    std::string m2 = std::string("device allocation/upload failed: ") + cudaGetErrorString(e);
    release(c);
    delete c;
    return fail(nullptr, e == cudaErrorMemoryAllocation ? TDDFT_ERR_NOMEM : TDDFT_ERR_CUDA, m2);
  }
  *out = c;
  return TDDFT_OK;
}

void tddft_destroy(tddft_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  release(c);
  delete c;
}

const char *tddft_last_error(const tddft_ctx *c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

tddft_status tddft_set_wait_timeout(tddft_ctx *c, int64_t ns) {
  if (!c) return TDDFT_ERR_INVALID_ARG;
  c->err.clear();
  if (ns < 0) return fail(c, TDDFT_ERR_INVALID_ARG, "wait_timeout_ns must be >= 0");
  CUDA_TRY(c, set_wait_limit(c, ns));
  c->opts.wait_timeout_ns = ns;
  return TDDFT_OK;
}

tddft_status tddft_kproduct_plan(const tddft_ctx *c, int32_t n_rhs, int32_t *ncl,
                                 int32_t *ksplit) {
  if (!c || !ncl || !ksplit || n_rhs < 1) return TDDFT_ERR_INVALID_ARG;
  *ncl = 1;
  *ksplit = 1;
  if (!c->lowprec) return TDDFT_OK;
  int ks = 1, nc = 1;
  tc_split_plan(c->lp.KpK, c->sys.n_prod, 2 * n_rhs, c->lp.bnK, &ks, &nc);
  *ncl = nc;
  *ksplit = ks;
  return TDDFT_OK;
}

tddft_status tddft_tuning(const tddft_ctx *c, int32_t *n_tiles) {
  if (!c || !n_tiles) return TDDFT_ERR_INVALID_ARG;
  n_tiles[0] = c->lowprec ? c->lp.bnK : 0;
  n_tiles[1] = c->lowprec ? c->lp.bn1 : 0;
  n_tiles[2] = c->lowprec ? c->lp.bn2 : 0;
  return TDDFT_OK;
}

tddft_status tddft_sizes(const tddft_ctx *c, int32_t *n_orb, int32_t *n_occ, int32_t *n_prod,
                         int32_t *n_blocks) {
  if (!c) return TDDFT_ERR_INVALID_ARG;
  if (n_orb) *n_orb = c->sys.n_orb;
  if (n_occ) *n_occ = c->sys.n_occ;
  if (n_prod) *n_prod = c->sys.n_prod;
  if (n_blocks) *n_blocks = c->sys.n_blocks;
  return TDDFT_OK;
}

static tddft_status check_device_error(tddft_ctx *c);

static tddft_status boundary_apply(tddft_ctx *c, OpMode mode, int32_t n_rhs, const double *omega,
                                   double eps, const double *z, double *out, int32_t flags) {
  if (!c) return TDDFT_ERR_INVALID_ARG;
  c->err.clear();
  if (!z || !out) return fail(c, TDDFT_ERR_INVALID_ARG, "z or out is NULL");
  if (n_rhs < 1 || n_rhs > c->wk.slots)
    return fail(c, TDDFT_ERR_SHAPE, "n_rhs must be in 1..batch");
  const bool dev = (flags & TDDFT_DEVICE_PTRS) != 0;
  if (mode != kKernel) {
    if (!(eps > 0.0) || !std::isfinite(eps)) return fail(c, TDDFT_ERR_INVALID_ARG, "eps must be > 0");
    tddft_status s = check_omega(c, n_rhs, omega, dev);
    if (s != TDDFT_OK) return s;
  }
  const int np = c->sys.n_prod;
  const size_t bytes = (size_t)n_rhs * np * 2 * sizeof(double);
  cudaStream_t st = c->st;
  if (mode != kKernel)
    CUDA_TRY(c, cudaMemcpyAsync(c->wk.omega, omega, n_rhs * sizeof(double),
                                dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  const double *zin = z;
  if (!dev) {
    CUDA_TRY(c, cudaMemcpyAsync(c->stage, z, bytes, cudaMemcpyHostToDevice, st));
    zin = c->stage;
  }
  CUDA_TRY(c, launch_interleaved_to_planar(st, n_rhs, np, zin, c->Zc));
  if (c->lowprec && mode != kKernel) {
    CUDA_TRY(c, cudaMemcpyAsync(c->lp.omega, c->wk.omega, n_rhs * sizeof(double),
                                cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(c, launch_apply_operator_lp(st, c->sys, c->lp, n_rhs, mode, eps, c->Zc, c->Wout));
  } else {
    CUDA_TRY(c, launch_apply_operator(st, c->sys, c->wk, n_rhs, mode, eps, c->Zc, c->Wout));
  }
  CUDA_TRY(c, launch_planar_to_interleaved(st, n_rhs, np, c->Wout, dev ? out : c->stage));
  if (!dev) {
    CUDA_TRY(c, cudaMemcpyAsync(out, c->stage, bytes, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    c->timer.resolve();
    return check_device_error(c);
  }
  return TDDFT_OK;
}

static tddft_status check_device_error(tddft_ctx *c) {
  for (int *flag : {c->lowprec ? c->lp.err : nullptr, c->emu ? c->oz.err : nullptr}) {
    if (!flag) continue;
    int h = 0;
    CUDA_TRY(c, cudaMemcpy(&h, flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0) {
      cudaMemset(flag, 0, sizeof(int));
      return fail(c, TDDFT_ERR_TIMEOUT,
                  "a tensor-core GEMM wait gave up (code " + std::to_string(h) + ")");
    }
  }
  return TDDFT_OK;
}

tddft_status tddft_chi0_apply(tddft_ctx *c, int32_t n_rhs, const double *omega, double eps,
                              const double *z, double *out, int32_t flags) {
  return boundary_apply(c, kChi0, n_rhs, omega, eps, z, out, flags);
}

tddft_status tddft_kernel_apply(tddft_ctx *c, int32_t n_rhs, const double *z, double *out,
                                int32_t flags) {
  return boundary_apply(c, kKernel, n_rhs, nullptr, 1.0, z, out, flags);
}

tddft_status tddft_apply_A(tddft_ctx *c, int32_t n_rhs, const double *omega, double eps,
                           const double *z, double *out, int32_t flags) {
  return boundary_apply(c, kA, n_rhs, omega, eps, z, out, flags);
}

static tddft_status polarizability_impl(tddft_ctx *c, int32_t n_omega, const double *omega,
                                        double eps, const double *x0, double *Xout, double *P,
                                        tddft_solve_stats *stats, int32_t flags);

// Without explicit guesses, a context whose guess mode is not zero runs the
// warm-started frequency sweep (sweep.cu), which calls polarizability_impl
// per chunk with the guesses it forms.
static tddft_status polarizability_entry(tddft_ctx *c, int32_t n_omega, const double *omega,
                                         double eps, const double *x0, double *X, double *P,
                                         tddft_solve_stats *stats, int32_t flags) {
  if (!c) return TDDFT_ERR_INVALID_ARG;
  c->err.clear();
  if (n_omega < 1) return fail(c, TDDFT_ERR_SHAPE, "n_omega must be >= 1");
  if (!P) return fail(c, TDDFT_ERR_INVALID_ARG, "P is NULL");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(c, TDDFT_ERR_INVALID_ARG, "eps must be > 0");
  tddft_status s0 = check_omega(c, n_omega, omega, (flags & TDDFT_DEVICE_PTRS) != 0);
  if (s0 != TDDFT_OK) return s0;
  if (!x0 && c->opts.guess != TDDFT_GUESS_ZERO)
    return sweep_polarizability(c, n_omega, omega, eps, X, P, stats, flags);
  return polarizability_impl(c, n_omega, omega, eps, x0, X, P, stats, flags);
}

tddft_status tddft_polarizability(tddft_ctx *c, int32_t n_omega, const double *omega, double eps,
                                  double *P, tddft_solve_stats *stats, int32_t flags) {
  return polarizability_entry(c, n_omega, omega, eps, nullptr, nullptr, P, stats, flags);
}

tddft_status tddft_polarizability_guess(tddft_ctx *c, int32_t n_omega, const double *omega,
                                        double eps, const double *x0, double *X, double *P,
                                        tddft_solve_stats *stats, int32_t flags) {
  if (c && !(flags & TDDFT_DEVICE_PTRS) && (x0 || X))
    return fail(c, TDDFT_ERR_INVALID_ARG, "x0 and X must be device pointers (flags bit 0)");
  return polarizability_entry(c, n_omega, omega, eps, x0, X, P, stats, flags);
}

tddft_status tddft_set_guess(tddft_ctx *c, int32_t guess) {
  if (!c) return TDDFT_ERR_INVALID_ARG;
  c->err.clear();
  if (guess < TDDFT_GUESS_ZERO || guess > TDDFT_GUESS_LEARNED_SUBSPACE)
    return fail(c, TDDFT_ERR_INVALID_ARG, "unknown initial guess");
  c->opts.guess = guess;
  return TDDFT_OK;
}

// One GMRES iteration of a group of n right-hand sides, captured once in a
// CUDA graph on the private stream and replayed: launch shapes are those of
// n live right-hand sides and every kernel reads the live counts on the
// device, so no host decision is needed between iterations.  The host reads
// the counts back every kReplays launches.
// Loop control of the device-driven GMRES loop (one WHILE node per group):
// right after the selection of each iteration, keep the node repeating while
// some right-hand side is live and the iteration bound holds; ctl[0] counts
// the iterations, ctl[1] = 1 records that the bound stopped the loop.
__global__ void loop_control_kernel(cudaGraphConditionalHandle h, const int *__restrict__ count,
                                    int *__restrict__ ctl, int max_iter) {
  const bool live = count[0] > 0 || count[1] > 0;
  const int it = ++ctl[0];
  bool go = live;
  if (live && it > max_iter) {
    ctl[1] = 1;
    go = false;
  }
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Enqueue one device-driven GMRES iteration of context c's current group of
// n right-hand sides on stream gs (no host decision, no synchronisation).
// With loop: the body of a WHILE node, whose condition the control kernel
// sets after the selection (the rest of the iteration then finds no live
// right-hand side and does no work).
static cudaError_t enqueue_iteration(tddft_ctx *c, cudaStream_t gs, int n, double eps, int split,
                                     int min_b, const cudaGraphConditionalHandle *loop = nullptr,
                                     int max_iter = 0) {
  GmresState &g = c->gs;
  OpWork wk = c->wk;
  LpWork lp = c->lp;
  wk.timer = nullptr;
  lp.timer = nullptr;
  wk.dcnt = g.count + (split ? 1 : 0);
  lp.dcnt = g.count;
  cudaError_t e = launch_gmres_select(gs, g, n, split, min_b);
  if (e == cudaSuccess && loop) {
    loop_control_kernel<<<1, 1, 0, gs>>>(*loop, g.count, g.loopctl, max_iter);
    e = cudaGetLastError();
  }
  if (split) {
    if (e == cudaSuccess) e = launch_gmres_gather(gs, c->sys, g, g.act, n, c->Zc, lp.omega, g.count);
    if (e == cudaSuccess) e = launch_apply_operator_lp(gs, c->sys, lp, n, kA, eps, c->Zc, c->Wout);
    if (e == cudaSuccess) e = launch_gmres_step(gs, c->sys, g, g.act, n, c->Wout, g.count);
    if (e == cudaSuccess)
      e = launch_gmres_gather(gs, c->sys, g, g.act2, n, c->Zc, wk.omega, g.count + 1);
    if (e == cudaSuccess) e = launch_apply_operator(gs, c->sys, wk, n, kA, eps, c->Zc, c->Wout);
    if (e == cudaSuccess) e = launch_gmres_step(gs, c->sys, g, g.act2, n, c->Wout, g.count + 1);
  } else {
    if (e == cudaSuccess) e = launch_gmres_gather(gs, c->sys, g, g.act, n, c->Zc, wk.omega, g.count);
    if (e == cudaSuccess) e = launch_apply_operator(gs, c->sys, wk, n, kA, eps, c->Zc, c->Wout);
    if (e == cudaSuccess) e = launch_gmres_step(gs, c->sys, g, g.act, n, c->Wout, g.count);
  }
  return e;
}

// Refinement forms: the float64 residual group runs once this many right-hand
// sides of a group of n await it (or nothing else is left), so that its fixed
// costs are shared.
static int residual_batch(int split, int n) {
  return split ? std::max(1, std::min(64, n / 3)) : 1;
}

// Add to graph `parent` a WHILE node (no dependencies) whose body, captured
// on stream cs, is one device-driven GMRES iteration of context c's group.
static cudaError_t add_device_loop(tddft_ctx *c, cudaGraph_t parent, cudaStream_t cs, int n,
                                   double eps, int split, int min_b, int max_iter) {
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, parent, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, parent, nullptr, nullptr, 0, &p);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = p.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t e1 = enqueue_iteration(c, cs, n, eps, split, min_b, &h, max_iter);
  cudaGraph_t captured = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
  return e1 != cudaSuccess ? e1 : e2;
}

// The whole GMRES loop of a group as one graph launch: a WHILE node repeats
// the iteration on the device until no right-hand side is live (or the
// iteration bound is hit: TIMEOUT); the host waits once, at the end.
static tddft_status run_group_device_loop(tddft_ctx *c, int n, double eps, int split, int min_b,
                                          long max_iter) {
  GmresState &g = c->gs;
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  struct Cleanup {
    cudaGraph_t &g; cudaGraphExec_t &e;
    ~Cleanup() { if (e) cudaGraphExecDestroy(e); if (g) cudaGraphDestroy(g); }
  } cleanup{graph, exec};
  CUDA_TRY(c, cudaGraphCreate(&graph, 0));
  cudaError_t e = add_device_loop(c, graph, c->gst, n, eps, split, min_b, (int)max_iter);
  if (e != cudaSuccess)
    return fail(c, TDDFT_ERR_CUDA, std::string("device loop capture failed: ") +
                                       cudaGetErrorString(e));
  CUDA_TRY(c, cudaGraphInstantiate(&exec, graph, 0));
  CUDA_TRY(c, cudaMemsetAsync(g.loopctl, 0, 2 * sizeof(int), c->st));
  CUDA_TRY(c, cudaGraphLaunch(exec, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(c->h_count, g.loopctl, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                              c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  if (c->h_count[1]) return fail(c, TDDFT_ERR_TIMEOUT, "GMRES driver exceeded its iteration bound");
  return TDDFT_OK;
}

static tddft_status run_group_graph(tddft_ctx *c, int n, double eps, int split, int min_b,
                                    long max_iter) {
  constexpr int kReplays = 4;
  GmresState &g = c->gs;
  cudaStream_t gs = c->gst;
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  struct Cleanup {
    cudaGraph_t &g; cudaGraphExec_t &e;
    ~Cleanup() { if (e) cudaGraphExecDestroy(e); if (g) cudaGraphDestroy(g); }
  } cleanup{graph, exec};
  CUDA_TRY(c, cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = enqueue_iteration(c, gs, n, eps, split, min_b);
  cudaError_t e2 = cudaStreamEndCapture(gs, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return fail(c, TDDFT_ERR_CUDA, std::string("graph capture failed: ") +
                                       cudaGetErrorString(e != cudaSuccess ? e : e2));
  CUDA_TRY(c, cudaGraphInstantiate(&exec, graph, 0));
  for (long it = 0;; it += kReplays) {
    if (it > max_iter + kReplays)
      return fail(c, TDDFT_ERR_TIMEOUT, "GMRES driver exceeded its iteration bound");
    for (int r = 0; r < kReplays; ++r) CUDA_TRY(c, cudaGraphLaunch(exec, gs));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_count, g.count, 2 * sizeof(int), cudaMemcpyDeviceToHost, gs));
    CUDA_TRY(c, cudaStreamSynchronize(gs));
    if (c->h_count[0] <= 0 && c->h_count[1] <= 0) {
      // the counts of the last replay's selection; one more selection confirms
      CUDA_TRY(c, launch_gmres_select(gs, g, n, split, min_b));
      CUDA_TRY(c, cudaMemcpyAsync(c->h_count, g.count, 2 * sizeof(int), cudaMemcpyDeviceToHost, gs));
      CUDA_TRY(c, cudaStreamSynchronize(gs));
      if (c->h_count[0] <= 0 && c->h_count[1] <= 0) break;
    }
  }
  return TDDFT_OK;
}

static tddft_status polarizability_impl(tddft_ctx *c, int32_t n_omega, const double *omega,
                                        double eps, const double *x0, double *Xout, double *P,
                                        tddft_solve_stats *stats, int32_t flags) {
  if (!c) return TDDFT_ERR_INVALID_ARG;
  c->err.clear();
  if (n_omega < 1) return fail(c, TDDFT_ERR_SHAPE, "n_omega must be >= 1");
  if (!P) return fail(c, TDDFT_ERR_INVALID_ARG, "P is NULL");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(c, TDDFT_ERR_INVALID_ARG, "eps must be > 0");
  const bool dev = (flags & TDDFT_DEVICE_PTRS) != 0;
  tddft_status s0 = check_omega(c, n_omega, omega, dev);
  if (s0 != TDDFT_OK) return s0;
  cudaStream_t st = c->st;
  const int total = 3 * n_omega;
  const int S = c->wk.slots;
  const int np = c->sys.n_prod;
  GmresState &g = c->gs;

  double *d_omega = nullptr;
  double2 *d_P = nullptr;
  CUDA_TRY(c, cudaMalloc(&d_omega, n_omega * sizeof(double)));
  cudaError_t e = cudaMalloc(&d_P, (size_t)n_omega * 9 * sizeof(double2));
  if (e != cudaSuccess) { cudaFree(d_omega); return fail(c, TDDFT_ERR_NOMEM, "P buffer"); }
  struct Free { void *a, *b; ~Free() { cudaFree(a); cudaFree(b); } } fr{d_omega, d_P};
  CUDA_TRY(c, cudaMemcpyAsync(d_omega, omega, n_omega * sizeof(double),
                              dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));

  bool all_conv = true;
  std::vector<int> h_mv(S), h_cy(S), h_cv(S), h_fl(S);
  std::vector<double> h_res(S), h_crit(g.stop ? (size_t)S * 10 : 0);
  const long max_iter = (long)(g.max_restarts + 1) * (g.m + 1) + 4;
  for (int g0 = 0; g0 < total; g0 += S) {
    const int n = std::min(S, total - g0);
    CUDA_TRY(c, launch_rhs_init(st, c->sys, n, g0, d_omega, c->Zc, c->wk.omega, g.omega, g.dir));
    CUDA_TRY(c, launch_rhs_formation(st, c->sys, c->wk, n, g0, d_omega, eps, c->Z3, c->a3,
                                     c->Wout));
    CUDA_TRY(c, launch_gmres_start(st, c->sys, g, n, c->Wout));
    if (x0) CUDA_TRY(c, launch_gmres_guess(st, c->sys, g, n, g0, x0));
    long it = 0;
    const int split = c->lowprec ? 1 : 0;
    // Float64 residuals that end a refinement cycle are batched: while reduced-
    // precision Arnoldi work remains, right-hand sides awaiting their residual
    // wait until enough of them have gathered to fill the float64 GEMM tiles.
    const int min_b = residual_batch(split, n);
    if (c->opts.graph == 2 && !c->timer.on) {
      tddft_status gs_ = run_group_device_loop(c, n, eps, split, min_b, max_iter);
      if (gs_ != TDDFT_OK) return gs_;
    } else if (c->opts.graph == 1 && !c->timer.on) {
      tddft_status gs_ = run_group_graph(c, n, eps, split, min_b, max_iter);
      if (gs_ != TDDFT_OK) return gs_;
    } else {
      for (;; ++it) {
        if (it > max_iter)
          return fail(c, TDDFT_ERR_TIMEOUT, "GMRES driver exceeded its iteration bound");
        {
          TimedLaunch tl(c->timer, st, kcGmresSelect);
          CUDA_TRY(c, launch_gmres_select(st, g, n, split, min_b));
        }
        CUDA_TRY(c, cudaMemcpyAsync(c->h_count, g.count, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(c, cudaStreamSynchronize(st));
        const int cntA = c->h_count[0], cntB = c->h_count[1];
        if (cntA <= 0 && cntB <= 0) break;
        if (cntA > 0) {
          // Arnoldi steps (reduced precision in the refinement forms)
          {
            TimedLaunch tl(c->timer, st, kcGmresGather);
            CUDA_TRY(c, launch_gmres_gather(st, c->sys, g, g.act, cntA, c->Zc,
                                            split ? c->lp.omega : c->wk.omega));
          }
          if (split)
            CUDA_TRY(c, launch_apply_operator_lp(st, c->sys, c->lp, cntA, kA, eps, c->Zc, c->Wout));
          else
            CUDA_TRY(c, launch_apply_operator(st, c->sys, c->wk, cntA, kA, eps, c->Zc, c->Wout));
          {
            TimedLaunch tl(c->timer, st, kcGmresStep);
            CUDA_TRY(c, launch_gmres_step(st, c->sys, g, g.act, cntA, c->Wout));
          }
        }
        if (cntB > 0) {
          // float64 residuals that end a refinement cycle
          {
            TimedLaunch tl(c->timer, st, kcGmresGather);
            CUDA_TRY(c, launch_gmres_gather(st, c->sys, g, g.act2, cntB, c->Zc, c->wk.omega));
          }
          CUDA_TRY(c, launch_apply_operator(st, c->sys, c->wk, cntB, kA, eps, c->Zc, c->Wout));
          {
            TimedLaunch tl(c->timer, st, kcGmresStep);
            CUDA_TRY(c, launch_gmres_step(st, c->sys, g, g.act2, cntB, c->Wout));
          }
        }
      }
    }
    {
      tddft_status se = check_device_error(c);
      if (se != TDDFT_OK) return se;
    }
    CUDA_TRY(c, launch_polarization(st, c->sys, g, n, g0, d_P));
    if (Xout) CUDA_TRY(c, launch_gmres_export(st, c->sys, g, n, g0, Xout));
    CUDA_TRY(c, cudaMemcpyAsync(h_mv.data(), g.matvecs, n * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaMemcpyAsync(h_cy.data(), g.cycles, n * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaMemcpyAsync(h_cv.data(), g.conv, n * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaMemcpyAsync(h_res.data(), g.resid, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaMemcpyAsync(h_fl.data(), g.flags, n * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (g.stop)
      CUDA_TRY(c, cudaMemcpyAsync(h_crit.data(), g.crit, (size_t)n * 10 * sizeof(double),
                                  cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    c->timer.resolve();
    for (int r = 0; r < n; ++r) {
      if (!h_cv[r]) all_conv = false;
      if (stats) {
        tddft_solve_stats &t = stats[g0 + r];
        t.matvecs = h_mv[r];
        t.cycles = h_cy[r];
        t.resid = h_res[r];
        t.converged = h_cv[r];
        t.flags = h_fl[r];
        t.eps_p = g.stop ? h_crit[(size_t)r * 10 + 7] : NAN;
        t.eps_x = g.stop ? h_crit[(size_t)r * 10 + 8] : NAN;
      }
    }
  }
  CUDA_TRY(c, cudaMemcpyAsync(P, d_P, (size_t)n_omega * 9 * sizeof(double2),
                              dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  if (!all_conv) return fail(c, TDDFT_ERR_NOT_CONVERGED, "some (omega, direction) missed tol");
  return TDDFT_OK;
}

tddft_status tddft_timing_enable(tddft_ctx *c, int32_t on) {
  if (!c) return TDDFT_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->st);
  c->timer.reset();
  c->timer.on = on != 0;
  return TDDFT_OK;
}

int32_t tddft_timing_count(const tddft_ctx *) { return kcCount; }

tddft_status tddft_timing_bytes(tddft_ctx *c, int32_t i, double *bytes) {
  if (!c || !bytes || i < 0 || i >= kcCount) return TDDFT_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->st);
  c->timer.resolve();
  *bytes = c->timer.bytes[i];
  return TDDFT_OK;
}

tddft_status tddft_timing_get(tddft_ctx *c, int32_t i, const char **name, int32_t *launches,
                              double *total_ms, double *flops) {
  if (!c || i < 0 || i >= kcCount) return TDDFT_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->st);
  c->timer.resolve();
  if (name) *name = kernel_class_name(i);
  if (launches) *launches = c->timer.launches[i];
  if (total_ms) *total_ms = c->timer.ms[i];
  if (flops) *flops = c->timer.flops[i];
  return TDDFT_OK;
}

}  // extern "C"

namespace tddft {
// Accessors for entry points defined in other translation units.
const DevSystem *ctx_system(const tddft_ctx *c) { return &c->sys; }
cudaStream_t ctx_stream(const tddft_ctx *c) { return c->st; }
void ctx_set_error(tddft_ctx *c, const char *msg) { c->err = msg; }
int ctx_slots(const tddft_ctx *c) { return c->wk.slots; }
const tddft_options *ctx_options(const tddft_ctx *c) { return &c->opts; }
int ctx_guess_mode(const tddft_ctx *c) { return c->opts.guess; }
tddft_mlp *ctx_guess_net(const tddft_ctx *c) { return c->guess_net; }
void ctx_set_guess_net(tddft_ctx *c, tddft_mlp *net) {
  if (c->guess_net) tddft_mlp_destroy(c->guess_net);
  c->guess_net = net;
}
tddft_status ctx_polarizability_groups(tddft_ctx *c, int32_t n_omega, const double *omega,
                                       double eps, const double *x0, double *X, double *P,
                                       tddft_solve_stats *stats, int32_t flags) {
  return polarizability_impl(c, n_omega, omega, eps, x0, X, P, stats, flags);
}
const float *ctx_product_features(const tddft_ctx *c) { return c->sys.pfeat; }
}  // namespace tddft

// ---------------------------------------------------------------------------
// Several molecules solved together
// ---------------------------------------------------------------------------
struct tddft_batch {
  std::vector<tddft_ctx *> ctx;
  std::vector<cudaStream_t> streams;
  cudaStream_t main = nullptr;
  int *h_counts = nullptr;   // pinned [2 n_mol]
  std::string err;
};

namespace {
thread_local std::string g_batch_error;

tddft_status bfail(tddft_batch *b, tddft_status s, const std::string &msg) {
  if (b) b->err = msg;
  else g_batch_error = msg;
  return s;
}

void batch_release(tddft_batch *b) {
  for (auto *c : b->ctx) tddft_destroy(c);
  b->ctx.clear();
  for (auto s : b->streams) cudaStreamDestroy(s);
  b->streams.clear();
  if (b->main) cudaStreamDestroy(b->main);
  b->main = nullptr;
  if (b->h_counts) cudaFreeHost(b->h_counts);
  b->h_counts = nullptr;
}

#define BCUDA(b, expr)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return bfail(b, TDDFT_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));   \
  } while (0)
}  // namespace

extern "C" {

tddft_status tddft_batch_create(int32_t n_mol, const tddft_system *systems,
                                const tddft_options *opts, tddft_batch **out) {
  g_batch_error.clear();
  if (!out || !systems || !opts || n_mol < 1)
    return bfail(nullptr, TDDFT_ERR_INVALID_ARG, "need n_mol >= 1, systems, options and out");
  *out = nullptr;
  tddft_batch *b = new tddft_batch();
  cudaError_t e = cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_counts, 2 * sizeof(int) * n_mol);
  if (e != cudaSuccess) {
    batch_release(b);
    delete b;
    return bfail(nullptr, TDDFT_ERR_CUDA, cudaGetErrorString(e));
  }
  for (int i = 0; i < n_mol; ++i) {
    cudaStream_t s = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      batch_release(b);
      delete b;
      return bfail(nullptr, TDDFT_ERR_CUDA, cudaGetErrorString(e));
    }
    b->streams.push_back(s);
    tddft_options o = *opts;
    o.stream = s;
    o.graph = 0;
    tddft_ctx *c = nullptr;
    tddft_status st = tddft_create(&systems[i], &o, &c);
    if (st != TDDFT_OK) {
      std::string m = "molecule " + std::to_string(i) + ": " + tddft_last_error(nullptr);
      batch_release(b);
      delete b;
      return bfail(nullptr, st, m);
    }
    b->ctx.push_back(c);
  }
  *out = b;
  return TDDFT_OK;
}

void tddft_batch_destroy(tddft_batch *b) {
  if (!b) return;
  batch_release(b);
  delete b;
}

const char *tddft_batch_last_error(const tddft_batch *b) {
  return b ? b->err.c_str() : g_batch_error.c_str();
}

tddft_ctx *tddft_batch_context(tddft_batch *b, int32_t i) {
  if (!b || i < 0 || i >= (int)b->ctx.size()) return nullptr;
  return b->ctx[i];
}

tddft_status tddft_batch_polarizability(tddft_batch *b, int32_t n_omega, const double *omega,
                                        double eps, double *P, tddft_solve_stats *stats) {
  if (!b) return TDDFT_ERR_INVALID_ARG;
  b->err.clear();
  if (n_omega < 1 || !omega || !P) return bfail(b, TDDFT_ERR_INVALID_ARG, "bad omega or P");
  if (!(eps > 0.0) || !std::isfinite(eps)) return bfail(b, TDDFT_ERR_INVALID_ARG, "eps must be > 0");
  if (!all_finite(omega, (size_t)n_omega))
    return bfail(b, TDDFT_ERR_INVALID_ARG, "omega holds NaN or Inf");
  const int nm = (int)b->ctx.size();
  const int total = 3 * n_omega;
  std::vector<double *> d_omega(nm, nullptr);
  std::vector<double2 *> d_P(nm, nullptr);
  struct Free {
    std::vector<double *> &a; std::vector<double2 *> &p;
    ~Free() { for (auto x : a) cudaFree(x); for (auto x : p) cudaFree(x); }
  } fr{d_omega, d_P};
  int rounds = 0;
  for (int i = 0; i < nm; ++i) {
    tddft_ctx *c = b->ctx[i];
    BCUDA(b, cudaMalloc(&d_omega[i], n_omega * sizeof(double)));
    BCUDA(b, cudaMalloc(&d_P[i], (size_t)n_omega * 9 * sizeof(double2)));
    BCUDA(b, cudaMemcpyAsync(d_omega[i], omega, n_omega * sizeof(double), cudaMemcpyHostToDevice,
                             c->st));
    rounds = std::max(rounds, (total + c->wk.slots - 1) / c->wk.slots);
  }
  std::vector<cudaEvent_t> ev(nm + 1, nullptr);
  struct EvFree {
    std::vector<cudaEvent_t> &e;
    ~EvFree() { for (auto x : e) if (x) cudaEventDestroy(x); }
  } efr{ev};
  for (auto &x : ev) BCUDA(b, cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
  bool all_conv = true;
  const long max_iter = 1000000;
  for (int r = 0; r < rounds; ++r) {
    std::vector<int> act, g0v, nv, splitv, minbv;
    for (int i = 0; i < nm; ++i) {
      tddft_ctx *c = b->ctx[i];
      const int S = c->wk.slots, g0 = r * S;
      if (g0 >= total) continue;
      const int n = std::min(S, total - g0);
      GmresState &g = c->gs;
      const int split = c->lowprec ? 1 : 0;
      act.push_back(i);
      g0v.push_back(g0);
      nv.push_back(n);
      splitv.push_back(split);
      minbv.push_back(residual_batch(split, n));
      // right-hand sides of this round, on the molecule's stream
      BCUDA(b, launch_rhs_init(c->st, c->sys, n, g0, d_omega[i], c->Zc, c->wk.omega, g.omega,
                               g.dir));
      BCUDA(b, launch_rhs_formation(c->st, c->sys, c->wk, n, g0, d_omega[i], eps, c->Z3, c->a3,
                                    c->Wout));
      BCUDA(b, launch_gmres_start(c->st, c->sys, g, n, c->Wout));
      BCUDA(b, cudaEventRecord(ev[i], c->st));
      BCUDA(b, cudaStreamWaitEvent(b->main, ev[i], 0));
    }
    // one graph launch per round: a WHILE node per molecule (independent
    // nodes, so the molecules' iterations run side by side), each repeating
    // that molecule's GMRES iteration on the device until its group is done
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    struct GFree {
      cudaGraph_t &g; cudaGraphExec_t &e;
      ~GFree() { if (e) cudaGraphExecDestroy(e); if (g) cudaGraphDestroy(g); }
    } gfr{graph, exec};
    BCUDA(b, cudaStreamSynchronize(b->main));
    BCUDA(b, cudaGraphCreate(&graph, 0));
    for (size_t a = 0; a < act.size(); ++a) {
      tddft_ctx *c = b->ctx[act[a]];
      const GmresState &g = c->gs;
      const long bound = (long)(g.max_restarts + 1) * (g.m + 1) + 4;
      const cudaError_t ce = add_device_loop(c, graph, b->main, nv[a], eps, splitv[a], minbv[a],
                                             (int)std::min(bound, max_iter));
      if (ce != cudaSuccess)
        return bfail(b, TDDFT_ERR_CUDA, std::string("graph capture failed: ") +
                                            cudaGetErrorString(ce));
    }
    BCUDA(b, cudaGraphInstantiate(&exec, graph, 0));
    for (size_t a = 0; a < act.size(); ++a)
      BCUDA(b, cudaMemsetAsync(b->ctx[act[a]]->gs.loopctl, 0, 2 * sizeof(int), b->main));
    BCUDA(b, cudaGraphLaunch(exec, b->main));
    for (size_t a = 0; a < act.size(); ++a)
      BCUDA(b, cudaMemcpyAsync(b->h_counts + 2 * a, b->ctx[act[a]]->gs.loopctl, 2 * sizeof(int),
                               cudaMemcpyDeviceToHost, b->main));
    BCUDA(b, cudaStreamSynchronize(b->main));
    for (size_t a = 0; a < act.size(); ++a)
      if (b->h_counts[2 * a + 1])
        return bfail(b, TDDFT_ERR_TIMEOUT, "molecule " + std::to_string(act[a]) +
                                               ": GMRES driver exceeded its iteration bound");
    // results of the round
    for (size_t a = 0; a < act.size(); ++a) {
      const int i = act[a];
      tddft_ctx *c = b->ctx[i];
      GmresState &g = c->gs;
      const int n = nv[a], g0 = g0v[a];
      BCUDA(b, launch_polarization(c->st, c->sys, g, n, g0, d_P[i]));
      std::vector<int> mv(n), cy(n), cv(n), fl(n);
      std::vector<double> rs(n), cr(g.stop ? (size_t)n * 10 : 0);
      BCUDA(b, cudaMemcpyAsync(mv.data(), g.matvecs, n * sizeof(int), cudaMemcpyDeviceToHost, c->st));
      BCUDA(b, cudaMemcpyAsync(cy.data(), g.cycles, n * sizeof(int), cudaMemcpyDeviceToHost, c->st));
      BCUDA(b, cudaMemcpyAsync(cv.data(), g.conv, n * sizeof(int), cudaMemcpyDeviceToHost, c->st));
      BCUDA(b, cudaMemcpyAsync(fl.data(), g.flags, n * sizeof(int), cudaMemcpyDeviceToHost, c->st));
      BCUDA(b, cudaMemcpyAsync(rs.data(), g.resid, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      if (g.stop)
        BCUDA(b, cudaMemcpyAsync(cr.data(), g.crit, (size_t)n * 10 * sizeof(double),
                                 cudaMemcpyDeviceToHost, c->st));
      BCUDA(b, cudaStreamSynchronize(c->st));
      if (check_device_error(c) != TDDFT_OK)
        return bfail(b, TDDFT_ERR_TIMEOUT, "molecule " + std::to_string(i) + ": " + c->err);
      for (int q = 0; q < n; ++q) {
        if (!cv[q]) all_conv = false;
        if (stats) {
          tddft_solve_stats &t = stats[(size_t)i * total + g0 + q];
          t.matvecs = mv[q];
          t.cycles = cy[q];
          t.resid = rs[q];
          t.converged = cv[q];
          t.flags = fl[q];
          t.eps_p = g.stop ? cr[(size_t)q * 10 + 7] : NAN;
          t.eps_x = g.stop ? cr[(size_t)q * 10 + 8] : NAN;
        }
      }
    }
  }
  for (int i = 0; i < nm; ++i) {
    tddft_ctx *c = b->ctx[i];
    BCUDA(b, cudaMemcpyAsync(P + (size_t)i * n_omega * 18, d_P[i], (size_t)n_omega * 9 * sizeof(double2),
                             cudaMemcpyDeviceToHost, c->st));
    BCUDA(b, cudaStreamSynchronize(c->st));
  }
  if (!all_conv) return bfail(b, TDDFT_ERR_NOT_CONVERGED, "some (molecule, omega, direction) missed tol");
  return TDDFT_OK;
}

}  // extern "C"
