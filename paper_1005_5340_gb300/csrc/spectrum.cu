// Adaptive frequency grid and pole extraction on top of tddft_polarizability
// (the step named as the next one in the paper's conclusions, Sec. 8).  Host
// code only: every frequency of a refinement round is solved by one batched
// call of the GPU solver; the rule and the fit are a few hundred flops.
//
// Absorption S(w) = Im alpha_tr(w), alpha_tr = -tr P / 3.  Grid: a uniform
// start, then rounds over flagged intervals (all of them at first): solve
// their midpoints, and flag both halves again where
// |S(mid) - (S(l) + S(r)) / 2| > rel_tol max|S|.  Poles: one pole plus a
// constant background, alpha_tr = g / (Omega^2 - z^2) + b (z = w + i eps),
// fitted on the five grid points around every local maximum of S by complex
// least squares in (p = Omega^2, b, q = g + b p): alpha p + z^2 b - q = alpha z^2.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

namespace tddft {
namespace {

using cplx = std::complex<double>;

// S and alpha_tr of one 3 x 3 block (complex interleaved, row i, column k)
void trace_of(const double *P, cplx &alpha_tr, double &S) {
  const cplx tr(P[0] + P[8] + P[16], P[1] + P[9] + P[17]);
  alpha_tr = -tr / 3.0;
  S = alpha_tr.imag();
}

// Least squares min ||A x - y|| for A [k][3] (k >= 3) by modified
// Gram-Schmidt QR; false if A is rank deficient.
bool lstsq3(std::vector<std::array<cplx, 3>> A, std::vector<cplx> y, cplx x[3]) {
  const size_t k = A.size();
  cplx R[3][3] = {};
  for (int j = 0; j < 3; ++j) {
    for (int i = 0; i < j; ++i) {
      cplx d = 0.0;
      for (size_t r = 0; r < k; ++r) d += std::conj(A[r][i]) * A[r][j];
      R[i][j] = d;
      for (size_t r = 0; r < k; ++r) A[r][j] -= d * A[r][i];
    }
    double nrm = 0.0;
    for (size_t r = 0; r < k; ++r) nrm += std::norm(A[r][j]);
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0)) return false;
    R[j][j] = nrm;
    for (size_t r = 0; r < k; ++r) A[r][j] /= nrm;
  }
  cplx qy[3];
  for (int i = 0; i < 3; ++i) {
    cplx d = 0.0;
    for (size_t r = 0; r < k; ++r) d += std::conj(A[r][i]) * y[r];
    qy[i] = d;
  }
  for (int i = 2; i >= 0; --i) {
    cplx v = qy[i];
    for (int j = i + 1; j < 3; ++j) v -= R[i][j] * x[j];
    x[i] = v / R[i][i];
  }
  return true;
}

}  // namespace
}  // namespace tddft

extern "C" tddft_status tddft_spectrum_adaptive(tddft_ctx *ctx, double w_lo, double w_hi,
                                                double eps, const tddft_adaptive_options *o,
                                                double *omega, double *P, int32_t *n_points,
                                                tddft_pole *poles, int32_t max_poles,
                                                int32_t *n_poles) {
  using namespace tddft;
  if (!ctx) return TDDFT_ERR_INVALID_ARG;
  if (!o || !omega || !P || !n_points || !n_poles || (max_poles > 0 && !poles) || max_poles < 0)
    return set_ctx_error(ctx, TDDFT_ERR_INVALID_ARG, "null output or options");
  if (!(w_hi > w_lo) || !std::isfinite(w_lo) || !std::isfinite(w_hi) || !(eps > 0.0))
    return set_ctx_error(ctx, TDDFT_ERR_INVALID_ARG, "need w_lo < w_hi and eps > 0");
  if (o->n_initial < 2 || o->max_points < o->n_initial || !(o->rel_tol > 0.0) ||
      !(o->min_step >= 0.0) || !(o->peak_floor >= 0.0 && o->peak_floor < 1.0))
    return set_ctx_error(ctx, TDDFT_ERR_INVALID_ARG,
                         "bad adaptive options (n_initial >= 2, max_points >= n_initial, "
                         "rel_tol > 0, min_step >= 0, peak_floor in [0, 1))");
  *n_points = 0;
  *n_poles = 0;
  // grid: frequency -> (S, 3 x 3 block)
  std::map<double, std::pair<double, std::array<double, 18>>> grid;
  std::vector<double> buf;
  auto solve = [&](const std::vector<double> &ws) -> tddft_status {
    buf.assign(ws.size() * 18, 0.0);
    const tddft_status st = tddft_polarizability(ctx, (int32_t)ws.size(), ws.data(), eps,
                                                 buf.data(), nullptr, 0);
    for (size_t i = 0; i < ws.size(); ++i) {
      std::array<double, 18> blk;
      std::copy(buf.begin() + 18 * i, buf.begin() + 18 * (i + 1), blk.begin());
      cplx a;
      double S;
      trace_of(blk.data(), a, S);
      grid[ws[i]] = {S, blk};
    }
    return st;
  };
  auto write_grid = [&]() {
    int32_t n = 0;
    for (const auto &kv : grid) {
      omega[n] = kv.first;
      std::copy(kv.second.second.begin(), kv.second.second.end(), P + 18 * (size_t)n);
      ++n;
    }
    *n_points = n;
  };

  // uniform start (the last point exactly w_hi)
  std::vector<double> ws(o->n_initial);
  const double step = (w_hi - w_lo) / (o->n_initial - 1);
  for (int i = 0; i < o->n_initial; ++i) ws[i] = w_lo + i * step;
  ws.back() = w_hi;
  tddft_status st = solve(ws);
  if (st != TDDFT_OK) {
    write_grid();
    return st;
  }
  std::vector<std::pair<double, double>> flagged;
  for (int i = 0; i + 1 < o->n_initial; ++i) flagged.push_back({ws[i], ws[i + 1]});
  while (!flagged.empty() && (int32_t)grid.size() < o->max_points) {
    std::vector<std::pair<double, double>> live;
    for (const auto &iv : flagged)
      if (iv.second - iv.first > 2.0 * o->min_step) live.push_back(iv);
    // an interval whose midpoint rounds onto a grid point cannot be split
    {
      std::vector<std::pair<double, double>> keep;
      for (const auto &iv : live)
        if (!grid.count(0.5 * (iv.first + iv.second))) keep.push_back(iv);
      live.swap(keep);
    }
    const size_t room = (size_t)(o->max_points - (int32_t)grid.size());
    if (live.size() > room) live.resize(room);
    if (live.empty()) break;
    std::vector<double> mids(live.size());
    for (size_t i = 0; i < live.size(); ++i) mids[i] = 0.5 * (live[i].first + live[i].second);
    st = solve(mids);
    if (st != TDDFT_OK) {
      write_grid();
      return st;
    }
    double scale = 0.0;
    for (const auto &kv : grid) scale = std::max(scale, std::fabs(kv.second.first));
    std::vector<std::pair<double, double>> next;
    for (size_t i = 0; i < live.size(); ++i) {
      const double sl = grid[live[i].first].first, sr = grid[live[i].second].first;
      const double sm = grid[mids[i]].first;
      if (std::fabs(sm - 0.5 * (sl + sr)) > o->rel_tol * scale) {
        next.push_back({live[i].first, mids[i]});
        next.push_back({mids[i], live[i].second});
      }
    }
    flagged.swap(next);
  }
  write_grid();

  // peaks and one-pole fits
  const int32_t n = *n_points;
  std::vector<double> S(n);
  std::vector<cplx> a(n);
  double top = -INFINITY;
  for (int32_t i = 0; i < n; ++i) {
    trace_of(P + 18 * (size_t)i, a[i], S[i]);
    top = std::max(top, S[i]);
  }
  int32_t found = 0;
  for (int32_t i = 0; i < n; ++i) {
    const double left = i > 0 ? S[i - 1] : -INFINITY;
    const double right = i + 1 < n ? S[i + 1] : -INFINITY;
    if (!(S[i] > left && S[i] >= right && S[i] > o->peak_floor * top)) continue;
    const int32_t lo = std::min(std::max(0, i - 2), std::max(0, n - 5));
    const int32_t hi = std::min(n, lo + 5);
    tddft_pole pl{};
    pl.peak = S[i];
    pl.omega_peak = omega[i];
    std::vector<std::array<cplx, 3>> A;
    std::vector<cplx> y;
    for (int32_t r = lo; r < hi; ++r) {
      const cplx z(omega[r], eps), z2 = z * z;
      A.push_back({a[r], z2, cplx(-1.0, 0.0)});
      y.push_back(a[r] * z2);
    }
    cplx x[3] = {};
    if (hi - lo >= 3 && lstsq3(A, y, x)) {
      const cplx p = x[0], b = x[1], q = x[2];
      const cplx g = q - b * p;
      pl.omega = std::sqrt(std::max(p.real(), 0.0));
      pl.g_re = g.real();
      pl.g_im = g.imag();
    } else {
      pl.omega = omega[i];
      pl.g_re = pl.g_im = NAN;
    }
    if (found < max_poles) poles[found] = pl;
    ++found;
  }
  *n_poles = found;
  return TDDFT_OK;
}
