// Checkpoint and resume of a spectrum.  Every (omega, direction) solve is
// independent (the paper distributes them freely, Sec. 6.2.3), so a spectrum
// can be computed in pieces: each finished frequency is appended to a file as
// one record, and a later call over the same grid skips the recorded
// frequencies and solves the rest.
//
// File: a 64-byte header (magic "TDDFTCKP", version 1, and the fingerprint of
// the problem: n_prod, n_orb, n_occ, precision, stopping rule, restart,
// tolerance), then records of 280 bytes, appended in the order the groups
// finish:
//   double omega, eps; double P[3][3][2];
//   int32 matvecs[3], cycles[3], converged[3], flags[3];
//   double resid[3], eps_p[3], eps_x[3]
// Each group's records are flushed and synced before the next group starts.
// A record cut short by an interruption is dropped (the file is truncated to
// the last whole record before appending).
#include <unistd.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

namespace tddft {
const DevSystem *ctx_system(const tddft_ctx *c);
void ctx_set_error(tddft_ctx *c, const char *msg);
int ctx_slots(const tddft_ctx *c);
const tddft_options *ctx_options(const tddft_ctx *c);
}  // namespace tddft

namespace {
using namespace tddft;

constexpr char kMagic[8] = {'T', 'D', 'D', 'F', 'T', 'C', 'K', 'P'};

struct Header {
  char magic[8];
  int32_t version, n_prod, n_orb, n_occ, prec, stop, restart, pad;
  double tol;
  char reserved[16];
};
static_assert(sizeof(Header) == 64, "checkpoint header layout");

struct Record {
  double omega, eps;
  double P[18];
  int32_t matvecs[3], cycles[3], converged[3], flags[3];
  double resid[3], eps_p[3], eps_x[3];
};
static_assert(sizeof(Record) == 280, "checkpoint record layout");

uint64_t bits(double x) {
  uint64_t u;
  std::memcpy(&u, &x, sizeof u);
  return u;
}

Header header_of(const tddft_ctx *c) {
  Header h;
  std::memset(&h, 0, sizeof h);
  std::memcpy(h.magic, kMagic, 8);
  const DevSystem &s = *ctx_system(c);
  const tddft_options &o = *ctx_options(c);
  h.version = 1;
  h.n_prod = s.n_prod;
  h.n_orb = s.n_orb;
  h.n_occ = s.n_occ;
  h.prec = o.prec;
  h.stop = o.stop;
  h.restart = o.restart;
  h.tol = o.tol;
  return h;
}

tddft_status fail(tddft_ctx *c, tddft_status s, const std::string &msg) {
  ctx_set_error(c, msg.c_str());
  return s;
}
}  // namespace

extern "C" tddft_status tddft_polarizability_resume(tddft_ctx *ctx, int32_t n_omega,
                                                    const double *omega, double eps, double *P,
                                                    tddft_solve_stats *stats, const char *path,
                                                    int32_t *n_solved) {
  if (!ctx) return TDDFT_ERR_INVALID_ARG;
  ctx_set_error(ctx, "");
  if (n_omega < 1 || !omega || !P || !path)
    return fail(ctx, TDDFT_ERR_INVALID_ARG, "n_omega >= 1 and non-NULL omega, P, path required");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(ctx, TDDFT_ERR_INVALID_ARG, "eps must be > 0");
  for (int i = 0; i < n_omega; ++i)
    if (!std::isfinite(omega[i])) return fail(ctx, TDDFT_ERR_INVALID_ARG, "omega holds NaN or Inf");
  const Header want = header_of(ctx);
  // read what the file holds
  std::map<std::pair<uint64_t, uint64_t>, Record> done;
  long keep = 0;   // bytes of whole records (and header) to keep
  if (FILE *f = std::fopen(path, "rb")) {
    Header h;
    const size_t got = std::fread(&h, 1, sizeof h, f);
    if (got == sizeof h) {
      if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != 1) {
        std::fclose(f);
        return fail(ctx, TDDFT_ERR_INVALID_ARG, std::string("not a checkpoint file: ") + path);
      }
      if (h.n_prod != want.n_prod || h.n_orb != want.n_orb || h.n_occ != want.n_occ ||
          h.prec != want.prec || h.stop != want.stop || h.restart != want.restart ||
          bits(h.tol) != bits(want.tol)) {
        std::fclose(f);
        return fail(ctx, TDDFT_ERR_INVALID_ARG,
                    "the checkpoint belongs to another problem or solver setting");
      }
      keep = sizeof h;
      Record r;
      while (std::fread(&r, 1, sizeof r, f) == sizeof r) {
        done[{bits(r.omega), bits(r.eps)}] = r;
        keep += (long)sizeof r;
      }
    }
    std::fclose(f);
  }
  // drop a trailing partial record (or a partial header), then append
  if (keep == 0) {
    FILE *f = std::fopen(path, "wb");
    if (!f || std::fwrite(&want, sizeof want, 1, f) != 1) {
      if (f) std::fclose(f);
      return fail(ctx, TDDFT_ERR_INVALID_ARG, std::string("cannot write ") + path);
    }
    std::fflush(f);
    fsync(fileno(f));
    std::fclose(f);
    keep = sizeof want;
  } else if (truncate(path, keep) != 0) {
    return fail(ctx, TDDFT_ERR_INVALID_ARG, std::string("cannot truncate ") + path);
  }
  FILE *out = std::fopen(path, "ab");
  if (!out) return fail(ctx, TDDFT_ERR_INVALID_ARG, std::string("cannot append to ") + path);

  std::vector<int> todo;
  for (int i = 0; i < n_omega; ++i)
    if (!done.count({bits(omega[i]), bits(eps)})) todo.push_back(i);
  const int cw = std::max(1, ctx_slots(ctx) / 3);
  tddft_status result = TDDFT_OK;
  std::vector<double> om, Pc;
  std::vector<tddft_solve_stats> st;
  for (size_t c0 = 0; c0 < todo.size(); c0 += cw) {
    const int m = (int)std::min<size_t>(cw, todo.size() - c0);
    om.resize(m);
    Pc.resize((size_t)m * 18);
    st.resize((size_t)3 * m);
    for (int w = 0; w < m; ++w) om[w] = omega[todo[c0 + w]];
    const tddft_status s = tddft_polarizability(ctx, m, om.data(), eps, Pc.data(), st.data(), 0);
    if (s != TDDFT_OK && s != TDDFT_ERR_NOT_CONVERGED) {
      std::fclose(out);
      return s;
    }
    if (s == TDDFT_ERR_NOT_CONVERGED) result = s;
    for (int w = 0; w < m; ++w) {
      Record r;
      std::memset(&r, 0, sizeof r);
      r.omega = om[w];
      r.eps = eps;
      std::memcpy(r.P, Pc.data() + (size_t)18 * w, sizeof r.P);
      for (int k = 0; k < 3; ++k) {
        const tddft_solve_stats &t = st[(size_t)3 * w + k];
        r.matvecs[k] = t.matvecs;
        r.cycles[k] = t.cycles;
        r.converged[k] = t.converged;
        r.flags[k] = t.flags;
        r.resid[k] = t.resid;
        r.eps_p[k] = t.eps_p;
        r.eps_x[k] = t.eps_x;
      }
      if (std::fwrite(&r, sizeof r, 1, out) != 1) {
        std::fclose(out);
        return fail(ctx, TDDFT_ERR_INVALID_ARG, std::string("cannot append to ") + path);
      }
      done[{bits(r.omega), bits(r.eps)}] = r;
    }
    std::fflush(out);
    fsync(fileno(out));
  }
  std::fclose(out);
  // every requested frequency from its record
  for (int i = 0; i < n_omega; ++i) {
    const Record &r = done.at({bits(omega[i]), bits(eps)});
    std::memcpy(P + (size_t)18 * i, r.P, sizeof r.P);
    bool conv = true;
    for (int k = 0; k < 3; ++k) {
      conv = conv && r.converged[k];
      if (stats) {
        tddft_solve_stats &t = stats[(size_t)3 * i + k];
        t.matvecs = r.matvecs[k];
        t.cycles = r.cycles[k];
        t.converged = r.converged[k];
        t.flags = r.flags[k];
        t.resid = r.resid[k];
        t.eps_p = r.eps_p[k];
        t.eps_x = r.eps_x[k];
      }
    }
    if (!conv) result = TDDFT_ERR_NOT_CONVERGED;
  }
  if (n_solved) *n_solved = (int32_t)todo.size();
  if (result == TDDFT_ERR_NOT_CONVERGED) ctx_set_error(ctx, "some (omega, direction) missed tol");
  return result;
}
