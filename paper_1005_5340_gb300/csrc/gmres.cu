// Device-resident restarted GMRES for a group of right-hand sides, one per
// (omega, field direction): eq. sle solved by the Krylov method of Sec. 4.1
// (basis of eq. orthogonal-krylov-basis, minimal residual in the subspace),
// float64 throughout.  Each right-hand side runs its own state machine:
//   Arnoldi step j : w = A v_j, classical Gram-Schmidt against v_0..v_j
//                    with the second (reorthogonalising) pass folded in
//                    through the basis Gram matrix, Givens QR of the
//                    Hessenberg column, residual estimate |g_{j+1}|;
//   end of a cycle : x += V y, then the next operator application computes
//                    A x so that the true residual b - A x decides between
//                    done, not converged (cycle limit) and a restart.
// Right-hand sides that are done drop out of the active list, so the batched
// operator only works on live ones.
// Stopping rules: the relative residual ||b - A x|| / ||b|| <= tol, or the
// error estimates of Sec. 4.1, eps_P = |A^-1| |<d|r>| / |<d|x>| (alone, or
// together with eps_X = |A^-1| ||r|| / ||x||) <= tol, where |A^-1| is the
// Frobenius norm of the inverse of the square Krylov representation H_j of A
// and d the dipole of the right-hand side's direction.  For those each step
// keeps, per right-hand side, delta_i = <d|v_i>, xi_i = <x0|v_i> and
// phi_i = <d|A v_i> of the cycle, and solves R_j [y, c] = [g, e_j] with the
// rotated Hessenberg triangle: y gives <d|x_j>, ||x_j|| and <d|r_j> =
// <d|r_0> - sum_i phi_i y_i, and c (the last column of R_j^-1) extends
// ||R_j^-1||_F^2; ||H_j^-1||_F follows because H_j and R_j differ by a unitary
// factor except in the last diagonal entry (before the last rotation in H_j).
#include <cooperative_groups.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace tddft {
namespace {

constexpr int NT = 256;
constexpr int kHsmemMaxM = 48;   // restart lengths whose Hessenberg matrix is staged in shared memory
constexpr int kStateArnoldi = 0, kStateResid = 1, kStateDone = 2;

__device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ inline double cabs2(double2 a) { return hypot(a.x, a.y); }
__device__ inline double2 cdiv(double2 a, double2 b) {
  // a / b with scaling by the larger component of b
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + r * b.y;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    double r = b.x / b.y, d = b.y + r * b.x;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}

// Sum of NV values over the CTA; every thread receives the totals.
template <int NV>
__device__ void block_sum(double (&v)[NV], double *red /* [NV][NT/32] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double t = v[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    v[q] = t;
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) red[q * (NT / 32) + warp] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) t += red[q * (NT / 32) + w];
    v[q] = t;
  }
}

// Per-right-hand-side scalars of the error estimates (crit[r][kCrit]).
constexpr int kCrit = 10;
constexpr int kCrFsum = 0;   // ||R_j^-1||_F^2 of the current cycle's rotated triangle
constexpr int kCrFsq = 1;    // ||H_j^-1||_F^2 of the latest step (infinity before any)
constexpr int kCrPd0 = 2;    // <d|x0> (complex) of the current cycle
constexpr int kCrXn0 = 4;    // ||x0||^2
constexpr int kCrDr0 = 5;    // <d|r0> (complex)
constexpr int kCrEpsP = 7;   // eps_P and eps_X at the latest residual check
constexpr int kCrEpsX = 8;

struct Gs {
  int m, max_restarts, n_prod;
  int stop;   // 0: relative residual, 1: eps_P, 2: eps_P and eps_X
  double tol, inner_tol;
  double *rho0;
  int *state, *jcur, *cycles, *matvecs, *conv, *flags;
  double *bnorm, *resid, *omega;
  double2 *H, *sn, *g;
  double *cs, *V, *x, *b;
  float *Vf;   // the basis in float32 (refinement forms), else NULL
  const int *act;
  unsigned long long *bytes;
  double2 *Gm;
  const double *dip;   // [3][n_prod] dipoles
  const int *dir;      // [cap] direction of each right-hand side
  double *crit;        // [cap][kCrit]
  double2 *cvec;       // [cap][3 m + 2]: delta_0..m, xi_0..m, phi_0..m-1
  const float *dipf;   // the dipoles in float32 (float32 basis with estimates), else NULL
  float *xf;           // x in float32 (float32 basis with the eps_X estimate), else NULL
};

Gs view(const GmresState &s, const DevSystem &sys) {
  const int n_prod = sys.n_prod;
  Gs v;
  v.m = s.m; v.max_restarts = s.max_restarts; v.n_prod = n_prod; v.tol = s.tol;
  v.inner_tol = s.inner_tol; v.rho0 = s.rho0;
  v.state = s.state; v.jcur = s.jcur; v.cycles = s.cycles; v.matvecs = s.matvecs; v.conv = s.conv;
  v.flags = s.flags;
  v.bnorm = s.bnorm; v.resid = s.resid; v.omega = s.omega;
  v.H = s.H; v.sn = s.sn; v.g = s.g; v.cs = s.cs; v.V = s.V; v.x = s.x; v.b = s.b; v.act = s.act;
  v.Vf = s.Vf;
  v.bytes = s.bytes;
  v.Gm = s.Gm;
  v.stop = s.stop;
  v.dip = sys.dip;
  v.dir = s.dir;
  v.crit = s.crit;
  v.cvec = s.cvec;
  v.dipf = s.dipf;
  v.xf = s.xf;
  return v;
}

template <class T> __device__ __forceinline__ T *basis(const Gs &G);
template <> __device__ __forceinline__ double *basis<double>(const Gs &G) { return G.V; }
template <> __device__ __forceinline__ float *basis<float>(const Gs &G) { return G.Vf; }
// the dipoles and x in the basis type, for the error-estimate dot products
template <class T> __device__ __forceinline__ const T *dip_t(const Gs &G);
template <> __device__ __forceinline__ const double *dip_t<double>(const Gs &G) { return G.dip; }
template <> __device__ __forceinline__ const float *dip_t<float>(const Gs &G) { return G.dipf; }
template <class T> __device__ __forceinline__ T *x_t(const Gs &G);
template <> __device__ __forceinline__ double *x_t<double>(const Gs &G) { return G.x; }
template <> __device__ __forceinline__ float *x_t<float>(const Gs &G) { return G.xf; }

// F num / den, read as 0 when num = 0 and as infinity when only den = 0.
__device__ inline double est_ratio(double F, double num, double den) {
  if (num == 0.0) return 0.0;
  if (den == 0.0) return __longlong_as_double(0x7ff0000000000000LL);
  return F * num / den;
}
__device__ inline bool stop_met(int stop, double ep, double ex, double tol) {
  return stop == 1 ? ep <= tol : (ep <= tol && ex <= tol);
}

// Start: store b, x = 0, v_0 = b / ||b||.
template <class T>
__global__ void __launch_bounds__(NT) gmres_start_kernel(Gs G, const double *__restrict__ Bp) {
  __shared__ double red[3 * (NT / 32)];
  const int r = blockIdx.x;
  const int N = G.n_prod;
  const double *bin = Bp + (int64_t)2 * r * N;
  double *b = G.b + (int64_t)2 * r * N;
  double *x = G.x + (int64_t)2 * r * N;
  T *v0 = basis<T>(G) + (int64_t)r * (G.m + 1) * 2 * N;
  double s[3] = {0.0, 0.0, 0.0};
  for (int e = threadIdx.x; e < 2 * N; e += NT) {
    double t = bin[e];
    b[e] = t;
    x[e] = 0.0;
    s[0] += t * t;
  }
  if (G.xf)
    for (int e = threadIdx.x; e < 2 * N; e += NT) G.xf[(int64_t)2 * r * N + e] = 0.0f;
  if (G.stop) {
    const double *d = G.dip + (int64_t)G.dir[r] * N;
    for (int e = threadIdx.x; e < N; e += NT) {
      s[1] = fma(d[e], bin[e], s[1]);
      s[2] = fma(d[e], bin[N + e], s[2]);
    }
  }
  block_sum<3>(s, red);
  const double nrm = sqrt(s[0]);
  if (nrm > 0.0) {
    const double inv = 1.0 / nrm;
    for (int e = threadIdx.x; e < 2 * N; e += NT) v0[e] = (T)(bin[e] * inv);
  }
  if (threadIdx.x == 0) {
    G.bnorm[r] = nrm;
    G.matvecs[r] = 0;
    G.jcur[r] = 0;
    G.flags[r] = 0;
    if (G.stop) {
      // x0 = 0, r0 = b: <d|x0> = 0, ||x0|| = 0, <d|r0> = <d|b>; |A^-1| unknown
      double *cr = G.crit + (int64_t)r * kCrit;
      const double nan = __longlong_as_double(0x7ff8000000000000LL);
      cr[kCrFsum] = 0.0;
      cr[kCrFsq] = __longlong_as_double(0x7ff0000000000000LL);
      cr[kCrPd0] = 0.0;
      cr[kCrPd0 + 1] = 0.0;
      cr[kCrXn0] = 0.0;
      cr[kCrDr0] = s[1];
      cr[kCrDr0 + 1] = s[2];
      cr[kCrEpsP] = nan;
      cr[kCrEpsX] = nan;
      double2 *cv = G.cvec + (int64_t)r * (3 * G.m + 2);
      cv[0] = nrm > 0.0 ? make_double2(s[1] / nrm, s[2] / nrm) : make_double2(0.0, 0.0);
      cv[G.m + 1] = make_double2(0.0, 0.0);
    }
    if (nrm > 0.0) {
      G.state[r] = kStateArnoldi;
      G.cycles[r] = 1;
      G.conv[r] = 0;
      G.resid[r] = 1.0;
      G.g[(int64_t)r * (G.m + 1)] = make_double2(nrm, 0.0);
      G.rho0[r] = nrm;
    } else {
      G.state[r] = kStateDone;
      G.cycles[r] = 0;
      G.conv[r] = 1;
      G.resid[r] = 0.0;
    }
  }
}

// Ordered list of right-hand sides that are not done (one CTA).
// With split, right-hand sides in an Arnoldi step go to act and those whose
// next product is the residual check go to act2.
__global__ void __launch_bounds__(1024) gmres_select_kernel(const int *__restrict__ state, int n,
                                                            int split, int min_b,
                                                            int *__restrict__ act,
                                                            int *__restrict__ act2,
                                                            int *__restrict__ count) {
  __shared__ int sums[2][1024];
  const int t = threadIdx.x;
  const int chunk = (n + 1023) / 1024;
  const int lo = min(n, t * chunk), hi = min(n, lo + chunk);
  int c1 = 0, c2 = 0;
  for (int i = lo; i < hi; ++i) {
    const int st = state[i];
    if (st == kStateDone) continue;
    if (split && st == kStateResid) ++c2;
    else ++c1;
  }
  sums[0][t] = c1;
  sums[1][t] = c2;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {   // inclusive Hillis-Steele scans
    int v1 = (t >= off) ? sums[0][t - off] : 0;
    int v2 = (t >= off) ? sums[1][t - off] : 0;
    __syncthreads();
    sums[0][t] += v1;
    sums[1][t] += v2;
    __syncthreads();
  }
  int p1 = sums[0][t] - c1, p2 = sums[1][t] - c2;
  for (int i = lo; i < hi; ++i) {
    const int st = state[i];
    if (st == kStateDone) continue;
    if (split && st == kStateResid) act2[p2++] = i;
    else act[p1++] = i;
  }
  if (t == 1023) {
    const int c0 = sums[0][1023], c1v = sums[1][1023];
    count[0] = c0;
    // the float64 group waits until it is worth a launch, unless nothing else is left
    count[1] = (c0 > 0 && c1v < min_b) ? 0 : c1v;
  }
}

// Operator input of each active right-hand side: v_j (Arnoldi) or x (residual).
template <class T>
__global__ void __launch_bounds__(NT) gmres_gather_kernel(Gs G, const int *__restrict__ list,
                                                          double *__restrict__ Zc,
                                                          double *__restrict__ slot_omega,
                                                          const int *__restrict__ dcnt) {
  const int s = blockIdx.x;
  if (dcnt && s >= *dcnt) return;
  const int r = list[s];
  const int N = G.n_prod;
  double *dst = Zc + (int64_t)2 * s * N;
  if (G.state[r] == kStateArnoldi) {
    const T *src = basis<T>(G) + ((int64_t)r * (G.m + 1) + G.jcur[r]) * 2 * N;
    for (int e = threadIdx.x; e < 2 * N; e += NT) dst[e] = (double)src[e];
  } else {
    const double *src = G.x + (int64_t)2 * r * N;
    for (int e = threadIdx.x; e < 2 * N; e += NT) dst[e] = src[e];
  }
  if (threadIdx.x == 0) slot_omega[s] = G.omega[r];
}

// Sum of NV values over the P CTAs of the cluster (after the block sums), in
// rank order, so every CTA gets bit-identical totals.
template <int P, int NV>
__device__ void cluster_sum(double (&v)[NV], double *red, double *clx) {
  block_sum<NV>(v, red);
  if (P == 1) return;
  cg::cluster_group cl = cg::this_cluster();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) clx[q] = v[q];
  }
  cl.sync();
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = 0.0;
  for (int rk = 0; rk < P; ++rk) {
    const double *rem = cl.map_shared_rank(clx, rk);
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += rem[q];
  }
  cl.sync();   // clx may be reused once every CTA has read it
}

// One GMRES step of the right-hand side in slot blockIdx.y, its vectors split
// over the P CTAs of a cluster (element range per CTA); dot products and norms
// are reduced across the cluster through distributed shared memory.  Every
// CTA takes the same decisions from the same totals; rank 0 writes the
// per-right-hand-side scalars.
// EST: 0 the residual rule; 1 and 2 the error estimates (eps_P; eps_P and
// eps_X), the latter also needing <x0|v_i>.
template <int P, class T, int EST>
__global__ void __launch_bounds__(NT, 4) gmres_step_kernel(Gs G, const int *__restrict__ list,
                                                        const double *__restrict__ Wout,
                                                        const int *__restrict__ dcnt,
                                                        int h_smem) {
  __shared__ double red[16 * (NT / 32)];
  __shared__ double clx[16];
  __shared__ double2 hs[257], hp[257], ys[257], hq[257], gq[257], gp[257];
  __shared__ float2 hT[257];   // coefficients in float32 for the float32 basis
  __shared__ int finish_flag;
  __shared__ double2 s_gj;
  // error estimates: this step's <d|A v_j>, <d|w>, <x0|w>, |a|^2 and |rho|^2
  // of the last diagonal before and after its rotation, |g_{j+1}|, the
  // cycle's scalars read at entry, and the updated Frobenius sums
  __shared__ double2 s_phi, s_dw, s_xw;
  __shared__ double s_a2, s_rho2, s_est, s_cr[6], s_F[2];
  extern __shared__ double2 hdyn[];   // the Hessenberg columns when h_smem
  const int s = blockIdx.y;
  if (dcnt && s >= *dcnt) return;          // the same for the whole cluster
  const int rank = (P > 1) ? (int)cg::this_cluster().block_rank() : 0;
  const int r = list[s];
  const int N = G.n_prod;
  const int m = G.m;
  const int tid = threadIdx.x;
  // element range of this CTA; starts on multiples of 4 (16-byte float4 access)
  const int chunk = ((N + P - 1) / P + 3) & ~3;
  const int lo = rank * chunk, hi = min(N, lo + chunk);
  const bool vec4 = sizeof(T) == 4 && (N & 3) == 0;
  const int n4 = max(0, hi - lo) >> 2;
  const double *win = Wout + (int64_t)2 * s * N;
  T *Vr = basis<T>(G) + (int64_t)r * (m + 1) * 2 * N;
  const int state = G.state[r];
  const int cyc = G.cycles[r];

  if (state == kStateResid) {
    // r = b - A x ; decide done / not converged / restart
    const double *b = G.b + (int64_t)2 * r * N;
    double *x = G.x + (int64_t)2 * r * N;
    // [0] ||r||^2; with the error estimates also <d|r>, <d|b>, <d|x>, <x|r>
    // (complex) and ||x||^2
    double s2[10] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const double *d = EST ? G.dip + (int64_t)G.dir[r] * N : nullptr;
    for (int e = lo + tid; e < hi; e += NT) {
      const double tr = b[e] - win[e], ti = b[N + e] - win[N + e];
      Vr[e] = (T)tr;
      Vr[N + e] = (T)ti;
      s2[0] += tr * tr + ti * ti;
      if constexpr (EST > 0) {
        const double de = d[e], xr = x[e], xi = x[N + e];
        s2[1] = fma(de, tr, s2[1]);
        s2[2] = fma(de, ti, s2[2]);
        s2[3] = fma(de, b[e], s2[3]);
        s2[4] = fma(de, b[N + e], s2[4]);
        s2[5] = fma(de, xr, s2[5]);
        s2[6] = fma(de, xi, s2[6]);
        s2[7] = fma(xr, tr, fma(xi, ti, s2[7]));
        s2[8] = fma(xr, ti, fma(-xi, tr, s2[8]));
        s2[9] = fma(xr, xr, fma(xi, xi, s2[9]));
      }
    }
    if constexpr (EST > 0) {
      cluster_sum<P, 10>(s2, red, clx);
    } else {
      double t1[1] = {s2[0]};
      cluster_sum<P, 1>(t1, red, clx);
      s2[0] = t1[0];
    }
    double rho = sqrt(s2[0]);
    bool rejected = false;
    if (cyc == 0 && rho > G.bnorm[r]) {
      // the residual of a supplied initial guess: zero is the fallback and the
      // arbiter, so a guess worse than zero is dropped
      for (int e = lo + tid; e < hi; e += NT) {
        Vr[e] = (T)b[e];
        Vr[N + e] = (T)b[N + e];
        x[e] = 0.0;
        x[N + e] = 0.0;
      }
      if constexpr (EST == 2 && sizeof(T) == 4) {
        float *xf = G.xf + (int64_t)2 * r * N;
        for (int e = lo + tid; e < hi; e += NT) {
          xf[e] = 0.0f;
          xf[N + e] = 0.0f;
        }
      }
      rho = G.bnorm[r];
      rejected = true;
      // r = b and x = 0
      s2[1] = s2[3];
      s2[2] = s2[4];
      for (int q = 5; q < 10; ++q) s2[q] = 0.0;
    }
    const double rel = rho / G.bnorm[r];
    double ep = 0.0, ex = 0.0;
    bool met;
    if constexpr (EST > 0) {
      // eps_P and eps_X of x with the |A^-1| of the last step of the last cycle
      const double Fn = sqrt(G.crit[(int64_t)r * kCrit + kCrFsq]);
      ep = est_ratio(Fn, hypot(s2[1], s2[2]), hypot(s2[5], s2[6]));
      ex = est_ratio(Fn, rho, sqrt(s2[9]));
      met = rho == 0.0 || stop_met(EST, ep, ex, G.tol);
    } else {
      met = rel <= G.tol;
    }
    int next;
    if (met) next = 0;
    else if (cyc >= G.max_restarts) next = 1;
    else next = 2;
    if (next == 2) {
      const double inv = 1.0 / rho;
      for (int e = lo + tid; e < hi; e += NT) {
        Vr[e] *= (T)inv;
        Vr[N + e] *= (T)inv;
      }
    }
    if (tid == 0 && rank == 0) {
      // algorithmic traffic: b and A x read, v_0 written and normalised
      atomicAdd(G.bytes, (2ull * 16ull + 3ull * 2ull * sizeof(T)) * (unsigned long long)N);
      G.matvecs[r] += 1;
      G.resid[r] = rel;
      if (rejected) G.flags[r] |= 1;
      if constexpr (EST > 0) {
        double *cr = G.crit + (int64_t)r * kCrit;
        cr[kCrEpsP] = ep;
        cr[kCrEpsX] = ex;
        if (next == 2) {
          // the next cycle starts from x0 = x, r0 = r, v_0 = r / rho
          cr[kCrFsum] = 0.0;
          cr[kCrPd0] = s2[5];
          cr[kCrPd0 + 1] = s2[6];
          cr[kCrXn0] = s2[9];
          cr[kCrDr0] = s2[1];
          cr[kCrDr0 + 1] = s2[2];
          double2 *cv = G.cvec + (int64_t)r * (3 * m + 2);
          cv[0] = make_double2(s2[1] / rho, s2[2] / rho);
          cv[m + 1] = make_double2(s2[7] / rho, s2[8] / rho);
        }
      }
      if (next == 0) { G.state[r] = kStateDone; G.conv[r] = 1; }
      else if (next == 1) { G.state[r] = kStateDone; G.conv[r] = 0; }
      else {
        G.state[r] = kStateArnoldi;
        G.jcur[r] = 0;
        G.cycles[r] = cyc + 1;
        G.g[(int64_t)r * (m + 1)] = make_double2(rho, 0.0);
        G.rho0[r] = rho;
      }
    }
    return;
  }
  if (state != kStateArnoldi) return;

  const int j = G.jcur[r];
  const double2 gj0 = G.g[(int64_t)r * (m + 1) + j];
  const double rho0 = G.rho0[r];
  if (EST > 0 && tid == 0) {
    // read before the first cluster synchronisation: rank 0 rewrites them
    const double *cr = G.crit + (int64_t)r * kCrit;
    s_cr[0] = cr[kCrFsum];
    s_cr[1] = cr[kCrPd0];
    s_cr[2] = cr[kCrPd0 + 1];
    s_cr[3] = cr[kCrXn0];
    s_cr[4] = cr[kCrDr0];
    s_cr[5] = cr[kCrDr0 + 1];
  }
  T *w = Vr + (int64_t)(j + 1) * 2 * N;
  const T *vj = Vr + (int64_t)j * 2 * N;
  const int warp = tid >> 5, lane = tid & 31;

  // Classical Gram-Schmidt with the reorthogonalisation folded in through the
  // Gram matrix of the basis, G_ik = <v_i, v_k>: one pass over v_0..v_j gives
  // h1_i = <v_i, A v_j> and the new column g_i = <v_i, v_j>; the second CGS
  // pass would add h2 = V^H (w - V h1) = h1 - G h1, so the coefficients are
  // h = 2 h1 - G h1 and w = A v_j - V h (one update pass).  Warp q streams
  // v_q, v_{q+8}, ... over this CTA's elements; the partial dots of all i
  // are reduced across the cluster at once, in rank order.
  // Arithmetic of the streaming passes in the basis type T: float32 in the
  // refinement forms (float64 would make these passes FP64-pipe bound; the
  // per-lane sums are short and every reduction across lanes, CTAs and the
  // Gram and Hessenberg algebra stay float64), float64 otherwise.
  const T *aw;   // A v_j in type T
  if constexpr (sizeof(T) == 4) {
    if (vec4) {
      const double2 *wr2 = (const double2 *)(win + lo), *wi2 = (const double2 *)(win + N + lo);
      float4 *o_r = (float4 *)(w + lo), *o_i = (float4 *)(w + N + lo);
      for (int q = tid; q < n4; q += NT) {
        const double2 a = wr2[2 * q], b = wr2[2 * q + 1], c = wi2[2 * q], d = wi2[2 * q + 1];
        o_r[q] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
        o_i[q] = make_float4((float)c.x, (float)c.y, (float)d.x, (float)d.y);
      }
    } else {
      for (int e = lo + tid; e < hi; e += NT) {
        w[e] = (T)win[e];
        w[N + e] = (T)win[N + e];
      }
    }
    __syncthreads();
    aw = w;
  } else {
    aw = win;
  }
  for (int i = warp; i <= j; i += NT / 32) {
    const T *vi_ = Vr + (int64_t)i * 2 * N;
    T pr = 0, pim = 0, gr = 0, gim = 0;
    if (vec4) {
      // four elements per lane and load (float32 basis)
      const float4 *v_r = (const float4 *)(vi_ + lo), *v_i = (const float4 *)(vi_ + N + lo);
      const float4 *w_r = (const float4 *)(aw + lo), *w_i = (const float4 *)(aw + N + lo);
      const float4 *j_r = (const float4 *)(vj + lo), *j_i = (const float4 *)(vj + N + lo);
#pragma unroll 1
      for (int q = lane; q < n4; q += 32) {
        const float4 a = v_r[q], b = v_i[q], c = w_r[q], d = w_i[q], f = j_r[q], g = j_i[q];
        pr = fmaf(a.x, c.x, fmaf(b.x, d.x, fmaf(a.y, c.y, fmaf(b.y, d.y,
             fmaf(a.z, c.z, fmaf(b.z, d.z, fmaf(a.w, c.w, fmaf(b.w, d.w, pr))))))));
        pim = fmaf(a.x, d.x, fmaf(-b.x, c.x, fmaf(a.y, d.y, fmaf(-b.y, c.y,
              fmaf(a.z, d.z, fmaf(-b.z, c.z, fmaf(a.w, d.w, fmaf(-b.w, c.w, pim))))))));
        gr = fmaf(a.x, f.x, fmaf(b.x, g.x, fmaf(a.y, f.y, fmaf(b.y, g.y,
             fmaf(a.z, f.z, fmaf(b.z, g.z, fmaf(a.w, f.w, fmaf(b.w, g.w, gr))))))));
        gim = fmaf(a.x, g.x, fmaf(-b.x, f.x, fmaf(a.y, g.y, fmaf(-b.y, f.y,
              fmaf(a.z, g.z, fmaf(-b.z, f.z, fmaf(a.w, g.w, fmaf(-b.w, f.w, gim))))))));
      }
    } else {
#pragma unroll 4
      for (int e = lo + lane; e < hi; e += 32) {
        const T wr = aw[e], wi = aw[N + e];
        const T ar = vj[e], ai = vj[N + e];
        const T vr = vi_[e], vi = vi_[N + e];
        pr = fma(vr, wr, fma(vi, wi, pr));
        pim = fma(vr, wi, fma(-vi, wr, pim));
        gr = fma(vr, ar, fma(vi, ai, gr));
        gim = fma(vr, ai, fma(-vi, ar, gim));
      }
    }
    // across the warp in type T (the float32 basis: float64 shuffles would load
    // the FP64 pipe with every vector), then float64 per warp
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      pr += __shfl_xor_sync(0xffffffffu, pr, off);
      pim += __shfl_xor_sync(0xffffffffu, pim, off);
      gr += __shfl_xor_sync(0xffffffffu, gr, off);
      gim += __shfl_xor_sync(0xffffffffu, gim, off);
    }
    if (lane == 0) {
      hq[i] = make_double2((double)pr, (double)pim);
      gq[i] = make_double2((double)gr, (double)gim);
    }
  }
  if (P == 1) {
    __syncthreads();
    for (int i = tid; i <= j; i += NT) {
      hp[i] = hq[i];
      gp[i] = gq[i];
    }
  } else {
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    for (int i = tid; i <= j; i += NT) {
      double2 t = make_double2(0.0, 0.0), u = make_double2(0.0, 0.0);
      for (int rk = 0; rk < P; ++rk) {
        const double2 a = cl.map_shared_rank(hq, rk)[i];
        const double2 b = cl.map_shared_rank(gq, rk)[i];
        t.x += a.x;
        t.y += a.y;
        u.x += b.x;
        u.y += b.y;
      }
      hp[i] = t;
      gp[i] = u;
    }
    cl.sync();   // hq, gq may be rewritten once every CTA has read them
  }
  __syncthreads();
  // h_i = 2 h1_i - sum_k G_ik h1_k (warp per row i, lanes over k); column k
  // of G (entries i <= k) is stored at Gr[k (m+1) + i], column j is gp
  double2 *Gr = G.Gm + (int64_t)r * (m + 1) * (m + 1);
  for (int i = warp; i <= j; i += NT / 32) {
    double sr = 0.0, si = 0.0;
    for (int k = lane; k <= j; k += 32) {
      double2 gik;
      if (k == j) gik = gp[i];
      else if (i == j) gik = cconj(gp[k]);
      else if (k >= i) gik = Gr[(int64_t)k * (m + 1) + i];
      else gik = cconj(Gr[(int64_t)i * (m + 1) + k]);
      const double2 t = cmul(gik, hp[k]);
      sr += t.x;
      si += t.y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, off);
      si += __shfl_xor_sync(0xffffffffu, si, off);
    }
    if (lane == 0) hs[i] = make_double2(2.0 * hp[i].x - sr, 2.0 * hp[i].y - si);
  }
  __syncthreads();
  if (rank == 0)
    for (int i = tid; i <= j; i += NT) Gr[(int64_t)j * (m + 1) + i] = gp[i];
  // w = A v_j - V h, with ||w||^2 (coefficients in type T)
  for (int i = tid; i <= j; i += NT) hT[i] = make_float2((float)hs[i].x, (float)hs[i].y);
  __syncthreads();
  // ||w||^2, and with the error estimates <d|A v_j>, <d|w> (and <x0|w>) from
  // the values in registers (d and x0 in the basis type)
  double q7[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const T *dT = nullptr, *x0T = nullptr;
  if constexpr (EST > 0) {
    dT = dip_t<T>(G) + (int64_t)G.dir[r] * N;
    if constexpr (EST == 2) x0T = x_t<T>(G) + (int64_t)2 * r * N;
  }
  if (vec4) {
    // four elements per thread and load (float32 basis); w holds A v_j here
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float4 *w_r = (float4 *)(w + lo), *w_i = (float4 *)(w + N + lo);
    for (int q = tid; q < n4; q += NT) {
      float4 ar = make_float4(0.f, 0.f, 0.f, 0.f), ai = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
      for (int i = 0; i <= j; ++i) {
        const float *vi_ = (const float *)(Vr + (int64_t)i * 2 * N);
        const float4 a = ((const float4 *)(vi_ + lo))[q], b = ((const float4 *)(vi_ + N + lo))[q];
        const float hx = hT[i].x, hy = hT[i].y;
        ar.x = fmaf(hx, a.x, fmaf(-hy, b.x, ar.x));
        ar.y = fmaf(hx, a.y, fmaf(-hy, b.y, ar.y));
        ar.z = fmaf(hx, a.z, fmaf(-hy, b.z, ar.z));
        ar.w = fmaf(hx, a.w, fmaf(-hy, b.w, ar.w));
        ai.x = fmaf(hx, b.x, fmaf(hy, a.x, ai.x));
        ai.y = fmaf(hx, b.y, fmaf(hy, a.y, ai.y));
        ai.z = fmaf(hx, b.z, fmaf(hy, a.z, ai.z));
        ai.w = fmaf(hx, b.w, fmaf(hy, a.w, ai.w));
      }
      const float4 c = w_r[q], d = w_i[q];
      const float4 nr = make_float4(c.x - ar.x, c.y - ar.y, c.z - ar.z, c.w - ar.w);
      const float4 ni = make_float4(d.x - ai.x, d.y - ai.y, d.z - ai.z, d.w - ai.w);
      w_r[q] = nr;
      w_i[q] = ni;
      acc[0] += nr.x * nr.x + nr.y * nr.y + nr.z * nr.z + nr.w * nr.w + ni.x * ni.x +
                ni.y * ni.y + ni.z * ni.z + ni.w * ni.w;
      if constexpr (EST > 0) {
        const float4 dp = ((const float4 *)((const float *)dT + lo))[q];
        acc[1] += dp.x * c.x + dp.y * c.y + dp.z * c.z + dp.w * c.w;
        acc[2] += dp.x * d.x + dp.y * d.y + dp.z * d.z + dp.w * d.w;
        acc[3] += dp.x * nr.x + dp.y * nr.y + dp.z * nr.z + dp.w * nr.w;
        acc[4] += dp.x * ni.x + dp.y * ni.y + dp.z * ni.z + dp.w * ni.w;
        if constexpr (EST == 2) {
          const float4 xr = ((const float4 *)((const float *)x0T + lo))[q];
          const float4 xi = ((const float4 *)((const float *)x0T + N + lo))[q];
          acc[5] += xr.x * nr.x + xi.x * ni.x + xr.y * nr.y + xi.y * ni.y + xr.z * nr.z +
                    xi.z * ni.z + xr.w * nr.w + xi.w * ni.w;
          acc[6] += xr.x * ni.x - xi.x * nr.x + xr.y * ni.y - xi.y * nr.y + xr.z * ni.z -
                    xi.z * nr.z + xr.w * ni.w - xi.w * nr.w;
        }
      }
    }
    constexpr int NQ = EST == 0 ? 1 : (EST == 1 ? 5 : 7);
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      float v = acc[k];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      q7[k] = lane == 0 ? (double)v : 0.0;   // the block sum adds the warps' totals
    }
  } else {
    T acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int e = lo + tid; e < hi; e += NT) {
      T ar = 0, ai = 0;
#pragma unroll 4
      for (int i = 0; i <= j; ++i) {
        const T *vi_ = Vr + (int64_t)i * 2 * N;
        T hx, hy;
        if constexpr (sizeof(T) == 4) {
          hx = hT[i].x;
          hy = hT[i].y;
        } else {
          hx = hs[i].x;
          hy = hs[i].y;
        }
        const T vr = vi_[e], vi = vi_[N + e];
        ar += hx * vr - hy * vi;
        ai += hx * vi + hy * vr;
      }
      const T avr = aw[e], avi = aw[N + e];
      const T nr = avr - ar, ni = avi - ai;
      w[e] = nr;
      w[N + e] = ni;
      acc[0] += nr * nr + ni * ni;
      if constexpr (EST > 0) {
        const T de = dT[e];
        acc[1] += de * avr;
        acc[2] += de * avi;
        acc[3] += de * nr;
        acc[4] += de * ni;
        if constexpr (EST == 2) {
          const T xr = x0T[e], xi = x0T[N + e];
          acc[5] += xr * nr + xi * ni;
          acc[6] += xr * ni - xi * nr;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) q7[k] = (double)acc[k];
  }
  if constexpr (EST > 0) {
    cluster_sum<P, 7>(q7, red, clx);   // synchronises: w complete
    if (tid == 0) {
      s_phi = make_double2(q7[1], q7[2]);
      s_dw = make_double2(q7[3], q7[4]);
      s_xw = make_double2(q7[5], q7[6]);
    }
  } else {
    double n1[1] = {q7[0]};
    cluster_sum<P, 1>(n1, red, clx);   // synchronises: w complete
    q7[0] = n1[0];
  }
  const double hn = sqrt(q7[0]);

  // the earlier rotations to shared memory (all threads), then thread 0
  // applies them to the new column in order
  {
    const double *csg = G.cs + (int64_t)r * m;
    const double2 *sng = G.sn + (int64_t)r * m;
    for (int i = tid; i < j; i += NT) {
      gq[i] = make_double2(csg[i], 0.0);
      hq[i] = sng[i];
    }
  }
  __syncthreads();
  if (tid == 0) {
    // every CTA rotates its own copy of the new column (identical inputs)
    for (int i = 0; i < j; ++i) {
      const double csi = gq[i].x;
      const double2 sni = hq[i];
      const double2 a = hs[i], bb = hs[i + 1];
      const double2 t = make_double2(csi * a.x + (sni.x * bb.x - sni.y * bb.y),
                                     csi * a.y + (sni.x * bb.y + sni.y * bb.x));
      const double2 cb = cmul(cconj(sni), a);
      hs[i + 1] = make_double2(-cb.x + csi * bb.x, -cb.y + csi * bb.y);
      hs[i] = t;
    }
    // new rotation mapping (hs[j], hn) to (rho, 0)
    const double2 a = hs[j];
    const double aa = cabs2(a);
    double c;
    double2 sv;
    if (hn == 0.0) { c = 1.0; sv = make_double2(0.0, 0.0); }
    else if (aa == 0.0) { c = 0.0; sv = make_double2(1.0, 0.0); }
    else {
      const double rr = hypot(aa, hn);
      c = aa / rr;
      sv = make_double2(a.x / aa * hn / rr, a.y / aa * hn / rr);
    }
    hs[j] = make_double2(c * a.x + sv.x * hn, c * a.y + sv.y * hn);
    const double2 t = cmul(cconj(sv), gj0);
    const double2 gnext = make_double2(-t.x, -t.y);
    const double2 gj = make_double2(c * gj0.x, c * gj0.y);
    const double est = cabs2(gnext);
    // a cycle ends at the tolerance (of the residual rule; the error
    // estimates decide below), at the restart length, on breakdown, or
    // (refinement forms) once it has reduced its own residual by inner_tol
    const bool fin = (!EST && est <= G.tol * G.bnorm[r]) || (j + 1 == m) || !(hn > 0.0) ||
                     (est <= G.inner_tol * rho0);
    finish_flag = fin ? 1 : 0;
    s_gj = gj;
    s_a2 = aa * aa;
    s_rho2 = aa * aa + hn * hn;
    s_est = est;
    gq[0] = make_double2(c, 0.0);   // the new rotation, kept for the writes below
    hq[0] = sv;
    hq[1] = gnext;
  }
  __syncthreads();
  const double c_new = gq[0].x;
  const double2 sv_new = hq[0], gnext_new = hq[1];
  if constexpr (EST > 0) {
    // R_j [y, c] = [g, e_j] (R_j: earlier rotated columns, shared memory when
    // they fit, and column j from this step), then the estimates of x_j
    const int k = j + 1;
    const double2 *Hr = G.H + (int64_t)r * (m + 1) * m;
    const double2 *gg = G.g + (int64_t)r * (m + 1);
    if (h_smem) {
      for (int idx = tid; idx < j * (m + 1); idx += NT) {
        const int l = idx / (m + 1), i = idx - l * (m + 1);
        if (i <= l) hdyn[idx] = Hr[idx];
      }
    }
    for (int i = tid; i < j; i += NT) hp[i] = gg[i];
    __syncthreads();
    const double2 *Hs = h_smem ? hdyn : Hr;
    if (warp == 0) {
      for (int i = k - 1; i >= 0; --i) {
        double sr = 0.0, si = 0.0, cr = 0.0, ci = 0.0;
        for (int l = i + 1 + lane; l < k; l += 32) {
          const double2 hil = (l == j) ? hs[i] : Hs[(int64_t)l * (m + 1) + i];
          const double2 p = cmul(hil, ys[l]), q = cmul(hil, gq[l]);
          sr += p.x;
          si += p.y;
          cr += q.x;
          ci += q.y;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          sr += __shfl_xor_sync(0xffffffffu, sr, off);
          si += __shfl_xor_sync(0xffffffffu, si, off);
          cr += __shfl_xor_sync(0xffffffffu, cr, off);
          ci += __shfl_xor_sync(0xffffffffu, ci, off);
        }
        if (lane == 0) {
          const double2 gi = (i == j) ? s_gj : hp[i];
          const double2 hii = (i == j) ? hs[j] : Hs[(int64_t)i * (m + 1) + i];
          ys[i] = cdiv(make_double2(gi.x - sr, gi.y - si), hii);
          gq[i] = cdiv(make_double2((i == j ? 1.0 : 0.0) - cr, -ci), hii);
        }
        __syncwarp();
      }
      // <d|x_j> = <d|x0> + sum delta_i y_i, <d|r_j> = <d|r0> - sum phi_i y_i,
      // ||x_j||^2 = ||x0||^2 + 2 Re sum xi_i y_i + sum |y_i|^2, and the
      // squared norm of the last column of R_j^-1
      const double2 *cv = G.cvec + (int64_t)r * (3 * m + 2);
      double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      for (int i = lane; i < k; i += 32) {
        const double2 yi = ys[i], ci = gq[i];
        const double2 dl = cv[i], xi = cv[m + 1 + i];
        const double2 ph = (i == j) ? s_phi : cv[2 * m + 2 + i];
        const double2 a = cmul(dl, yi), bq = cmul(ph, yi), cq = cmul(xi, yi);
        acc[0] += a.x;
        acc[1] += a.y;
        acc[2] += bq.x;
        acc[3] += bq.y;
        acc[4] += cq.x;
        acc[5] += yi.x * yi.x + yi.y * yi.y;
        acc[6] += ci.x * ci.x + ci.y * ci.y;
      }
#pragma unroll
      for (int q = 0; q < 7; ++q)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
      if (lane == 0) {
        const double Pr = s_cr[1] + acc[0], Pi = s_cr[2] + acc[1];
        const double dr = s_cr[4] - acc[2], di = s_cr[5] - acc[3];
        const double xx = fmax(0.0, s_cr[3] + 2.0 * acc[4] + acc[5]);
        const double Fsum = s_cr[0] + acc[6];
        // H_j differs from R_j only in the last diagonal entry: a instead of rho
        const double Fsq = s_a2 > 0.0 ? s_cr[0] + acc[6] * (s_rho2 / s_a2)
                                      : __longlong_as_double(0x7ff0000000000000LL);
        const double Fn = sqrt(Fsq);
        const double ep = est_ratio(Fn, hypot(dr, di), hypot(Pr, Pi));
        const double ex = est_ratio(Fn, s_est, sqrt(xx));
        if (stop_met(EST, ep, ex, G.tol)) finish_flag = 1;
        s_F[0] = Fsum;
        s_F[1] = Fsq;
      }
    }
    __syncthreads();
  }
  if (tid == 0 && rank == 0) {
    const bool fin = finish_flag != 0;
    double2 *Hc = G.H + (int64_t)r * (m + 1) * m + (int64_t)j * (m + 1);
    for (int i = 0; i <= j; ++i) Hc[i] = hs[i];
    G.cs[(int64_t)r * m + j] = c_new;
    G.sn[(int64_t)r * m + j] = sv_new;
    G.g[(int64_t)r * (m + 1) + j] = s_gj;
    G.g[(int64_t)r * (m + 1) + j + 1] = gnext_new;
    G.matvecs[r] += 1;
    if (fin) G.state[r] = kStateResid;
    else G.jcur[r] = j + 1;
    // algorithmic traffic of this step: basis vectors (2 N sizeof(T) bytes)
    // v_0..v_j read twice, v_{j+1} written and normalised, A v_j read
    // (16 N); at a cycle end v_0..v_j read again and x read and written
    const unsigned long long nb = 2ull * (j + 1) + 3ull + (fin ? (unsigned long long)j + 1ull : 0ull);
    const unsigned long long nd = 1ull + (fin ? 2ull : 0ull);
    // the error estimates read d (and x0) in the basis type; x0's float32
    // copy is rewritten with x at a cycle end
    const unsigned long long ne =
        (EST == 0 ? 0ull : (EST == 1 ? 1ull : 3ull)) * sizeof(T) +
        (EST == 2 && sizeof(T) == 4 && fin ? 8ull : 0ull);
    atomicAdd(G.bytes, (nb * 2ull * sizeof(T) + nd * 16ull + ne) * (unsigned long long)N);
    if constexpr (EST > 0) {
      double *cr = G.crit + (int64_t)r * kCrit;
      cr[kCrFsum] = s_F[0];
      cr[kCrFsq] = s_F[1];
      double2 *cv = G.cvec + (int64_t)r * (3 * m + 2);
      cv[2 * m + 2 + j] = s_phi;
      if (hn > 0.0) {
        // v_{j+1} = w / hn
        const double inv = 1.0 / hn;
        cv[j + 1] = make_double2(s_dw.x * inv, s_dw.y * inv);
        cv[m + 1 + j + 1] = make_double2(s_xw.x * inv, s_xw.y * inv);
      }
    }
  }
  __syncthreads();
  if (finish_flag && !EST) {
    // back substitution R y = g (with the error estimates, ys holds y already) with the rotated (upper triangular)
    // Hessenberg matrix: its earlier columns (shared memory when they fit)
    // and g_0..g_{j-1} staged by all threads, column j and g_j from this
    // step; warp 0 solves, lanes over the columns l > i
    const int k = j + 1;
    const double2 *Hr = G.H + (int64_t)r * (m + 1) * m;
    const double2 *gg = G.g + (int64_t)r * (m + 1);
    if (h_smem) {
      for (int idx = tid; idx < j * (m + 1); idx += NT) {
        const int l = idx / (m + 1), i = idx - l * (m + 1);
        if (i <= l) hdyn[idx] = Hr[idx];
      }
    }
    for (int i = tid; i < j; i += NT) hp[i] = gg[i];
    __syncthreads();
    const double2 *Hs = h_smem ? hdyn : Hr;
    if (warp == 0) {
      for (int i = k - 1; i >= 0; --i) {
        double sr = 0.0, si = 0.0;
        for (int l = i + 1 + lane; l < k; l += 32) {
          const double2 hil = (l == j) ? hs[i] : Hs[(int64_t)l * (m + 1) + i];
          const double2 p = cmul(hil, ys[l]);
          sr += p.x;
          si += p.y;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          sr += __shfl_xor_sync(0xffffffffu, sr, off);
          si += __shfl_xor_sync(0xffffffffu, si, off);
        }
        if (lane == 0) {
          const double2 gi = (i == j) ? s_gj : hp[i];
          const double2 hii = (i == j) ? hs[j] : Hs[(int64_t)i * (m + 1) + i];
          ys[i] = cdiv(make_double2(gi.x - sr, gi.y - si), hii);
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
  if (!finish_flag) {
    const T inv = (T)(1.0 / hn);
    if (vec4) {
      float4 *w_r = (float4 *)(w + lo), *w_i = (float4 *)(w + N + lo);
      const float fi = (float)inv;
      for (int q = tid; q < n4; q += NT) {
        float4 a = w_r[q], b = w_i[q];
        a.x *= fi; a.y *= fi; a.z *= fi; a.w *= fi;
        b.x *= fi; b.y *= fi; b.z *= fi; b.w *= fi;
        w_r[q] = a;
        w_i[q] = b;
      }
    } else {
      for (int e = lo + tid; e < hi; e += NT) {
        w[e] *= inv;
        w[N + e] *= inv;
      }
    }
  } else {
    const int k = j + 1;
    double *x = G.x + (int64_t)2 * r * N;
    for (int i = tid; i < k; i += NT) hT[i] = make_float2((float)ys[i].x, (float)ys[i].y);
    __syncthreads();
    if (vec4) {
      double2 *x_r = (double2 *)(x + lo), *x_i = (double2 *)(x + N + lo);
      for (int q = tid; q < n4; q += NT) {
        float4 ar = make_float4(0.f, 0.f, 0.f, 0.f), ai = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
        for (int i = 0; i < k; ++i) {
          const float *vi_ = (const float *)(Vr + (int64_t)i * 2 * N);
          const float4 a = ((const float4 *)(vi_ + lo))[q], b = ((const float4 *)(vi_ + N + lo))[q];
          const float yx = hT[i].x, yy = hT[i].y;
          ar.x = fmaf(yx, a.x, fmaf(-yy, b.x, ar.x));
          ar.y = fmaf(yx, a.y, fmaf(-yy, b.y, ar.y));
          ar.z = fmaf(yx, a.z, fmaf(-yy, b.z, ar.z));
          ar.w = fmaf(yx, a.w, fmaf(-yy, b.w, ar.w));
          ai.x = fmaf(yx, b.x, fmaf(yy, a.x, ai.x));
          ai.y = fmaf(yx, b.y, fmaf(yy, a.y, ai.y));
          ai.z = fmaf(yx, b.z, fmaf(yy, a.z, ai.z));
          ai.w = fmaf(yx, b.w, fmaf(yy, a.w, ai.w));
        }
        double2 p0 = x_r[2 * q], p1 = x_r[2 * q + 1], q0 = x_i[2 * q], q1 = x_i[2 * q + 1];
        p0.x += (double)ar.x; p0.y += (double)ar.y; p1.x += (double)ar.z; p1.y += (double)ar.w;
        q0.x += (double)ai.x; q0.y += (double)ai.y; q1.x += (double)ai.z; q1.y += (double)ai.w;
        x_r[2 * q] = p0; x_r[2 * q + 1] = p1; x_i[2 * q] = q0; x_i[2 * q + 1] = q1;
        if constexpr (EST == 2) {
          // the float32 copy of x for the next cycle's <x0|w>
          float *xf = G.xf + (int64_t)2 * r * N;
          ((float4 *)(xf + lo))[q] = make_float4((float)p0.x, (float)p0.y, (float)p1.x, (float)p1.y);
          ((float4 *)(xf + N + lo))[q] = make_float4((float)q0.x, (float)q0.y, (float)q1.x, (float)q1.y);
        }
      }
    } else
    for (int e = lo + tid; e < hi; e += NT) {
      T ar = 0, ai = 0;
#pragma unroll 4
      for (int i = 0; i < k; ++i) {
        const T *vi_ = Vr + (int64_t)i * 2 * N;
        T yx, yy;
        if constexpr (sizeof(T) == 4) {
          yx = hT[i].x;
          yy = hT[i].y;
        } else {
          yx = ys[i].x;
          yy = ys[i].y;
        }
        const T vr = vi_[e], vi = vi_[N + e];
        ar += yx * vr - yy * vi;
        ai += yx * vi + yy * vr;
      }
      x[e] += (double)ar;
      x[N + e] += (double)ai;
      if constexpr (EST == 2 && sizeof(T) == 4) {
        float *xf = G.xf + (int64_t)2 * r * N;
        xf[e] = (float)x[e];
        xf[N + e] = (float)x[N + e];
      }
    }
  }
}

// Initial guesses: x = x0 (interleaved complex rows g0..g0+n-1), and the first
// operator product is A x0 (state "awaiting A x", no cycle started yet).
__global__ void __launch_bounds__(NT) gmres_guess_kernel(Gs G, int g0,
                                                         const double *__restrict__ x0) {
  const int r = blockIdx.x;
  const int N = G.n_prod;
  if (G.state[r] == kStateDone) return;   // b = 0: x stays 0
  const double *src = x0 + (int64_t)(g0 + r) * 2 * N;
  double *x = G.x + (int64_t)2 * r * N;
  for (int e = threadIdx.x; e < N; e += NT) {
    x[e] = src[2 * e];
    x[N + e] = src[2 * e + 1];
  }
  if (G.xf) {
    float *xf = G.xf + (int64_t)2 * r * N;
    for (int e = threadIdx.x; e < N; e += NT) {
      xf[e] = (float)src[2 * e];
      xf[N + e] = (float)src[2 * e + 1];
    }
  }
  if (threadIdx.x == 0) {
    G.state[r] = kStateResid;
    G.cycles[r] = 0;
  }
}

// X rows g0..g0+n-1 (interleaved complex) = x of each right-hand side.
__global__ void __launch_bounds__(NT) gmres_export_kernel(Gs G, int g0, double *__restrict__ X) {
  const int r = blockIdx.x;
  const int N = G.n_prod;
  const double *x = G.x + (int64_t)2 * r * N;
  double *dst = X + (int64_t)(g0 + r) * 2 * N;
  for (int e = threadIdx.x; e < N; e += NT) {
    dst[2 * e] = x[e];
    dst[2 * e + 1] = x[N + e];
  }
}

// Right-hand sides g0 .. g0+n-1 of a spectrum: index g -> (omega g/3, direction g%3).
__global__ void rhs_init_kernel(int n, int g0, int n_prod, const double *__restrict__ omega_all,
                                const double *__restrict__ dip, double *__restrict__ Zc,
                                double *__restrict__ slot_omega, double *__restrict__ gs_omega,
                                int *__restrict__ gs_dir) {
  const int r = blockIdx.x;
  const int g = g0 + r;
  const int k = g % 3;
  const double *d = dip + (int64_t)k * n_prod;
  double *z = Zc + (int64_t)2 * r * n_prod;
  for (int e = threadIdx.x; e < n_prod; e += blockDim.x) {
    z[e] = d[e];
    z[n_prod + e] = 0.0;
  }
  if (threadIdx.x == 0) {
    slot_omega[r] = omega_all[g / 3];
    gs_omega[r] = omega_all[g / 3];
    if (gs_dir) gs_dir[r] = k;
  }
}

// P[w][i][k] = d_i . x_{(w,k)} for the right-hand sides g0 .. g0+n-1.
__global__ void __launch_bounds__(NT) polarization_kernel(int g0, int n_prod,
                                                          const double *__restrict__ dip,
                                                          const double *__restrict__ X,
                                                          double2 *__restrict__ P) {
  __shared__ double red[6 * (NT / 32)];
  const int r = blockIdx.x;
  const int g = g0 + r;
  const double *x = X + (int64_t)2 * r * n_prod;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int e = threadIdx.x; e < n_prod; e += NT) {
    const double xr = x[e], xi = x[n_prod + e];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double d = dip[(int64_t)i * n_prod + e];
      acc[2 * i] = fma(d, xr, acc[2 * i]);
      acc[2 * i + 1] = fma(d, xi, acc[2 * i + 1]);
    }
  }
  block_sum<6>(acc, red);
  if (threadIdx.x == 0) {
    const int w = g / 3, k = g % 3;
    for (int i = 0; i < 3; ++i) P[((int64_t)w * 3 + i) * 3 + k] = make_double2(acc[2 * i], acc[2 * i + 1]);
  }
}

template <class T, int EST>
cudaError_t launch_step_e(cudaStream_t st, const Gs &G, int P, int S, const int *list,
                          const double *Wout, const int *dcnt, int h_smem, size_t dyn) {
  static bool attr_set = false;
  if (!attr_set) {
    const int mx = (int)((size_t)kHsmemMaxM * (kHsmemMaxM + 1) * sizeof(double2));
    cudaFuncSetAttribute(gmres_step_kernel<1, T, EST>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(gmres_step_kernel<2, T, EST>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(gmres_step_kernel<4, T, EST>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(gmres_step_kernel<8, T, EST>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    attr_set = true;
  }
  if (P == 1) {
    gmres_step_kernel<1, T, EST><<<dim3(1, S), NT, dyn, st>>>(G, list, Wout, dcnt, h_smem);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P, S);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (P == 8) return cudaLaunchKernelEx(&cfg, gmres_step_kernel<8, T, EST>, G, list, Wout, dcnt, h_smem);
  return P == 4 ? cudaLaunchKernelEx(&cfg, gmres_step_kernel<4, T, EST>, G, list, Wout, dcnt, h_smem)
                : cudaLaunchKernelEx(&cfg, gmres_step_kernel<2, T, EST>, G, list, Wout, dcnt, h_smem);
}

template <class T>
cudaError_t launch_step_t(cudaStream_t st, const Gs &G, int P, int S, const int *list,
                          const double *Wout, const int *dcnt, int h_smem, size_t dyn) {
  switch (G.stop) {
    case 0: return launch_step_e<T, 0>(st, G, P, S, list, Wout, dcnt, h_smem, dyn);
    case 1: return launch_step_e<T, 1>(st, G, P, S, list, Wout, dcnt, h_smem, dyn);
    default: return launch_step_e<T, 2>(st, G, P, S, list, Wout, dcnt, h_smem, dyn);
  }
}

// Float32 copies of the dipoles for the float32-basis estimates.
__global__ void dip_to_f32_kernel(int n, const double *__restrict__ src, float *__restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

}  // namespace

cudaError_t launch_gmres_start(cudaStream_t st, const DevSystem &sys, GmresState &gs, int n,
                               const double *Bplanar) {
  if (n <= 0) return cudaSuccess;
  if (!gs.V && !gs.Vf) return cudaErrorInvalidValue;
  if (gs.Vf)
    gmres_start_kernel<float><<<n, NT, 0, st>>>(view(gs, sys), Bplanar);
  else
    gmres_start_kernel<double><<<n, NT, 0, st>>>(view(gs, sys), Bplanar);
  return cudaGetLastError();
}

cudaError_t launch_gmres_prepare(cudaStream_t st, const DevSystem &sys, GmresState &gs) {
  if (gs.dipf) {
    dip_to_f32_kernel<<<64, 256, 0, st>>>(3 * sys.n_prod, sys.dip, gs.dipf);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

cudaError_t launch_gmres_select(cudaStream_t st, GmresState &gs, int n, int split, int min_b) {
  gmres_select_kernel<<<1, 1024, 0, st>>>(gs.state, n, split, min_b, gs.act, gs.act2, gs.count);
  return cudaGetLastError();
}

cudaError_t launch_gmres_gather(cudaStream_t st, const DevSystem &sys, GmresState &gs,
                                const int *list, int S, double *Zc, double *slot_omega,
                                const int *dcnt) {
  if (S <= 0) return cudaSuccess;
  if (!gs.V && !gs.Vf) return cudaErrorInvalidValue;
  if (gs.Vf)
    gmres_gather_kernel<float><<<S, NT, 0, st>>>(view(gs, sys), list, Zc, slot_omega, dcnt);
  else
    gmres_gather_kernel<double><<<S, NT, 0, st>>>(view(gs, sys), list, Zc, slot_omega, dcnt);
  return cudaGetLastError();
}

cudaError_t launch_gmres_step(cudaStream_t st, const DevSystem &sys, GmresState &gs,
                              const int *list, int S, const double *Wout, const int *dcnt) {
  if (S <= 0) return cudaSuccess;
  if (S > 65535) return cudaErrorInvalidConfiguration;
  if (!gs.V && !gs.Vf) return cudaErrorInvalidValue;
  const Gs G = view(gs, sys);
  // Long vectors: a cluster of CTAs per right-hand side, so that the FP64
  // work of the orthogonalisation is spread over more SMs than there are
  // live right-hand sides.
  const int P = sys.n_prod >= 8192 ? 8 : (sys.n_prod >= 4096 ? 4 : (sys.n_prod >= 2048 ? 2 : 1));
  // the Hessenberg columns go to shared memory for the back substitution
  // when the restart length allows (m (m+1) complex values)
  const int h_smem = gs.m <= kHsmemMaxM ? 1 : 0;
  const size_t dyn = h_smem ? (size_t)gs.m * (gs.m + 1) * sizeof(double2) : 0;
  return gs.Vf ? launch_step_t<float>(st, G, P, S, list, Wout, dcnt, h_smem, dyn)
               : launch_step_t<double>(st, G, P, S, list, Wout, dcnt, h_smem, dyn);
}

cudaError_t launch_rhs_init(cudaStream_t st, const DevSystem &sys, int n, int g0,
                            const double *omega_all, double *Zc, double *slot_omega,
                            double *gs_omega, int *gs_dir) {
  if (n <= 0) return cudaSuccess;
  rhs_init_kernel<<<n, 256, 0, st>>>(n, g0, sys.n_prod, omega_all, sys.dip, Zc, slot_omega,
                                     gs_omega, gs_dir);
  return cudaGetLastError();
}

cudaError_t launch_gmres_guess(cudaStream_t st, const DevSystem &sys, GmresState &gs, int n, int g0,
                               const double *x0) {
  if (n <= 0) return cudaSuccess;
  gmres_guess_kernel<<<n, NT, 0, st>>>(view(gs, sys), g0, x0);
  return cudaGetLastError();
}

cudaError_t launch_gmres_export(cudaStream_t st, const DevSystem &sys, GmresState &gs, int n, int g0,
                                double *X) {
  if (n <= 0) return cudaSuccess;
  gmres_export_kernel<<<n, NT, 0, st>>>(view(gs, sys), g0, X);
  return cudaGetLastError();
}

cudaError_t launch_polarization(cudaStream_t st, const DevSystem &sys, GmresState &gs, int n,
                                int g0, double2 *P) {
  if (n <= 0) return cudaSuccess;
  polarization_kernel<<<n, NT, 0, st>>>(g0, sys.n_prod, sys.dip, gs.x, P);
  return cudaGetLastError();
}

}  // namespace tddft
