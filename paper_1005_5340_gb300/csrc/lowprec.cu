// Reduced-precision application of A(omega) z = z - chi0(omega) (K z)
// (Sec. 4.1, chi0 . y by steps 1-5 of Table t:flops on the stored transition
// vertex) used for the inner GMRES iterations of the refinement forms.  Every
// product runs on the tensor cores in split bf16 (or, in the TF32 forms, in
// tf32; the same buffers hold Kp floats per row instead of the [hi | lo]
// planes) with float32 accumulation (gemm_tc.cu): K z, step 2 (per
// 16-orbital chunk in per-atom parts, alpha.cu), X_virt^T beta with the D(omega) epilogue,
// X_virt a into the per-atom Gcat rows, step 5 (per atom).
// Layouts (n = right-hand-side column, complex planes interleaved per
// occupied state):
//   Zb     [2S][2 KpK]          z split, row c = 2 s + p
//   Yt     [2S][n_prod]         K z
//   betaT  [2 S n_occ][2 Kp1]   beta^T split, row E nc + 2 s + p (E-major;
//                               nc = 2 x the live right-hand sides)
//   aT     [2 S n_occ][2 Kp2]   (D . X_virt^T beta)^T split
#include <cuda_bf16.h>

#include "internal.h"
#include "tc_ptx.h"

namespace tddft {
namespace {

int grid_for(int64_t total, int threads) {
  int64_t g = (total + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (int)(g < 1 ? 1 : g);
}

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

// dst[r][k] = hi(src[r, k]), dst[r][Kp + k] = lo(src[r, k]); zero for k >= cols.
// With tf32: dst is float [r][Kp], the value rounded to tf32 (same bytes per row).
__global__ void split_rows_kernel(const double *__restrict__ src, int64_t rs, int64_t cs, int rows,
                                  int cols, int Kp, void *__restrict__ dstv, bool tf32,
                                  const int *__restrict__ dcnt = nullptr, int mul_r = 0) {
  if (dcnt) rows = min(rows, mul_r * *dcnt);
  const int64_t total = (int64_t)rows * Kp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / Kp;
    const int k = (int)(i % Kp);
    double x = (k < cols) ? src[r * rs + (int64_t)k * cs] : 0.0;
    if (tf32) {
      ((float *)dstv)[i] = ptx::tf32_round((float)x);
      continue;
    }
    __nv_bfloat16 *dst = (__nv_bfloat16 *)dstv;
    const __nv_bfloat16 hi = __double2bfloat16(x);
    const __nv_bfloat16 lo = __double2bfloat16(x - (double)__bfloat162float(hi));
    dst[r * 2 * Kp + k] = hi;
    dst[r * 2 * Kp + Kp + k] = lo;
  }
}

__global__ void split_f32_pairs_kernel(const double *__restrict__ src, int n,
                                       float2 *__restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float hi = (float)src[i];
    dst[i] = make_float2(hi, (float)(src[i] - (double)hi));
  }
}

// dterm[s][F] = (hi, lo) of omega_s - e_F and of omega_s + e_F, e_F the
// energy of virtual state F (float64 differences, float pairs)
__global__ void dterm_kernel(int S, int n_virt, int n_occ, const double *__restrict__ energy,
                             const double *__restrict__ omega, float4 *__restrict__ dterm,
                             const int *__restrict__ dcnt) {
  if (dcnt) S = min(S, *dcnt);
  const int64_t total = (int64_t)S * n_virt;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(i / n_virt), F = (int)(i - (int64_t)s * n_virt);
    const double w = omega[s], e = energy[n_occ + F];
    const double am = w - e, ap = w + e;
    const float amh = (float)am, aph = (float)ap;
    dterm[i] = make_float4(amh, (float)(am - (double)amh), aph, (float)(ap - (double)aph));
  }
}

}  // namespace

cudaError_t lp_prepare_constants(cudaStream_t st, const DevSystem &sys, LpWork &lp) {
  const int g = 152 * 8;
  split_rows_kernel<<<g, 256, 0, st>>>(sys.K, sys.n_prod, 1, sys.n_prod, sys.n_prod, lp.KpK, lp.Ks,
                                       lp.tf32);
  split_rows_kernel<<<g, 256, 0, st>>>(sys.XvT, sys.n_orb, 1, sys.n_virt, sys.n_orb, lp.Kp1, lp.XvTs,
                                       lp.tf32);
  split_rows_kernel<<<g, 256, 0, st>>>(sys.Xv, sys.n_virt, 1, sys.n_orb, sys.n_virt, lp.Kp2, lp.Xvs,
                                       lp.tf32);
  split_f32_pairs_kernel<<<4, 256, 0, st>>>(sys.energy, sys.n_occ, lp.eocc2);
  const size_t rows = (size_t)2 * lp.slots * sys.n_occ;
  cudaMemsetAsync(lp.Zb, 0, (size_t)2 * lp.slots * 2 * lp.KpK * sizeof(__nv_bfloat16), st);
  cudaMemsetAsync(lp.betaT, 0, rows * 2 * lp.Kp1 * sizeof(__nv_bfloat16), st);
  cudaMemsetAsync(lp.aT, 0, rows * 2 * lp.Kp2 * sizeof(__nv_bfloat16), st);
  cudaMemsetAsync(lp.err, 0, sizeof(int), st);
  return cudaGetLastError();
}

cudaError_t lp_autotune(cudaStream_t st, const DevSystem &sys, LpWork &lp) {
  // The workspace holds zeros here; timing does not depend on the values.
  const int S = lp.slots, ncols = 2 * S;
  const int64_t N1 = (int64_t)ncols * sys.n_occ;
  if (N1 > INT32_MAX) return cudaErrorInvalidValue;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  auto time_one = [&](int which, int bn, float &ms) -> cudaError_t {
    TcEpilogue ep;
    cudaError_t r = cudaSuccess;
    float best = 1e30f;
    for (int rep = 0; rep < 5 && r == cudaSuccess; ++rep) {
      r = cudaEventRecord(a, st);
      if (which == 0) {
        ep.outF = lp.Yt;
        ep.ldo = sys.n_prod;
        ep.split_ok = 1;   // as in the operator: split K and clusters where they apply
        // the live count shrinks as right-hand sides converge: the full and
        // the half batch, back to back
        if (r == cudaSuccess)
          r = launch_gemm_tc(st, lp.opK, lp.opZ, sys.n_prod, ncols, kStoreF32, ep, lp.err, nullptr,
                             0, bn);
        if (r == cudaSuccess)
          r = launch_gemm_tc(st, lp.opK, lp.opZ, sys.n_prod, (ncols / 2 + 1) & ~1, kStoreF32, ep,
                             lp.err, nullptr, 0, bn);
      } else if (which == 1) {
        ep.outB = lp.aT;
        ep.ldo = 2 * (int64_t)lp.Kp2;
        ep.lo_off = lp.Kp2;
        ep.rows_out = lp.Kp2;
        ep.energy = sys.energy;
        ep.eocc2 = lp.eocc2;
        ep.dterm = lp.dterm;
        ep.omega = lp.omega;
        ep.eps = 0.01;
        ep.occ_value = sys.occ_value;
        ep.n_occ = sys.n_occ;
        if (r == cudaSuccess)
          r = launch_gemm_tc(st, lp.opXvT, lp.opBeta, sys.n_virt, (int)N1, kDscaleSplit, ep, lp.err,
                             nullptr, 0, bn);
      } else {
        const AlphaRoute &ar = *lp.ar;
        ep.outB = ar.gcat_q;
        ep.ldo = 2 * (int64_t)ar.kcat5;
        ep.lo_off = ar.kcat5;
        ep.n_occ = sys.n_occ;
        ep.aoff = sys.aoff;
        ep.orb_atom = ar.orb_atom;
        ep.xoff5 = ar.xoff5;
        if (r == cudaSuccess)
          r = launch_gemm_tc(st, lp.opXv, lp.opA, sys.n_orb, (int)N1, kGammaCatSplit, ep, lp.err,
                             nullptr, 0, bn);
      }
      if (r == cudaSuccess) r = cudaEventRecord(b, st);
      if (r == cudaSuccess) r = cudaEventSynchronize(b);
      float t = 0.f;
      if (r == cudaSuccess) r = cudaEventElapsedTime(&t, a, b);
      if (rep > 0) best = fminf(best, t);   // first launch is a warm-up
    }
    ms = best;
    return r;
  };
  dterm_kernel<<<grid_for((int64_t)S * sys.n_virt, 256), 256, 0, st>>>(
      S, sys.n_virt, sys.n_occ, sys.energy, lp.omega, lp.dterm, nullptr);
  int *pick[3] = {&lp.bnK, &lp.bn1, &lp.bn2};
  for (int which = 0; which < 3 && e == cudaSuccess; ++which) {
    float t128 = 0.f, t64 = 0.f, t256 = 0.f;
    e = time_one(which, 128, t128);
    if (e == cudaSuccess) e = time_one(which, 64, t64);
    if (e == cudaSuccess) e = time_one(which, 256, t256);
    if (e == cudaSuccess) {
      int bn = 128;
      float best = t128;
      if (t64 < best) { bn = 64; best = t64; }
      if (t256 < best) { bn = 256; best = t256; }
      *pick[which] = bn;
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  // the timing runs wrote the workspace; the pads of aT must be zero again
  if (e == cudaSuccess)
    e = cudaMemsetAsync(lp.aT, 0, (size_t)N1 * 2 * lp.Kp2 * sizeof(__nv_bfloat16), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(lp.err, 0, sizeof(int), st);
  return e;
}

cudaError_t launch_apply_operator_lp(cudaStream_t st, const DevSystem &sys, LpWork &lp, int S,
                                     OpMode mode, double eps, const double *Zin, double *Out) {
  if (S <= 0) return cudaSuccess;
  if (S > lp.slots || mode == kKernel) return cudaErrorInvalidValue;
  const int ncols = 2 * S;
  const int np = sys.n_prod;
  cudaError_t err;
  const int64_t N1 = (int64_t)ncols * sys.n_occ;
  if (N1 > INT32_MAX) return cudaErrorInvalidValue;
  TcEpilogue ep;
  if (mode == kA) {
    {
      Scope sc(lp.timer, st, kcLpSplit, 0.0);
      split_rows_kernel<<<grid_for((int64_t)ncols * lp.KpK, 256), 256, 0, st>>>(
          Zin, np, 1, ncols, np, lp.KpK, lp.Zb, lp.tf32, lp.dcnt, 2);
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    {
      Scope sc(lp.timer, st, kcTcK, 2.0 * ncols * (double)np * np);
      ep.outF = lp.Yt;
      ep.ldo = np;
      ep.split_ok = 1;
      err = launch_gemm_tc(st, lp.opK, lp.opZ, np, ncols, kStoreF32, ep, lp.err, lp.dcnt, 2,
                           lp.bnK);
      if (err != cudaSuccess) return err;
    }
  }
  if (!lp.ar) return cudaErrorInvalidValue;
  const AlphaRoute &ar = *lp.ar;
  // steps 1-2 on the stored transition vertex: gather v^nu per atom, then
  // beta^T per 16-orbital chunk, part by part, on the tensor cores
  {
    Scope sc(lp.timer, st, kcAlphaGather, 0.0);
    err = launch_alpha_gather_lp(st, ar, ncols, mode == kA ? (const void *)lp.Yt : Zin,
                                 mode != kA, np, lp.dcnt);
    if (err != cudaSuccess) return err;
  }
  {
    Scope sc(lp.timer, st, kcTcStep2, ncols * ar.flops2);
    TcEpilogue eb;
    eb.outB = lp.betaT;
    eb.ldo = 2 * (int64_t)lp.Kp1;
    eb.lo_off = lp.Kp1;
    eb.n_occ = sys.n_occ;
    eb.parts = ar.parts;
    err = launch_gemm_tc_grouped(st, ar.ycat, ar.a2, ar.tiles2p, ar.n_tiles2p, ncols,
                                 kBetaPartSplit, eb, lp.err, lp.dcnt, 2, 256);
    if (err != cudaSuccess) return err;
  }
  const double tflops = 2.0 * sys.n_virt * (double)sys.n_orb * (double)N1;
  {
    Scope sc(lp.timer, st, kcDterm, 0.0);
    dterm_kernel<<<grid_for((int64_t)S * sys.n_virt, 256), 256, 0, st>>>(
        S, sys.n_virt, sys.n_occ, sys.energy, lp.omega, lp.dterm, lp.dcnt);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  {
    Scope sc(lp.timer, st, kcTcT1, tflops);
    TcEpilogue e1;
    e1.outB = lp.aT;
    e1.ldo = 2 * (int64_t)lp.Kp2;
    e1.lo_off = lp.Kp2;
    e1.rows_out = lp.Kp2;
    e1.energy = sys.energy;
    e1.eocc2 = lp.eocc2;
    e1.dterm = lp.dterm;
    e1.omega = lp.omega;
    e1.eps = eps;
    e1.occ_value = sys.occ_value;
    e1.n_occ = sys.n_occ;
    err = launch_gemm_tc(st, lp.opXvT, lp.opBeta, sys.n_virt, (int)N1, kDscaleSplit, e1, lp.err,
                         lp.dcnt, 2 * sys.n_occ, lp.bn1);
    if (err != cudaSuccess) return err;
  }
  // gamma into the per-atom Gcat rows, then step 5 per atom and the sum
  // of each product's (one or two) partials
  {
    Scope sc(lp.timer, st, kcTcT2, tflops);
    TcEpilogue e2;
    e2.outB = ar.gcat_q;
    e2.ldo = 2 * (int64_t)ar.kcat5;
    e2.lo_off = ar.kcat5;
    e2.n_occ = sys.n_occ;
    e2.aoff = sys.aoff;
    e2.orb_atom = ar.orb_atom;
    e2.xoff5 = ar.xoff5;
    err = launch_gemm_tc(st, lp.opXv, lp.opA, sys.n_orb, (int)N1, kGammaCatSplit, e2, lp.err,
                         lp.dcnt, 2 * sys.n_occ, lp.bn2);
    if (err != cudaSuccess) return err;
  }
  {
    Scope sc(lp.timer, st, kcTcStep5, ncols * ar.flops5);
    TcEpilogue e5;
    e5.outF = ar.P2f;
    e5.ldo = ar.ldp;
    err = launch_gemm_tc_grouped(st, ar.a5, ar.gcat, ar.tiles5lp, ar.n_tiles5lp, ncols, kPartialF32,
                                 e5, lp.err, lp.dcnt, 2);
    if (err != cudaSuccess) return err;
  }
  {
    Scope sc(lp.timer, st, kcCombine, 0.0);
    err = launch_alpha_combine(st, ar, ncols, np, false, Zin, mode == kA ? 1 : 0, Out, lp.dcnt);
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

}  // namespace tddft
