// Step 5 of the chi0 product (Table t:flops): on every orbital block
// k = (A, B) and for every real column c,
//   G[a][b] = sum_E Xo[A+a][E] gamma_c[B+b][E]   (+ gamma_c[A+a][E] Xo[B+b][E] if A != B)
//   n_c[mu] = sum_ab V_mu[a][b] G[a][b]            for the products mu of block k
//   Out[c][mu] = Zin[c][mu] - n_c[mu]  (A operator)  or  n_c[mu]  (chi0 only).
// One CTA handles one block and 16 columns; each thread owns a 4 x 4 (a, b)
// tile of one column, so every shared-memory operand feeds two FMAs per
// load, and each vertex block is read once for 16 columns in the dot phase.
// float64 throughout; gamma is laid out [n_orb][ncols][n_occ].
#include "internal.h"

namespace tddft {
namespace {

constexpr int BD_COLS = 16;

__global__ void __launch_bounds__(256, 2) block_dot_kernel(
    int ncols, int n_occ, int n_prod, int n_orb, const int *__restrict__ aoff,
    const int2 *__restrict__ blk_atoms, const int *__restrict__ blk_ptr,
    const int *__restrict__ blk_prod, const double *__restrict__ Vpad,
    const double *__restrict__ Xo, const double *__restrict__ gamma, const double *__restrict__ Zin, int subtract,
    double *__restrict__ Out, const int *__restrict__ dcnt) {
  using T = double;
  // E-slices of 8 keep the static shared memory < 48 KB
  constexpr int BD_E = 8;
  __shared__ T XA[BD_E][kMaxOrb + 1], XB[BD_E][kMaxOrb + 1];
  // gamma slices of the A and B rows, [2][BD_COLS][BD_E][kMaxOrb + 1], reused for G
  __shared__ T gbuf[2 * BD_COLS * BD_E * (kMaxOrb + 1)];
  // G is stored with rows of 17 (bank-conflict free): 16 columns x 16 x 17
  constexpr int GS = kMaxOrb * (kMaxOrb + 1);
  static_assert(2 * BD_COLS * BD_E * (kMaxOrb + 1) >= BD_COLS * GS, "G must fit in gbuf");
  auto gA = [&](int c, int e, int r) -> T & {
    return gbuf[(c * BD_E + e) * (kMaxOrb + 1) + r];
  };
  auto gB = [&](int c, int e, int r) -> T & {
    return gbuf[((BD_COLS + c) * BD_E + e) * (kMaxOrb + 1) + r];
  };
  const int k = blockIdx.x;
  const int c0 = blockIdx.y * BD_COLS;
  const int nact = dcnt ? min(ncols, 2 * *dcnt) : ncols;   // ncols: stride; nact: live
  if (c0 >= nact) return;
  const int t = threadIdx.x;
  const int cl = t >> 4;                  // column of this thread within the CTA
  const int a0 = ((t >> 2) & 3) * 4;      // 4 rows a
  const int b0 = (t & 3) * 4;             // 4 columns b
  const int2 AB = blk_atoms[k];
  const int aoA = aoff[AB.x], nA = aoff[AB.x + 1] - aoA;
  const int aoB = aoff[AB.y], nB = aoff[AB.y + 1] - aoB;
  const bool bilocal = AB.x != AB.y;
  T G[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) G[i][j] = T(0);

  for (int E0 = 0; E0 < n_occ; E0 += BD_E) {
    __syncthreads();
    for (int i = t; i < BD_E * kMaxOrb; i += 256) {
      const int e = i / kMaxOrb, r = i % kMaxOrb, E = E0 + e;
      XA[e][r] = (r < nA && E < n_occ) ? Xo[(int64_t)(aoA + r) * n_occ + E] : T(0);
      XB[e][r] = (r < nB && E < n_occ) ? Xo[(int64_t)(aoB + r) * n_occ + E] : T(0);
    }
    for (int i = t; i < BD_COLS * BD_E * kMaxOrb; i += 256) {
      // e fastest: contiguous in gamma
      const int c = i / (BD_E * kMaxOrb);
      const int rem = i % (BD_E * kMaxOrb);
      const int r = rem / BD_E, e = rem % BD_E;
      const int E = E0 + e, cc = c0 + c;
      T va = T(0), vb = T(0);
      if (cc < nact && E < n_occ) {
        if (r < nA) va = gamma[((int64_t)(aoA + r) * ncols + cc) * n_occ + E];
        if (r < nB) vb = gamma[((int64_t)(aoB + r) * ncols + cc) * n_occ + E];
      }
      gA(c, e, r) = va;
      gB(c, e, r) = vb;
    }
    __syncthreads();
#pragma unroll 4
    for (int e = 0; e < BD_E; ++e) {
      T xa[4], xb[4], ga[4], gb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        xa[i] = XA[e][a0 + i];
        xb[i] = XB[e][b0 + i];
        ga[i] = gA(cl, e, a0 + i);
        gb[i] = gB(cl, e, b0 + i);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          G[i][j] = fma(xa[i], gb[j], G[i][j]);
          if (bilocal) G[i][j] = fma(ga[i], xb[j], G[i][j]);
        }
    }
  }
  // G of all 16 columns to shared memory (reusing gbuf), then the block dots
  __syncthreads();
  T *Gs = gbuf;   // [BD_COLS][kMaxOrb][kMaxOrb + 1]
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) Gs[cl * GS + (a0 + i) * (kMaxOrb + 1) + b0 + j] = G[i][j];
  __syncthreads();
  const int warp = t >> 5, lane = t & 31;
  const int p0 = blk_ptr[k], p1 = blk_ptr[k + 1];
  for (int q = p0 + warp; q < p1; q += 8) {
    T part[BD_COLS];
#pragma unroll
    for (int c = 0; c < BD_COLS; ++c) part[c] = T(0);
    for (int i = lane; i < kBlk; i += 32) {
      const T v = Vpad[(int64_t)q * kBlk + i];
      const int gi = (i >> 4) * (kMaxOrb + 1) + (i & 15);
#pragma unroll
      for (int c = 0; c < BD_COLS; ++c) part[c] = fma(v, Gs[c * GS + gi], part[c]);
    }
#pragma unroll
    for (int c = 0; c < BD_COLS; ++c) {
      T v = part[c];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      part[c] = v;
    }
    const int mu = blk_prod[q];
    // lane c writes column c
    T mine = T(0);
#pragma unroll
    for (int c = 0; c < BD_COLS; ++c)
      if (lane == c) mine = part[c];
    if (lane < BD_COLS && c0 + lane < nact) {
      const int64_t o = (int64_t)(c0 + lane) * n_prod + mu;
      Out[o] = subtract ? Zin[o] - mine : mine;
    }
  }
}

}  // namespace

cudaError_t launch_block_dot(cudaStream_t st, int ncols, const DevSystem &sys,
                             const double *Vpad, const double *Xo, const double *gamma,
                             const double *Zin, int subtract, double *Out, const int *dcnt) {
  dim3 grid(sys.n_blocks, (ncols + BD_COLS - 1) / BD_COLS);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  block_dot_kernel<<<grid, 256, 0, st>>>(ncols, sys.n_occ, sys.n_prod, sys.n_orb, sys.aoff,
                                         sys.blk_atoms, sys.blk_ptr, sys.blk_prod, Vpad, Xo,
                                         gamma, Zin, subtract, Out, dcnt);
  return cudaGetLastError();
}

}  // namespace tddft
