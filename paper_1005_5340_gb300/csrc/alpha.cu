// Steps 1, 2 and 5 of the chi0 product (Table t:flops) on the stored
// transition vertex alpha_nu^{cE} = sum_d V_nu^{cd} X_d^E (step 1, formed
// once at create in float64), laid out as per-atom dense operands so that
// steps 2 and 5 are grouped tensor-core products (split bf16 in the
// reduced-precision operator, integer slices in the emulated float64 one):
//   step 2  beta^{cE} = sum_{nu in L_A} alpha_nu^{cE} v^nu        (c in atom A)
//   step 5  n_mu = sum_{B of mu} sum_{b in B, E} alpha_mu^{bE} gamma_b^E
// L_A: the products whose block (A, B) or (B, A) holds atom A.  For a
// bilocal product mu on (A, B) the vertex block V_mu^{ab} (a in A, b in B)
// gives alpha_mu^{aE} = sum_b V^{ab} X_b^E and alpha_mu^{bE} = sum_a V^{ab} X_a^E;
// a local product (A, A) has alpha_mu^{aE} = sum_{a'} V^{aa'} X_a'^E.
//
// The reduced-precision step 2 runs over 16-orbital chunks of the orbital
// axis: chunk k holds orbitals 16k .. 16k+15, split into parts, the runs of
// its orbitals on one atom (one to three parts for atoms of 13 orbitals).
// Its operand rows, per block of 16 occupied states, are ordered (c16, e):
// row ((k nEB + b) 16 + c16) 16 + e holds alpha^{cE} of orbital 16k + c16
// and occupied state E = 16b + e over the per-atom list L_A of that
// orbital's atom (zero past n_orb or n_occ).  The product of a tile (the
// right-hand-side columns as M, one chunk and one E block as the 256 N
// columns, c16-major in tensor memory) runs part by part: each part's MMAs
// cover its own columns with N = 16 x its orbitals and its own atom's K
// range, so no MMA work is spent on products outside an orbital's list.  The
// epilogue gathers, for each thread's E, the 16 orbitals of the chunk (16
// 4-column tensor-memory loads) and writes them as one whole 32-byte sector
// of a beta^T row per plane.  (A per-atom output segment of 13 orbitals is
// 26 bytes and fills no sector; its 2-byte stores made step 2 store bound.)
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "tc_ptx.h"

namespace tddft {
namespace {

int grid_for(int64_t total, int threads) {
  int64_t g = (total + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (int)(g < 1 ? 1 : g);
}

// One CTA per product (Vpad row q): every (side, c, E) of alpha_mu, written
// to the step-2 operand (row (ao_X n_occ + E n_X + c), column pos_X) and to
// the step-5 operand (row rowoff5_X + pos_X, column c n_occ + E).
__global__ void alpha_build_kernel(int n_prod, int n_occ, int K2max, int K5max,
                                   const int4 *__restrict__ pinfo, const int *__restrict__ aoff,
                                   const int *__restrict__ rowoff5, const double *__restrict__ Vpad,
                                   const double *__restrict__ Xo, double *__restrict__ a2,
                                   double *__restrict__ a5) {
  const int q = blockIdx.x;
  const int4 pi = pinfo[q];   // (A, B, pos in L_A, pos in L_B)
  const int A = pi.x, B = pi.y;
  const int aoA = aoff[A], nA = aoff[A + 1] - aoA;
  const int aoB = aoff[B], nB = aoff[B + 1] - aoB;
  const double *V = Vpad + (int64_t)q * kBlk;   // V[a][b] at a * 16 + b
  const int sides = (A == B) ? 1 : 2;
  const int per0 = nA * n_occ;
  const int total = per0 + (sides == 2 ? nB * n_occ : 0);
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int side = i < per0 ? 0 : 1;
    const int li = side ? i - per0 : i;
    const int X = side ? B : A, aoX = side ? aoB : aoA, nX = side ? nB : nA;
    const int pos = side ? pi.w : pi.z;
    const int c = li / n_occ, E = li - c * n_occ;
    double s = 0.0;
    if (side == 0) {
      // c in A: sum over d in B (= A for a local product) of V[c][d] X_d^E
      for (int d = 0; d < nB; ++d) s = fma(V[c * kMaxOrb + d], Xo[(int64_t)(aoB + d) * n_occ + E], s);
    } else {
      // c in B: sum over d in A of V[d][c] X_d^E
      for (int d = 0; d < nA; ++d) s = fma(V[d * kMaxOrb + c], Xo[(int64_t)(aoA + d) * n_occ + E], s);
    }
    a2[((int64_t)aoX * n_occ + (int64_t)E * nX + c) * K2max + pos] = s;
    a5[((int64_t)rowoff5[X] + pos) * K5max + (int64_t)c * n_occ + E] = s;
  }
}

// dst[r][k] = hi(src[r][k]), dst[r][Kp + k] = lo(src[r][k])   (rows of length Kp)
// With tf32: float dst[r][k] = src[r][k] rounded to tf32.
__global__ void split_dense_kernel(const double *__restrict__ src, int64_t rows, int Kp,
                                   void *__restrict__ dstv, bool tf32) {
  const int64_t total = rows * Kp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / Kp;
    const int k = (int)(i - r * Kp);
    const double x = src[i];
    if (tf32) {
      ((float *)dstv)[i] = ptx::tf32_round((float)x);
      continue;
    }
    __nv_bfloat16 *dst = (__nv_bfloat16 *)dstv;
    const __nv_bfloat16 hi = __double2bfloat16(x);
    dst[r * 2 * Kp + k] = hi;
    dst[r * 2 * Kp + Kp + k] = __double2bfloat16(x - (double)__bfloat162float(hi));
  }
}

// The part operand of the reduced-precision step 2: row r = ((k nEB + b) 16
// + c16) 16 + e holds the per-atom row of orbital o = 16k + c16 and occupied
// state E = 16b + e (the K2max columns of alpha over L_{A(o)}), zero past
// n_orb or n_occ; split bf16 [rows][2 K2max] or tf32 [rows][K2max].
__global__ void alpha_part_kernel(int64_t rows, int K2max, int n_occ, int n_orb, int nEB,
                                  const int *__restrict__ aoff, const int *__restrict__ orb_atom,
                                  const double *__restrict__ a2, void *__restrict__ dstv,
                                  bool tf32) {
  const int64_t total = rows * K2max;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / K2max;
    const int q = (int)(i - r * K2max);
    const int e = (int)(r & 15), c16 = (int)((r >> 4) & 15);
    const int64_t kb = r >> 8;   // k nEB + b
    const int k = (int)(kb / nEB), b = (int)(kb - (int64_t)k * nEB);
    const int o = 16 * k + c16, E = 16 * b + e;
    double x = 0.0;
    if (o < n_orb && E < n_occ) {
      const int A = orb_atom[o], aoA = aoff[A], nA = aoff[A + 1] - aoA;
      x = a2[((int64_t)aoA * n_occ + (int64_t)E * nA + (o - aoA)) * K2max + q];
    }
    if (tf32) {
      ((float *)dstv)[i] = ptx::tf32_round((float)x);
      continue;
    }
    __nv_bfloat16 *dst = (__nv_bfloat16 *)dstv;
    const __nv_bfloat16 hi = __double2bfloat16(x);
    dst[r * 2 * K2max + q] = hi;
    dst[r * 2 * K2max + K2max + q] = __double2bfloat16(x - (double)__bfloat162float(hi));
  }
}

// Ycat[c][k] = Y[c][lcat[k]] (0 where lcat[k] < 0), split bf16 (or tf32)
template <class T>
__global__ void gather_split_kernel(int ncols, int kcat, const int *__restrict__ lcat,
                                    const T *__restrict__ Y, int64_t ld,
                                    void *__restrict__ dstv, bool tf32, const int *dcnt) {
  if (dcnt) ncols = min(ncols, 2 * *dcnt);
  const int64_t total = (int64_t)ncols * kcat;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / kcat;
    const int k = (int)(i - c * kcat);
    const int mu = lcat[k];
    const float x = mu >= 0 ? (float)Y[c * ld + mu] : 0.f;
    if (tf32) {
      ((float *)dstv)[i] = ptx::tf32_round(x);
      continue;
    }
    __nv_bfloat16 *dst = (__nv_bfloat16 *)dstv;
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    dst[c * 2 * kcat + k] = hi;
    dst[c * 2 * kcat + kcat + k] = __float2bfloat16_rn(x - __bfloat162float(hi));
  }
}

template <class TP>
__global__ void combine_kernel(int ncols, int n_prod, const int2 *__restrict__ pos5,
                               const TP *__restrict__ P2, int ldp, const double *__restrict__ Zin,
                               int subtract, double *__restrict__ Out, const int *dcnt) {
  if (dcnt) ncols = min(ncols, 2 * *dcnt);
  const int64_t total = (int64_t)ncols * n_prod;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / n_prod;
    const int mu = (int)(i - c * n_prod);
    const int2 p = pos5[mu];
    double n = (double)P2[(int64_t)p.x * ldp + c];
    if (p.y >= 0) n += (double)P2[(int64_t)p.y * ldp + c];
    Out[i] = subtract ? Zin[i] - n : n;
  }
}

}  // namespace

cudaError_t alpha_setup(cudaStream_t st, const tddft_system *h, const DevSystem &sys,
                        AlphaRoute &ar, int slots, bool lp, bool emu, int slices,
                        std::vector<void *> &allocs) {
  const int na = sys.n_atoms, np = sys.n_prod, nocc = sys.n_occ, no = sys.n_orb;
  const int32_t *ao = h->atom_orb_offset;
  // lists L_A in increasing product order and each product's positions
  std::vector<std::vector<int>> L(na);
  std::vector<int4> pinfo_by_mu(np);
  for (int mu = 0; mu < np; ++mu) {
    const int A = h->prod_atoms[2 * mu], B = h->prod_atoms[2 * mu + 1];
    pinfo_by_mu[mu] = make_int4(A, B, (int)L[A].size(), -1);
    L[A].push_back(mu);
    if (B != A) {
      pinfo_by_mu[mu].w = (int)L[B].size();
      L[B].push_back(mu);
    }
  }
  std::vector<int> xoff2(na), rowoff5(na + 1, 0), xoff5(na);
  std::vector<int> lcat;
  int k2max = 0, k5max = 0, kcat5 = 0;
  for (int A = 0; A < na; ++A) {
    const int nA = ao[A + 1] - ao[A];
    xoff2[A] = (int)lcat.size();
    for (int mu : L[A]) lcat.push_back(mu);
    while (lcat.size() % 64) lcat.push_back(-1);
    k2max = std::max(k2max, (int)L[A].size());
    rowoff5[A + 1] = rowoff5[A] + (int)L[A].size();
    xoff5[A] = kcat5;
    kcat5 += round_up(nA * nocc, 64);
    k5max = std::max(k5max, nA * nocc);
  }
  ar.K2max = round_up(std::max(k2max, 1), 64);
  ar.K5max = round_up(std::max(k5max, 1), 64);
  ar.rows2 = (int64_t)no * nocc;
  ar.rows5 = rowoff5[na];
  ar.kcat2 = std::max((int)lcat.size(), 64);
  while ((int)lcat.size() < ar.kcat2) lcat.push_back(-1);
  ar.kcat5 = kcat5;
  ar.ldp = 2 * std::max(slots, 3);
  // tiles (128 rows of the per-atom operands), atom by atom
  std::vector<GTile> t2, t5, t5lp;   // t5lp: 256-row entries (two M blocks per tile)
  ar.flops2 = ar.flops5 = 0.0;
  for (int A = 0; A < na; ++A) {
    const int nA = ao[A + 1] - ao[A], K = (int)L[A].size();
    if (K == 0) continue;   // no product on A: beta of its orbitals stays zero
    const int rows = nA * nocc;
    for (int m = 0; m < rows; m += 128)
      t2.push_back(GTile{ao[A] * nocc + m, xoff2[A], (K + 63) / 64, std::min(128, rows - m), A,
                         0, 0, 0});
    for (int m = 0; m < K; m += 128)
      t5.push_back(GTile{rowoff5[A] + m, xoff5[A], (rows + 63) / 64, std::min(128, K - m), A, 0,
                         0, 0});
    for (int m = 0; m < K; m += 256)
      t5lp.push_back(GTile{rowoff5[A] + m, xoff5[A], (rows + 63) / 64, std::min(256, K - m), A, 0,
                           0, 0});
    ar.flops2 += 2.0 * rows * K;
    ar.flops5 += 2.0 * rows * K;
  }
  ar.n_tiles2 = (int)t2.size();
  ar.n_tiles5 = (int)t5.size();
  ar.n_tiles5lp = (int)t5lp.size();
  ar.max_nkb2 = ar.K2max / 64;
  ar.max_nkb5 = ar.K5max / 64;
  std::vector<int2> pos5(np);
  std::vector<int4> pinfo_q(np);   // by Vpad row (block order)
  for (int mu = 0; mu < np; ++mu) {
    const int4 p = pinfo_by_mu[mu];
    pos5[mu] = make_int2(rowoff5[p.x] + p.z, p.w >= 0 ? rowoff5[p.y] + p.w : -1);
  }
  std::vector<int> orb_atom(no);
  for (int A = 0; A < na; ++A)
    for (int a = ao[A]; a < ao[A + 1]; ++a) orb_atom[a] = A;
  // the parts of the 16-orbital chunks of the reduced-precision step 2
  // (runs of a chunk's orbitals on one atom; past n_orb, one zero part) and
  // its tiles, one per (chunk, block of 16 occupied states): bands of 16
  // chunks, the E blocks of a band run block by block across its chunks
  const int nch = (no + 15) / 16, nEB = (nocc + 15) / 16;
  std::vector<int4> parts;   // {c16 start | n << 8, atom, Ycat K offset, K blocks}
  std::vector<int> pptr(nch + 1, 0);
  std::vector<GTile> t2p;
  if (lp) {
    for (int k = 0; k < nch; ++k) {
      for (int c = 0; c < 16;) {
        const int o = 16 * k + c;
        const int A = o < no ? orb_atom[o] : -1;
        int n = 1;
        while (c + n < 16 && (16 * k + c + n < no ? orb_atom[16 * k + c + n] : -1) == A) ++n;
        // an atom without products, or the zero tail: one K block of zero
        // vertex rows, so that its columns are written (as zeros) too
        const int nkb = A >= 0 ? std::max(1, ((int)L[A].size() + 63) / 64) : 1;
        parts.push_back(make_int4(c | (n << 8), A, A >= 0 ? xoff2[A] : 0, nkb));
        c += n;
      }
      pptr[k + 1] = (int)parts.size();
    }
    ar.rows2p = (int64_t)nch * nEB * 256;
    constexpr int kBand = 16;
    for (int b0 = 0; b0 < nch; b0 += kBand)
      for (int b = 0; b < nEB; ++b)
        for (int k = b0; k < std::min(nch, b0 + kBand); ++k)
          t2p.push_back(GTile{(k * nEB + b) * 256, pptr[k], pptr[k + 1] - pptr[k],
                              std::min(16, nocc - 16 * b), k, 0, 0, 0});
    ar.n_tiles2p = (int)t2p.size();
  }

  cudaError_t e = cudaSuccess;
  auto up = [&](void **p, const void *src, size_t bytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(p, bytes + 16);
    if (e != cudaSuccess) return;
    allocs.push_back(*p);
    e = cudaMemcpy(*p, src, bytes, cudaMemcpyHostToDevice);
  };
  auto al = [&](void **p, size_t bytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(p, bytes + 16);
    if (e == cudaSuccess) allocs.push_back(*p);
  };
  if (ar.n_tiles2 == 0) {
    // no products at all: keep one empty tile list
    t2.push_back(GTile{0, 0, 0, 0, 0, 0, 0, 0});
    t5.push_back(GTile{0, 0, 0, 0, 0, 0, 0, 0});
    t5lp.push_back(GTile{0, 0, 0, 0, 0, 0, 0, 0});
  }
  up((void **)&ar.tiles2, t2.data(), t2.size() * sizeof(GTile));
  up((void **)&ar.tiles5, t5.data(), t5.size() * sizeof(GTile));
  if (lp) up((void **)&ar.tiles5lp, t5lp.data(), t5lp.size() * sizeof(GTile));
  up((void **)&ar.lcat, lcat.data(), lcat.size() * sizeof(int));
  up((void **)&ar.pos5, pos5.data(), pos5.size() * sizeof(int2));
  up((void **)&ar.xoff5, xoff5.data(), xoff5.size() * sizeof(int));
  up((void **)&ar.orb_atom, orb_atom.data(), orb_atom.size() * sizeof(int));
  if (lp) {
    up((void **)&ar.tiles2p, t2p.data(), t2p.size() * sizeof(GTile));
    up((void **)&ar.parts, parts.data(), parts.size() * sizeof(int4));
  }
  // product info in Vpad (block) order: blk_prod[q] = mu
  int *rowoff5_d = nullptr;
  int4 *pinfo_d = nullptr;
  std::vector<int> blk_prod(np);
  if (e == cudaSuccess) e = cudaMemcpy(blk_prod.data(), sys.blk_prod, np * sizeof(int),
                                       cudaMemcpyDeviceToHost);
  for (int q = 0; q < np; ++q) pinfo_q[q] = pinfo_by_mu[blk_prod[q]];
  up((void **)&rowoff5_d, rowoff5.data(), rowoff5.size() * sizeof(int));
  up((void **)&pinfo_d, pinfo_q.data(), pinfo_q.size() * sizeof(int4));
  // step 1 in float64 (temporary buffers)
  double *a2 = nullptr, *a5 = nullptr;
  const size_t n2 = (size_t)ar.rows2 * ar.K2max, n5 = (size_t)std::max(ar.rows5, 1) * ar.K5max;
  if (e == cudaSuccess) e = cudaMalloc(&a2, n2 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&a5, n5 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(a2, 0, n2 * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a5, 0, n5 * sizeof(double), st);
  if (e == cudaSuccess && np > 0) {
    alpha_build_kernel<<<np, 128, 0, st>>>(np, nocc, ar.K2max, ar.K5max, pinfo_d, sys.aoff,
                                           rowoff5_d, sys.Vpad, sys.Xo, a2, a5);
    e = cudaGetLastError();
  }
  const int64_t rows5 = std::max(ar.rows5, 1);
  const int64_t ncap = 2 * (int64_t)std::max(slots, 3);
  if (lp) {
    ar.lp = true;
    __nv_bfloat16 *q2 = nullptr, *q5 = nullptr, *qy = nullptr, *qg = nullptr;
    al((void **)&q2, (size_t)ar.rows2p * 2 * ar.K2max * sizeof(__nv_bfloat16));
    al((void **)&q5, n5 * 2 * sizeof(__nv_bfloat16));
    al((void **)&qy, (size_t)ncap * 2 * ar.kcat2 * sizeof(__nv_bfloat16));
    al((void **)&qg, (size_t)ncap * 2 * ar.kcat5 * sizeof(__nv_bfloat16));
    al((void **)&ar.P2f, (size_t)rows5 * ar.ldp * sizeof(float));
    if (e == cudaSuccess) {
      alpha_part_kernel<<<152 * 8, 256, 0, st>>>(ar.rows2p, ar.K2max, nocc, no, nEB, sys.aoff,
                                                 ar.orb_atom, a2, q2, ar.tf32);
      split_dense_kernel<<<152 * 8, 256, 0, st>>>(a5, rows5, ar.K5max, q5, ar.tf32);
      e = cudaGetLastError();
    }
    // Gcat pads (never written) must read as zero
    if (e == cudaSuccess)
      e = cudaMemsetAsync(qg, 0, (size_t)ncap * 2 * ar.kcat5 * sizeof(__nv_bfloat16), st);
    if (e == cudaSuccess) e = make_operand_map(ar.a2, q2, ar.rows2p, ar.K2max, 128, ar.tf32);
    if (e == cudaSuccess) e = make_operand_map(ar.a5, q5, rows5, ar.K5max, 128, ar.tf32);
    if (e == cudaSuccess) e = make_operand_map(ar.ycat, qy, ncap, ar.kcat2, 128, ar.tf32);
    if (e == cudaSuccess) e = make_operand_map(ar.gcat, qg, ncap, ar.kcat5, 128, ar.tf32);
    ar.ycat_q = qy;
    ar.gcat_q = qg;
  }
  if (emu) {
    ar.emu = true;
    __nv_bfloat16 *q2 = nullptr, *q5 = nullptr, *qy = nullptr, *qg = nullptr;
    int *ex = nullptr;
    const int s = slices;
    al((void **)&q2, n2 * s * sizeof(__nv_bfloat16));
    al((void **)&q5, n5 * s * sizeof(__nv_bfloat16));
    al((void **)&qy, (size_t)ncap * s * ar.kcat2 * sizeof(__nv_bfloat16));
    al((void **)&qg, (size_t)ncap * s * ar.kcat5 * sizeof(__nv_bfloat16));
    al((void **)&ex, (size_t)(ar.rows2 + rows5 + 2 * ncap) * sizeof(int));
    al((void **)&ar.gcat64, (size_t)ncap * ar.kcat5 * sizeof(double));
    al((void **)&ar.P2d, (size_t)rows5 * ar.ldp * sizeof(double));
    if (e == cudaSuccess) e = oz_operand(ar.oa2, q2, ex, ar.rows2, ar.K2max, s, 128);
    if (e == cudaSuccess) e = oz_operand(ar.oa5, q5, ex + ar.rows2, rows5, ar.K5max, s, 128);
    if (e == cudaSuccess)
      e = oz_operand(ar.oycat, qy, ex + ar.rows2 + rows5, ncap, ar.kcat2, s, 64);
    if (e == cudaSuccess)
      e = oz_operand(ar.ogcat, qg, ex + ar.rows2 + rows5 + ncap, ncap, ar.kcat5, s, 64);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(ar.gcat64, 0, (size_t)ncap * ar.kcat5 * sizeof(double), st);
    if (e == cudaSuccess) e = launch_oz_slice_rows(st, a2, ar.K2max, (int)ar.rows2, ar.K2max, ar.oa2);
    if (e == cudaSuccess) e = launch_oz_slice_rows(st, a5, ar.K5max, (int)rows5, ar.K5max, ar.oa5);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(a2);
  cudaFree(a5);
  return e;
}

cudaError_t launch_alpha_gather_lp(cudaStream_t st, const AlphaRoute &ar, int ncols, const void *Y,
                                   bool y_f64, int64_t ld, const int *dcnt) {
  const int g = grid_for((int64_t)ncols * ar.kcat2, 256);
  __nv_bfloat16 *dst = ar.ycat_q;
  if (y_f64)
    gather_split_kernel<double><<<g, 256, 0, st>>>(ncols, ar.kcat2, ar.lcat, (const double *)Y, ld,
                                                   dst, ar.tf32, dcnt);
  else
    gather_split_kernel<float><<<g, 256, 0, st>>>(ncols, ar.kcat2, ar.lcat, (const float *)Y, ld,
                                                  dst, ar.tf32, dcnt);
  return cudaGetLastError();
}

cudaError_t launch_alpha_combine(cudaStream_t st, const AlphaRoute &ar, int ncols, int n_prod,
                                 bool p_f64, const double *Zin, int subtract, double *Out,
                                 const int *dcnt) {
  const int g = grid_for((int64_t)ncols * n_prod, 256);
  if (p_f64)
    combine_kernel<double><<<g, 256, 0, st>>>(ncols, n_prod, ar.pos5, ar.P2d, ar.ldp, Zin,
                                              subtract, Out, dcnt);
  else
    combine_kernel<float><<<g, 256, 0, st>>>(ncols, n_prod, ar.pos5, ar.P2f, ar.ldp, Zin, subtract,
                                             Out, dcnt);
  return cudaGetLastError();
}

}  // namespace tddft
