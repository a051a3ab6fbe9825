// Tensor-core GEMM for the reduced-precision operator (sm_103a, tcgen05 +
// TMA + mbarrier, inline PTX).
//
//   C^T[n][m] = sum_k A[m][k] * B[n][k]          (both operands K-major bf16)
//
// Split-bf16 ("bf16x3"): every real operand x is stored as two bf16 planes
// x = hi + lo (+ O(2^-17 |x|)), each row laid out [hi | lo] with Kp columns
// per plane (Kp a multiple of 64, zero padded).  The product is accumulated
// in float32 in tensor memory as A_hi B_hi + A_hi B_lo + A_lo B_hi.
// TF32 (template flag TF): every operand row is Kp floats rounded to tf32,
// the same 4 bytes per K entry; a 64-deep K block is two 32-wide boxes of
// 128-byte rows, where split bf16 has the hi and lo boxes, and the product
// is one tcgen05 kind::tf32 MMA chain (8 MMAs of K = 8 per block, against 12
// of K = 16 for split bf16; the tf32 rate is half the bf16 rate).  The
// kernel is persistent (one CTA per SM over its share of the 128 x BN output
// tiles) and warp-specialised: a TMA producer, an MMA issuer and eight
// epilogue warps that drain one TMEM accumulator while the next tile is
// accumulated in the other.  Epilogues, fused per use (the split-bf16 next
// operands are written as tf32 floats in the TF32 form):
//     kStoreF32      plain float32 C^T
//     kDscaleSplit   the D(omega) scaling of eq. response-mat on (re, im)
//                    column pairs, written back as split bf16 for the next GEMM
//                    (E-major input columns, slot-major output rows)
//     kBetaPartSplit step 2 on the stored transition vertex (16-orbital
//                    chunks in per-atom parts, right-hand-side columns as M):
//                    beta^T, split bf16, one 32-byte run per thread and plane
//     kGammaCatSplit transform 2 into the per-atom Gcat rows, split bf16
//     kPartialF32    step 5 partial sums, float32
// Grouped products take a tile table (per-atom operands: A rows, B K offset
// and length per 128-row tile; for step 2, per (chunk, E block) entries and
// the chunks' parts).  Every mbarrier wait is bounded by a wall-clock
// limit; on expiry the CTA records an error code, stops issuing work, waits
// (bounded) for its copies in flight and still frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.h"
#include "tc_ptx.h"

namespace tddft {
namespace {
using namespace ptx;

constexpr int TC_BM = 128, TC_BK = 64;
constexpr int TC_EPI_WARPS = 8;                     // two per TMEM lane quadrant
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;   // producer, MMA issuer, epilogue
constexpr uint32_t TC_A_BYTES = TC_BM * TC_BK * 2;    // 16 KB per plane
constexpr int TC_EOCC_MAX = 1024;   // occupied energies staged in shared memory (D(omega) epilogue)
// The N tile (TMEM columns per accumulator, B box rows, MMA N) is a template
// parameter, 64, 128 or 256, chosen per product by the autotuner; wider tiles
// read fewer operand bytes per MMA from L2.  A stage holds
// both planes of the A and B tiles of one 64-deep K block.
template <int BN> struct TcShape {
  static constexpr uint32_t B_BYTES = BN * TC_BK * 2;
  static constexpr uint32_t STAGE_BYTES = 2 * TC_A_BYTES + 2 * B_BYTES;
  static constexpr int STAGES = BN == 64 ? 4 : (BN == 128 ? 3 : 2);
  static constexpr size_t SMEM = STAGES * STAGE_BYTES + 1024 + 256 + TC_EOCC_MAX * 8;
};
// Per epilogue: step 5 (kPartialF32) runs two M blocks per tile (M2): the
// tile's B (the atom's Gcat rows) is loaded once for 256 vertex rows, whose
// two A tiles share the stage; two accumulators per TMEM buffer (4 BN
// columns, so BN <= 128) and two stages.
template <int EPI, int BN> struct TcCfg {
  static constexpr bool M2 = EPI == kPartialF32;
  static constexpr uint32_t B_BYTES = TcShape<BN>::B_BYTES;
  static constexpr uint32_t STAGE_BYTES = (M2 ? 4 : 2) * TC_A_BYTES + 2 * B_BYTES;
  static constexpr int STAGES = M2 ? 2 : TcShape<BN>::STAGES;
  static constexpr int ACC = M2 ? 2 * BN : BN;                  // TMEM columns per buffer
  static constexpr int TCOLS = 2 * ACC > 512 ? 512 : 2 * ACC;   // allocated (M2 needs BN <= 128)
  static constexpr size_t SMEM = STAGES * STAGE_BYTES + 1024 + 256 + TC_EOCC_MAX * 8;
};

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__device__ __forceinline__ void store_split(__nv_bfloat16 *p, int64_t lo_off, float x) {
  __nv_bfloat16 h, l;
  split_bf16(x, h, l);
  p[0] = h;
  p[lo_off] = l;
}

// Row stride, in elements, of a next-GEMM operand written by an epilogue:
// ep.ldo counts bf16 elements of a split row ([hi | lo], 2 Kp); a TF32 row
// holds the same bytes as Kp floats, so its stride in floats is ep.ldo / 2.
template <bool TF>
__device__ __forceinline__ int64_t operand_ld(const TcEpilogue &ep) {
  return TF ? ep.ldo / 2 : ep.ldo;
}

// element idx of a next-GEMM operand: split bf16 (hi at idx, lo at idx +
// lo_off) or, in the TF32 form, one tf32-rounded float at idx (idx computed
// with operand_ld)
template <bool TF>
__device__ __forceinline__ void put_operand(void *base, int64_t idx, int64_t lo_off, float x) {
  if (TF)
    ((float *)base)[idx] = tf32_round(x);
  else
    store_split((__nv_bfloat16 *)base + idx, lo_off, x);
}

// One 16-column chunk of the epilogue: row m (local row lr of the tile),
// columns n0 + j0 .. n0 + j0 + 15, fused per use.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// kDscaleSplit: the (omega -+ e_F) terms of the chunk's first slot (loaded
// before the chunk's TMEM read) and the occupied energies (shared memory)
struct DscaleIn {
  float4 dt;
  const float2 *eocc;
};

template <int EPI, bool TF>
__device__ __forceinline__ void epilogue16(const float (&v)[16], int m, int lr, int rows_valid,
                                           int atom, int M, int N, int n0, int j0,
                                           const TcEpilogue &ep, const DscaleIn &di) {
  if (EPI == kStoreF32) {
    if (m < M) {
      if (ep.ksplit > 1) {
        // two K halves add into the zeroed output (0 + a + b: either order)
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + j0 + j;
          if (n < N) atomicAdd(ep.outF + (int64_t)n * ep.ldo + m, v[j]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + j0 + j;
          if (n < N) ep.outF[(int64_t)n * ep.ldo + m] = v[j];
        }
      }
    }
  } else if (EPI == kPartialF32) {
    // C layout, rows of the grouped operand
    if (lr < rows_valid) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = n0 + j0 + j;
        if (n < N) ep.outF[(int64_t)m * ep.ldo + n] = v[j];
      }
    }
  } else if (EPI == kBetaPartSplit) {
    // (written by the kernel's own epilogue loop)
  } else if (EPI == kGammaCatSplit) {
    // row m = orbital (atom B, b); column n = (s n_occ + E) 2 + p, j = 2 s + p:
    // Gcat[j][xoff5_B + b n_occ + E]
    if (m < M) {
      const int B = ep.orb_atom[m], b = m - ep.aoff[B];
      const int64_t xo = ep.xoff5[B] + (int64_t)b * ep.n_occ;
      const int pair0 = (n0 + j0) >> 1;
      if (ep.n_occ % 8 == 0 && n0 + j0 + 16 <= N) {
        // the 16 columns are E0 .. E0+7 of one slot, both planes: four
        // 16-byte stores (hi and lo of p = 0 and p = 1)
        const int sl = pair0 / ep.n_occ, E0 = pair0 - sl * ep.n_occ;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const int64_t at = (int64_t)(2 * sl + p) * operand_ld<TF>(ep) + xo + E0;
          if (TF) {
            // eight floats: two 16-byte stores
            float *dst = (float *)ep.outB + at;
            *(float4 *)dst = make_float4(tf32_round(v[p]), tf32_round(v[2 + p]),
                                         tf32_round(v[4 + p]), tf32_round(v[6 + p]));
            *(float4 *)(dst + 4) = make_float4(tf32_round(v[8 + p]), tf32_round(v[10 + p]),
                                               tf32_round(v[12 + p]), tf32_round(v[14 + p]));
          } else {
            __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) split_bf16(v[2 * e + p], h[e], l[e]);
            __nv_bfloat16 *dst = (__nv_bfloat16 *)ep.outB + at;
            *(uint4 *)dst = *(const uint4 *)h;
            *(uint4 *)(dst + ep.lo_off) = *(const uint4 *)l;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + j0 + j;
          if (n < N) {
            const int pair = n >> 1, p = n & 1;
            const int sl = pair / ep.n_occ, E = pair - sl * ep.n_occ;
            put_operand<TF>(ep.outB, (int64_t)(2 * sl + p) * operand_ld<TF>(ep) + xo + E, ep.lo_off,
                            v[j]);
          }
        }
      }
    }
  } else {
    // (re, im) pairs: columns n (even) and n+1 of the same (slot, E).
    // omega -+ Delta, Delta = e_F - e_E, cancel near a resonance: they are
    // formed as (omega -+ e_F) +- e_E from float (hi, lo) pairs, the
    // first precomputed in float64 per (slot, F); the rest of D in
    // float32 (its rounding, ~1e-7, is far below the split-bf16 error).
    // The B operand (beta^T) rows, the columns n here, are E-major:
    // n = (E hs + s) 2 + p for hs = N / (2 n_occ) live slots; the output
    // rows are slot-major, (s n_occ + E) 2 + p, the order transform 2 and
    // its Gcat epilogue take.
    if (m < ep.rows_out) {
      const bool live = m < M;
      const float ef = (float)ep.eps, e2 = ef * ef, occ = (float)ep.occ_value;
      const int hs = max(1, N / (2 * ep.n_occ));
      const int pair0 = (n0 + j0) >> 1;
      int E = pair0 / hs, sl = pair0 - E * hs;
      // (omega -+ e_F) of each pair's slot as float (hi, lo) pairs,
      // precomputed per (slot, F) for this product; the first is loaded
      // before the chunk's TMEM read
      float4 dt = di.dt;
      int dsl = sl;
#pragma unroll
      for (int j = 0; j < 16; j += 2) {
        const int n = n0 + j0 + j;
        if (n >= N) continue;
        float re = 0.f, im = 0.f;
        if (live) {
          if (sl != dsl) {
            dt = ep.dterm[(int64_t)sl * M + m];
            dsl = sl;
          }
          const float2 eE = di.eocc[E];
          const float xm = (dt.x + eE.x) + (dt.y + eE.y);
          const float xp = (dt.z - eE.x) + (dt.w - eE.y);
          const float im2 = rcp_approx(fmaf(xm, xm, e2)), ip2 = rcp_approx(fmaf(xp, xp, e2));
          const float dre = occ * (xm * im2 - xp * ip2);
          const float dim = occ * ef * (ip2 - im2);
          re = dre * v[j] - dim * v[j + 1];
          im = dre * v[j + 1] + dim * v[j];
        }
        const int64_t nout = ((int64_t)sl * ep.n_occ + E) * 2;
        put_operand<TF>(ep.outB, nout * operand_ld<TF>(ep) + m, ep.lo_off, re);
        put_operand<TF>(ep.outB, (nout + 1) * operand_ld<TF>(ep) + m, ep.lo_off, im);
        if (++sl == hs) {
          sl = 0;
          ++E;
        }
      }
    }
  }
}

// Persistent warp-specialised kernel: one CTA per SM walks its share of the
// output tiles (tile t = blockIdx.x + i gridDim.x).
//   warp 0 lane 0 : TMA producer; one ring stage holds the four planes
//                   (A_hi, A_lo, B_hi, B_lo) of a 64-deep K block
//   warp 1 lane 0 : tcgen05.mma issuer: A_hi B_hi + A_hi B_lo + A_lo B_hi
//                   (M=128, N=BN, K=16) into one of two TMEM accumulators
//   warps 2-9     : epilogue, TMEM -> registers -> global, two warps per
//                   TMEM lane quadrant (half of the columns each); draining
//                   tile i while the MMA warp fills tile i+1 in the other buffer
template <int EPI, int TC_BN, bool TF>
__global__ void __launch_bounds__(TC_THREADS, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const __grid_constant__ CUtensorMap mapB64,
                   const __grid_constant__ CUtensorMap mapB128, int M, int N, int KpA, int KpB,
                   TcEpilogue ep, int *err, const int *dcnt, int mul_n, const GTile *tiles,
                   int n_mtiles) {
  // graph replays: right-hand-side columns beyond the live count are
  // skipped (whole tiles); they are the M axis of step 2, else the N axis
  constexpr bool kPart = EPI == kBetaPartSplit;
  // the part-based step 2 is built for the 256-wide tile (16 c16 x 16 e)
  if (kPart && TC_BN != 256) return;
  if (dcnt) {
    const int live = (int)min((int64_t)(kPart ? M : N), (int64_t)mul_n * (*dcnt));
    if (kPart)
      M = live;
    else
      N = live;
  }
  // step 2: n_ntiles counts the M tiles of the columns, run fastest
  const int n_ntiles = kPart ? (M + TC_BM - 1) / TC_BM : (N + TC_BN - 1) / TC_BN;
  // the N tiles share the columns evenly (multiples of 16, at most TC_BN):
  // tiles of one M row block then run at the same pace, so the second one
  // finds the A tile (the large operand of the K product) still in L2
  const int tn = kPart ? TC_BN : min(TC_BN, ((N + n_ntiles - 1) / n_ntiles + 15) & ~15);
  const int ksplit = ep.ksplit;
  const int n_tiles = n_mtiles * n_ntiles * ksplit;
  if ((int)blockIdx.x >= n_tiles) return;
  constexpr bool kM2 = TcCfg<EPI, TC_BN>::M2;
  constexpr uint32_t SB = TcCfg<EPI, TC_BN>::STAGE_BYTES;
  constexpr int NS = TcCfg<EPI, TC_BN>::STAGES;
  constexpr uint32_t B_BYTES = TcCfg<EPI, TC_BN>::B_BYTES;
  constexpr int ACC = TcCfg<EPI, TC_BN>::ACC;
  constexpr int TCOLS = TcCfg<EPI, TC_BN>::TCOLS;
  // B tile offset in a stage (after the one or two A tiles, both planes)
  constexpr uint32_t B_OFF = (kM2 ? 4 : 2) * TC_A_BYTES;
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned stage ring (required by the 128-byte swizzle atoms)
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(smem + NS * SB);
  uint64_t *empty = full + NS;
  uint64_t *tfull = empty + NS;     // [2]
  uint64_t *tempty = tfull + 2;     // [2]
  uint64_t *drain = tempty + 2;     // completion of every MMA this CTA issued
  uint32_t *tslot = (uint32_t *)(drain + 1);
  __shared__ int abort_flag;
  const uint64_t lim = wait_limit(err);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // tile t: M tile fastest, then the K slice (split K), then the N tile of
  // tn columns (the small A of the transforms stays in L2 while each B tile
  // is read once); in a cluster launch (ep.ncl > 1) and in a grouped product
  // (per-atom A operands, the large operand of steps 2 and 5) the N tile is
  // fastest, so consecutive CTAs (in a cluster: one GPC, one L2 partition)
  // read the same A tile, which DRAM then supplies once;
  // xa / xb: K offsets (elements) of the A and B tiles within a plane
  // step 2 (kPart): the table runs over (chunk, E block) entries, the M
  // tiles of the columns fastest, so that DRAM supplies each B block once;
  // xa = the first part, nkb = the part count, rows_valid = the valid E,
  // n0 = the B row base of the entry
  auto tile_of = [&](int t, int &m0, int &xa, int &xb, int &nkb, int &rows_valid, int &atom,
                     int &n0) {
    if (kPart) {
      const GTile g = tiles[t / n_ntiles];
      m0 = (t % n_ntiles) * TC_BM;
      xa = g.xoff;
      xb = 0;
      nkb = g.nkb;
      rows_valid = g.rows;
      atom = g.atom;
      n0 = g.row0;
      return;
    }
    int mt, ks, nt;
    if (ep.ncl > 1 || tiles) {
      nt = t % n_ntiles;
      const int rest = t / n_ntiles;
      mt = rest % n_mtiles;
      ks = rest / n_mtiles;
    } else {
      mt = t % n_mtiles;
      const int rest = t / n_mtiles;
      ks = rest % ksplit;
      nt = rest / ksplit;
    }
    n0 = nt * tn;
    if (tiles) {
      const GTile g = tiles[mt];
      m0 = g.row0;
      xa = 0;
      xb = g.xoff;
      nkb = g.nkb;
      rows_valid = g.rows;
      atom = g.atom;
    } else {
      const int nkb_all = KpA / TC_BK;
      const int kb0 = ks * nkb_all / ksplit, kb1 = (ks + 1) * nkb_all / ksplit;
      m0 = mt * TC_BM;
      xa = kb0 * TC_BK;
      xb = kb0 * TC_BK;
      nkb = kb1 - kb0;
      rows_valid = min(TC_BM, M - m0);
      atom = -1;
    }
  };

  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], TC_EPI_WARPS);   // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      // producer
      int g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        int m0, xa, xoff, nkb, rv, at, n0;
        tile_of(t, m0, xa, xoff, nkb, rv, at, n0);
        // step 2: one K loop per part (its atom's Ycat segment, its B rows)
        const int nparts = kPart ? nkb : 1;
        for (int p = 0; p < nparts && ok; ++p) {
        int pxa = xa, pxb = xoff, prow = n0, pnkb = nkb, pncol = TC_BN;
        if (kPart) {
          const int4 pi = ep.parts[xa + p];
          pxa = pi.z;
          pxb = 0;
          prow = n0 + (pi.x & 255) * 16;
          pnkb = pi.w;
          pncol = (pi.x >> 8) * 16;
        }
        for (int kb = 0; kb < pnkb; ++kb, ++g) {
          const int s = g % NS;
          const uint32_t ph = (uint32_t)(g / NS) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, lim)) {
            atomicExch(err, 1);
            abort_flag = 1;
            ok = false;
            break;
          }
          if (*(volatile int *)&abort_flag) {
            ok = false;
            break;
          }
          uint8_t *st = smem + s * SB;
          // second box of each operand: the lo plane (split bf16) or the
          // upper 32 entries of the K block (TF32)
          const int secA = TF ? 32 : KpA, secB = TF ? 32 : KpB;
          // step 2: the smallest B box that holds the part's rows (64, 128 or
          // 256), whose bytes the stage then expects
          const CUtensorMap *mb = &mapB;
          uint32_t bbytes = B_BYTES;
          if (kPart && pncol <= 64) {
            mb = &mapB64;
            bbytes = 64 * TC_BK * 2;
          } else if (kPart && pncol <= 128) {
            mb = &mapB128;
            bbytes = 128 * TC_BK * 2;
          }
          mbar_expect_tx(&full[s], SB - 2 * (B_BYTES - bbytes));
          tma_load_2d(st, &mapA, &full[s], pxa + kb * TC_BK, m0);                      // A_hi / A_0
          tma_load_2d(st + TC_A_BYTES, &mapA, &full[s], secA + pxa + kb * TC_BK, m0);  // A_lo / A_1
          if (kM2) {   // the second M block's A tile
            tma_load_2d(st + 2 * TC_A_BYTES, &mapA, &full[s], pxa + kb * TC_BK, m0 + TC_BM);
            tma_load_2d(st + 3 * TC_A_BYTES, &mapA, &full[s], secA + pxa + kb * TC_BK,
                        m0 + TC_BM);
          }
          tma_load_2d(st + B_OFF, mb, &full[s], pxb + kb * TC_BK, prow);           // B_hi / B_0
          tma_load_2d(st + B_OFF + B_BYTES, mb, &full[s], secB + pxb + kb * TC_BK,
                      prow);                                                     // B_lo / B_1
        }
        }
      }
      // copies in flight: the last NS stages issued must land before exit
      for (int h = max(0, g - NS); h < g; ++h)
        mbar_wait(&full[h % NS], (uint32_t)(h / NS) & 1u);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      const uint32_t idesc = TF ? idesc_tf32(TC_BM, tn) : idesc_bf16(TC_BM, tn);
      const uint32_t base = smem_u32(smem);
      int g = 0, lt = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++lt) {
        int m0, xa, xoff, nkb, rv, at, n0;
        tile_of(t, m0, xa, xoff, nkb, rv, at, n0);
        const int buf = lt & 1, use = lt >> 1;
        if (use > 0) {
          // the epilogue has drained this buffer's previous tile
          if (!mbar_wait(&tempty[buf], (uint32_t)(use - 1) & 1u, lim)) {
            atomicExch(err, 2);
            abort_flag = 1;
            ok = false;
            break;
          }
          fence_after();
        }
        const uint32_t d0 = tmem + (uint32_t)(buf * ACC);
        // M2: the second M block (accumulator d + TC_BN) only where the
        // table entry has rows there
        const int nblk = (kM2 && rv > TC_BM) ? 2 : 1;
        // step 2: one K loop per part, into the part's own columns
        // (c16 start x 16, N = 16 x its orbitals) with its own descriptor
        const int nparts = kPart ? nkb : 1;
        for (int p = 0; p < nparts && ok; ++p) {
        int pnkb = nkb;
        uint32_t pidesc = idesc, d = d0;
        if (kPart) {
          const int4 pi = ep.parts[xa + p];
          const int ncol = (pi.x >> 8) * 16;
          pnkb = pi.w;
          d = d0 + (uint32_t)((pi.x & 255) * 16);
          pidesc = TF ? idesc_tf32(TC_BM, ncol) : idesc_bf16(TC_BM, ncol);
        }
        for (int kb = 0; kb < pnkb; ++kb, ++g) {
          const int s = g % NS;
          if (!mbar_wait(&full[s], (uint32_t)(g / NS) & 1u, lim)) {
            atomicExch(err, 2);
            abort_flag = 1;
            ok = false;
            break;
          }
          fence_after();
          const uint32_t bhi = base + (uint32_t)s * SB + B_OFF, blo = bhi + B_BYTES;
          for (int blk = 0; blk < nblk; ++blk) {
            const uint32_t ahi = base + (uint32_t)s * SB + (uint32_t)blk * 2 * TC_A_BYTES,
                           alo = ahi + TC_A_BYTES;
            const uint32_t db = d + (uint32_t)(blk * TC_BN);
            if (TF) {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const uint32_t a0 = h ? alo : ahi, b0 = h ? blo : bhi;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                  mma_tf32(db, desc_sw128(a0 + 32 * k), desc_sw128(b0 + 32 * k), pidesc,
                           (kb > 0 || h > 0 || k > 0) ? 1u : 0u);
              }
            } else {
#pragma unroll
              for (int k = 0; k < TC_BK / 16; ++k) {
                mma_bf16(db, desc_sw128(ahi + 32 * k), desc_sw128(bhi + 32 * k), pidesc,
                         (kb > 0 || k > 0) ? 1u : 0u);
                mma_bf16(db, desc_sw128(ahi + 32 * k), desc_sw128(blo + 32 * k), pidesc, 1u);
                mma_bf16(db, desc_sw128(alo + 32 * k), desc_sw128(bhi + 32 * k), pidesc, 1u);
              }
            }
          }
          mma_commit(&empty[s]);
        }
        }
        if (ok) mma_commit(&tfull[buf]);
      }
      // every MMA issued here (also after an abort) completes before the
      // tensor memory is freed
      mma_commit(drain);
      mbar_wait(drain, 0u);
    }
    __syncwarp();
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (rows of the tile)
    const int q = warp & 3;
    const int lr = q * 32 + lane;
    const float2 *eocc = ep.eocc2;
    if (EPI == kDscaleSplit && ep.n_occ <= TC_EOCC_MAX) {
      // the occupied energies to shared memory (the four epilogue warps)
      float2 *es = (float2 *)(tslot + 4);
      for (int i = threadIdx.x - 64; i < ep.n_occ; i += 32 * TC_EPI_WARPS) es[i] = ep.eocc2[i];
      asm volatile("bar.sync 1, %0;" ::"n"(32 * TC_EPI_WARPS) : "memory");
      eocc = es;
    }
    int lt = 0;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++lt) {
      int m0, xa, xoff, nkb, rows_valid, atom, n0;
      tile_of(t, m0, xa, xoff, nkb, rows_valid, atom, n0);
      const int buf = lt & 1, use = lt >> 1;
      bool have = mbar_wait(&tfull[buf], (uint32_t)use & 1u, lim);
      // tcgen05.ld is warp-collective: one decision per warp
      have = __all_sync(0xffffffffu, have && !*(volatile int *)&abort_flag);
      if (!have) {
        if (lane == 0) atomicExch(err, 3);
        abort_flag = 1;
        break;
      }
      fence_after();
      // the two warps of a lane quadrant take the two halves of the columns
      // (M2: the two M blocks, all columns each)
      const int blk = (kM2 && warp >= 6) ? 1 : 0;
      const int m = m0 + blk * TC_BM + lr;
      const int rv_blk = kM2 ? min(TC_BM, rows_valid - blk * TC_BM) : rows_valid;
      const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * ACC + blk * TC_BN);
      const int half = ((tn >> 4) + 1) / 2 * 16;
      const int j_lo = kM2 ? 0 : ((warp >= 6) ? half : 0);
      const int j_hi = kM2 ? tn : ((warp >= 6) ? tn : half);
      if (kPart) {
        // step 2: tensor-memory column c16 16 + e holds orbital 16 k + c16
        // (k = atom, the chunk) and occupied state E = 16 eb + e of column
        // m = m0 + lr; each warp of a lane quadrant takes 8 of the 16 e, four
        // at a time, and writes each E's 16 orbitals as one 32-byte run of
        // the beta^T row E M + m per plane (M: the live columns)
        const int eb = n0 / 256 - atom * ((ep.n_occ + 15) / 16);
        const int mm = m0 + lr;
#pragma unroll 1
        for (int r = 0; r < 2; ++r) {
          const int e0 = ((warp >= 6) ? 8 : 0) + 4 * r;
          float v[16][4];
          tmem_ld4x16(trow + (uint32_t)e0, v);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (mm >= M || e0 + e >= rows_valid) continue;
            const int64_t row = (int64_t)(16 * eb + e0 + e) * M + mm;
            const int64_t at = row * operand_ld<TF>(ep) + 16 * (int64_t)atom;
            if (TF) {
              float4 *dst = (float4 *)((float *)ep.outB + at);
#pragma unroll
              for (int c = 0; c < 4; ++c)
                dst[c] = make_float4(tf32_round(v[4 * c][e]), tf32_round(v[4 * c + 1][e]),
                                     tf32_round(v[4 * c + 2][e]), tf32_round(v[4 * c + 3][e]));
            } else {
              __align__(16) __nv_bfloat16 hh[16], ll[16];
#pragma unroll
              for (int c = 0; c < 16; ++c) split_bf16(v[c][e], hh[c], ll[c]);
              __nv_bfloat16 *dst = (__nv_bfloat16 *)ep.outB + at;
              *(uint4 *)dst = *(const uint4 *)hh;
              *(uint4 *)(dst + 8) = *(const uint4 *)(hh + 8);
              *(uint4 *)(dst + ep.lo_off) = *(const uint4 *)ll;
              *(uint4 *)(dst + ep.lo_off + 8) = *(const uint4 *)(ll + 8);
            }
          }
        }
      }
      for (int j0 = j_lo; j0 < j_hi && !kPart; j0 += 16) {
        DscaleIn di;
        di.eocc = eocc;
        if (EPI == kDscaleSplit) {
          const int hs = max(1, N / (2 * ep.n_occ));   // live slots (E-major columns)
          const int sl0 = ((n0 + j0) >> 1) % hs;
          di.dt = (m < M && n0 + j0 < N) ? ep.dterm[(int64_t)sl0 * M + m]
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float v[16];
        tmem_ld16(trow + (uint32_t)j0, v);
        epilogue16<EPI, TF>(v, m, lr, rv_blk, atom, M, N, n0, j0, ep, di);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TCOLS));
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}
}  // namespace

// Row-major bf16 matrix [rows][cols] as a TMA map with 128-byte swizzled
// boxes of 64 columns x box_rows rows.
cudaError_t encode_bf16_map(CUtensorMap *map, const void *base, int64_t rows, int64_t cols,
                            int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if (cols % TC_BK != 0 || ((uintptr_t)base & 15) != 0) return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t estr[2] = {1, 1};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Row-major float32 matrix [rows][cols] (cols a multiple of 64) with
// 128-byte swizzled boxes of 32 columns x box_rows rows (tf32 operands).
cudaError_t encode_f32_map(CUtensorMap *map, const void *base, int64_t rows, int64_t cols,
                           int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if (cols % TC_BK != 0 || ((uintptr_t)base & 15) != 0) return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
  cuuint32_t estr[2] = {1, 1};
  cuuint32_t box[2] = {32u, (cuuint32_t)box_rows};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// A 2-D operand of Kp entries per row (Kp a multiple of 64): split bf16
// [rows][2*Kp] ([hi | lo] planes, boxes of 64 x box_rows) or, with tf32,
// float32 [rows][Kp] (boxes of 32 x box_rows); the same bytes per row.
cudaError_t make_operand_map(TcOperand &op, const void *base, int64_t rows, int Kp, int box_rows,
                             bool tf32) {
  if (Kp % TC_BK != 0) return cudaErrorInvalidValue;
  auto enc = [&](CUtensorMap *m, int br) {
    return tf32 ? encode_f32_map(m, base, rows, (int64_t)Kp, br)
                : encode_bf16_map(m, base, rows, 2 * (int64_t)Kp, br);
  };
  // box_rows for the A role (128) or the 128-wide B tile; 64 and 256 for the other B tiles
  cudaError_t e = enc(&op.map, box_rows);
  if (e == cudaSuccess) e = enc(&op.map64, 64);
  if (e == cudaSuccess) e = enc(&op.map256, 256);
  if (e != cudaSuccess) return e;
  op.has64 = true;
  op.rows = rows;
  op.Kp = Kp;
  op.tf32 = tf32;
  return cudaSuccess;
}

namespace {
template <int EPI, int BN>
void set_attr() {
  // (two M blocks need BN <= 128; the other instances are never launched,
  // and a refused attribute would leave an error for the next check)
  if constexpr (TcCfg<EPI, BN>::M2 && BN > 128) return;
  cudaFuncSetAttribute(gemm_tc_kernel<EPI, BN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)TcCfg<EPI, BN>::SMEM);
  cudaFuncSetAttribute(gemm_tc_kernel<EPI, BN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)TcCfg<EPI, BN>::SMEM);
}

template <int BN>
void set_attr_all() {
  set_attr<kStoreF32, BN>();
  set_attr<kDscaleSplit, BN>();
  set_attr<kBetaPartSplit, BN>();
  set_attr<kGammaCatSplit, BN>();
  set_attr<kPartialF32, BN>();
}
}  // namespace

void tc_init_attributes() {
  static bool done = false;
  if (done) return;
  set_attr_all<128>();
  set_attr_all<64>();
  set_attr_all<256>();
  done = true;
}

namespace {
int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 1;
  }
  return n;
}

template <int EPI, int BN, bool TF>
cudaError_t launch_tc(cudaStream_t st, int grid, const CUtensorMap &mA, const CUtensorMap &mB,
                      const CUtensorMap &mB64, const CUtensorMap &mB128, int M, int N, int KpA,
                      int KpB, const TcEpilogue &ep, int *err, const int *dcnt, int mul_n,
                      const GTile *tiles, int n_mtiles) {
  if (ep.ncl <= 1) {
    gemm_tc_kernel<EPI, BN, TF><<<grid, TC_THREADS, TcCfg<EPI, BN>::SMEM, st>>>(
        mA, mB, mB64, mB128, M, N, KpA, KpB, ep, err, dcnt, mul_n, tiles, n_mtiles);
    return cudaGetLastError();
  }
  // clusters of ncl CTAs; the grid is at most the clusters that fit at once
  // (a persistent CTA that waited for a slot would run its tiles last)
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = TcCfg<EPI, BN>::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ep.ncl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  static int fit[5] = {0, 0, 0, 0, 0};   // co-resident clusters per cluster size
  if (ep.ncl > 4) return cudaErrorInvalidValue;
  if (fit[ep.ncl] == 0) {
    cfg.gridDim = dim3(ep.ncl * sm_count());
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, gemm_tc_kernel<EPI, BN, TF>, &cfg) != cudaSuccess ||
        n < 1)
      return cudaErrorInvalidConfiguration;
    fit[ep.ncl] = n;
  }
  cfg.gridDim = dim3(std::min(grid / ep.ncl, fit[ep.ncl]) * ep.ncl);
  return cudaLaunchKernelEx(&cfg, gemm_tc_kernel<EPI, BN, TF>, mA, mB, mB64, mB128, M, N, KpA, KpB,
                            ep, err, dcnt, mul_n, tiles, n_mtiles);
}

template <int BN, bool TF>
cudaError_t launch_tc_epi(cudaStream_t st, int epi, int M, int N, const CUtensorMap &mA,
                          const CUtensorMap &mB, const CUtensorMap &mB64, const CUtensorMap &mB128,
                          int KpA, int KpB, const TcEpilogue &ep, int *err,
                          const int *dcnt, int mul_n, const GTile *tiles, int n_mtiles) {
  // persistent: one CTA per SM at most, each walking its share of the tiles
  const int64_t n_tiles = epi == kBetaPartSplit
                              ? (int64_t)n_mtiles * ((M + TC_BM - 1) / TC_BM)
                              : (int64_t)n_mtiles * ((N + BN - 1) / BN) * ep.ksplit;
  const int grid = (int)std::min<int64_t>(n_tiles, sm_count());
  switch (epi) {
    case kStoreF32:
      return launch_tc<kStoreF32, BN, TF>(st, grid, mA, mB, mB64, mB128, M, N, KpA, KpB, ep, err,
                                    dcnt, mul_n, tiles, n_mtiles);
    case kDscaleSplit:
      return launch_tc<kDscaleSplit, BN, TF>(st, grid, mA, mB, mB64, mB128, M, N, KpA, KpB, ep, err,
                                    dcnt, mul_n, tiles, n_mtiles);
    case kBetaPartSplit:
      return launch_tc<kBetaPartSplit, BN, TF>(st, grid, mA, mB, mB64, mB128, M, N, KpA, KpB, ep,
                                               err, dcnt, mul_n, tiles, n_mtiles);
    case kGammaCatSplit:
      return launch_tc<kGammaCatSplit, BN, TF>(st, grid, mA, mB, mB64, mB128, M, N, KpA, KpB, ep,
                                               err, dcnt, mul_n, tiles, n_mtiles);
    case kPartialF32:
      return launch_tc<kPartialF32, BN, TF>(st, grid, mA, mB, mB64, mB128, M, N, KpA, KpB, ep, err,
                                    dcnt, mul_n, tiles, n_mtiles);
    default:
      return cudaErrorInvalidValue;
  }
}
// the N tile's B map and the operand format select the kernel
cudaError_t dispatch_bn(cudaStream_t st, int epi, int M, int N, const TcOperand &A,
                        const TcOperand &B, const TcEpilogue &e, int *err, const int *dcnt,
                        int mul_n, const GTile *tiles, int n_mtiles, int bn) {
  // (the 64- and 128-row B maps go along for step 2's per-part boxes)
  if (A.tf32) {
    if (bn == 64)
      return launch_tc_epi<64, true>(st, epi, M, N, A.map, B.map64, B.map64, B.map, A.Kp, B.Kp, e,
                                     err, dcnt, mul_n, tiles, n_mtiles);
    if (bn == 256)
      return launch_tc_epi<256, true>(st, epi, M, N, A.map, B.map256, B.map64, B.map, A.Kp, B.Kp,
                                      e, err, dcnt, mul_n, tiles, n_mtiles);
    return launch_tc_epi<128, true>(st, epi, M, N, A.map, B.map, B.map64, B.map, A.Kp, B.Kp, e,
                                    err, dcnt, mul_n, tiles, n_mtiles);
  }
  if (bn == 64)
    return launch_tc_epi<64, false>(st, epi, M, N, A.map, B.map64, B.map64, B.map, A.Kp, B.Kp, e,
                                    err, dcnt, mul_n, tiles, n_mtiles);
  if (bn == 256)
    return launch_tc_epi<256, false>(st, epi, M, N, A.map, B.map256, B.map64, B.map, A.Kp, B.Kp, e,
                                     err, dcnt, mul_n, tiles, n_mtiles);
  return launch_tc_epi<128, false>(st, epi, M, N, A.map, B.map, B.map64, B.map, A.Kp, B.Kp, e, err,
                                   dcnt, mul_n, tiles, n_mtiles);
}
}  // namespace

void tc_split_plan(int Kp, int M, int N, int bn, int *ksplit, int *ncl) {
  const int n_mtiles = (M + TC_BM - 1) / TC_BM;
  *ksplit = 1;
  *ncl = 1;
  if (Kp / TC_BK < 32) return;
  const int nnt = (N + bn - 1) / bn;
  // too few tiles for the SMs: two K halves, added into the zeroed output
  if ((int64_t)n_mtiles * nnt < 2 * (int64_t)sm_count()) *ksplit = 2;
  // a long shared A (the kernel matrix) and a few N tiles: one cluster per
  // M row block (and K half), so that A comes from DRAM once
  if (nnt >= 2 && nnt <= 4) *ncl = nnt;
}

cudaError_t launch_gemm_tc(cudaStream_t st, const TcOperand &A, const TcOperand &B, int M, int N,
                           int epi, const TcEpilogue &ep, int *err, const int *dcnt, int mul_n,
                           int bn) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (A.Kp != B.Kp || A.tf32 != B.tf32) return cudaErrorInvalidValue;
  tc_init_attributes();
  if (bn == 64 && !B.has64) return cudaErrorInvalidValue;
  const int n_mtiles = (M + TC_BM - 1) / TC_BM;
  TcEpilogue e = ep;
  e.ksplit = 1;
  if (epi == kStoreF32 && ep.split_ok) {
    tc_split_plan(A.Kp, M, N, bn, &e.ksplit, &e.ncl);
    if (e.ksplit > 1) {
      cudaError_t r = cudaMemsetAsync(ep.outF, 0, (size_t)N * ep.ldo * sizeof(float), st);
      if (r != cudaSuccess) return r;
    }
  }
  return dispatch_bn(st, epi, M, N, A, B, e, err, dcnt, mul_n, nullptr, n_mtiles, bn);
}

cudaError_t launch_gemm_tc_grouped(cudaStream_t st, const TcOperand &A, const TcOperand &B,
                                   const GTile *tiles, int n_tiles, int N, int epi,
                                   const TcEpilogue &ep, int *err, const int *dcnt, int mul_n,
                                   int bn) {
  if (n_tiles <= 0 || N <= 0) return cudaSuccess;
  tc_init_attributes();
  if (bn == 64 && !B.has64) return cudaErrorInvalidValue;
  if (A.tf32 != B.tf32) return cudaErrorInvalidValue;
  // two M blocks need 4 bn TMEM columns; the part-based step 2 needs 16 x 16
  if (epi == kPartialF32 && bn > 128) return cudaErrorInvalidValue;
  if (epi == kBetaPartSplit && bn != 256) return cudaErrorInvalidValue;
  TcEpilogue e = ep;
  e.ksplit = 1;
  // step 2: the N columns of the launch are the M axis (rows of A = Ycat)
  return dispatch_bn(st, epi, epi == kBetaPartSplit ? N : 0, N, A, B, e, err, dcnt, mul_n, tiles,
                     n_tiles, bn);
}

}  // namespace tddft

// ---------------------------------------------------------------------------
// Self-test of the split-bf16 tensor-core GEMM against a float64 product on
// the same deterministic operands (entries uniform in [-1, 1) from a hash of
// the index and the seed).
// ---------------------------------------------------------------------------
namespace tddft {
namespace {
__device__ __forceinline__ double hash_uniform(uint64_t i, uint64_t seed) {
  uint64_t z = i * 0x9E3779B97F4A7C15ull + seed * 0xD1B54A32D192ED03ull + 0x632BE59BD9B4E019ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}
__global__ void st_fill_split(int rows, int K, int Kp, uint64_t seed, double *full,
                              __nv_bfloat16 *split, bool tf32) {
  const int64_t total = (int64_t)rows * Kp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / Kp;
    const int k = (int)(i % Kp);
    const double x = (k < K) ? hash_uniform((uint64_t)(r * K + k), seed) : 0.0;
    if (k < K) full[r * K + k] = x;
    if (tf32) {
      ((float *)split)[i] = ptx::tf32_round((float)x);
      continue;
    }
    const __nv_bfloat16 hi = __double2bfloat16(x);
    split[r * 2 * Kp + k] = hi;
    split[r * 2 * Kp + Kp + k] = __double2bfloat16(x - (double)__bfloat162float(hi));
  }
}
__global__ void st_ref(int M, int N, int K, const double *A, const double *B, const float *C,
                       double *err2) {
  // err2[0] = max |C - ref|, err2[1] = max |ref| (as ordered bit patterns of non-negative doubles)
  const int64_t total = (int64_t)M * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(i / M), m = (int)(i % M);
    double acc = 0.0;
    for (int k = 0; k < K; ++k) acc = fma(A[(int64_t)m * K + k], B[(int64_t)n * K + k], acc);
    double d = fabs((double)C[(int64_t)n * M + m] - acc);
    if (!(d == d)) d = 1e300;   // an unwritten (NaN) entry is a failure
    atomicMax((unsigned long long *)&err2[0], __double_as_longlong(d));
    atomicMax((unsigned long long *)&err2[1], __double_as_longlong(fabs(acc)));
  }
}
}  // namespace
}  // namespace tddft

namespace {
tddft_status selftest_gemm(int32_t M, int32_t N, int32_t K, uint64_t seed, double *max_rel_err,
                           bool tf32) {
  using namespace tddft;
  if (M < 1 || N < 1 || K < 1 || !max_rel_err) return TDDFT_ERR_INVALID_ARG;
  const int Kp = round_up(K, 64);
  double *A = nullptr, *B = nullptr, *e2 = nullptr;
  __nv_bfloat16 *As = nullptr, *Bs = nullptr;
  float *C = nullptr;
  int *err = nullptr;
  tddft_status status = TDDFT_OK;
  cudaError_t e = cudaMalloc(&A, (size_t)M * K * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&B, (size_t)N * K * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&As, (size_t)M * 2 * Kp * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&Bs, (size_t)N * 2 * Kp * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&C, (size_t)N * M * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&e2, 2 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&err, ptx::kErrInts * sizeof(int));
  TcOperand *opA = new TcOperand(), *opB = new TcOperand();
  if (e == cudaSuccess) {
    cudaMemset(e2, 0, 2 * sizeof(double));
    cudaMemset(err, 0, ptx::kErrInts * sizeof(int));
    st_fill_split<<<304, 256>>>(M, K, Kp, seed, A, As, tf32);
    st_fill_split<<<304, 256>>>(N, K, Kp, seed + 1, B, Bs, tf32);
    e = make_operand_map(*opA, As, M, Kp, 128, tf32);
    if (e == cudaSuccess) e = make_operand_map(*opB, Bs, N, Kp, 128, tf32);
  }
  // both N-tile widths, each checked against the float64 product
  for (int bn : {128, 64, 256}) {
    if (e == cudaSuccess) {
      cudaMemset(C, 0xFF, (size_t)N * M * sizeof(float));   // NaN: unwritten entries fail
      TcEpilogue ep;
      ep.outF = C;
      ep.ldo = M;
      e = launch_gemm_tc(0, *opA, *opB, M, N, kStoreF32, ep, err, nullptr, 0, bn);
    }
    if (e == cudaSuccess) {
      st_ref<<<304, 256>>>(M, N, K, A, B, C, e2);
      e = cudaDeviceSynchronize();
    }
  }
  if (e == cudaSuccess) {
    double h[2];
    int herr = 0;
    cudaMemcpy(h, e2, sizeof(h), cudaMemcpyDeviceToHost);
    cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    *max_rel_err = h[1] > 0 ? h[0] / h[1] : h[0];
    if (herr) status = TDDFT_ERR_TIMEOUT;
  } else {
    status = TDDFT_ERR_CUDA;
  }
  delete opA;
  delete opB;
  cudaFree(A); cudaFree(B); cudaFree(As); cudaFree(Bs); cudaFree(C); cudaFree(e2); cudaFree(err);
  return status;
}
}  // namespace

extern "C" tddft_status tddft_selftest_gemm(int32_t M, int32_t N, int32_t K, uint64_t seed,
                                            double *max_rel_err) {
  return selftest_gemm(M, N, K, seed, max_rel_err, false);
}

extern "C" tddft_status tddft_selftest_gemm_tf32(int32_t M, int32_t N, int32_t K, uint64_t seed,
                                                 double *max_rel_err) {
  return selftest_gemm(M, N, K, seed, max_rel_err, true);
}
