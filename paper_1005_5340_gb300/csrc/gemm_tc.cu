// Tensor-core GEMM for the reduced-precision operator (sm_103a, tcgen05 +
// TMA + mbarrier, inline PTX).
//
//   C^T[n][m] = sum_k A[m][k] * B[n][k]          (both operands K-major bf16)
//
// Split-bf16 ("bf16x3"): every real operand x is stored as two bf16 planes
// x = hi + lo (+ O(2^-17 |x|)), each row laid out [hi | lo] with Kp columns
// per plane (Kp a multiple of 64, zero padded).  The product is accumulated
// in float32 in tensor memory over three segments,
//   A_hi B_hi + A_hi B_lo + A_lo B_hi ,
// i.e. segment g reads A plane aseg[g] and B plane bseg[g].  One launch
// computes a 128 x 128 tile of C^T per CTA:
//   warp 0 lane 0 : TMA producer (3-stage ring of 64-deep K slices, SW128)
//   warp 1 lane 0 : issues tcgen05.mma (M=128, N=128, K=16) into TMEM
//   warps 0-3     : epilogue, TMEM -> registers -> global, fused per use:
//     kStoreF32    plain float32 C^T
//     kDscaleSplit the D(omega) scaling of eq. response-mat on (re, im)
//                  column pairs, written back as split bf16 for the next GEMM
// Every mbarrier wait is bounded by a wall-clock limit; on expiry the CTA
// records an error code, stops issuing work and still frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.h"
#include "tc_ptx.h"

namespace tddft {
namespace {
using namespace ptx;

constexpr int TC_BM = 128, TC_BK = 64, TC_STAGES = 3;
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_A_BYTES = TC_BM * TC_BK * 2;    // 16 KB
// The N tile (TMEM columns, B box rows, MMA N) is a template parameter: 128
// (2 CTAs per SM) or 64 (3 CTAs per SM), chosen per product by the autotuner.
template <int BN> struct TcShape {
  static constexpr uint32_t B_BYTES = BN * TC_BK * 2;
  static constexpr uint32_t STAGE_BYTES = TC_A_BYTES + B_BYTES;
  static constexpr size_t SMEM = TC_STAGES * STAGE_BYTES + 1024 + 256;
  static constexpr int MIN_CTAS = BN == 64 ? 3 : 2;
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

template <int EPI, int TC_BN>
__global__ void __launch_bounds__(TC_THREADS, TcShape<TC_BN>::MIN_CTAS)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   int M, int N, int KpA, int KpB, int nseg, int4 segs, TcEpilogue ep, int *err,
                   const int *dcnt, int mul_n, const GTile *tiles) {
  // graph replays: columns beyond the live count are skipped (whole CTAs)
  if (dcnt) N = (int)min((int64_t)N, (int64_t)mul_n * (*dcnt));
  if ((int)blockIdx.y * TC_BN >= N) return;
  // this CTA's rows of A and K range of B (grouped products: from the tile table)
  int m0, xoff, nkb, rows_valid, atom;
  if (tiles) {
    const GTile t = tiles[blockIdx.x];
    m0 = t.row0;
    xoff = t.xoff;
    nkb = t.nkb;
    rows_valid = t.rows;
    atom = t.atom;
  } else {
    m0 = blockIdx.x * TC_BM;
    xoff = 0;
    nkb = KpA / TC_BK;
    rows_valid = min(TC_BM, M - m0);
    atom = -1;
  }
  constexpr uint32_t TC_STAGE_BYTES = TcShape<TC_BN>::STAGE_BYTES;
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned stage ring (required by the 128-byte swizzle atoms)
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(smem + TC_STAGES * TC_STAGE_BYTES);
  uint64_t *empty = full + TC_STAGES;
  uint64_t *tfull = empty + TC_STAGES;
  uint32_t *tslot = (uint32_t *)(tfull + 1);
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.y * TC_BN;
  const int total = nseg * nkb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(TC_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // producer
    for (int it = 0; it < total; ++it) {
      const int s = it % TC_STAGES;
      const uint32_t ph = (uint32_t)(it / TC_STAGES) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u)) {
        atomicExch(err, 1);
        abort_flag = 1;
        break;
      }
      if (*(volatile int *)&abort_flag) break;
      const int g = it / nkb, kb = it % nkb;
      const int ka = ((g == 0) ? segs.x : (g == 1) ? segs.y : segs.z) & 0xFF;
      const int kbp = (((g == 0) ? segs.x : (g == 1) ? segs.y : segs.z) >> 8) & 0xFF;
      uint8_t *sa = smem + s * TC_STAGE_BYTES;
      uint8_t *sb = sa + TC_A_BYTES;
      mbar_expect_tx(&full[s], TC_STAGE_BYTES);
      tma_load_2d(sa, &mapA, &full[s], ka * KpA + kb * TC_BK, m0);
      tma_load_2d(sb, &mapB, &full[s], kbp * KpB + xoff + kb * TC_BK, n0);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = idesc_bf16(TC_BM, TC_BN);
    bool ok = true;
    for (int it = 0; it < total; ++it) {
      const int s = it % TC_STAGES;
      const uint32_t ph = (uint32_t)(it / TC_STAGES) & 1u;
      if (!mbar_wait(&full[s], ph)) {
        atomicExch(err, 2);
        abort_flag = 1;
        ok = false;
        break;
      }
      fence_after();
      const uint32_t sa = smem_u32(smem + s * TC_STAGE_BYTES);
      const uint32_t sb = sa + TC_A_BYTES;
#pragma unroll
      for (int k = 0; k < TC_BK / 16; ++k)
        mma_bf16(tmem, desc_sw128(sa + 32 * k), desc_sw128(sb + 32 * k), idesc,
                 (it > 0 || k > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    if (ok) mma_commit(tfull);
  }
  __syncwarp();

  // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w+31
  bool have = mbar_wait(tfull, 0);
  if (!have) atomicExch(err, 3);
  fence_after();
  // tcgen05.ld is warp-collective: take the decision once per warp
  have = __all_sync(0xffffffffu, have && !*(volatile int *)&abort_flag);
  const int lr = warp * 32 + lane;
  const int m = m0 + lr;
  if (have) {
    for (int j0 = 0; j0 < TC_BN; j0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j0, v);
      if (EPI == kStoreF32) {
        if (m < M) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = n0 + j0 + j;
            if (n < N) ep.outF[(int64_t)n * ep.ldo + m] = v[j];
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
      } else if (EPI == kBetaTSplit) {
        // row m = (atom A, E, c) of the step-2 operand; column n = 2 s + p:
        // beta^T row (s n_occ + E) 2 + p, column ao_A + c
        if (lr < rows_valid) {
          const int aoA = ep.aoff[atom], nA = ep.aoff[atom + 1] - aoA;
          const int r = m - aoA * ep.n_occ, E = r / nA, c = r - E * nA;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = n0 + j0 + j;
            if (n < N) {
              const int64_t row = ((int64_t)(n >> 1) * ep.n_occ + E) * 2 + (n & 1);
              store_split(ep.outB + row * ep.ldo + aoA + c, ep.lo_off, v[j]);
            }
          }
        }
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
              __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) split_bf16(v[2 * e + p], h[e], l[e]);
              __nv_bfloat16 *dst = ep.outB + (int64_t)(2 * sl + p) * ep.ldo + xo + E0;
              *(uint4 *)dst = *(const uint4 *)h;
              *(uint4 *)(dst + ep.lo_off) = *(const uint4 *)l;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int n = n0 + j0 + j;
              if (n < N) {
                const int pair = n >> 1, p = n & 1;
                const int sl = pair / ep.n_occ, E = pair - sl * ep.n_occ;
                store_split(ep.outB + (int64_t)(2 * sl + p) * ep.ldo + xo + E, ep.lo_off, v[j]);
              }
            }
          }
        }
      } else {
        // (re, im) pairs: columns n (even) and n+1 of the same (slot, E).
        // omega -+ Delta, Delta = e_F - e_E, cancel near a resonance: they are
        // formed as (omega -+ e_F) +- e_E from float (hi, lo) pairs, the
        // first once per slot in float64; the rest of D in float32 (its
        // rounding, ~1e-7, is far below the split-bf16 error).
        if (m < ep.rows_out) {
          const bool live = m < M;
          const float ef = (float)ep.eps, e2 = ef * ef, occ = (float)ep.occ_value;
          const int pair0 = (n0 + j0) >> 1;
          const int sl0 = pair0 / ep.n_occ, E0 = pair0 - sl0 * ep.n_occ;
          // (omega -+ e_F) of the chunk's slot, once (the usual case: all 8
          // pairs in one slot); otherwise per pair, with identical arithmetic
          // so that no result depends on a right-hand side's slot
          float am_hi = 0.f, am_lo = 0.f, ap_hi = 0.f, ap_lo = 0.f;
          const bool one_slot = E0 + 8 <= ep.n_occ;
          double eF = 0.0;
          if (live) {
            eF = ep.energy[ep.n_occ + m];
            if (one_slot) {
              const double w = ep.omega[sl0];
              const double am = w - eF, ap = w + eF;
              am_hi = (float)am;
              am_lo = (float)(am - (double)am_hi);
              ap_hi = (float)ap;
              ap_lo = (float)(ap - (double)ap_hi);
            }
          }
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const int n = n0 + j0 + j;
            if (n >= N) continue;
            float re = 0.f, im = 0.f;
            if (live) {
              float xm, xp;
              if (one_slot) {
                const float2 eE = ep.eocc2[E0 + (j >> 1)];
                xm = (am_hi + eE.x) + (am_lo + eE.y);
                xp = (ap_hi - eE.x) + (ap_lo - eE.y);
              } else {
                // the same arithmetic with this pair's slot (chunks that cross a slot)
                const int pair = n >> 1;
                const int sl = pair / ep.n_occ, E = pair - sl * ep.n_occ;
                const double w = ep.omega[sl];
                const double am = w - eF, ap = w + eF;
                const float bm_hi = (float)am, bm_lo = (float)(am - (double)bm_hi);
                const float bp_hi = (float)ap, bp_lo = (float)(ap - (double)bp_hi);
                const float2 eE = ep.eocc2[E];
                xm = (bm_hi + eE.x) + (bm_lo + eE.y);
                xp = (bp_hi - eE.x) + (bp_lo - eE.y);
              }
              const float im2 = __frcp_rn(fmaf(xm, xm, e2)), ip2 = __frcp_rn(fmaf(xp, xp, e2));
              const float dre = occ * (xm * im2 - xp * ip2);
              const float dim = occ * ef * (ip2 - im2);
              re = dre * v[j] - dim * v[j + 1];
              im = dre * v[j + 1] + dim * v[j];
            }
            __nv_bfloat16 h, l;
            split_bf16(re, h, l);
            ep.outB[(int64_t)n * ep.ldo + m] = h;
            ep.outB[(int64_t)n * ep.ldo + ep.lo_off + m] = l;
            split_bf16(im, h, l);
            ep.outB[(int64_t)(n + 1) * ep.ldo + m] = h;
            ep.outB[(int64_t)(n + 1) * ep.ldo + ep.lo_off + m] = l;
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN));
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

// A 2-D bf16 operand [rows][2*Kp] ([hi | lo] planes), boxes of 64 x box_rows.
cudaError_t make_operand_map(TcOperand &op, const void *base, int64_t rows, int Kp, int box_rows) {
  if (Kp % TC_BK != 0) return cudaErrorInvalidValue;
  // box_rows for the A role (128) or the 128-wide B tile; 64 for the 64-wide B tile
  cudaError_t e = encode_bf16_map(&op.map, base, rows, 2 * (int64_t)Kp, box_rows);
  if (e == cudaSuccess) e = encode_bf16_map(&op.map64, base, rows, 2 * (int64_t)Kp, 64);
  if (e != cudaSuccess) return e;
  op.has64 = true;
  op.rows = rows;
  op.Kp = Kp;
  return cudaSuccess;
}

namespace {
template <int EPI, int BN>
void set_attr() {
  cudaFuncSetAttribute(gemm_tc_kernel<EPI, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)TcShape<BN>::SMEM);
}

template <int BN>
void set_attr_all() {
  set_attr<kStoreF32, BN>();
  set_attr<kDscaleSplit, BN>();
  set_attr<kBetaTSplit, BN>();
  set_attr<kGammaCatSplit, BN>();
  set_attr<kPartialF32, BN>();
}
}  // namespace

void tc_init_attributes() {
  static bool done = false;
  if (done) return;
  set_attr_all<128>();
  set_attr_all<64>();
  done = true;
}

namespace {
template <int EPI, int BN>
cudaError_t launch_tc(cudaStream_t st, dim3 grid, const CUtensorMap &mA, const CUtensorMap &mB,
                      int M, int N, int KpA, int KpB, const TcEpilogue &ep, int *err,
                      const int *dcnt, int mul_n, const GTile *tiles) {
  // segments: A_hi B_hi, A_hi B_lo, A_lo B_hi  (low byte: A plane, next byte: B plane)
  const int4 segs = make_int4(0 | (0 << 8), 0 | (1 << 8), 1 | (0 << 8), 0);
  gemm_tc_kernel<EPI, BN><<<grid, TC_THREADS, TcShape<BN>::SMEM, st>>>(
      mA, mB, M, N, KpA, KpB, 3, segs, ep, err, dcnt, mul_n, tiles);
  return cudaGetLastError();
}

template <int BN>
cudaError_t launch_tc_epi(cudaStream_t st, int epi, dim3 grid, const CUtensorMap &mA,
                          const CUtensorMap &mB, int M, int N, int KpA, int KpB,
                          const TcEpilogue &ep, int *err, const int *dcnt, int mul_n,
                          const GTile *tiles) {
  switch (epi) {
    case kStoreF32:
      return launch_tc<kStoreF32, BN>(st, grid, mA, mB, M, N, KpA, KpB, ep, err, dcnt, mul_n, tiles);
    case kDscaleSplit:
      return launch_tc<kDscaleSplit, BN>(st, grid, mA, mB, M, N, KpA, KpB, ep, err, dcnt, mul_n,
                                         tiles);
    case kBetaTSplit:
      return launch_tc<kBetaTSplit, BN>(st, grid, mA, mB, M, N, KpA, KpB, ep, err, dcnt, mul_n,
                                        tiles);
    case kGammaCatSplit:
      return launch_tc<kGammaCatSplit, BN>(st, grid, mA, mB, M, N, KpA, KpB, ep, err, dcnt, mul_n,
                                           tiles);
    case kPartialF32:
      return launch_tc<kPartialF32, BN>(st, grid, mA, mB, M, N, KpA, KpB, ep, err, dcnt, mul_n,
                                        tiles);
    default:
      return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t launch_gemm_tc(cudaStream_t st, const TcOperand &A, const TcOperand &B, int M, int N,
                           int epi, const TcEpilogue &ep, int *err, const int *dcnt, int mul_n,
                           int bn) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (A.Kp != B.Kp) return cudaErrorInvalidValue;
  tc_init_attributes();
  if (bn == 64 && !B.has64) return cudaErrorInvalidValue;
  dim3 grid((M + TC_BM - 1) / TC_BM, (N + bn - 1) / bn);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  if (bn == 64)
    return launch_tc_epi<64>(st, epi, grid, A.map, B.map64, M, N, A.Kp, B.Kp, ep, err, dcnt, mul_n,
                             nullptr);
  return launch_tc_epi<128>(st, epi, grid, A.map, B.map, M, N, A.Kp, B.Kp, ep, err, dcnt, mul_n,
                            nullptr);
}

cudaError_t launch_gemm_tc_grouped(cudaStream_t st, const TcOperand &A, const TcOperand &B,
                                   const GTile *tiles, int n_tiles, int N, int epi,
                                   const TcEpilogue &ep, int *err, const int *dcnt, int mul_n,
                                   int bn) {
  if (n_tiles <= 0 || N <= 0) return cudaSuccess;
  tc_init_attributes();
  if (bn == 64 && !B.has64) return cudaErrorInvalidValue;
  dim3 grid(n_tiles, (N + bn - 1) / bn);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  if (bn == 64)
    return launch_tc_epi<64>(st, epi, grid, A.map, B.map64, 0, N, A.Kp, B.Kp, ep, err, dcnt, mul_n,
                             tiles);
  return launch_tc_epi<128>(st, epi, grid, A.map, B.map, 0, N, A.Kp, B.Kp, ep, err, dcnt, mul_n,
                            tiles);
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
                              __nv_bfloat16 *split) {
  const int64_t total = (int64_t)rows * Kp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / Kp;
    const int k = (int)(i % Kp);
    const double x = (k < K) ? hash_uniform((uint64_t)(r * K + k), seed) : 0.0;
    if (k < K) full[r * K + k] = x;
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

extern "C" tddft_status tddft_selftest_gemm(int32_t M, int32_t N, int32_t K, uint64_t seed,
                                            double *max_rel_err) {
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
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  TcOperand *opA = new TcOperand(), *opB = new TcOperand();
  if (e == cudaSuccess) {
    cudaMemset(e2, 0, 2 * sizeof(double));
    cudaMemset(err, 0, sizeof(int));
    st_fill_split<<<304, 256>>>(M, K, Kp, seed, A, As);
    st_fill_split<<<304, 256>>>(N, K, Kp, seed + 1, B, Bs);
    e = make_operand_map(*opA, As, M, Kp, 128);
    if (e == cudaSuccess) e = make_operand_map(*opB, Bs, N, Kp, 128);
  }
  // both N-tile widths, each checked against the float64 product
  for (int bn : {128, 64}) {
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
