// Float64 matrix products emulated on the bf16 tensor cores (sm_103a,
// tcgen05 + TMA + mbarrier, inline PTX) by error-free splitting of both
// operands into integer slices (the Ozaki scheme).
//
// Every row of an operand is scaled by a power of two 2^e (|x| < 2^e over the
// row) and cut into s integer slices,
//     x = 2^e sum_{i=1..s} q_i 2^(-7 i),   q_1 in [-128, 128], q_i in [-64, 64],
// each q_i an exact bf16.  The product of two rows is then
//     2^(eA+eB) sum_t 2^(-7 t) G_t,        G_t = sum_{i+j=t} sum_k qA_i qB_j ,
// kept for t <= s+1 (pairs below the last slice's weight are dropped).  The
// t-1 pairs of a group contribute at most 2^12 (s+2) per k, so over a K chunk
// of L <= 2^12 / (s+2) entries every partial sum of G_t is an integer of at
// most 2^24 and the float32 accumulation in tensor memory is exact.  The
// epilogue warps read each G_t of a chunk, convert it to an integer and add
// it, shifted to its weight, into one 64-bit integer accumulator per output;
// u = max(0, 7s - 35) low bits are dropped so that the accumulator stays below
// 2^63 over up to 1024 chunks.  The float64 result is 2^(eA+eB+u-7(s+1)) acc,
// with an error of about (1 + (s+1)/4) 2^(-7s) 2^(eA+eB) K at most (2^-42
// relative for s = 6).
//
// One CTA computes a 128 x 64 output tile:
//   warp 0     TMA producer: per 64-deep K block, the s slices of the A tile
//              (16 KB each) and of the B tile (8 KB each), one stage per
//              slice index, into a 9-stage ring (128-byte swizzle)
//   warp 1     tcgen05.mma issuer (M=128, N=64, K=16): once slice i of a K
//              block has landed, every pair (i, j) and (j, i) with j <= i and
//              i + j <= s+1 goes to the TMEM accumulator of group i+j (s
//              groups x 64 columns); a slice's stage is released after the
//              last pair that reads it, and a group of the next chunk starts
//              as soon as the epilogue has drained it
//   warps 2-9  epilogue (two warps per TMEM lane quadrant, 32 columns each):
//              per chunk, TMEM -> registers -> int64 accumulators; at the end
//              the float64 tile is stored (C or C^T)
// Every mbarrier wait is bounded; on expiry the CTA records an error code,
// stops issuing work, waits (bounded) for its TMA copies in flight and still
// frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "internal.h"
#include "tc_ptx.h"

namespace tddft {
namespace {
using namespace ptx;

constexpr int OZ_BM = 128, OZ_BN = 64, OZ_BK = 64;
constexpr int OZ_EPI_WARPS = 8;                        // 2 per TMEM lane quadrant
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;      // producer, MMA, epilogue
constexpr uint32_t OZ_A_BYTES = OZ_BM * OZ_BK * 2;   // 16 KB
// The N tile: 96 columns where the s groups fit in tensor memory (s x 96 <=
// 512, s <= 5), else 64; each MMA then does 1.5x the work for the same A
// tile read from shared memory.  9 stages of 24 KB, or 8 of 28 KB.
template <int BN> struct OzShape {
  static constexpr int EPI_COLS = BN / 2;                      // columns per epilogue thread
  static constexpr uint32_t B_BYTES = BN * OZ_BK * 2;
  static constexpr uint32_t STAGE_BYTES = OZ_A_BYTES + B_BYTES;
  static constexpr int STAGES = BN == 64 ? 9 : 8;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
};
__host__ __device__ constexpr int oz_bn(int S) { return S * 96 <= 512 ? 96 : 64; }

struct OzArgs {
  int M, N;
  int KpA, KpB; // slice-plane widths of the two operands
  int ns;       // slices (the kernel's template argument)
  int cb;       // K blocks per exact chunk
  const int *eA, *eB;
  OzEpilogue ep;
  int vec;      // kOzC with 16-byte aligned rows: double2 stores
  const GTile *tiles;   // grouped product: one entry per M tile (NULL: plain row tiles)
  int mgroup;           // M tiles per group of the L2-aware tile order
  int Mt, Nt;           // M tiles (rows / 128, or table entries) and N tiles
  int *err;
  const int *dcnt;
  int mul_n;
};

// Low bits dropped from the integer accumulator for S slices: with u(S) the
// largest value, 2^(24 + 7(S-1) - u) summed over up to 1024 chunks (and the
// lower groups, < 1% more) stays below 2^63.
__host__ __device__ constexpr int oz_drop_bits(int S) { return 7 * S - 35 > 0 ? 7 * S - 35 : 0; }
constexpr int kOzMaxChunks = 1024;

// acc += G_t of every group (t = grp + 2) read from tensor memory (this
// thread's 32 columns at tcol), at weight 2^(7 (S - 1 - grp) - u); a negative
// weight is a rounded right shift of the (exact, < 2^25) group sum.  One
// group's values are live at a time (the loop is not unrolled).
// (ns == S, passed at run time so that the loop stays rolled)
// Columns j0 .. j0 + n - 1 of acc from v (n = 16 or 32).
template <int N, int EC>
__device__ __forceinline__ void add_group(long long (&acc)[EC], const float *v, int j0, int sh) {
  if (sh >= 0) {
#pragma unroll
    for (int j = 0; j < N; ++j) acc[j0 + j] += (long long)__float2int_rn(v[j]) << sh;
  } else {
    const int r = -sh, half = 1 << (r - 1);
#pragma unroll
    for (int j = 0; j < N; ++j) acc[j0 + j] += (long long)((__float2int_rn(v[j]) + half) >> r);
  }
}

// tcol: this thread's lane and its first column (h EPI_COLS) in group 0.
// With 96-wide groups, half h = 0 reads 32 + 16 columns, h = 1 reads 16 +
// 32, so that every 32-column load starts on a multiple of 32 columns.
template <int S, int BN>
__device__ __forceinline__ void read_groups(uint32_t tcol, int h,
                                            long long (&acc)[OzShape<BN>::EPI_COLS], int ns,
                                            uint64_t *tempty) {
#pragma unroll 1
  for (int grp = 0; grp < ns; ++grp) {
    const int sh = 7 * (S - 1 - grp) - oz_drop_bits(S);
    const uint32_t g0 = tcol + (uint32_t)(grp * BN);
    float v[32], u[16];
    if (BN == 64) {
      tmem_ld32(g0, v);
    } else if (h == 0) {
      tmem_ld32(g0, v);
      tmem_ld16(g0 + 32, u);
    } else {
      tmem_ld16(g0, u);
      tmem_ld32(g0 + 16, v);
    }
    // this group's accumulator may be overwritten by the next chunk
    fence_before();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&tempty[grp]);
    if (BN == 64) {
      add_group<32>(acc, v, 0, sh);
    } else if (h == 0) {
      add_group<32>(acc, v, 0, sh);
      add_group<16>(acc, u, 32, sh);
    } else {
      add_group<16>(acc, u, 0, sh);
      add_group<32>(acc, v, 16, sh);
    }
  }
}

// 2^e for a normal-range exponent (clamped to [-1022, 1023])
__device__ __forceinline__ double pow2(int e) {
  e = max(-1022, min(1023, e));
  return __longlong_as_double((long long)(e + 1023) << 52);
}

template <int S, int BN>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    ozaki_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                      const __grid_constant__ CUtensorMap mapB, OzArgs a) {
  int N = a.N;
  if (a.dcnt) N = (int)min((int64_t)N, (int64_t)a.mul_n * (*a.dcnt));
  constexpr int OZ_STAGES = OzShape<BN>::STAGES;
  constexpr uint32_t OZ_STAGE_BYTES = OzShape<BN>::STAGE_BYTES;
  constexpr int OZ_EPI_COLS = OzShape<BN>::EPI_COLS;
  // Persistent: CTA b walks tiles t = b, b + gridDim.x, ...  Tile t -> (mt,
  // nt) in an L2-aware order: the M tiles (rows of A, or entries of the tile
  // table) in groups of a.mgroup (A panels that fit in L2 together), every N
  // tile of a group before the next group, the M tile fastest within it, so
  // that each A panel is read from DRAM about once.  Tiles past the live
  // columns are skipped by every role alike.
  const int Mt = a.Mt, Nt = a.Nt, n_tiles = Mt * Nt;
  struct Tile {
    int m0, xoff, nkb, rows_valid, atom, n0;
  };
  auto tile_of = [&](int t, Tile &T) -> bool {
    const int G = a.mgroup;
    const int g = t / (G * Nt), r = t - g * (G * Nt);
    const int Gg = min(G, Mt - g * G);
    const int mt = g * G + r % Gg, nt = r / Gg;
    T.n0 = nt * BN;
    if (T.n0 >= N) return false;
    if (a.tiles) {
      const GTile gt = a.tiles[mt];
      T.m0 = gt.row0;
      T.xoff = gt.xoff;
      T.nkb = gt.nkb;
      T.rows_valid = gt.rows;
      T.atom = gt.atom;
    } else {
      T.m0 = mt * OZ_BM;
      T.xoff = 0;
      T.nkb = a.KpA / OZ_BK;
      T.rows_valid = min(OZ_BM, a.M - T.m0);
      T.atom = -1;
    }
    return true;
  };
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(smem + OZ_STAGES * OZ_STAGE_BYTES);
  uint64_t *empty = full + OZ_STAGES;
  uint64_t *tfull = empty + OZ_STAGES;
  uint64_t *tempty = tfull + 1;   // [kOzMaxSlices] one per TMEM group
  uint64_t *drain = tempty + kOzMaxSlices;   // completion of every MMA this CTA issued
  uint32_t *tslot = (uint32_t *)(drain + 1);
  __shared__ int abort_flag;
  const uint64_t lim = wait_limit(a.err);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int s = S;
  const int cb = a.cb;
  constexpr uint32_t tcols = S * BN <= 256 ? 256u : 512u;

  if (threadIdx.x == 0) {
    for (int i = 0; i < OZ_STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(tfull, 1);
    for (int q = 0; q < kOzMaxSlices; ++q)
      mbar_init(&tempty[q], OZ_EPI_WARPS);   // one arrival per epilogue warp
    mbar_init(drain, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      // producer: stage g = (kb * s + i) counted over this CTA's tiles holds
      // slice i of K block kb
      int g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        Tile T;
        if (!tile_of(t, T)) continue;
        for (int kb = 0; kb < T.nkb && ok; ++kb) {
          for (int i = 0; i < s; ++i, ++g) {
            const int slot = g % OZ_STAGES;
            const uint32_t ph = (uint32_t)(g / OZ_STAGES) & 1u;
            if (!mbar_wait(&empty[slot], ph ^ 1u, lim)) {
              atomicExch(a.err, 21);
              abort_flag = 1;
              ok = false;
              break;
            }
            if (*(volatile int *)&abort_flag) {
              ok = false;
              break;
            }
            uint8_t *sa = smem + slot * OZ_STAGE_BYTES;
            mbar_expect_tx(&full[slot], OZ_STAGE_BYTES);
            tma_load_2d(sa, &mapA, &full[slot], i * a.KpA + kb * OZ_BK, T.m0);
            tma_load_2d(sa + OZ_A_BYTES, &mapB, &full[slot], i * a.KpB + T.xoff + kb * OZ_BK,
                        T.n0);
          }
        }
      }
      // copies in flight: the last OZ_STAGES stages issued (each the latest
      // use of its slot) must have landed before the CTA may exit
      for (int h = max(0, g - OZ_STAGES); h < g; ++h)
        mbar_wait(&full[h % OZ_STAGES], (uint32_t)(h / OZ_STAGES) & 1u);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(OZ_BM, BN);
      const uint32_t base = smem_u32(smem);
      int g = 0;
      int gc = 0;   // chunks issued by this CTA (over its tiles)
      bool ok = true;
      for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        Tile T;
        if (!tile_of(t, T)) continue;
        const int nchunks = (T.nkb + cb - 1) / cb;
        for (int c = 0; c < nchunks && ok; ++c, ++gc) {
          const int kb1 = min(T.nkb, (c + 1) * cb);
          for (int kb = c * cb; kb < kb1 && ok; ++kb) {
            const bool first_kb = kb == c * cb;
            // slice pairs (i, j), i >= j, i + j <= S - 1, in the order i, then
            // j; the unrolled schedule is fixed by S.  (i, j) is the first
            // pair of its group (i + j) in that order exactly when i - j <= 1.
#pragma unroll
            for (int i = 0; i < S; ++i) {
              const int gi = g + i;
              if (!mbar_wait(&full[gi % OZ_STAGES], (uint32_t)(gi / OZ_STAGES) & 1u, lim)) {
                atomicExch(a.err, 23);
                abort_flag = 1;
                ok = false;
                break;
              }
              // each group of the previous chunk (of this tile or the one
              // before) drained by the epilogue, which drains them in order,
              // before its first MMA of this chunk: the groups first used at
              // step i are 2i - 1 and 2i, so the MMAs of the first groups
              // overlap the drain of the later ones
              if (first_kb && gc > 0) {
#pragma unroll
                for (int grp = (i == 0 ? 0 : 2 * i - 1); grp <= 2 * i && grp < S; ++grp)
                  if (ok && !mbar_wait(&tempty[grp], (uint32_t)(gc - 1) & 1u, lim)) {
                    atomicExch(a.err, 22);
                    abort_flag = 1;
                    ok = false;
                  }
                if (!ok) break;
              }
              fence_after();
              const uint32_t si = base + (uint32_t)(gi % OZ_STAGES) * OZ_STAGE_BYTES;
#pragma unroll
              for (int j = 0; j <= (i < S - 1 - i ? i : S - 1 - i); ++j) {
                const uint32_t sj = base + (uint32_t)((g + j) % OZ_STAGES) * OZ_STAGE_BYTES;
                const uint32_t d = tmem + (uint32_t)((i + j) * BN);
                const bool overwrite = first_kb && (i - j <= 1);
                // A slice i x B slice j
#pragma unroll
                for (int k = 0; k < OZ_BK / 16; ++k)
                  mma_bf16(d, desc_sw128(si + 32 * k), desc_sw128(sj + OZ_A_BYTES + 32 * k),
                           idesc, (overwrite && k == 0) ? 0u : 1u);
                if (j < i) {
                  // A slice j x B slice i
#pragma unroll
                  for (int k = 0; k < OZ_BK / 16; ++k)
                    mma_bf16(d, desc_sw128(sj + 32 * k), desc_sw128(si + OZ_A_BYTES + 32 * k),
                             idesc, 1u);
                }
              }
              // slice q is last used at step max(q, S-1-q): release what step i
              // finished (the stage frees once these MMAs complete)
              if (i >= S - 1 - i) mma_commit(&empty[gi % OZ_STAGES]);
              if (S - 1 - i < i) mma_commit(&empty[(g + S - 1 - i) % OZ_STAGES]);
            }
            if (!ok) break;
            g += S;
          }
          if (ok) mma_commit(tfull);
        }
      }
      // every MMA issued here (also after an abort) completes before the
      // tensor memory is freed
      mma_commit(drain);
      mbar_wait(drain, 0u);
    }
    __syncwarp();
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (rows of the tile)
    // and columns 32 h .. 32 h + 31 of every group, h = (w - 2) / 4
    const int q = warp & 3, h = (warp - 2) >> 2;
    const int lr = q * 32 + lane;
    const uint32_t tcol = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * OZ_EPI_COLS);
    int gc = 0;   // chunks drained (over this CTA's tiles)
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
      Tile T;
      if (!tile_of(t, T)) continue;
      const int m = T.m0 + lr;
      const int nc = T.n0 + h * OZ_EPI_COLS;
      const int nchunks = (T.nkb + cb - 1) / cb;
      long long acc[OZ_EPI_COLS];
#pragma unroll
      for (int j = 0; j < OZ_EPI_COLS; ++j) acc[j] = 0;
      bool ok = true;
      for (int c = 0; c < nchunks; ++c, ++gc) {
        bool have = mbar_wait(tfull, (uint32_t)gc & 1u, lim);
        // tcgen05.ld is warp-collective: one decision per warp
        have = __all_sync(0xffffffffu, have && !*(volatile int *)&abort_flag);
        if (!have) {
          if (lane == 0) atomicExch(a.err, 24);
          abort_flag = 1;
          ok = false;
          break;
        }
        fence_after();
        read_groups<S, BN>(tcol, h, acc, a.ns, tempty);
      }
      if (!ok) break;
      if (lr < T.rows_valid && nc < N) {
        // C = acc 2^(eA + eB + u - 7(S+1)), as two exact power-of-two factors
        const double fa = pow2(a.eA[m] + oz_drop_bits(S) - 7 * (S + 1));
        const OzEpilogue &ep = a.ep;
        if (ep.mode == kOzC) {
          double *crow = ep.C + (int64_t)m * ep.ldc + nc;
          if (a.vec && nc + OZ_EPI_COLS <= N) {
#pragma unroll
            for (int j = 0; j < OZ_EPI_COLS; j += 2) {
              double2 w;
              w.x = (double)acc[j] * fa * pow2(__ldg(a.eB + nc + j));
              w.y = (double)acc[j + 1] * fa * pow2(__ldg(a.eB + nc + j + 1));
              *(double2 *)(crow + j) = w;
            }
          } else {
#pragma unroll
            for (int j = 0; j < OZ_EPI_COLS; ++j)
              if (nc + j < N) crow[j] = (double)acc[j] * fa * pow2(__ldg(a.eB + nc + j));
          }
        } else if (ep.mode == kOzCT) {
#pragma unroll
          for (int j = 0; j < OZ_EPI_COLS; ++j)
            if (nc + j < N)
              ep.C[(int64_t)(nc + j) * ep.ldc + m] =
                  (double)acc[j] * fa * pow2(__ldg(a.eB + nc + j));
        } else if (ep.mode == kOzBetaT) {
          // row m = (atom A, E, c): beta^T[(j n_occ + E)][ao_A + c] for column j
          const int aoA = ep.aoff[T.atom], nA = ep.aoff[T.atom + 1] - aoA;
          const int r = m - aoA * ep.n_occ, E = r / nA, c = r - E * nA;
          double *dst = ep.C + (int64_t)E * ep.ldc + aoA + c;
          const int64_t step = (int64_t)ep.n_occ * ep.ldc;
#pragma unroll
          for (int j = 0; j < OZ_EPI_COLS; ++j)
            if (nc + j < N)
              dst[(int64_t)(nc + j) * step] = (double)acc[j] * fa * pow2(__ldg(a.eB + nc + j));
        } else {
          // kOzGammaCat: row m = orbital (atom B, b), column n = j n_occ + E ->
          // Gcat[j][xoff_B + b n_occ + E]
          const int B = ep.orb_atom[m], b = m - ep.aoff[B];
          const int64_t xo = ep.xoff5[B] + (int64_t)b * ep.n_occ;
          int jj = nc / ep.n_occ, E = nc - jj * ep.n_occ;
#pragma unroll
          for (int j = 0; j < OZ_EPI_COLS; ++j) {
            if (nc + j < N)
              ep.C[(int64_t)jj * ep.ldc + xo + E] =
                  (double)acc[j] * fa * pow2(__ldg(a.eB + nc + j));
            if (++E == ep.n_occ) {
              E = 0;
              ++jj;
            }
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
  }
}

// ---------------------------------------------------------------------------
// Slicing, in integer arithmetic on the float64 bit patterns (float64 ops run
// at 1/64 of the float32 rate on this part).  The row exponent is e = f - 1022
// for the largest biased exponent field f of the row (so |x| < 2^e); each x
// becomes the fixed-point integer F = round(x 2^(7s - e)), |F| <= 2^(7s),
// and F is written as balanced base-128 digits, most significant first:
//   F = sum_i q_i 128^(s-i),   q_1 in [-128, 128],  q_i in [-64, 63] (i > 1),
// so x = 2^e sum_i q_i 2^(-7i) up to the rounding of F.  Zero and subnormal
// values (below 2^-1022, far under any row's scale) count as zero.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int exp_field(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}
__device__ __forceinline__ int row_exponent_of_field(int fmax) {
  return fmax > 0 ? fmax - 1022 : 0;
}
__device__ __forceinline__ long long fixed_point(double x, int e, int s) {
  const long long b = __double_as_longlong(x);
  const int f = (int)((b >> 52) & 0x7FF);
  if (f == 0) return 0;
  const long long M = (b & 0xFFFFFFFFFFFFFll) | (1ll << 52);   // x = +-M 2^(f - 1075)
  const int sh = f - 1075 + 7 * s - e;
  long long F;
  if (sh >= 0) F = M << sh;                       // only for s = 8 (sh <= 3)
  else if (sh < -62) F = 0;
  else F = (M + (1ll << (-sh - 1))) >> (-sh);     // round half up in magnitude
  return b < 0 ? -F : F;
}
// bf16 bit pattern of an integer with |q| <= 128 (exact)
__device__ __forceinline__ unsigned int bf16_bits_small(int q) {
  if (q == 0) return 0u;
  const unsigned int sign = q < 0 ? 0x8000u : 0u;
  const unsigned int a = (unsigned int)(q < 0 ? -q : q);
  const int p = 31 - __clz(a);                    // 2^p <= a < 2^(p+1), p <= 7
  return sign | ((unsigned int)(127 + p) << 7) | ((a << (7 - p)) & 0x7Fu);
}
// slices of two neighbouring entries (x0, x1) of a row with exponent e,
// stored as bf16 pairs at dst + i*Kp for slice i
__device__ __forceinline__ void store_slices(double x0, double x1, int e, int s, int Kp,
                                             __nv_bfloat16 *dst) {
  long long F0 = fixed_point(x0, e, s), F1 = fixed_point(x1, e, s);
  unsigned int w[kOzMaxSlices];
  for (int i = s - 1; i >= 1; --i) {
    const int d0 = (int)(((F0 + 64) & 127) - 64), d1 = (int)(((F1 + 64) & 127) - 64);
    w[i] = bf16_bits_small(d0) | (bf16_bits_small(d1) << 16);
    F0 = (F0 - d0) >> 7;
    F1 = (F1 - d1) >> 7;
  }
  w[0] = bf16_bits_small((int)F0) | (bf16_bits_small((int)F1) << 16);
  for (int i = 0; i < s; ++i) *(unsigned int *)(dst + (int64_t)i * Kp) = w[i];
}

// Block-wide max of an int (all threads receive it); red holds >= 32 ints.
__device__ __forceinline__ int block_max_int(int v, int *red) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    int t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) t = max(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  const int r = red[0];
  __syncthreads();
  return r;
}

// Row r of the operand: X[r][k] for k < Kdim, or, with a column map,
// X[r][cols[k]] (zero where cols[k] < 0).
__device__ __forceinline__ double gathered(const double *x, const int *cols, int k, int Kdim) {
  if (k >= Kdim) return 0.0;
  if (!cols) return x[k];
  const int c = cols[k];
  return c >= 0 ? x[c] : 0.0;
}

__global__ void oz_slice_rows_kernel(int rows, int Kdim, const double *__restrict__ X, int64_t ldx,
                                     const int *__restrict__ cols, int s, int Kp,
                                     __nv_bfloat16 *__restrict__ Q, int *__restrict__ E,
                                     const int *dcnt, int mul) {
  __shared__ int red[32];
  int live = rows;
  if (dcnt) live = min(rows, mul * (*dcnt));
  for (int r = blockIdx.x; r < live; r += gridDim.x) {
    const double *x = X + (int64_t)r * ldx;
    int fm = 0;
    for (int k = threadIdx.x; k < Kdim; k += blockDim.x) fm = max(fm, exp_field(gathered(x, cols, k, Kdim)));
    const int e = row_exponent_of_field(block_max_int(fm, red));
    if (threadIdx.x == 0) E[r] = e;
    __nv_bfloat16 *qr = Q + (int64_t)r * s * Kp;
    for (int k = 2 * threadIdx.x; k < Kp; k += 2 * blockDim.x)
      store_slices(gathered(x, cols, k, Kdim), gathered(x, cols, k + 1, Kdim), e, s, Kp, qr + k);
  }
}

// Long rows: grid (chunks, rows).  Pass 1 raises E[r] (preset to a large
// negative value) to the exponent of each chunk's largest entry; pass 2
// slices every chunk with the row's exponent (a row of zeros keeps the preset
// value and gives zero slices).
constexpr int OZ_CHUNK = 4096;

__global__ void __launch_bounds__(256) oz_rowmax_kernel(int rows, int Kdim,
                                                        const double *__restrict__ X, int64_t ldx,
                                                        const int *__restrict__ cols,
                                                        int *__restrict__ E, const int *dcnt,
                                                        int mul) {
  __shared__ int red[32];
  int live = rows;
  if (dcnt) live = min(rows, mul * (*dcnt));
  const int r = blockIdx.y;
  if (r >= live) return;
  const double *x = X + (int64_t)r * ldx;
  const int k0 = blockIdx.x * OZ_CHUNK, k1 = min(Kdim, k0 + OZ_CHUNK);
  int fm = 0;
  for (int k = k0 + threadIdx.x; k < k1; k += 256) fm = max(fm, exp_field(gathered(x, cols, k, Kdim)));
  fm = block_max_int(fm, red);
  if (threadIdx.x == 0 && fm > 0) atomicMax(E + r, row_exponent_of_field(fm));
}

__global__ void __launch_bounds__(256) oz_slice_chunks_kernel(int rows, int Kdim,
                                                              const double *__restrict__ X,
                                                              int64_t ldx,
                                                              const int *__restrict__ cols, int s,
                                                              int Kp, __nv_bfloat16 *__restrict__ Q,
                                                              const int *__restrict__ E,
                                                              const int *dcnt, int mul) {
  int live = rows;
  if (dcnt) live = min(rows, mul * (*dcnt));
  const int r = blockIdx.y;
  if (r >= live) return;
  const double *x = X + (int64_t)r * ldx;
  const int e = E[r];   // a row of zeros: every entry gives F = 0 whatever e is
  __nv_bfloat16 *qr = Q + (int64_t)r * s * Kp;
  const int k0 = blockIdx.x * OZ_CHUNK, k1 = min(Kp, k0 + OZ_CHUNK);
  for (int k = k0 + 2 * threadIdx.x; k < k1; k += 512)
    store_slices(gathered(x, cols, k, Kdim), gathered(x, cols, k + 1, Kdim), e, s, Kp, qr + k);
}

// 32 columns per CTA (256 threads): column exponents, then 64-row tiles staged
// through shared memory and written as rows of the transposed operand.
__global__ void __launch_bounds__(256) oz_slice_cols_kernel(int Kdim, int N,
                                                            const double *__restrict__ X,
                                                            int64_t ldx, int s, int Kp,
                                                            __nv_bfloat16 *__restrict__ Q,
                                                            int *__restrict__ E, const int *dcnt,
                                                            int mul) {
  __shared__ double tile[32][65];
  __shared__ int red[8][32];
  __shared__ int ecol[32];
  int live = N;
  if (dcnt) live = (int)min((int64_t)N, (int64_t)mul * (*dcnt));
  const int n0 = blockIdx.x * 32;
  if (n0 >= live) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int n = n0 + tx;
  int fm = 0;
  if (n < live)
    for (int k = ty; k < Kdim; k += 8) fm = max(fm, exp_field(X[(int64_t)k * ldx + n]));
  red[ty][tx] = fm;
  __syncthreads();
  if (ty == 0) {
    int v = 0;
    for (int i = 0; i < 8; ++i) v = max(v, red[i][tx]);
    const int e = row_exponent_of_field(v);
    if (n < live) E[n] = e;
    ecol[tx] = e;
  }
  __syncthreads();
  for (int k0 = 0; k0 < Kp; k0 += 64) {
    for (int rr = ty; rr < 64; rr += 8) {
      const int k = k0 + rr;
      tile[tx][rr] = (k < Kdim && n < live) ? X[(int64_t)k * ldx + n] : 0.0;
    }
    __syncthreads();
    for (int cc = 0; cc < 4; ++cc) {
      const int col = ty * 4 + cc;
      if (n0 + col < live)
        store_slices(tile[col][2 * tx], tile[col][2 * tx + 1], ecol[col], s, Kp,
                     Q + (int64_t)(n0 + col) * s * Kp + k0 + 2 * tx);
    }
    __syncthreads();
  }
}

int chunk_blocks(int s) { return std::max(1, 4096 / (s + 2) / OZ_BK); }

template <int S>
cudaError_t launch_oz_kernel(cudaStream_t st, dim3 grid, const CUtensorMap &mA,
                             const OzOperand &B, const OzArgs &a) {
  constexpr int BN = oz_bn(S);
  ozaki_gemm_kernel<S, BN><<<grid, OZ_THREADS, OzShape<BN>::SMEM, st>>>(
      mA, BN == 64 ? B.map : B.map96, a);
  return cudaGetLastError();
}

template <int S>
cudaError_t set_smem_attr() {
  constexpr int BN = oz_bn(S);
  return cudaFuncSetAttribute(ozaki_gemm_kernel<S, BN>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)OzShape<BN>::SMEM);
}
}  // namespace

// Dynamic shared memory limits of every slice count (once; outside any
// stream capture).
cudaError_t oz_init_attributes() {
  static cudaError_t done = cudaErrorNotReady;
  if (done == cudaSuccess) return done;
  cudaError_t e = set_smem_attr<3>();
  if (e == cudaSuccess) e = set_smem_attr<4>();
  if (e == cudaSuccess) e = set_smem_attr<5>();
  if (e == cudaSuccess) e = set_smem_attr<6>();
  if (e == cudaSuccess) e = set_smem_attr<7>();
  if (e == cudaSuccess) e = set_smem_attr<8>();
  done = e;
  return e;
}

cudaError_t oz_operand(OzOperand &op, __nv_bfloat16 *q, int *e, int64_t rows, int Kdim, int s,
                       int box_rows) {
  if (s < kOzMinSlices || s > kOzMaxSlices || rows < 1 || Kdim < 1) return cudaErrorInvalidValue;
  op.q = q;
  op.e = e;
  op.rows = rows;
  op.Kp = round_up(Kdim, OZ_BK);
  op.s = s;
  cudaError_t r = encode_bf16_map(&op.map, q, rows, (int64_t)s * op.Kp, box_rows);
  // the B role also gets 96-row boxes (the N tile of 3 to 5 slices)
  op.has96 = false;
  if (r == cudaSuccess && box_rows == OZ_BN) {
    r = encode_bf16_map(&op.map96, q, rows, (int64_t)s * op.Kp, 96);
    op.has96 = r == cudaSuccess;
  }
  return r;
}

cudaError_t launch_oz_slice_rows(cudaStream_t st, const double *X, int64_t ldx, int rows, int Kdim,
                                 OzOperand &op, const int *dcnt, int mul, const int *cols) {
  if (rows <= 0) return cudaSuccess;
  if (rows > op.rows || Kdim > op.Kp) return cudaErrorInvalidValue;
  if (op.Kp >= 2 * OZ_CHUNK && rows <= 65535) {
    // long rows: chunks of a row on separate CTAs (exponent by atomic max)
    cudaError_t e = cudaMemsetAsync(op.e, 0x80, (size_t)rows * sizeof(int), st);
    if (e != cudaSuccess) return e;
    dim3 g1((Kdim + OZ_CHUNK - 1) / OZ_CHUNK, rows), g2((op.Kp + OZ_CHUNK - 1) / OZ_CHUNK, rows);
    oz_rowmax_kernel<<<g1, 256, 0, st>>>(rows, Kdim, X, ldx, cols, op.e, dcnt, mul);
    oz_slice_chunks_kernel<<<g2, 256, 0, st>>>(rows, Kdim, X, ldx, cols, op.s, op.Kp, op.q, op.e,
                                               dcnt, mul);
    return cudaGetLastError();
  }
  const int grid = std::min(rows, 152 * 8);
  oz_slice_rows_kernel<<<grid, 256, 0, st>>>(rows, Kdim, X, ldx, cols, op.s, op.Kp, op.q, op.e,
                                             dcnt, mul);
  return cudaGetLastError();
}

cudaError_t launch_oz_slice_cols(cudaStream_t st, const double *X, int64_t ldx, int Kdim, int N,
                                 OzOperand &op, const int *dcnt, int mul) {
  if (N <= 0) return cudaSuccess;
  if (N > op.rows || Kdim > op.Kp) return cudaErrorInvalidValue;
  oz_slice_cols_kernel<<<(N + 31) / 32, 256, 0, st>>>(Kdim, N, X, ldx, op.s, op.Kp, op.q, op.e,
                                                      dcnt, mul);
  return cudaGetLastError();
}

cudaError_t launch_gemm_oz_ex(cudaStream_t st, const OzOperand &A, const OzOperand &B, int M,
                              int N, const OzEpilogue &ep, const GTile *tiles, int n_tiles,
                              int max_nkb, int *err, const int *dcnt, int mul_n) {
  if (N <= 0 || (tiles ? n_tiles <= 0 : M <= 0)) return cudaSuccess;
  if (A.s != B.s || N > B.rows || (!tiles && (A.Kp != B.Kp || M > A.rows)))
    return cudaErrorInvalidValue;
  cudaError_t e = oz_init_attributes();
  if (e != cudaSuccess) return e;
  OzArgs a;
  a.M = M;
  a.N = N;
  a.KpA = A.Kp;
  a.KpB = B.Kp;
  a.ns = A.s;
  a.cb = chunk_blocks(A.s);
  const int nkb = tiles ? max_nkb : A.Kp / OZ_BK;
  if ((nkb + a.cb - 1) / a.cb > kOzMaxChunks) return cudaErrorInvalidValue;
  a.eA = A.e;
  a.eB = B.e;
  a.ep = ep;
  a.vec = (ep.mode == kOzC && (ep.ldc % 2) == 0 && ((uintptr_t)ep.C & 15) == 0) ? 1 : 0;
  a.tiles = tiles;
  {
    // M tiles whose A panels (s slices of the whole K) fill about 40 MB of L2
    // (grid.x = Mt, the tiles or 128-row blocks)
    const double panel = (double)OZ_BM * A.s * A.Kp * sizeof(__nv_bfloat16);
    const int Mt = tiles ? n_tiles : (M + OZ_BM - 1) / OZ_BM;
    a.mgroup = std::max(1, std::min(Mt, (int)(40.0e6 / panel)));
  }
  a.err = err;
  a.dcnt = dcnt;
  a.mul_n = mul_n;
  const int bn = oz_bn(A.s);
  if (bn == 96 && !B.has96) return cudaErrorInvalidValue;
  // persistent grid: one CTA per SM at most, each walking its share of the tiles
  a.Mt = tiles ? n_tiles : (M + OZ_BM - 1) / OZ_BM;
  a.Nt = (N + bn - 1) / bn;
  if ((int64_t)a.Mt * a.Nt > INT32_MAX) return cudaErrorInvalidConfiguration;
  static int n_sm = 0;
  if (n_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n_sm < 1)
      n_sm = 1;
  }
  dim3 grid((unsigned)std::min<int64_t>((int64_t)a.Mt * a.Nt, n_sm));
  switch (A.s) {
    case 3: return launch_oz_kernel<3>(st, grid, A.map, B, a);
    case 4: return launch_oz_kernel<4>(st, grid, A.map, B, a);
    case 5: return launch_oz_kernel<5>(st, grid, A.map, B, a);
    case 6: return launch_oz_kernel<6>(st, grid, A.map, B, a);
    case 7: return launch_oz_kernel<7>(st, grid, A.map, B, a);
    case 8: return launch_oz_kernel<8>(st, grid, A.map, B, a);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gemm_oz(cudaStream_t st, const OzOperand &A, const OzOperand &B, int M, int N,
                           double *C, int64_t ldc, int trans, int *err, const int *dcnt,
                           int mul_n) {
  OzEpilogue ep;
  ep.mode = trans ? kOzCT : kOzC;
  ep.C = C;
  ep.ldc = ldc;
  return launch_gemm_oz_ex(st, A, B, M, N, ep, nullptr, 0, 0, err, dcnt, mul_n);
}

// Constants sliced once; dynamic operands sized for `slots` right-hand sides.
cudaError_t oz_setup(cudaStream_t st, const DevSystem &sys, OzWork &oz, int slots,
                     std::vector<void *> &allocs) {
  const int s = oz.s, np = sys.n_prod, no = sys.n_orb, nv = sys.n_virt;
  const int64_t rowsB = 2 * (int64_t)slots * sys.n_occ;
  const int64_t rows6 = 6 * (int64_t)sys.n_occ;   // the three dipole columns
  const int64_t rowsT = std::max(rowsB, rows6);
  const int KpK = round_up(np, OZ_BK), Kp1 = round_up(no, OZ_BK), Kp2 = round_up(nv, OZ_BK);
  auto alloc = [&](size_t bytes, void **p) -> cudaError_t {
    cudaError_t e = cudaMalloc(p, bytes + 16);
    if (e == cudaSuccess) allocs.push_back(*p);
    return e;
  };
  void *qK, *qXvT, *qXv, *qZ, *qT, *e;
  const size_t bf = sizeof(__nv_bfloat16);
  const int64_t rowsZ = 2 * (int64_t)slots;
  cudaError_t r = alloc((size_t)np * s * KpK * bf, &qK);
  if (r == cudaSuccess) r = alloc((size_t)nv * s * Kp1 * bf, &qXvT);
  if (r == cudaSuccess) r = alloc((size_t)no * s * Kp2 * bf, &qXv);
  if (r == cudaSuccess) r = alloc((size_t)rowsZ * s * KpK * bf, &qZ);
  if (r == cudaSuccess) r = alloc((size_t)rowsT * s * std::max(Kp1, Kp2) * bf, &qT);
  const int64_t ne = (int64_t)np + nv + no + rowsZ + 2 * rowsT;
  if (r == cudaSuccess) r = alloc((size_t)ne * sizeof(int), &e);
  if (r == cudaSuccess) r = alloc(ptx::kErrInts * sizeof(int), (void **)&oz.err);
  if (r != cudaSuccess) return r;
  int *ep = (int *)e;
  auto bq = [](void *p) { return (__nv_bfloat16 *)p; };
  r = oz_operand(oz.K, bq(qK), ep, np, np, s, OZ_BM);
  ep += np;
  if (r == cudaSuccess) r = oz_operand(oz.XvT, bq(qXvT), ep, nv, no, s, OZ_BM);
  ep += nv;
  if (r == cudaSuccess) r = oz_operand(oz.Xv, bq(qXv), ep, no, nv, s, OZ_BM);
  ep += no;
  if (r == cudaSuccess) r = oz_operand(oz.Z, bq(qZ), ep, rowsZ, np, s, OZ_BN);
  ep += rowsZ;
  if (r == cudaSuccess) r = oz_operand(oz.Bt1, bq(qT), ep, rowsT, no, s, OZ_BN);
  ep += rowsT;
  if (r == cudaSuccess) r = oz_operand(oz.Bt2, bq(qT), ep, rowsT, nv, s, OZ_BN);
  if (r == cudaSuccess) r = oz_init_attributes();
  if (r == cudaSuccess) r = cudaMemsetAsync(oz.err, 0, ptx::kErrInts * sizeof(int), st);
  if (r == cudaSuccess) r = launch_oz_slice_rows(st, sys.K, np, np, np, oz.K);
  if (r == cudaSuccess) r = launch_oz_slice_rows(st, sys.XvT, no, nv, no, oz.XvT);
  if (r == cudaSuccess) r = launch_oz_slice_rows(st, sys.Xv, nv, no, nv, oz.Xv);
  return r;
}

}  // namespace tddft

// ---------------------------------------------------------------------------
// C boundary: one emulated float64 product on device buffers
// ---------------------------------------------------------------------------
extern "C" tddft_status tddft_gemm_f64_emulated(int32_t M, int32_t N, int32_t K, const double *A,
                                                int64_t lda, const double *B, int64_t ldb,
                                                double *C, int64_t ldc, int32_t slices,
                                                void *stream) {
  using namespace tddft;
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C) return TDDFT_ERR_INVALID_ARG;
  if (slices < kOzMinSlices || slices > kOzMaxSlices) return TDDFT_ERR_INVALID_ARG;
  if (lda < K || ldb < N || ldc < N) return TDDFT_ERR_SHAPE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int Kp = round_up(K, OZ_BK);
  std::vector<void *> allocs;
  auto alloc = [&](size_t bytes, void **p) -> cudaError_t {
    cudaError_t e = cudaMalloc(p, bytes + 16);
    if (e == cudaSuccess) allocs.push_back(*p);
    return e;
  };
  void *qa = nullptr, *qb = nullptr, *ea = nullptr, *eb = nullptr, *err = nullptr;
  cudaError_t e = alloc((size_t)M * slices * Kp * sizeof(__nv_bfloat16), &qa);
  if (e == cudaSuccess) e = alloc((size_t)N * slices * Kp * sizeof(__nv_bfloat16), &qb);
  if (e == cudaSuccess) e = alloc((size_t)M * sizeof(int), &ea);
  if (e == cudaSuccess) e = alloc((size_t)N * sizeof(int), &eb);
  if (e == cudaSuccess) e = alloc(ptx::kErrInts * sizeof(int), &err);
  OzOperand oa, ob;
  if (e == cudaSuccess) e = oz_operand(oa, (__nv_bfloat16 *)qa, (int *)ea, M, K, slices, OZ_BM);
  if (e == cudaSuccess) e = oz_operand(ob, (__nv_bfloat16 *)qb, (int *)eb, N, K, slices, OZ_BN);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, ptx::kErrInts * sizeof(int), st);
  if (e == cudaSuccess) e = launch_oz_slice_rows(st, A, lda, M, K, oa);
  if (e == cudaSuccess) e = launch_oz_slice_cols(st, B, ldb, K, N, ob);
  if (e == cudaSuccess) e = launch_gemm_oz(st, oa, ob, M, N, C, ldc, 0, (int *)err);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (void *p : allocs) cudaFree(p);
  if (e == cudaErrorMemoryAllocation) return TDDFT_ERR_NOMEM;
  if (e != cudaSuccess) return TDDFT_ERR_CUDA;
  return herr ? TDDFT_ERR_TIMEOUT : TDDFT_OK;
}
