// chi0 . z without any allocation: the float64 product of tddft_chi0_apply
// with every intermediate (planar copies of z and of the result, the block
// sums W, beta, a, gamma and the per-column frequencies) carved out of one
// block of device memory that the library reserves as a static array when it
// is loaded on a GPU.  The caller passes device pointers for z, omega and out.
#include <mutex>

#include "internal.h"

namespace {

// 16 MiB reserved on every GPU that loads the library, held until exit.
constexpr size_t kNoallocDoubles = (size_t)2 * 1024 * 1024;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current (the host-side symbol is only a stand-in).
std::mutex g_mutex;
double *g_scratch_ptr[128] = {};

size_t up256(size_t doubles) { return (doubles + 31) / 32 * 32; }

}  // namespace

namespace tddft {
const DevSystem *ctx_system(const tddft_ctx *c);
cudaStream_t ctx_stream(const tddft_ctx *c);
void ctx_set_error(tddft_ctx *c, const char *msg);
}  // namespace tddft

extern "C" tddft_status tddft_chi0_apply_noalloc(tddft_ctx *ctx, int32_t n_rhs,
                                                 const double *omega, double eps,
                                                 const double *z, double *out, int32_t flags) {
  using namespace tddft;
  if (!ctx) return TDDFT_ERR_INVALID_ARG;
  ctx_set_error(ctx, "");   // no stale message from an earlier failed call
  if (!(flags & TDDFT_DEVICE_PTRS) || !omega || !z || !out) {
    ctx_set_error(ctx, "tddft_chi0_apply_noalloc takes device pointers only (flags bit 0)");
    return TDDFT_ERR_INVALID_ARG;
  }
  if (!(eps > 0.0) || eps != eps || eps > 1e300) {
    ctx_set_error(ctx, "eps must be > 0");
    return TDDFT_ERR_INVALID_ARG;
  }
  if (n_rhs < 1) {
    ctx_set_error(ctx, "n_rhs must be >= 1");
    return TDDFT_ERR_SHAPE;
  }
  const DevSystem &sys = *ctx_system(ctx);
  const size_t S = (size_t)n_rhs, np = (size_t)sys.n_prod;
  const size_t nZ = up256(2 * S * np);                                  // planar z
  const size_t nO = up256(2 * S * np);                                  // planar result
  const size_t nW = up256(2 * S * (size_t)sys.n_blocks * kBlk);         // W blocks
  const size_t nB = up256((size_t)sys.n_orb * 2 * S * sys.n_occ);       // beta
  const size_t nA = up256((size_t)sys.n_virt * 2 * S * sys.n_occ);      // a
  const size_t nG = up256((size_t)sys.n_orb * 2 * S * sys.n_occ);       // gamma
  const size_t nM = up256(S);                                           // omega per column
  const size_t need = nZ + nO + nW + nB + nA + nG + nM;
  if (need > kNoallocDoubles) {
    char msg[200];
    snprintf(msg, sizeof msg,
             "n_rhs = %d needs %zu bytes of scratch; the reserved block holds %zu bytes",
             n_rhs, need * sizeof(double), kNoallocDoubles * sizeof(double));
    ctx_set_error(ctx, msg);
    return TDDFT_ERR_SHAPE;
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
    ctx_set_error(ctx, "cudaGetDevice failed");
    return TDDFT_ERR_CUDA;
  }
  double *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        ctx_set_error(ctx, cudaGetErrorString(e));
        return TDDFT_ERR_CUDA;
      }
      g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    base = g_scratch_ptr[dev];
  }

  // Every scratch region below is written in full before it is read, so
  // nothing has to be cleared between calls.
  OpWork wk;
  wk.slots = n_rhs;
  double *Zc = base;
  double *Wout = Zc + nZ;
  wk.W = Wout + nO;
  wk.beta = wk.W + nW;
  wk.abuf = wk.beta + nB;
  wk.gamma = wk.abuf + nA;
  wk.omega = wk.gamma + nG;
  wk.Y = nullptr;        // chi0 only: no K product
  wk.timer = nullptr;

  cudaStream_t st = ctx_stream(ctx);
  cudaError_t e = cudaMemcpyAsync(wk.omega, omega, S * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = launch_interleaved_to_planar(st, n_rhs, sys.n_prod, z, Zc);
  if (e == cudaSuccess) e = launch_apply_operator(st, sys, wk, n_rhs, kChi0, eps, Zc, Wout);
  if (e == cudaSuccess) e = launch_planar_to_interleaved(st, n_rhs, sys.n_prod, Wout, out);
  if (e != cudaSuccess) {
    ctx_set_error(ctx, cudaGetErrorString(e));
    return TDDFT_ERR_CUDA;
  }
  return TDDFT_OK;
}
