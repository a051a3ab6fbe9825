// Learned initial guess for the frequency sweep: a small network, shared by
// all products mu, that corrects the linear interpolation between the
// solutions X(omega-) and X(omega+) of two already solved neighbouring
// frequencies.  Hand-written kernels for the features, the forward pass
// (float32, or bf16 weights for inference), the backward pass, the Adam
// update and the guess loss.
//
// Network: n_in -> width -> width -> n_out, tanh after the two hidden
// layers, parameters packed as [W1 (width x n_in), b1, W2 (width x width),
// b2, W3 (n_out x width), b3].  W3 and b3 start at zero, so an untrained
// network returns the interpolation itself.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"

struct tddft_mlp {
  int n_in = 0, width = 0, n_out = 0;
  int64_t n_params = 0, cap_rows = 0, step = 0;
  float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *params_bf16 = nullptr;
  float *H1 = nullptr, *H2 = nullptr, *dH1 = nullptr, *dH2 = nullptr, *Y = nullptr;
  cudaStream_t st = nullptr;
  std::vector<void *> allocs;
  std::string err;
  // offsets into the packed parameter vector
  int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
};

namespace tddft {
namespace {

thread_local std::string g_mlp_error;

constexpr int MG = 64, MK = 16;
enum MlpEpi { kPlain = 0, kBiasTanh = 1, kTimesDtanh = 2, kAtomicAdd = 3, kBias = 4 };

__device__ __forceinline__ float ld(const float *p) { return *p; }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// C[m][n] = epi(sum_k A(m,k) B(k,n)), A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn].
// 64 x 64 tile, 16-deep K slices in shared memory, 4 x 4 outputs per thread.
// kAtomicAdd: blockIdx.z covers K in slices of ksplit and adds into C.
template <int EPI, class TB>
__global__ void __launch_bounds__(256) mlp_gemm(int M, int N, int K, const float *__restrict__ A,
                                                int64_t sam, int64_t sak, const TB *__restrict__ B,
                                                int64_t sbk, int64_t sbn, float *__restrict__ C,
                                                int64_t ldc, const float *__restrict__ bias,
                                                const float *__restrict__ H, int ksplit) {
  __shared__ float As[MK][MG + 1];
  __shared__ float Bs[MK][MG + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * MG, n0 = (int64_t)blockIdx.x * MG;
  const int kb = (EPI == kAtomicAdd) ? blockIdx.z * ksplit : 0;
  const int ke = (EPI == kAtomicAdd) ? min(K, kb + ksplit) : K;
  float acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += MK) {
    for (int i = tid; i < MG * MK; i += 256) {
      const int mm = i / MK, kk = i % MK;
      const int64_t gm = m0 + mm;
      const int gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < ke) ? A[gm * sam + (int64_t)gk * sak] : 0.f;
      const int kk2 = i / MG, nn = i % MG;
      const int64_t gn = n0 + nn;
      const int gk2 = k0 + kk2;
      Bs[kk2][nn] = (gn < N && gk2 < ke) ? ld(B + (int64_t)gk2 * sbk + gn * sbn) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < MK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      float x = acc[i][j];
      float *dst = C + gm * ldc + gn;
      if (EPI == kBiasTanh) *dst = tanhf(x + bias[gn]);
      else if (EPI == kBias) *dst = x + bias[gn];
      else if (EPI == kTimesDtanh) {
        const float h = H[gm * ldc + gn];
        *dst = x * (1.f - h * h);
      } else if (EPI == kAtomicAdd) atomicAdd(dst, x);
      else *dst = x;
    }
  }
}

// out[n] += sum_m X[m][n]  (column sums, partial per CTA then atomics)
__global__ void colsum_kernel(int64_t M, int N, const float *__restrict__ X, float *__restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int64_t m = blockIdx.y; m < M; m += gridDim.y) s += X[m * N + n];
  atomicAdd(out + n, s);
}

__global__ void adam_kernel(int64_t n, float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void to_bf16_kernel(int64_t n, const float *__restrict__ src, __nv_bfloat16 *__restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

__global__ void init_params_kernel(int64_t n, float *__restrict__ p, int64_t oW1, int64_t ob1,
                                   int64_t oW2, int64_t ob2, int64_t oW3, float a1, float a2,
                                   uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + seed * 0xD1B54A32D192ED03ull + 1;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u = (float)((z >> 40) * (1.0 / 16777216.0)) * 2.f - 1.f;
    float val = 0.f;
    if (i >= oW1 && i < ob1) val = a1 * u;
    else if (i >= oW2 && i < ob2) val = a2 * u;
    else val = 0.f;   // biases, W3 and b3 start at zero
    (void)oW3;
    p[i] = val;
  }
}

int grid1(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 152 * 16);
}

template <int EPI, class TB>
cudaError_t gemm(cudaStream_t st, int M, int N, int K, const float *A, int64_t sam, int64_t sak,
                 const TB *B, int64_t sbk, int64_t sbn, float *C, int64_t ldc,
                 const float *bias = nullptr, const float *H = nullptr) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  int ksplit = K, splits = 1;
  if (EPI == kAtomicAdd) {
    // spread the long reduction (over rows) across CTAs
    const int tiles = ((M + MG - 1) / MG) * ((N + MG - 1) / MG);
    splits = std::max(1, std::min((K + 2047) / 2048, (152 * 8) / std::max(1, tiles)));
    ksplit = (K + splits - 1) / splits;
    ksplit = (ksplit + MK - 1) / MK * MK;
    splits = (K + ksplit - 1) / ksplit;
  }
  dim3 grid((N + MG - 1) / MG, (M + MG - 1) / MG, splits);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  mlp_gemm<EPI, TB><<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, H, ksplit);
  return cudaGetLastError();
}

// Features of target right-hand side r (one CTA): neighbours X- = X[nb[2r]],
// X+ = X[nb[2r+1]] (interleaved complex rows of n_prod), interpolation
// weight t, frequency omega, spacing (omega+ - omega-) / eps, direction k.
__global__ void __launch_bounds__(256) features_kernel(
    int n_prod, const int *__restrict__ nb, const double *__restrict__ t,
    const double *__restrict__ omega, const int *__restrict__ dir, double h_over_eps,
    const double *__restrict__ X, const double *__restrict__ dip, const float *__restrict__ pfeat,
    float *__restrict__ F, double *__restrict__ lin, double *__restrict__ scale) {
  __shared__ double red[2][8];
  const int r = blockIdx.x;
  const double *xm = X + (int64_t)nb[2 * r] * 2 * n_prod;
  const double *xp = X + (int64_t)nb[2 * r + 1] * 2 * n_prod;
  const double *d = dip + (int64_t)dir[r] * n_prod;
  double s1 = 0.0, s2 = 0.0;
  for (int e = threadIdx.x; e < n_prod; e += 256) {
    s1 += xm[2 * e] * xm[2 * e] + xm[2 * e + 1] * xm[2 * e + 1] + xp[2 * e] * xp[2 * e] +
          xp[2 * e + 1] * xp[2 * e + 1];
    s2 += d[e] * d[e];
  }
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s1;
    red[1][threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  s1 = 0.0;
  s2 = 0.0;
  for (int w = 0; w < 8; ++w) {
    s1 += red[0][w];
    s2 += red[1][w];
  }
  double sc = sqrt(s1 / (2.0 * n_prod));
  if (!(sc > 0.0)) sc = 1.0;
  const double dr = s2 > 0.0 ? sqrt(s2 / n_prod) : 1.0;
  if (threadIdx.x == 0) scale[r] = sc;
  const double tr = t[r];
  const float tf = (float)tr, wf = (float)omega[r], hf = (float)h_over_eps;
  for (int e = threadIdx.x; e < n_prod; e += 256) {
    float *f = F + ((int64_t)r * n_prod + e) * 10;
    f[0] = (float)(xm[2 * e] / sc);
    f[1] = (float)(xm[2 * e + 1] / sc);
    f[2] = (float)(xp[2 * e] / sc);
    f[3] = (float)(xp[2 * e + 1] / sc);
    f[4] = tf;
    f[5] = wf;
    f[6] = hf;
    f[7] = pfeat[2 * e];
    f[8] = (float)(d[e] / dr);
    f[9] = pfeat[2 * e + 1];
    double *l = lin + ((int64_t)r * n_prod + e) * 2;
    l[0] = (1.0 - tr) * xm[2 * e] + tr * xp[2 * e];
    l[1] = (1.0 - tr) * xm[2 * e + 1] + tr * xp[2 * e + 1];
  }
}

// dY = d/dY of sum_r w_r |lin + s_r Y - x*|^2 / |x*|^2 (mean over targets);
// loss[r] = the relative squared error of target r (one CTA per target).
__global__ void __launch_bounds__(256) guess_loss_kernel(int n_prod, int n_target,
                                                         const float *__restrict__ Y,
                                                         const double *__restrict__ lin,
                                                         const double *__restrict__ xs,
                                                         const double *__restrict__ scale,
                                                         float *__restrict__ dY,
                                                         double *__restrict__ loss) {
  __shared__ double red[2][8];
  const int r = blockIdx.x;
  const double s = scale[r];
  double e2 = 0.0, n2 = 0.0;
  for (int e = threadIdx.x; e < n_prod; e += 256) {
    const int64_t i = (int64_t)r * n_prod + e;
    const double gr = lin[2 * i] + s * Y[2 * i] - xs[2 * i];
    const double gi = lin[2 * i + 1] + s * Y[2 * i + 1] - xs[2 * i + 1];
    e2 += gr * gr + gi * gi;
    n2 += xs[2 * i] * xs[2 * i] + xs[2 * i + 1] * xs[2 * i + 1];
  }
  for (int off = 16; off > 0; off >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, off);
    n2 += __shfl_xor_sync(0xffffffffu, n2, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = e2;
    red[1][threadIdx.x >> 5] = n2;
  }
  __syncthreads();
  e2 = 0.0;
  n2 = 0.0;
  for (int w = 0; w < 8; ++w) {
    e2 += red[0][w];
    n2 += red[1][w];
  }
  const double inv = n2 > 0.0 ? 1.0 / n2 : 0.0;
  if (threadIdx.x == 0) loss[r] = e2 * inv;
  const double c = 2.0 * s * inv / n_target;
  for (int e = threadIdx.x; e < n_prod; e += 256) {
    const int64_t i = (int64_t)r * n_prod + e;
    dY[2 * i] = (float)(c * (lin[2 * i] + s * Y[2 * i] - xs[2 * i]));
    dY[2 * i + 1] = (float)(c * (lin[2 * i + 1] + s * Y[2 * i + 1] - xs[2 * i + 1]));
  }
}

__global__ void combine_kernel(int64_t n, const float *__restrict__ Y, const double *__restrict__ lin,
                               const double *__restrict__ scale, int n_prod, double *__restrict__ x0) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double s = scale[i / n_prod];
    x0[2 * i] = lin[2 * i] + s * Y[2 * i];
    x0[2 * i + 1] = lin[2 * i + 1] + s * Y[2 * i + 1];
  }
}

tddft_status mfail(tddft_mlp *p, tddft_status s, const std::string &msg) {
  if (p) p->err = msg;
  else g_mlp_error = msg;
  return s;
}

cudaError_t forward(tddft_mlp *p, int64_t rows, const float *F, float *Y, bool bf16) {
  const int W = p->width, R = (int)rows;
  cudaError_t e;
  if (bf16) {
    const __nv_bfloat16 *q = p->params_bf16;
    e = gemm<kBiasTanh>(p->st, R, W, p->n_in, F, p->n_in, 1, q + p->oW1, 1, p->n_in, p->H1, W,
                        p->params + p->ob1);
    if (e == cudaSuccess)
      e = gemm<kBiasTanh>(p->st, R, W, W, p->H1, W, 1, q + p->oW2, 1, W, p->H2, W, p->params + p->ob2);
    if (e == cudaSuccess)
      e = gemm<kBias>(p->st, R, p->n_out, W, p->H2, W, 1, q + p->oW3, 1, W, Y, p->n_out,
                      p->params + p->ob3);
    return e;
  }
  const float *q = p->params;
  e = gemm<kBiasTanh>(p->st, R, W, p->n_in, F, p->n_in, 1, q + p->oW1, 1, p->n_in, p->H1, W,
                      q + p->ob1);
  if (e == cudaSuccess)
    e = gemm<kBiasTanh>(p->st, R, W, W, p->H1, W, 1, q + p->oW2, 1, W, p->H2, W, q + p->ob2);
  if (e == cudaSuccess)
    e = gemm<kBias>(p->st, R, p->n_out, W, p->H2, W, 1, q + p->oW3, 1, W, Y, p->n_out, q + p->ob3);
  return e;
}

// grad = d/dparams of sum_rows dY . Y(rows), using H1, H2 of the last forward
cudaError_t backward(tddft_mlp *p, int64_t rows, const float *F, const float *dY) {
  const int W = p->width, R = (int)rows, no = p->n_out, ni = p->n_in;
  const float *q = p->params;
  float *g = p->grad;
  cudaError_t e = cudaMemsetAsync(g, 0, p->n_params * sizeof(float), p->st);
  // layer 3: dW3 = dY^T H2, db3 = colsum dY, dH2 = (dY W3) * (1 - H2^2)
  if (e == cudaSuccess)
    e = gemm<kAtomicAdd>(p->st, no, W, R, dY, 1, no, p->H2, W, 1, g + p->oW3, W);
  if (e == cudaSuccess) {
    colsum_kernel<<<dim3((no + 255) / 256, 256), 256, 0, p->st>>>(rows, no, dY, g + p->ob3);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = gemm<kTimesDtanh>(p->st, R, W, no, dY, no, 1, q + p->oW3, W, 1, p->dH2, W, nullptr, p->H2);
  // layer 2
  if (e == cudaSuccess)
    e = gemm<kAtomicAdd>(p->st, W, W, R, p->dH2, 1, W, p->H1, W, 1, g + p->oW2, W);
  if (e == cudaSuccess) {
    colsum_kernel<<<dim3((W + 255) / 256, 256), 256, 0, p->st>>>(rows, W, p->dH2, g + p->ob2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = gemm<kTimesDtanh>(p->st, R, W, W, p->dH2, W, 1, q + p->oW2, W, 1, p->dH1, W, nullptr, p->H1);
  // layer 1
  if (e == cudaSuccess)
    e = gemm<kAtomicAdd>(p->st, W, ni, R, p->dH1, 1, W, F, ni, 1, g + p->oW1, ni);
  if (e == cudaSuccess) {
    colsum_kernel<<<dim3((W + 255) / 256, 256), 256, 0, p->st>>>(rows, W, p->dH1, g + p->ob1);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace

// accessor defined with the context
const DevSystem *ctx_system(const tddft_ctx *c);
cudaStream_t ctx_stream(const tddft_ctx *c);
void ctx_set_error(tddft_ctx *c, const char *msg);
const float *ctx_product_features(const tddft_ctx *c);
int ctx_slots(const tddft_ctx *c);
void ctx_set_guess_net(tddft_ctx *c, tddft_mlp *net);

}  // namespace tddft

using namespace tddft;

// File layout of tddft_mlp_save / tddft_mlp_load.
namespace {
constexpr char kMlpMagic[8] = {'T', 'D', 'D', 'F', 'T', 'M', 'L', 'P'};
struct MlpFileHeader {
  char magic[8];
  int32_t version, n_in, width, n_out;
  int64_t n_params;
};
static_assert(sizeof(MlpFileHeader) == 32, "file header layout");
}  // namespace

extern "C" {

tddft_status tddft_mlp_create(int32_t n_in, int32_t width, int32_t n_out, int64_t max_rows,
                              uint64_t seed, void *stream, tddft_mlp **out) {
  if (!out) return mfail(nullptr, TDDFT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_in < 1 || width < 1 || n_out < 1 || max_rows < 1 || max_rows > INT32_MAX)
    return mfail(nullptr, TDDFT_ERR_INVALID_ARG, "bad network shape or max_rows");
  tddft_mlp *p = new tddft_mlp();
  p->n_in = n_in;
  p->width = width;
  p->n_out = n_out;
  p->cap_rows = max_rows;
  p->st = static_cast<cudaStream_t>(stream);
  p->oW1 = 0;
  p->ob1 = p->oW1 + (int64_t)width * n_in;
  p->oW2 = p->ob1 + width;
  p->ob2 = p->oW2 + (int64_t)width * width;
  p->oW3 = p->ob2 + width;
  p->ob3 = p->oW3 + (int64_t)n_out * width;
  p->n_params = p->ob3 + n_out;
  cudaError_t e = cudaSuccess;
  auto al = [&](auto **ptr, size_t bytes) {
    if (e != cudaSuccess) return;
    void *q = nullptr;
    e = cudaMalloc(&q, bytes);
    if (e == cudaSuccess) {
      p->allocs.push_back(q);
      *ptr = static_cast<std::remove_reference_t<decltype(**ptr)> *>(q);
    }
  };
  al(&p->params, p->n_params * sizeof(float));
  al(&p->grad, p->n_params * sizeof(float));
  al(&p->m, p->n_params * sizeof(float));
  al(&p->v, p->n_params * sizeof(float));
  al(&p->params_bf16, p->n_params * sizeof(__nv_bfloat16));
  al(&p->H1, (size_t)max_rows * width * sizeof(float));
  al(&p->H2, (size_t)max_rows * width * sizeof(float));
  al(&p->dH1, (size_t)max_rows * width * sizeof(float));
  al(&p->dH2, (size_t)max_rows * width * sizeof(float));
  al(&p->Y, (size_t)max_rows * n_out * sizeof(float));
  if (e == cudaSuccess) {
    init_params_kernel<<<grid1(p->n_params), 256, 0, p->st>>>(
        p->n_params, p->params, p->oW1, p->ob1, p->oW2, p->ob2, p->oW3,
        (float)(1.0 / std::sqrt((double)n_in)), (float)(1.0 / std::sqrt((double)width)), seed);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(p->m, 0, p->n_params * sizeof(float), p->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->v, 0, p->n_params * sizeof(float), p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) {
    for (void *q : p->allocs) cudaFree(q);
    delete p;
    return mfail(nullptr, e == cudaErrorMemoryAllocation ? TDDFT_ERR_NOMEM : TDDFT_ERR_CUDA,
                 cudaGetErrorString(e));
  }
  *out = p;
  return TDDFT_OK;
}

void tddft_mlp_destroy(tddft_mlp *p) {
  if (!p) return;
  cudaStreamSynchronize(p->st);
  for (void *q : p->allocs) cudaFree(q);
  delete p;
}

const char *tddft_mlp_last_error(const tddft_mlp *p) {
  return p ? p->err.c_str() : g_mlp_error.c_str();
}

int64_t tddft_mlp_num_params(const tddft_mlp *p) { return p ? p->n_params : 0; }

tddft_status tddft_mlp_params(tddft_mlp *p, float *host, int64_t n, int32_t set) {
  if (!p || !host || n != p->n_params) return mfail(p, TDDFT_ERR_INVALID_ARG, "bad parameter buffer");
  cudaError_t e = set ? cudaMemcpyAsync(p->params, host, n * sizeof(float), cudaMemcpyHostToDevice, p->st)
                      : cudaMemcpyAsync(host, p->params, n * sizeof(float), cudaMemcpyDeviceToHost, p->st);
  if (e == cudaSuccess && set) e = cudaMemsetAsync(p->m, 0, n * sizeof(float), p->st);
  if (e == cudaSuccess && set) e = cudaMemsetAsync(p->v, 0, n * sizeof(float), p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return mfail(p, TDDFT_ERR_CUDA, cudaGetErrorString(e));
  if (set) p->step = 0;
  return TDDFT_OK;
}

tddft_status tddft_mlp_save(tddft_mlp *p, const char *path) {
  if (!p || !path) return mfail(p, TDDFT_ERR_INVALID_ARG, "null network or path");
  std::vector<float> h((size_t)p->n_params);
  const tddft_status st = tddft_mlp_params(p, h.data(), p->n_params, 0);
  if (st != TDDFT_OK) return st;
  MlpFileHeader hd;
  std::memcpy(hd.magic, kMlpMagic, 8);
  hd.version = 1;
  hd.n_in = p->n_in;
  hd.width = p->width;
  hd.n_out = p->n_out;
  hd.n_params = p->n_params;
  FILE *f = std::fopen(path, "wb");
  if (!f) return mfail(p, TDDFT_ERR_INVALID_ARG, std::string("cannot open ") + path);
  bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 &&
            std::fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? TDDFT_OK : mfail(p, TDDFT_ERR_INVALID_ARG, std::string("cannot write ") + path);
}

tddft_status tddft_mlp_load(tddft_mlp *p, const char *path) {
  if (!p || !path) return mfail(p, TDDFT_ERR_INVALID_ARG, "null network or path");
  FILE *f = std::fopen(path, "rb");
  if (!f) return mfail(p, TDDFT_ERR_INVALID_ARG, std::string("cannot open ") + path);
  MlpFileHeader hd;
  if (std::fread(&hd, sizeof(hd), 1, f) != 1 || std::memcmp(hd.magic, kMlpMagic, 8) != 0 ||
      hd.version != 1) {
    std::fclose(f);
    return mfail(p, TDDFT_ERR_INVALID_ARG, "not a network file of version 1");
  }
  if (hd.n_in != p->n_in || hd.width != p->width || hd.n_out != p->n_out ||
      hd.n_params != p->n_params) {
    std::fclose(f);
    return mfail(p, TDDFT_ERR_SHAPE,
                 "the file holds a " + std::to_string(hd.n_in) + "-" + std::to_string(hd.width) +
                     "-" + std::to_string(hd.n_out) + " network, this one is " +
                     std::to_string(p->n_in) + "-" + std::to_string(p->width) + "-" +
                     std::to_string(p->n_out));
  }
  std::vector<float> h((size_t)p->n_params);
  const bool ok = std::fread(h.data(), sizeof(float), h.size(), f) == h.size();
  std::fclose(f);
  if (!ok) return mfail(p, TDDFT_ERR_INVALID_ARG, "truncated network file");
  return tddft_mlp_params(p, h.data(), p->n_params, 1);
}

tddft_status tddft_mlp_forward(tddft_mlp *p, int64_t rows, const float *F, float *Y, int32_t bf16) {
  if (!p || !F || !Y) return mfail(p, TDDFT_ERR_INVALID_ARG, "null pointer");
  if (rows < 1 || rows > p->cap_rows) return mfail(p, TDDFT_ERR_SHAPE, "rows beyond max_rows");
  cudaError_t e = cudaSuccess;
  if (bf16) {
    to_bf16_kernel<<<grid1(p->n_params), 256, 0, p->st>>>(p->n_params, p->params, p->params_bf16);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = forward(p, rows, F, Y, bf16 != 0);
  if (e != cudaSuccess) return mfail(p, TDDFT_ERR_CUDA, cudaGetErrorString(e));
  return TDDFT_OK;
}

tddft_status tddft_mlp_backward(tddft_mlp *p, int64_t rows, const float *F, const float *dY,
                                float *grad_host) {
  if (!p || !F || !dY) return mfail(p, TDDFT_ERR_INVALID_ARG, "null pointer");
  if (rows < 1 || rows > p->cap_rows) return mfail(p, TDDFT_ERR_SHAPE, "rows beyond max_rows");
  cudaError_t e = forward(p, rows, F, p->Y, false);
  if (e == cudaSuccess) e = backward(p, rows, F, dY);
  if (e == cudaSuccess && grad_host)
    e = cudaMemcpyAsync(grad_host, p->grad, p->n_params * sizeof(float), cudaMemcpyDeviceToHost, p->st);
  if (e == cudaSuccess && grad_host) e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return mfail(p, TDDFT_ERR_CUDA, cudaGetErrorString(e));
  return TDDFT_OK;
}

tddft_status tddft_mlp_train_step(tddft_mlp *p, int32_t n_target, int32_t n_prod, const float *F,
                                  const double *lin, const double *xstar, const double *scale,
                                  double *loss, float lr) {
  if (!p || !F || !lin || !xstar || !scale || !loss)
    return mfail(p, TDDFT_ERR_INVALID_ARG, "null pointer");
  if (p->n_out != 2) return mfail(p, TDDFT_ERR_UNSUPPORTED, "the guess network has 2 outputs");
  const int64_t rows = (int64_t)n_target * n_prod;
  if (n_target < 1 || n_prod < 1 || rows > p->cap_rows)
    return mfail(p, TDDFT_ERR_SHAPE, "rows beyond max_rows");
  cudaError_t e = forward(p, rows, F, p->Y, false);
  if (e == cudaSuccess) {
    // dY reuses dH1's storage (rows x 2 <= rows x width)
    guess_loss_kernel<<<n_target, 256, 0, p->st>>>(n_prod, n_target, p->Y, lin, xstar, scale,
                                                    p->dH1, loss);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    // dY is copied aside: backward overwrites dH1
    float *dY = p->Y;   // Y is no longer needed once the loss gradient exists
    e = cudaMemcpyAsync(dY, p->dH1, rows * 2 * sizeof(float), cudaMemcpyDeviceToDevice, p->st);
    if (e == cudaSuccess) e = backward(p, rows, F, dY);
  }
  if (e == cudaSuccess) {
    p->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)p->step), c2 = 1.f - std::pow(b2, (float)p->step);
    adam_kernel<<<grid1(p->n_params), 256, 0, p->st>>>(p->n_params, p->params, p->grad, p->m, p->v,
                                                       lr, b1, b2, 1e-8f, c1, c2);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return mfail(p, TDDFT_ERR_CUDA, cudaGetErrorString(e));
  return TDDFT_OK;
}

tddft_status tddft_guess_features(tddft_ctx *ctx, int32_t n_target, const int32_t *nb,
                                  const double *t, const double *omega, const int32_t *dir,
                                  double h_over_eps, const double *X, float *F, double *lin,
                                  double *scale) {
  if (!ctx) return TDDFT_ERR_INVALID_ARG;
  if (!nb || !t || !omega || !dir || !X || !F || !lin || !scale || n_target < 1) {
    ctx_set_error(ctx, "tddft_guess_features: null pointer or n_target < 1");
    return TDDFT_ERR_INVALID_ARG;
  }
  const DevSystem &s = *ctx_system(ctx);
  features_kernel<<<n_target, 256, 0, ctx_stream(ctx)>>>(s.n_prod, nb, t, omega, dir, h_over_eps,
                                                         X, s.dip, ctx_product_features(ctx), F,
                                                         lin, scale);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx_set_error(ctx, cudaGetErrorString(e));
    return TDDFT_ERR_CUDA;
  }
  return TDDFT_OK;
}

tddft_status tddft_guess_load(tddft_ctx *ctx, const char *path) {
  if (!ctx) return TDDFT_ERR_INVALID_ARG;
  ctx_set_error(ctx, "");
  if (!path) {
    ctx_set_error(ctx, "path is NULL");
    return TDDFT_ERR_INVALID_ARG;
  }
  FILE *f = std::fopen(path, "rb");
  MlpFileHeader hd;
  const bool ok = f && std::fread(&hd, sizeof(hd), 1, f) == 1 &&
                  std::memcmp(hd.magic, kMlpMagic, 8) == 0 && hd.version == 1;
  if (f) std::fclose(f);
  if (!ok) {
    ctx_set_error(ctx, (std::string("not a readable network file of version 1: ") + path).c_str());
    return TDDFT_ERR_INVALID_ARG;
  }
  if (hd.n_in != 10 || hd.n_out != 2) {
    ctx_set_error(ctx, "the guess network maps 10 features to 2 outputs");
    return TDDFT_ERR_SHAPE;
  }
  const DevSystem &s = *ctx_system(ctx);
  const int64_t rows = 3 * (int64_t)sweep_chunk_freqs(ctx_slots(ctx), s.n_prod) * s.n_prod;
  tddft_mlp *net = nullptr;
  tddft_status st = tddft_mlp_create(hd.n_in, hd.width, hd.n_out, rows, 0, ctx_stream(ctx), &net);
  if (st == TDDFT_OK) st = tddft_mlp_load(net, path);
  if (st != TDDFT_OK) {
    ctx_set_error(ctx, net ? net->err.c_str() : g_mlp_error.c_str());
    if (net) tddft_mlp_destroy(net);
    return st;
  }
  ctx_set_guess_net(ctx, net);
  return TDDFT_OK;
}

tddft_status tddft_guess_combine(int64_t n_target, int32_t n_prod, const float *Y, const double *lin,
                                 const double *scale, double *x0, void *stream) {
  if (!Y || !lin || !scale || !x0 || n_target < 1 || n_prod < 1) return TDDFT_ERR_INVALID_ARG;
  const int64_t n = n_target * n_prod;
  combine_kernel<<<grid1(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, Y, lin, scale, n_prod, x0);
  return cudaGetLastError() == cudaSuccess ? TDDFT_OK : TDDFT_ERR_CUDA;
}

}  // extern "C"
