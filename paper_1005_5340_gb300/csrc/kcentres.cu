// Matrix-free K z from the product centres: a labelled variant of the
// matrix-free Hartree product that the paper names as future work (Sec. 8),
// in the multipole form of Sec. 5 restricted to its monopole term.
//
// The paper forms f_Hxc^{mu nu} once and applies it as a dense matrix (Sec.
// 4.1); for distant products the Hartree part is the interaction of the
// products' multipole moments.  Here every product mu is a point charge at
// its centre C_{c(mu)} (an atom for a local product, a pair midpoint for a
// bilocal one) with the softened interaction g(r) = 1 / sqrt(r^2 + a^2) plus
// a diagonal term, which is the kernel of the synthetic inputs:
//     K_{mu nu} = g(|C_{c(mu)} - C_{c(nu)}|) + diag delta_{mu nu}.
// For point charges the monopole term is the whole expansion, so products
// sharing a centre interact through the centre's total charge
//     Q_c = sum_{mu at c} z_mu ,   (K z)_mu = diag z_mu + sum_c g(|C_{c(mu)} - C_c|) Q_c ,
// exactly (up to rounding): n_centres^2 kernel evaluations per vector instead
// of the n_prod^2 stored entries.  The multipole moments of extended product
// functions (l > 0) are not built: they need the products' radial functions.
//
// Three kernels, float64 throughout, deterministic:
//   charges    Q[r][c] (complex) summed over the centre's products in a fixed order
//   potential  H[r][c] = sum_c' g(|C_c - C_c'|) Q[r][c'] (source centres staged in
//              shared memory in tiles, every target centre for a chunk of columns)
//   scatter    out[r][mu] = diag z[r][mu] + H[r][c(mu)]
#include <algorithm>
#include <vector>

#include "internal.h"

namespace {

constexpr int KC_TILE = 128;   // source centres staged per tile
constexpr int KC_COLS = 4;     // complex columns per thread in the potential kernel

__global__ void kc_charges(int n_rhs, int n_prod, int n_centres, const int *__restrict__ cptr,
                           const int *__restrict__ members, const double2 *__restrict__ z,
                           double2 *__restrict__ Q) {
  const int c = blockIdx.x;
  if (c >= n_centres) return;
  const int b = cptr[c], e = cptr[c + 1];
  for (int r = threadIdx.x; r < n_rhs; r += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int i = b; i < e; ++i) {
      const double2 v = z[(int64_t)r * n_prod + members[i]];
      re += v.x;
      im += v.y;
    }
    Q[(int64_t)r * n_centres + c] = make_double2(re, im);
  }
}

// One thread per (target centre, chunk of KC_COLS columns); the source
// centres and their charges for the chunk pass through shared memory.
__global__ void __launch_bounds__(KC_TILE) kc_potential(int n_rhs, int n_centres,
                                                         const double *__restrict__ C,
                                                         double a2, const double2 *__restrict__ Q,
                                                         double2 *__restrict__ H) {
  __shared__ double sx[KC_TILE], sy[KC_TILE], sz[KC_TILE];
  __shared__ double2 sq[KC_COLS][KC_TILE];
  const int t = blockIdx.x * KC_TILE + threadIdx.x;
  const int r0 = blockIdx.y * KC_COLS;
  const bool live = t < n_centres;
  const double x = live ? C[3 * t] : 0.0, y = live ? C[3 * t + 1] : 0.0,
               zc = live ? C[3 * t + 2] : 0.0;
  double2 acc[KC_COLS];
#pragma unroll
  for (int j = 0; j < KC_COLS; ++j) acc[j] = make_double2(0.0, 0.0);
  for (int s0 = 0; s0 < n_centres; s0 += KC_TILE) {
    const int s = s0 + threadIdx.x;
    if (s < n_centres) {
      sx[threadIdx.x] = C[3 * s];
      sy[threadIdx.x] = C[3 * s + 1];
      sz[threadIdx.x] = C[3 * s + 2];
    }
#pragma unroll
    for (int j = 0; j < KC_COLS; ++j)
      sq[j][threadIdx.x] = (s < n_centres && r0 + j < n_rhs)
                               ? Q[(int64_t)(r0 + j) * n_centres + s]
                               : make_double2(0.0, 0.0);
    __syncthreads();
    const int ns = min(KC_TILE, n_centres - s0);
    for (int k = 0; k < ns; ++k) {
      const double dx = x - sx[k], dy = y - sy[k], dz = zc - sz[k];
      const double g = rsqrt(fma(dx, dx, fma(dy, dy, fma(dz, dz, a2))));
#pragma unroll
      for (int j = 0; j < KC_COLS; ++j) {
        acc[j].x = fma(g, sq[j][k].x, acc[j].x);
        acc[j].y = fma(g, sq[j][k].y, acc[j].y);
      }
    }
    __syncthreads();
  }
  if (live)
#pragma unroll
    for (int j = 0; j < KC_COLS; ++j)
      if (r0 + j < n_rhs) H[(int64_t)(r0 + j) * n_centres + t] = acc[j];
}

__global__ void kc_scatter(int64_t total, int n_prod, int n_centres, double diag,
                           const int *__restrict__ pc, const double2 *__restrict__ z,
                           const double2 *__restrict__ H, double2 *__restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / n_prod;
    const int mu = (int)(i - r * n_prod);
    const double2 h = H[r * n_centres + pc[mu]], v = z[i];
    out[i] = make_double2(fma(diag, v.x, h.x), fma(diag, v.y, h.y));
  }
}

}  // namespace

extern "C" tddft_status tddft_kernel_apply_centres(int32_t n_prod, int32_t n_centres,
                                                   const double *centres,
                                                   const int32_t *prod_centre, double softening,
                                                   double diag, int32_t n_rhs, const double *z,
                                                   double *out, void *stream) {
  if (n_prod < 1 || n_centres < 1 || n_rhs < 1 || !centres || !prod_centre || !z || !out)
    return TDDFT_ERR_INVALID_ARG;
  if (!(softening >= 0.0) || softening != softening || diag != diag) return TDDFT_ERR_INVALID_ARG;
  std::vector<int> count(n_centres + 1, 0);
  for (int mu = 0; mu < n_prod; ++mu) {
    const int c = prod_centre[mu];
    if (c < 0 || c >= n_centres) return TDDFT_ERR_SHAPE;
    ++count[c + 1];
  }
  for (int c = 0; c < n_centres; ++c) count[c + 1] += count[c];
  std::vector<int> members(n_prod), fill(count.begin(), count.end() - 1);
  for (int mu = 0; mu < n_prod; ++mu) members[fill[prod_centre[mu]]++] = mu;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<void *> allocs;
  auto alloc = [&](size_t bytes, void **p) -> cudaError_t {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) allocs.push_back(*p);
    return e;
  };
  void *d_c = nullptr, *d_ptr = nullptr, *d_mem = nullptr, *d_pc = nullptr, *d_Q = nullptr,
       *d_H = nullptr;
  cudaError_t e = alloc((size_t)n_centres * 3 * sizeof(double), &d_c);
  if (e == cudaSuccess) e = alloc(count.size() * sizeof(int), &d_ptr);
  if (e == cudaSuccess) e = alloc((size_t)n_prod * sizeof(int), &d_mem);
  if (e == cudaSuccess) e = alloc((size_t)n_prod * sizeof(int), &d_pc);
  if (e == cudaSuccess) e = alloc((size_t)n_rhs * n_centres * sizeof(double2), &d_Q);
  if (e == cudaSuccess) e = alloc((size_t)n_rhs * n_centres * sizeof(double2), &d_H);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_c, centres, (size_t)n_centres * 3 * sizeof(double),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_ptr, count.data(), count.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_mem, members.data(), members.size() * sizeof(int), cudaMemcpyHostToDevice,
                        st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_pc, prod_centre, (size_t)n_prod * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    kc_charges<<<n_centres, 128, 0, st>>>(n_rhs, n_prod, n_centres, (const int *)d_ptr,
                                          (const int *)d_mem, (const double2 *)z, (double2 *)d_Q);
    dim3 grid((n_centres + KC_TILE - 1) / KC_TILE, (n_rhs + KC_COLS - 1) / KC_COLS);
    kc_potential<<<grid, KC_TILE, 0, st>>>(n_rhs, n_centres, (const double *)d_c,
                                           softening * softening, (const double2 *)d_Q,
                                           (double2 *)d_H);
    const int64_t total = (int64_t)n_rhs * n_prod;
    const int g = (int)std::min<int64_t>((total + 255) / 256, 152 * 32);
    kc_scatter<<<g, 256, 0, st>>>(total, n_prod, n_centres, diag, (const int *)d_pc,
                                  (const double2 *)z, (const double2 *)d_H, (double2 *)out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (void *p : allocs) cudaFree(p);
  if (e == cudaErrorMemoryAllocation) return TDDFT_ERR_NOMEM;
  return e == cudaSuccess ? TDDFT_OK : TDDFT_ERR_CUDA;
}
