// Chebyshev-Jacobi smoothing and the power iteration that tunes it (the smoother of the paper's
// hybrid multigrid, Sec. 4.1: Chebyshev iteration preconditioned by the diagonal, here in any of
// the library's precisions through the same matrix-free apply).
//
// Chebyshev iteration on [lam_min, lam_max] (theta = centre, delta = half width, sigma =
// theta / delta), three-term form: d_0 = D^-1 r_0 / theta; rho_0 = 1 / sigma,
// rho_k = 1 / (2 sigma - rho_{k-1}), d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) D^-1 r_k;
// x_{k+1} = x_k + d_k with r_k = b - A x_k.  The scalar coefficients are formed on the host; each
// step is one apply and one fused vector kernel (r, d and x in one pass).
#include <cmath>
#include <vector>

#include "common.cuh"

namespace tetmf {
namespace {

constexpr int kRed = 256;        // threads per reduction block
constexpr int kRedBlocks = 1024; // blocks of the first reduction pass

#define CHEB_GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < (n); i += int64_t(gridDim.x) * blockDim.x)

// r = b - Ax (in place of Ax); d = c_d d + c_r r / diag (FIRST: d = c_r r / diag); x += d
template <typename T, bool FIRST>
__global__ void k_cheb_step(T* __restrict__ x, T* __restrict__ d, const T* __restrict__ ax, const T* __restrict__ b,
                            const T* __restrict__ diag, T c_d, T c_r, int64_t n) {
  CHEB_GRID_STRIDE(i, n) {
    const T r = b[i] - ax[i];
    const T di = FIRST ? c_r * r / diag[i] : c_d * d[i] + c_r * r / diag[i];
    d[i] = di;
    x[i] += di;
  }
}

// per-block partial sums of (v . av, v . (diag v), |av / diag|^2) in FP64, fixed order
template <typename T>
__global__ void __launch_bounds__(kRed) k_power_dots(const T* __restrict__ v, const T* __restrict__ av,
                                                     const T* __restrict__ diag, int64_t n, double* partials) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  CHEB_GRID_STRIDE(i, n) {
    const double vi = v[i], ai = av[i], di = diag[i];
    s0 = fma(vi, ai, s0);
    s1 = fma(vi * di, vi, s1);
    const double wi = ai / di;
    s2 = fma(wi, wi, s2);
  }
  __shared__ double sh[3][kRed];
  sh[0][threadIdx.x] = s0;
  sh[1][threadIdx.x] = s1;
  sh[2][threadIdx.x] = s2;
  __syncthreads();
  for (int w = kRed / 2; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w)
      for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) partials[3 * blockIdx.x + k] = sh[k][0];
}

// one block: out[k] = sum of the partials, fixed order
__global__ void __launch_bounds__(kRed) k_power_finish(const double* __restrict__ partials, int nb,
                                                       double* __restrict__ out) {
  __shared__ double sh[3][kRed];
  double s[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < nb; i += kRed)
    for (int k = 0; k < 3; ++k) s[k] += partials[3 * i + k];
  for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int w = kRed / 2; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w)
      for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) out[k] = sh[k][0];
}

// v = av / diag * scale
template <typename T>
__global__ void k_power_next(T* __restrict__ v, const T* __restrict__ av, const T* __restrict__ diag, double scale,
                             int64_t n) {
  CHEB_GRID_STRIDE(i, n) v[i] = T(double(av[i]) / double(diag[i]) * scale);
}

// v = v0 * scale
template <typename T>
__global__ void k_scale_copy(T* __restrict__ v, const T* __restrict__ v0, double scale, int64_t n) {
  CHEB_GRID_STRIDE(i, n) v[i] = T(double(v0[i]) * scale);
}

// per-block partial sums of |v|^2 (first slot of each triple of partials)
template <typename T>
__global__ void __launch_bounds__(kRed) k_norm2(const T* __restrict__ v, int64_t n, double* partials) {
  double s = 0.0;
  CHEB_GRID_STRIDE(i, n) s = fma(double(v[i]), double(v[i]), s);
  __shared__ double sh[kRed];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kRed / 2; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x] = sh[0];
    partials[3 * blockIdx.x + 1] = 0.0;
    partials[3 * blockIdx.x + 2] = 0.0;
  }
}

int ew_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  const int64_t cap = int64_t(sm_count()) * 16;
  return int(b < cap ? (b < 1 ? 1 : b) : cap);
}

int red_blocks(int64_t n) {
  int64_t b = (n + kRed - 1) / kRed;
  return int(b < kRedBlocks ? (b < 1 ? 1 : b) : kRedBlocks);
}

size_t vec_bytes(int64_t n, size_t es) { return (size_t(n) * es + 255) / 256 * 256; }

template <typename T>
int chebyshev_t(Ctx& c, int prec, const T* b, T* x, const T* diag, int degree, double lam_max, double lam_min,
                T* work, cudaStream_t st) {
  const int64_t n = c.ndofs;
  T* ax = work;
  T* d = reinterpret_cast<T*>(reinterpret_cast<char*>(work) + vec_bytes(n, sizeof(T)));
  const double theta = 0.5 * (lam_max + lam_min), delta = 0.5 * (lam_max - lam_min), sigma = theta / delta;
  double rho = 1.0 / sigma;
  for (int k = 0; k < degree; ++k) {
    if (int e = apply_op(c, prec, x, ax, st)) return e;
    if (k == 0) {
      k_cheb_step<T, true><<<ew_blocks(n), 256, 0, st>>>(x, d, ax, b, diag, T(0), T(1.0 / theta), n);
    } else {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      k_cheb_step<T, false><<<ew_blocks(n), 256, 0, st>>>(x, d, ax, b, diag, T(rho_new * rho),
                                                         T(2.0 * rho_new / delta), n);
      rho = rho_new;
    }
    TETMF_LAUNCH_CK();
  }
  return FEM_OK;
}

template <typename T>
int lambda_max_t(Ctx& c, int prec, const T* diag, const T* v0, int iterations, T* work, double* lam,
                 cudaStream_t st) {
  const int64_t n = c.ndofs;
  T* v = work;
  T* av = reinterpret_cast<T*>(reinterpret_cast<char*>(work) + vec_bytes(n, sizeof(T)));
  double* partials = reinterpret_cast<double*>(reinterpret_cast<char*>(work) + 2 * vec_bytes(n, sizeof(T)));
  double* res = partials + 3 * kRedBlocks;
  double h[3];
  auto reduce_read = [&]() -> int {
    k_power_finish<<<1, kRed, 0, st>>>(partials, red_blocks(n), res);
    TETMF_LAUNCH_CK();
    TETMF_CK(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st));
    TETMF_CK(cudaStreamSynchronize(st));
    return FEM_OK;
  };
  k_norm2<T><<<red_blocks(n), kRed, 0, st>>>(v0, n, partials);
  TETMF_LAUNCH_CK();
  if (int e = reduce_read()) return e;
  if (!(h[0] > 0.0)) {
    set_error("fem_lambda_max: v0 is zero");
    return FEM_EINVAL;
  }
  k_scale_copy<T><<<ew_blocks(n), 256, 0, st>>>(v, v0, 1.0 / std::sqrt(h[0]), n);
  TETMF_LAUNCH_CK();
  double l = 0.0;
  for (int it = 0; it < iterations; ++it) {
    if (int e = apply_op(c, prec, v, av, st)) return e;
    k_power_dots<T><<<red_blocks(n), kRed, 0, st>>>(v, av, diag, n, partials);
    TETMF_LAUNCH_CK();
    if (int e = reduce_read()) return e;
    l = h[0] / h[1];
    if (!(h[2] > 0.0)) break;
    k_power_next<T><<<ew_blocks(n), 256, 0, st>>>(v, av, diag, 1.0 / std::sqrt(h[2]), n);
    TETMF_LAUNCH_CK();
  }
  *lam = l;
  return FEM_OK;
}

}  // namespace

size_t lambda_max_work_bytes(const Ctx& c, int prec) {
  const size_t es = prec == FEM_FP64 ? 8 : 4;
  return 2 * vec_bytes(c.ndofs, es) + (3 * kRedBlocks + 3) * sizeof(double);
}

int chebyshev(Ctx& c, int prec, const void* b, void* x, const void* diag, int degree, double lam_max,
              double lam_min, void* work, void* stream) {
  cudaStream_t st = as_stream(stream);
  if (prec == FEM_FP64)
    return chebyshev_t<double>(c, prec, static_cast<const double*>(b), static_cast<double*>(x),
                               static_cast<const double*>(diag), degree, lam_max, lam_min,
                               static_cast<double*>(work), st);
  return chebyshev_t<float>(c, prec, static_cast<const float*>(b), static_cast<float*>(x),
                            static_cast<const float*>(diag), degree, lam_max, lam_min, static_cast<float*>(work),
                            st);
}

int lambda_max(Ctx& c, int prec, const void* diag, const void* v0, int iterations, void* work, double* lam,
               void* stream) {
  cudaStream_t st = as_stream(stream);
  if (prec == FEM_FP64)
    return lambda_max_t<double>(c, prec, static_cast<const double*>(diag), static_cast<const double*>(v0),
                                iterations, static_cast<double*>(work), lam, st);
  return lambda_max_t<float>(c, prec, static_cast<const float*>(diag), static_cast<const float*>(v0), iterations,
                             static_cast<float*>(work), lam, st);
}

}  // namespace tetmf
