// Device BLAS-1 pieces shared by the solvers: deterministic single-kernel reductions (each block
// writes a partial sum, the last block to finish adds the partials in block order) and the fused
// kernels of Jacobi-preconditioned CG with the scalars kept on the device.
#pragma once

#include "common.cuh"

namespace tetmf {
namespace {

constexpr int kBlock = 256;
constexpr int kMaxRedBlocks = 1024;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-reduce two values; the last block adds all partials and stores them
__device__ void finish2(double v0, double v1, double* partials, unsigned* ticket, double* out0, double* out1) {
  __shared__ double s0[kBlock / 32], s1[kBlock / 32];
  __shared__ bool last;
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    s0[w] = v0;
    s1[w] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < kBlock / 32; ++i) {
      a += s0[i];
      b += s1[i];
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < int(gridDim.x); i += kBlock) {
    a += partials[2 * i];
    b += partials[2 * i + 1];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if (l == 0) {
    s0[w] = a;
    s1[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int i = 0; i < kBlock / 32; ++i) {
      x += s0[i];
      y += s1[i];
    }
    if (out0) *out0 = x;
    if (out1) *out1 = y;
    *ticket = 0u;
  }
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < (n); i += int64_t(gridDim.x) * blockDim.x)

// out0 = a . b
template <typename T>
__global__ void __launch_bounds__(kBlock) k_dot(const T* __restrict__ a, const T* __restrict__ b, int64_t n,
                                                double* partials, unsigned* ticket, double* out0) {
  double s = 0.0;
  GRID_STRIDE(i, n) s = fma(double(a[i]), double(b[i]), s);
  finish2(s, 0.0, partials, ticket, out0, nullptr);
}

// PCG start: z = r / diag, p = z, rz = r . z, rr = r . r
template <typename T>
__global__ void __launch_bounds__(kBlock) k_pcg_start(const T* __restrict__ r, const T* __restrict__ diag,
                                                      T* __restrict__ z, T* __restrict__ p, int64_t n,
                                                      double* partials, unsigned* ticket, double* rz, double* rr) {
  double a = 0.0, b = 0.0;
  GRID_STRIDE(i, n) {
    const T ri = r[i];
    const T zi = ri / diag[i];
    z[i] = zi;
    p[i] = zi;
    a = fma(double(ri), double(zi), a);
    b = fma(double(ri), double(ri), b);
  }
  finish2(a, b, partials, ticket, rz, rr);
}

// alpha = rz / pq; x += alpha p; r -= alpha q; z = r / diag; rz' = r . z; rr = r . r
template <typename T>
__global__ void __launch_bounds__(kBlock) k_pcg_update(T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
                                                       const T* __restrict__ p, const T* __restrict__ q,
                                                       const T* __restrict__ diag, int64_t n, const double* rz,
                                                       const double* pq, double* partials, unsigned* ticket,
                                                       double* rz_next, double* rr) {
  const double pqv = *pq;
  const T alpha = pqv != 0.0 ? T(*rz / pqv) : T(0);
  double a = 0.0, b = 0.0;
  GRID_STRIDE(i, n) {
    x[i] = fma(alpha, p[i], x[i]);
    const T ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    const T zi = ri / diag[i];
    z[i] = zi;
    a = fma(double(ri), double(zi), a);
    b = fma(double(ri), double(ri), b);
  }
  finish2(a, b, partials, ticket, rz_next, rr);
}

// beta = rz' / rz; p = z + beta p
template <typename T>
__global__ void k_pcg_direction(T* __restrict__ p, const T* __restrict__ z, int64_t n, const double* rz_next,
                                const double* rz) {
  const double rzv = *rz;
  const T beta = rzv != 0.0 ? T(*rz_next / rzv) : T(0);
  GRID_STRIDE(i, n) p[i] = fma(beta, p[i], z[i]);
}

template <typename T>
__global__ void k_cast(const double* __restrict__ a, T* __restrict__ b, int64_t n) {
  GRID_STRIDE(i, n) b[i] = T(a[i]);
}

int red_grid(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  const int64_t cap = std::min<int64_t>(kMaxRedBlocks, int64_t(sm_count()) * 4);
  return int(g < 1 ? 1 : (g > cap ? cap : g));
}

int ew_grid(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  const int64_t cap = int64_t(sm_count()) * 8;
  return int(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace
}  // namespace tetmf
