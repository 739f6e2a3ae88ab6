// Helpers shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

#define TETMF_CK(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      ::tetmf::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? FEM_ENOMEM : FEM_ECUDA;                       \
    }                                                                                        \
  } while (0)

#define TETMF_LAUNCH_CK()                                                                     \
  do {                                                                                       \
    cudaError_t e_ = cudaGetLastError();                                                     \
    if (e_ != cudaSuccess) {                                                                 \
      ::tetmf::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
      return FEM_ECUDA;                                                                      \
    }                                                                                        \
  } while (0)

namespace tetmf {

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Number of SMs of the current device (cached per process for device 0..15).
int sm_count();

// Launch a kernel that may start while the kernel before it in the stream still runs (programmatic
// dependent launch, once that kernel has executed griddepcontrol.launch_dependents or exited): the
// launched kernel must execute griddepcontrol.wait before it touches anything its predecessor writes.
template <typename... P, typename... A>
inline cudaError_t launch_early(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<P>(args)...);
}

// Opt a kernel into more than 48 KB of dynamic shared memory (once per call site).
template <typename K>
inline int allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e != cudaSuccess) {
      set_error("cudaFuncSetAttribute(%zu bytes of shared memory): %s", bytes, cudaGetErrorString(e));
      return FEM_ECUDA;
    }
  }
  return FEM_OK;
}

// y[i] = mask && mask[i] ? u[i] * diag_one : 0  (Dirichlet identity rows, or zero fill).  A kernel
// launched after it with programmatic stream serialization may start at once; it must execute
// griddepcontrol.wait before it touches y.
template <typename T>
__global__ void k_init_rows(T* __restrict__ y, const T* __restrict__ u, const uint8_t* __restrict__ mask, int64_t n,
                            T fixed) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    T v = T(0);
    if (mask && mask[i]) v = u ? u[i] : fixed;
    y[i] = v;
  }
}

template <typename T>
inline int init_rows(T* y, const T* u, const uint8_t* mask, int64_t n, T fixed, cudaStream_t s) {
  if (n <= 0) return FEM_OK;
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = int64_t(sm_count()) * 8;
  if (blocks > cap) blocks = cap;
  k_init_rows<T><<<unsigned(blocks), 256, 0, s>>>(y, u, mask, n, fixed);
  TETMF_LAUNCH_CK();
  return FEM_OK;
}

}  // namespace tetmf

// Compile-time shapes of the supported spaces: degree p (ND = (p+1)(p+2)(p+3)/6 DoFs per cell)
// with the standard cell rule (Grundmann-Moeller s = p, NQ points) or the modified one of Sec. 3.3
// (s = p - 1); NQF = face points (always s = p).  CALL may use ND, NQ and NQF.
#define TETMF_DISPATCH_SPACE(p, nq, CALL)                                                        \
  switch ((p) * 100 + (nq)) {                                                                   \
    case 105: { constexpr int ND = 4, NQ = 5, NQF = 4; (void)NQF; return CALL; }                \
    case 101: { constexpr int ND = 4, NQ = 1, NQF = 4; (void)NQF; return CALL; }                \
    case 215: { constexpr int ND = 10, NQ = 15, NQF = 10; (void)NQF; return CALL; }             \
    case 205: { constexpr int ND = 10, NQ = 5, NQF = 10; (void)NQF; return CALL; }              \
    case 335: { constexpr int ND = 20, NQ = 35, NQF = 20; (void)NQF; return CALL; }             \
    case 315: { constexpr int ND = 20, NQ = 15, NQF = 20; (void)NQF; return CALL; }             \
    case 470: { constexpr int ND = 35, NQ = 70, NQF = 35; (void)NQF; return CALL; }             \
    case 435: { constexpr int ND = 35, NQ = 35, NQF = 35; (void)NQF; return CALL; }             \
    default:                                                                                    \
      ::tetmf::set_error("degree %d with %d cell quadrature points not supported", int(p), int(nq)); \
      return FEM_EUNSUPPORTED;                                                                  \
  }
