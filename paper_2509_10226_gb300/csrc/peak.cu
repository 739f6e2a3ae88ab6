// Arithmetic-throughput probe: the denominators of the FP64 and FP32 rooflines, measured on the
// GPU that runs the operator (the SIMT applies are bound by the FP64 and FP32 FMA pipes).
//
// Every thread runs a fixed number of iterations over eight independent FMA chains
// a_i <- a_i * b + c (b slightly below one, so the chains converge and stay finite); eight chains
// per thread and 32 warps per SM keep the pipe fed past its latency, and eight iterations per
// loop trip keep the loop's own instructions from taking dispatch slots from the FMAs.  Kind 0:
// FP64 fma.rn.f64; kind 1: FP32 fma.rn.f32; kind 2: packed fma.rn.f32x2 (two FP32 FMAs per
// instruction, the form the tensor-core apply's metric step uses).  The result is stored only if
// it equals a value the caller passes and the chains never reach, so the compiler has to keep
// every FMA while the kernel writes nothing in practice.
//
// Measured on GB300: the FP64 loop issues about 1.6 DP instructions per clock and SM whatever the
// chain count, occupancy or operand pattern, while the FP64 apply itself issues about 1.94; the
// probe is therefore reported as a measured lower bound of the FP64 peak, next to the nominal
// 1.25 TFLOP/s.  The FP32 loops reach 95-99 % of 128 FMA lanes per SM at 2.07 GHz.
#include <cstdint>

#include "common.cuh"

namespace tetmf {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;
constexpr int kChains = 8;
constexpr int kUnroll = 8;  // iterations per loop trip

__global__ void __launch_bounds__(kProbeThreads) k_fma_f64(int64_t iters, double never, double* sink) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 1.0 + 1e-3 * (threadIdx.x + i);
  const double b = 0.999999, c = 1e-6;
  for (int64_t it = 0; it < iters; it += kUnroll) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == never) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_fma_f32(int64_t iters, float never, double* sink) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 1.0f + 1e-3f * (threadIdx.x + i);
  const float b = 0.9999f, c = 1e-4f;
  for (int64_t it = 0; it < iters; it += kUnroll) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == never) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_fma_f32x2(int64_t iters, float never, double* sink) {
  uint64_t a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    const float lo = 1.0f + 1e-3f * (threadIdx.x + i), hi = lo + 0.5f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a[i]) : "f"(lo), "f"(hi));
  }
  uint64_t b, c;
  asm("mov.b64 %0, {%1, %1};" : "=l"(b) : "f"(0.9999f));
  asm("mov.b64 %0, {%1, %1};" : "=l"(c) : "f"(1e-4f));
  for (int64_t it = 0; it < iters; it += kUnroll) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int i = 0; i < kChains; ++i) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[i]) : "l"(b), "l"(c));
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[i]));
    s += lo + hi;
  }
  if (s == never) sink[0] = s;
}

}  // namespace
}  // namespace tetmf

using namespace tetmf;

extern "C" int fem_fma_probe(int32_t kind, int64_t iters, double* sink, double* flops, void* stream) {
  if (kind < 0 || kind > 2 || iters < 1 || iters > (int64_t(1) << 30) || iters % kUnroll || !sink || !flops) {
    set_error("fem_fma_probe: need kind 0..2, iters a multiple of 8 in [8, 2^30] and non-null sink and flops");
    return FEM_EINVAL;
  }
  int dev = -1;
  TETMF_CK(cudaGetDevice(&dev));
  const int blocks = sm_count() * kProbeBlocksPerSm;
  cudaStream_t st = as_stream(stream);
  // a value the converging chains (all near 1) never sum to
  const double never = -12345.678;
  if (kind == 0)
    k_fma_f64<<<blocks, kProbeThreads, 0, st>>>(iters, never, sink);
  else if (kind == 1)
    k_fma_f32<<<blocks, kProbeThreads, 0, st>>>(iters, float(never), sink);
  else
    k_fma_f32x2<<<blocks, kProbeThreads, 0, st>>>(iters, float(never), sink);
  TETMF_LAUNCH_CK();
  *flops = double(blocks) * kProbeThreads * double(iters) * kChains * 2.0 * (kind == 2 ? 2.0 : 1.0);
  return FEM_OK;
}
