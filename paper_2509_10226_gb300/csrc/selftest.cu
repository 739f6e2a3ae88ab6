// Diagnostics of the bounded-wait protocol of the tensor-core kernels, run without a GPU fault.
//
// One CTA of two warpgroups allocates TMEM like the apply kernels, then each warpgroup's first
// thread waits on an mbarrier that nothing ever arrives on, through the same helpers the kernels
// use (mbar_wait_ab with a shared abort flag).  The first wait gives up after limit_ns and raises
// the flag; the other wait then returns at once; the CTA frees its TMEM, records bit 0 in the
// context's device status word (as the kernels do) and returns, leaving the context usable.
#include <cuda_runtime.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace tetmf {
namespace {

__global__ void __launch_bounds__(256, 1)
    k_selftest_wait(uint64_t limit_ns, int32_t* __restrict__ status, int64_t* __restrict__ waited) {
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar[0]));
    mbar_init(smem_u32(&bar[1]));
    abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(32));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  bool ok = true;
  if (threadIdx.x % 128 == 0) {
    const int g = threadIdx.x / 128;
    const uint64_t t0 = global_ns();
    ok = mbar_wait_ab(smem_u32(&bar[g]), 0, &abort_flag, limit_ns);
    waited[g] = int64_t(global_ns() - t0);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tslot), "r"(32));
  if (!ok) atomicOr(status, 1);
}

}  // namespace

int selftest_wait(Ctx& c, int64_t limit_ns, int64_t* waited_ns) {
  int64_t* d_w = nullptr;
  TETMF_CK(cudaMalloc(&d_w, 2 * sizeof(int64_t)));
  k_selftest_wait<<<1, 256>>>(uint64_t(limit_ns), c.d_status, d_w);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int64_t w[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(w, d_w, sizeof(w), cudaMemcpyDeviceToHost);
  cudaFree(d_w);
  if (e != cudaSuccess) {
    set_error("self-test kernel: %s", cudaGetErrorString(e));
    return FEM_ECUDA;
  }
  waited_ns[0] = w[0];
  waited_ns[1] = w[1];
  return FEM_OK;
}

}  // namespace tetmf
