// Host-buffer apply: a sequence of host vectors y_b = A u_b streamed through the device.
//
// The operator is the one of fem_apply (Eq. 3 for CG, Eq. 5 for DG, no coefficient); this file
// only moves data.  Two device input and two device output buffers owned by the context take
// vector b in slot b % 2, and three streams of the context overlap the copy of vector b + 1 in,
// the apply of vector b and the copy of vector b - 1 out:
//   in  stream: [wait: apply of b - 2 has read u slot]  u_host[b] -> u slot       record in[b % 2]
//   cmp stream: [wait in[b % 2], copy-out of b - 2 has read y slot]  apply      record cmp[b % 2]
//   out stream: [wait cmp[b % 2]]  y slot -> y_host[b]                          record out[b % 2]
// Host-to-device and device-to-host copies use separate copy engines, so in steady state the two
// directions of the host link and the SMs are busy at the same time.
#include <cuda_runtime.h>

#include "common.cuh"

namespace tetmf {
namespace {

struct HostPipe {
  size_t bytes = 0;  // capacity of each slot
  void* d_u[2] = {nullptr, nullptr};
  void* d_y[2] = {nullptr, nullptr};
  cudaStream_t s_in = nullptr, s_cmp = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_cmp[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
};

void pipe_free(HostPipe* p) {
  if (!p) return;
  for (cudaStream_t s : {p->s_in, p->s_cmp, p->s_out})
    if (s) cudaStreamSynchronize(s);
  for (int i = 0; i < 2; ++i) {
    for (cudaEvent_t e : {p->ev_in[i], p->ev_cmp[i], p->ev_out[i]})
      if (e) cudaEventDestroy(e);
    if (p->d_u[i]) cudaFree(p->d_u[i]);
    if (p->d_y[i]) cudaFree(p->d_y[i]);
  }
  for (cudaStream_t s : {p->s_in, p->s_cmp, p->s_out})
    if (s) cudaStreamDestroy(s);
  cudaGetLastError();
  delete p;
}

int pipe_create(size_t bytes, HostPipe** out) {
  HostPipe* p = new HostPipe;
  p->bytes = bytes;
  auto fail = [&](cudaError_t e, const char* what) {
    set_error("%s failed: %s", what, cudaGetErrorString(e));
    pipe_free(p);
    return e == cudaErrorMemoryAllocation ? FEM_ENOMEM : FEM_ECUDA;
  };
  cudaError_t e;
  for (int i = 0; i < 2; ++i) {
    if ((e = cudaMalloc(&p->d_u[i], bytes)) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&p->d_y[i], bytes)) != cudaSuccess) return fail(e, "cudaMalloc");
    for (cudaEvent_t* ev : {&p->ev_in[i], &p->ev_cmp[i], &p->ev_out[i]})
      if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
        return fail(e, "cudaEventCreateWithFlags");
  }
  for (cudaStream_t* s : {&p->s_in, &p->s_cmp, &p->s_out})
    if ((e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking)) != cudaSuccess)
      return fail(e, "cudaStreamCreateWithFlags");
  *out = p;
  return FEM_OK;
}

}  // namespace

int apply_host(Ctx& c, int prec, int64_t nvec, const void* const* u_host, void* const* y_host) {
  const size_t bytes = size_t(c.ndofs) * (prec == FEM_FP64 ? sizeof(double) : sizeof(float));
  HostPipe* p = static_cast<HostPipe*>(c.host_pipe);
  if (p && p->bytes < bytes) {  // FP64 after a narrower precision: larger slots
    pipe_free(p);
    c.host_pipe = p = nullptr;
  }
  if (!p) {
    if (int s = pipe_create(bytes, &p)) return s;
    c.host_pipe = p;
  }
  for (int64_t b = 0; b < nvec; ++b) {
    const int i = int(b & 1);
    // slot i was last used by vector b - 2: its apply must have read u, its copy-out read y
    if (b >= 2) TETMF_CK(cudaStreamWaitEvent(p->s_in, p->ev_cmp[i], 0));
    TETMF_CK(cudaMemcpyAsync(p->d_u[i], u_host[b], bytes, cudaMemcpyHostToDevice, p->s_in));
    TETMF_CK(cudaEventRecord(p->ev_in[i], p->s_in));
    TETMF_CK(cudaStreamWaitEvent(p->s_cmp, p->ev_in[i], 0));
    if (b >= 2) TETMF_CK(cudaStreamWaitEvent(p->s_cmp, p->ev_out[i], 0));
    if (int s = apply_op(c, prec, p->d_u[i], p->d_y[i], p->s_cmp)) {
      cudaStreamSynchronize(p->s_in);
      cudaStreamSynchronize(p->s_out);
      return s;
    }
    TETMF_CK(cudaEventRecord(p->ev_cmp[i], p->s_cmp));
    TETMF_CK(cudaStreamWaitEvent(p->s_out, p->ev_cmp[i], 0));
    TETMF_CK(cudaMemcpyAsync(y_host[b], p->d_y[i], bytes, cudaMemcpyDeviceToHost, p->s_out));
    TETMF_CK(cudaEventRecord(p->ev_out[i], p->s_out));
  }
  // the last copy-out follows every earlier copy and apply of this call
  TETMF_CK(cudaStreamSynchronize(p->s_out));
  return FEM_OK;
}

void host_pipe_release(Ctx& c) {
  pipe_free(static_cast<HostPipe*>(c.host_pipe));
  c.host_pipe = nullptr;
}

}  // namespace tetmf
