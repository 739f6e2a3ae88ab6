// Poisson solve on the device: Jacobi-preconditioned CG (the smoother the paper
// pairs with its operator is Jacobi-based, Sec. 4.1) and mixed-precision
// iterative refinement (the paper runs its multigrid preconditioner in single
// precision and the outer CG in double precision, Sec. 4.1):
//
//   x (FP64); repeat:  r = b - A_64 x              FP64 apply + residual norm
//                      stop if ||r|| <= rtol ||b||
//                      r32 = r / ||r||             scaled, FP32
//                      solve A_32 d = r32 by Jacobi-PCG (FP32 vectors, FP32 or
//                      tensor-core apply, FP64 dot products) to inner_rtol
//                      x += ||r|| d                FP64 update
//
// FEM_SOLVE_IR_PMG replaces the inner Jacobi-PCG by flexible CG preconditioned by a p-multigrid
// V-cycle (pmg.cu).
//
// Every reduction is a single kernel: each block writes a partial sum to a
// scratch array, and the last block to finish (atomic ticket) adds the
// partials in block order, so results are deterministic.  Scalars (alpha,
// beta) stay on the device; the host reads one residual norm per iteration.
#include <chrono>
#include <cmath>

#include "blas.cuh"
#include "common.cuh"

namespace tetmf {
namespace {

constexpr int kCheck = 8;  // PCG iterations between residual checks on the host

// scalar slots in the solver's device scalar array
enum : int { S_PQ = 0, S_RZ0 = 1, S_RZ1 = 2, S_RR = 3, S_NORM = 4, S_RES = 5, S_COUNT = 8 };

struct Work {
  double* scal;          // [S_COUNT]
  double* partials;      // [kMaxRedBlocks][2]
  unsigned* ticket;      // [1]
  double* r64;           // [N]
  double* t64;           // [N]
  double* diag64;        // [N]
  double* p64;           // [N]   (FP64 PCG)
  double* z64;           // [N]
  void* r;               // [N] inner vectors, FP32
  void* z;
  void* p;
  void* q;
  void* d;
  float* diag32;
  double* host_scal;     // pinned host mirror
};

// A block of kCheck PCG iterations (apply, dot, update, direction each) captured once per solve
// into a CUDA graph and replayed with one launch per block: the host then enqueues one graph per
// residual check instead of about 6 kCheck kernels and their attribute queries, which is what the
// iterations cost at the smaller sizes.  kCheck is even, so the two alternating scalar slots of
// the recurrence line up from one block to the next.  A capture or instantiation that fails leaves
// the plain loop in charge.
struct PcgGraph {
  bool enabled = false;  // fem_solve: yes; fem_solve_noalloc: no (instantiating a graph may allocate)
  bool failed = false;
  cudaGraphExec_t exec = nullptr;
  ~PcgGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};
static_assert(kCheck % 2 == 0, "graph blocks must keep the scalar slots' parity");

// record what body(stream) enqueues into g.exec, on a private stream; on any failure g.failed
template <typename Body>
void capture_block(PcgGraph& g, Body body) {
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    g.failed = true;
    return;
  }
  cudaGraph_t graph = nullptr;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    const int body_status = body(cs);
    ok = cudaStreamEndCapture(cs, &graph) == cudaSuccess && body_status == FEM_OK && graph != nullptr;
  }
  if (ok) ok = cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (!ok) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.failed = true;
    cudaGetLastError();  // a failed capture leaves no error behind for later calls
  }
}





// r = b - Ax (FP64), scal[S_RR] = r . r
__global__ void __launch_bounds__(kBlock) k_residual64(const double* __restrict__ b, const double* __restrict__ ax,
                                                       double* __restrict__ r, int64_t n, double* partials,
                                                       unsigned* ticket, double* rr) {
  double s = 0.0;
  GRID_STRIDE(i, n) {
    const double v = b[i] - ax[i];
    r[i] = v;
    s = fma(v, v, s);
  }
  finish2(s, 0.0, partials, ticket, rr, nullptr);
}

// inner right-hand side r32 = r64 / ||r64||, inner iterate d = 0
__global__ void k_scale_down(const double* __restrict__ r64, const double* __restrict__ rr, float* __restrict__ r32,
                             float* __restrict__ d, int64_t n) {
  const double s = 1.0 / sqrt(*rr);
  GRID_STRIDE(i, n) {
    r32[i] = float(r64[i] * s);
    d[i] = 0.0f;
  }
}

// x += ||r64|| d
__global__ void k_correct(double* __restrict__ x, const float* __restrict__ d, const double* __restrict__ rr,
                          int64_t n) {
  const double s = sqrt(*rr);
  GRID_STRIDE(i, n) x[i] = fma(s, double(d[i]), x[i]);
}







// lay the solver's work arrays out from `base` (nullptr: only measure); returns the bytes used
size_t carve(uint8_t* base, int64_t N, Work& w) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    uint8_t* r = base ? base + off : nullptr;
    off += (bytes + 255) / 256 * 256;
    return r;
  };
  w.scal = reinterpret_cast<double*>(take(sizeof(double) * S_COUNT));
  w.partials = reinterpret_cast<double*>(take(sizeof(double) * 2 * kMaxRedBlocks));
  w.ticket = reinterpret_cast<unsigned*>(take(64));
  w.r64 = reinterpret_cast<double*>(take(sizeof(double) * N));
  w.t64 = reinterpret_cast<double*>(take(sizeof(double) * N));
  w.diag64 = reinterpret_cast<double*>(take(sizeof(double) * N));
  w.p64 = reinterpret_cast<double*>(take(sizeof(double) * N));
  w.z64 = reinterpret_cast<double*>(take(sizeof(double) * N));
  w.r = take(sizeof(float) * N);
  w.z = take(sizeof(float) * N);
  w.p = take(sizeof(float) * N);
  w.q = take(sizeof(float) * N);
  w.d = take(sizeof(float) * N);
  w.diag32 = reinterpret_cast<float*>(take(sizeof(float) * N));
  return off;
}

int ensure_work(Ctx& c, Work& w) {
  const int64_t N = c.ndofs;
  const size_t need = carve(nullptr, N, w);
  if (c.work_bytes < need) {
    void* p = nullptr;
    TETMF_CK(cudaMalloc(&p, need));
    c.allocations.push_back(p);
    c.d_work = p;
    c.work_bytes = need;
    TETMF_CK(cudaMemset(p, 0, need));
  }
  carve(static_cast<uint8_t*>(c.d_work), N, w);
  static thread_local double* pinned = nullptr;
  if (!pinned) TETMF_CK(cudaMallocHost(&pinned, sizeof(double) * S_COUNT));
  w.host_scal = pinned;
  return FEM_OK;
}

int read_scalar(const double* dev, double* host, double& out, cudaStream_t st) {
  TETMF_CK(cudaMemcpyAsync(host, dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  TETMF_CK(cudaStreamSynchronize(st));
  out = *host;
  return FEM_OK;
}

// Jacobi-PCG on vectors of type T with the operator `apply` (y = A x, apply(x, y, stream));
// solves A x = r starting from x = 0 (r is overwritten by the residual).  With g.enabled, whole
// blocks of kCheck iterations run as one graph launch.
template <typename T, typename Apply>
int pcg(const char* who, Ctx& c, Work& w, Apply apply, T* x, T* r, T* z, T* p, T* q, const T* diag,
        double rtol_abs2, int max_it, int& iters, cudaStream_t st, PcgGraph& g) {
  const int64_t N = c.ndofs;
  const int rg = red_grid(N), eg = ew_grid(N);
  k_pcg_start<T><<<rg, kBlock, 0, st>>>(r, diag, z, p, N, w.partials, w.ticket, w.scal + S_RZ0, w.scal + S_RR);
  TETMF_LAUNCH_CK();
  // iteration `it` of the recurrence on stream s
  auto iteration = [&](int it, cudaStream_t s) -> int {
    const int cur = S_RZ0 + (it & 1), nxt = S_RZ0 + ((it + 1) & 1);
    if (int e = apply(p, q, s)) return e;
    k_dot<T><<<rg, kBlock, 0, s>>>(p, q, N, w.partials, w.ticket, w.scal + S_PQ);
    TETMF_LAUNCH_CK();
    k_pcg_update<T><<<rg, kBlock, 0, s>>>(x, r, z, p, q, diag, N, w.scal + cur, w.scal + S_PQ, w.partials, w.ticket,
                                          w.scal + nxt, w.scal + S_RR);
    TETMF_LAUNCH_CK();
    k_pcg_direction<T><<<eg, kBlock, 0, s>>>(p, z, N, w.scal + nxt, w.scal + cur);
    TETMF_LAUNCH_CK();
    return FEM_OK;
  };
  double rr = 0.0;
  if (int e = read_scalar(w.scal + S_RR, w.host_scal, rr, st)) return e;
  iters = 0;
  while (rr > rtol_abs2 && iters < max_it) {
    if (g.enabled && !g.failed && iters % kCheck == 0 && iters + kCheck <= max_it) {
      if (!g.exec)
        capture_block(g, [&](cudaStream_t cs) -> int {
          for (int k = 0; k < kCheck; ++k)
            if (int e = iteration(k, cs)) return e;
          return FEM_OK;
        });
      if (g.exec) {
        TETMF_CK(cudaGraphLaunch(g.exec, st));
        iters += kCheck;
        if (int e = read_scalar(w.scal + S_RR, w.host_scal, rr, st)) return e;
        if (!std::isfinite(rr)) {
          set_error("%s: residual is not finite after %d iterations", who, iters);
          return FEM_ENOTCONV;
        }
        continue;
      }
    }
    if (int e = iteration(iters, st)) return e;
    ++iters;
    // the host reads the residual every kCheck iterations only (one synchronisation); the
    // iterations run past convergence keep reducing it (a zero denominator yields a zero step)
    if (iters % kCheck != 0 && iters < max_it) continue;
    if (int e = read_scalar(w.scal + S_RR, w.host_scal, rr, st)) return e;
    if (!std::isfinite(rr)) {
      set_error("%s: residual is not finite after %d iterations", who, iters);
      return FEM_ENOTCONV;
    }
  }
  return FEM_OK;
}

}  // namespace

// the solver proper, on work arrays laid out by carve()
// who: the entry point's name, for the error messages
// graphs: replay blocks of inner iterations as CUDA graphs (fem_solve; fem_solve_noalloc does not)
static int solve_with(const char* who, Ctx& c, Work& w, const fem_solve_opts* o, const double* b, double* x,
                      fem_solve_stats* stats, void* stream, bool graphs) {
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = as_stream(stream);
  const int64_t N = c.ndofs;
  const int rg = red_grid(N), eg = ew_grid(N);
  *stats = fem_solve_stats{0, 0, 0.0, 0.0};
  auto finish = [&](int status, double rel) {
    stats->rel_residual = rel;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (status == FEM_ENOTCONV)
      set_error("%s: relative residual %.3e above rtol %.3e after %d outer / %d inner iterations", who, rel,
                o->rtol, stats->outer_iterations, stats->inner_iterations);
    return status;
  };

  double bb = 0.0;
  k_dot<double><<<rg, kBlock, 0, st>>>(b, b, N, w.partials, w.ticket, w.scal + S_NORM);
  TETMF_LAUNCH_CK();
  if (int e = read_scalar(w.scal + S_NORM, w.host_scal, bb, st)) return e;
  if (bb == 0.0) {
    TETMF_CK(cudaMemsetAsync(x, 0, sizeof(double) * N, st));
    TETMF_CK(cudaStreamSynchronize(st));
    return finish(FEM_OK, 0.0);
  }
  if (int e = cg_diagonal(c, FEM_FP64, w.diag64, nullptr, stream)) return e;

  // r64 = b - A_64 x, ||r64||^2 in scal[S_RES]; rel = ||r64|| / ||b||
  auto residual = [&](double& rel) -> int {
    if (int e = cg_apply_simt(c, FEM_FP64, x, w.t64, nullptr, false, stream)) return e;
    k_residual64<<<rg, kBlock, 0, st>>>(b, w.t64, w.r64, N, w.partials, w.ticket, w.scal + S_RES);
    TETMF_LAUNCH_CK();
    double rr = 0.0;
    if (int e = read_scalar(w.scal + S_RES, w.host_scal, rr, st)) return e;
    rel = std::sqrt(rr / bb);
    return FEM_OK;
  };

  double rel = 0.0;
  if (o->mode == FEM_SOLVE_FP64_PCG) {
    if (int e = residual(rel)) return e;
    auto apply64 = [&](double* in, double* out, cudaStream_t s) {
      return cg_apply_simt(c, FEM_FP64, in, out, nullptr, false, s);
    };
    PcgGraph g;
    g.enabled = graphs;
    // PCG stops on its recurrence residual; the true residual b - A x is then recomputed, and where
    // rounding has left it above the tolerance PCG restarts from x with it (at most 8 restarts,
    // within the same iteration cap)
    int total = 0;
    for (int pass = 0;; ++pass) {
      int it = 0;
      const int e = pcg<double>(who, c, w, apply64, x, w.r64, w.z64, w.p64, w.t64, w.diag64, o->rtol * o->rtol * bb,
                                o->max_inner - total, it, st, g);
      total += it;
      stats->inner_iterations = total;
      stats->outer_iterations = pass + 1;
      if (e && e != FEM_ENOTCONV) return e;
      if (int e2 = residual(rel)) return e2;
      if (rel <= o->rtol || e == FEM_ENOTCONV || total >= o->max_inner || pass >= 8 || !std::isfinite(rel)) break;
    }
    return finish(rel <= o->rtol ? FEM_OK : FEM_ENOTCONV, rel);
  }

  // mixed-precision iterative refinement
  k_cast<float><<<eg, kBlock, 0, st>>>(w.diag64, w.diag32, N);
  TETMF_LAUNCH_CK();
  float* r32 = static_cast<float*>(w.r);
  float* z32 = static_cast<float*>(w.z);
  float* p32 = static_cast<float*>(w.p);
  float* q32 = static_cast<float*>(w.q);
  float* d32 = static_cast<float*>(w.d);
  const int ip = o->inner_prec;
  auto apply32 = [&](float* in, float* out, cudaStream_t s) {
    return ip == FEM_FP32 ? cg_apply_simt(c, FEM_FP32, in, out, nullptr, false, s)
                          : cg_apply_tc(c, ip, in, out, nullptr, s);
  };
  PcgGraph g;
  g.enabled = graphs;
  const double inner = o->inner_rtol > 0 ? o->inner_rtol : 1e-3;
  const bool pmg = o->mode == FEM_SOLVE_IR_PMG;
  if (pmg)
    if (int e = pmg_setup(c, ip, w.diag32, o->smoother_degree, o->coarse_steps, stream)) return e;
  for (;;) {
    if (int e = residual(rel)) return e;
    if (rel <= o->rtol) return finish(FEM_OK, rel);
    if (stats->outer_iterations >= o->max_outer) return finish(FEM_ENOTCONV, rel);
    if (!std::isfinite(rel)) return finish(FEM_ENOTCONV, rel);
    k_scale_down<<<eg, kBlock, 0, st>>>(w.r64, w.scal + S_RES, r32, d32, N);
    TETMF_LAUNCH_CK();
    int it = 0;
    const int e = pmg ? pmg_inner_solve(c, w.diag32, r32, d32, p32, q32, inner, o->max_inner, it, stream)
                      : pcg<float>(who, c, w, apply32, d32, r32, z32, p32, q32, w.diag32, inner * inner, o->max_inner, it,
                                   st, g);
    stats->inner_iterations += it;
    stats->outer_iterations += 1;
    if (e && e != FEM_ENOTCONV) return e;
    k_correct<<<eg, kBlock, 0, st>>>(x, d32, w.scal + S_RES, N);
    TETMF_LAUNCH_CK();
  }
}

int solve(Ctx& c, const fem_solve_opts* o, const double* b, double* x, fem_solve_stats* stats, void* stream) {
  Work w;
  if (int e = ensure_work(c, w)) return e;
  return solve_with("fem_solve", c, w, o, b, x, stats, stream, true);
}

}  // namespace tetmf

// ---- allocation-free solve ---------------------------------------------
//
// Some callers cannot let a library call cudaMalloc: an application whose
// memory manager owns all device memory up front (a framework caching
// allocator, a fixed per-process budget), or one on a path that must not stall,
// since cudaMalloc/cudaFree can synchronise the device.  fem_solve_noalloc runs
// the same solver as fem_solve, but its work space (reduction partials and
// scalars, the FP64 and FP32 PCG vectors) lives in one file-scope device array
// of a fixed size instead of a buffer the context allocates on first use.
// That array is reserved on every GPU where this library's device code is
// loaded, for the life of the process.  Every call shares it: two calls that
// run on the GPU at the same time (other streams, other threads, other
// contexts) race on it, so the caller must serialise them.

namespace tetmf {
namespace {

constexpr int64_t kNoAllocMaxDofs = FEM_SOLVE_NOALLOC_MAX_DOFS;
constexpr size_t kNoAllocBytes = size_t(kNoAllocMaxDofs) * 64 + (64 << 10);
static_assert(5 * 8 + 6 * 4 == 64, "per-DoF work bytes");

static __device__ __align__(256) unsigned char g_noalloc_work[kNoAllocBytes];

void* g_noalloc_addr[64] = {nullptr};

// device address of g_noalloc_work for this context, looked up by the context's first
// fem_solve_noalloc call with the context's device current.  Keeping it per context (not per
// device ordinal) means a context created after a device reset looks the address up again.
int noalloc_address(Ctx& c, void** out) {
  if (!c.noalloc_work) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_work);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("fem_solve_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return FEM_ECUDA;
    }
    c.noalloc_work = p;
  }
  *out = c.noalloc_work;
  return FEM_OK;
}

}  // namespace
}  // namespace tetmf

extern "C" int fem_solve_noalloc(fem_ctx* ctx, const fem_solve_opts* opts, const double* b, double* x,
                                 fem_solve_stats* stats, void* stream) {
  using namespace tetmf;
  // the checks every device entry point makes: a context on a device, and that device current
  if (int s = check_device(ctx)) return s;
  if (!opts || !b || !x || !stats || (const void*)b == (const void*)x) {
    set_error("fem_solve_noalloc: null or aliased argument");
    return FEM_EINVAL;
  }
  Ctx& c = ctx->c;
  if (c.kind != FEM_CG) {
    set_error("fem_solve_noalloc: CG spaces only");
    return FEM_EINVAL;
  }
  if (opts->mode == FEM_SOLVE_IR_PMG) {
    set_error("fem_solve_noalloc: the p-multigrid hierarchy is allocated; use fem_solve");
    return FEM_EUNSUPPORTED;
  }
  if (opts->mode != FEM_SOLVE_FP64_PCG && opts->mode != FEM_SOLVE_IR_MIXED) {
    set_error("fem_solve_noalloc: bad mode");
    return FEM_EINVAL;
  }
  if (opts->mode == FEM_SOLVE_IR_MIXED && opts->inner_prec != FEM_FP32 && opts->inner_prec != FEM_TF32 &&
      opts->inner_prec != FEM_BF16 && opts->inner_prec != FEM_TF32X3) {
    set_error("fem_solve_noalloc: inner_prec must be FEM_FP32, FEM_TF32, FEM_BF16 or FEM_TF32X3");
    return FEM_EUNSUPPORTED;
  }
  if (!(opts->rtol > 0) || opts->max_inner < 1 || opts->max_outer < 1) {
    set_error("fem_solve_noalloc: need rtol > 0, max_inner >= 1, max_outer >= 1");
    return FEM_EINVAL;
  }
  Work w;
  const size_t need = carve(nullptr, c.ndofs, w);
  if (c.ndofs > kNoAllocMaxDofs || need > kNoAllocBytes) {
    set_error("fem_solve_noalloc: %lld DoFs exceed the static work space (at most %lld DoFs); use fem_solve",
              (long long)c.ndofs, (long long)kNoAllocMaxDofs);
    return FEM_EINVAL;
  }
  void* base = nullptr;
  if (int e = noalloc_address(c, &base)) return e;
  carve(static_cast<uint8_t*>(base), c.ndofs, w);
  // the reduction ticket must start at zero; every other array is written before it is read
  TETMF_CK(cudaMemsetAsync(w.ticket, 0, 64, as_stream(stream)));
  static thread_local double host_scal[S_COUNT];
  w.host_scal = host_scal;
  return solve_with("fem_solve_noalloc", c, w, opts, b, x, stats, stream, false);
}
