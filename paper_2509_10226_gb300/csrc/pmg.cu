// p-multigrid preconditioner for the inner solve of the mixed-precision refinement: a two-level
// V-cycle over the polynomial degree (the p-levels of the paper's hybrid multigrid, Sec. 4.1),
// fine level = the context's space, coarse level = linear elements on the same mesh.
//
//   V(r):  z = Chebyshev-Jacobi(A, r, 0)            `degree` steps, fine level
//          r_c = P^T (r - A z)                      restriction
//          e_c = Jacobi-PCG(A_c, r_c), fixed steps  coarse level, scalars on the device
//          z += P e_c                               prolongation
//          z = Chebyshev-Jacobi(A, r, z)            post-smoothing
//
// The fixed-step coarse CG makes V(r) depend nonlinearly on r, so the fine iteration is the
// flexible CG variant (beta from r_{k+1} . (z_{k+1} - z_k)).  All vectors are FP32 with FP64
// reductions; the fine applies run in the inner precision, the coarse ones on the FP32 units.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "blas.cuh"
#include "common.cuh"

namespace tetmf {

struct Pmg {
  fem_ctx* coarse = nullptr;
  Transfer* tr = nullptr;
  int prec = -1;       // inner precision of the fine applies
  double lam = 0.0;    // safety factor x lambda_max of D^-1 A on the fine level
  int degree = 5, coarse_steps = 20;
  void* mem = nullptr;
  float *zn = nullptr, *zo = nullptr, *t = nullptr, *cw = nullptr;
  float *xc = nullptr, *rc = nullptr, *zc = nullptr, *pc = nullptr, *qc = nullptr, *dc = nullptr;
  double *scal = nullptr, *partials = nullptr;
  unsigned* ticket = nullptr;
  double* host = nullptr;  // pinned, 4 doubles
};

namespace {

enum : int { P_PQ = 0, P_RZ0 = 1, P_RZ1 = 2, P_RR = 3, P_A = 4, P_B = 5, P_COUNT = 8 };

// out0 = a . b, out1 = c . d (FP64 sums)
__global__ void __launch_bounds__(kBlock) k_dot2(const float* __restrict__ a, const float* __restrict__ b,
                                                 const float* __restrict__ c, const float* __restrict__ d, int64_t n,
                                                 double* partials, unsigned* ticket, double* out0, double* out1) {
  double s0 = 0.0, s1 = 0.0;
  GRID_STRIDE(i, n) {
    s0 = fma(double(a[i]), double(b[i]), s0);
    s1 = fma(double(c[i]), double(d[i]), s1);
  }
  finish2(s0, s1, partials, ticket, out0, out1);
}

// x += alpha p; r -= alpha q; out = r . r
__global__ void __launch_bounds__(kBlock) k_fcg_update(float* __restrict__ x, float* __restrict__ r,
                                                       const float* __restrict__ p, const float* __restrict__ q,
                                                       float alpha, int64_t n, double* partials, unsigned* ticket,
                                                       double* rr) {
  double s = 0.0;
  GRID_STRIDE(i, n) {
    x[i] = fmaf(alpha, p[i], x[i]);
    const float ri = fmaf(-alpha, q[i], r[i]);
    r[i] = ri;
    s = fma(double(ri), double(ri), s);
  }
  finish2(s, 0.0, partials, ticket, rr, nullptr);
}

// p = z + beta p
__global__ void k_xpby(float* __restrict__ p, const float* __restrict__ z, float beta, int64_t n) {
  GRID_STRIDE(i, n) p[i] = fmaf(beta, p[i], z[i]);
}

// t = r - t
__global__ void k_rsub(float* __restrict__ t, const float* __restrict__ r, int64_t n) {
  GRID_STRIDE(i, n) t[i] = r[i] - t[i];
}

// z += e
__global__ void k_add(float* __restrict__ z, const float* __restrict__ e, int64_t n) {
  GRID_STRIDE(i, n) z[i] += e[i];
}

size_t al(size_t b) { return (b + 255) / 256 * 256; }

int read2(Pmg& m, const double* dev, double& a, double& b, cudaStream_t st) {
  TETMF_CK(cudaMemcpyAsync(m.host, dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  TETMF_CK(cudaStreamSynchronize(st));
  a = m.host[0];
  b = m.host[1];
  return FEM_OK;
}

int fine_apply(Ctx& c, int prec, const float* in, float* out, cudaStream_t st) {
  return prec == FEM_FP32 ? cg_apply_simt(c, FEM_FP32, in, out, nullptr, false, st)
                          : cg_apply_tc(c, prec, in, out, nullptr, st);
}

// z = V(r) (r is not modified)
int vcycle(Ctx& c, Pmg& m, const float* r, float* z, const float* diag, cudaStream_t st) {
  Ctx& cc = m.coarse->c;
  const int64_t N = c.ndofs, Nc = cc.ndofs;
  TETMF_CK(cudaMemsetAsync(z, 0, sizeof(float) * N, st));
  if (int e = chebyshev(c, m.prec, r, z, diag, m.degree, m.lam, m.lam / 15.0, m.cw, st)) return e;
  if (int e = fine_apply(c, m.prec, z, m.t, st)) return e;
  k_rsub<<<ew_grid(N), kBlock, 0, st>>>(m.t, r, N);
  TETMF_LAUNCH_CK();
  if (int e = transfer_apply(*m.tr, FEM_FP32, false, m.t, m.rc, st)) return e;
  // coarse Jacobi-PCG from x = 0, a fixed number of steps, scalars on the device
  TETMF_CK(cudaMemsetAsync(m.xc, 0, sizeof(float) * Nc, st));
  const int rg = red_grid(Nc), eg = ew_grid(Nc);
  k_pcg_start<float><<<rg, kBlock, 0, st>>>(m.rc, m.dc, m.zc, m.pc, Nc, m.partials, m.ticket, m.scal + P_RZ0,
                                            m.scal + P_RR);
  TETMF_LAUNCH_CK();
  for (int k = 0; k < m.coarse_steps; ++k) {
    const int cur = P_RZ0 + (k & 1), nxt = P_RZ0 + ((k + 1) & 1);
    if (int e = cg_apply_simt(cc, FEM_FP32, m.pc, m.qc, nullptr, false, st)) return e;
    k_dot<float><<<rg, kBlock, 0, st>>>(m.pc, m.qc, Nc, m.partials, m.ticket, m.scal + P_PQ);
    TETMF_LAUNCH_CK();
    k_pcg_update<float><<<rg, kBlock, 0, st>>>(m.xc, m.rc, m.zc, m.pc, m.qc, m.dc, Nc, m.scal + cur, m.scal + P_PQ,
                                               m.partials, m.ticket, m.scal + nxt, m.scal + P_RR);
    TETMF_LAUNCH_CK();
    k_pcg_direction<float><<<eg, kBlock, 0, st>>>(m.pc, m.zc, Nc, m.scal + nxt, m.scal + cur);
    TETMF_LAUNCH_CK();
  }
  if (int e = transfer_apply(*m.tr, FEM_FP32, true, m.xc, m.t, st)) return e;
  k_add<<<ew_grid(N), kBlock, 0, st>>>(z, m.t, N);
  TETMF_LAUNCH_CK();
  return chebyshev(c, m.prec, r, z, diag, m.degree, m.lam, m.lam / 15.0, m.cw, st);
}

}  // namespace

void pmg_release(Ctx& c) {
  Pmg* m = static_cast<Pmg*>(c.pmg);
  if (!m) return;
  if (m->tr) transfer_destroy(m->tr);
  if (m->coarse) fem_destroy(m->coarse);
  if (m->mem) cudaFree(m->mem);
  if (m->host) cudaFreeHost(m->host);
  delete m;
  c.pmg = nullptr;
}

int pmg_setup(Ctx& c, int prec, const float* diag, int degree, int coarse_steps, void* stream) {
  cudaStream_t st = as_stream(stream);
  if (c.p < 2) return set_error("p-multigrid needs degree >= 2 (the coarse level is linear)"), FEM_EUNSUPPORTED;
  if (c.curved || !c.colour_start.empty())
    return set_error("p-multigrid: straight cells and atomic scatter only"), FEM_EUNSUPPORTED;
  Pmg* m = static_cast<Pmg*>(c.pmg);
  if (!m) {
    m = new (std::nothrow) Pmg;
    if (!m) return set_error("p-multigrid: out of host memory"), FEM_ENOMEM;
    c.pmg = m;
    fem_mesh_desc md{c.nv, c.xyz.data(), c.nc, c.ucells.data(), nullptr};
    fem_space_desc sd{};
    sd.kind = FEM_CG;
    sd.degree = 1;
    sd.dirichlet = c.dirichlet;
    sd.reorder = c.reorder;
    sd.device = c.device;
    if (int s = fem_create(&md, &sd, &m->coarse)) return s;
    if (int s = transfer_create(c, m->coarse->c, &m->tr)) return s;
    const int64_t N = c.ndofs, Nc = m->coarse->c.ndofs;
    const size_t vf = al(sizeof(float) * N), vc = al(sizeof(float) * Nc);
    const size_t cheb = lambda_max_work_bytes(c, FEM_FP32);
    const size_t bytes = 3 * vf + al(cheb) + 6 * vc + al(sizeof(double) * P_COUNT) +
                         al(sizeof(double) * 2 * kMaxRedBlocks) + 256;
    TETMF_CK(cudaMalloc(&m->mem, bytes));
    TETMF_CK(cudaMemset(m->mem, 0, bytes));
    uint8_t* p = static_cast<uint8_t*>(m->mem);
    auto take = [&](size_t b) {
      uint8_t* r = p;
      p += al(b);
      return r;
    };
    m->zn = reinterpret_cast<float*>(take(sizeof(float) * N));
    m->zo = reinterpret_cast<float*>(take(sizeof(float) * N));
    m->t = reinterpret_cast<float*>(take(sizeof(float) * N));
    m->cw = reinterpret_cast<float*>(take(cheb));
    m->xc = reinterpret_cast<float*>(take(sizeof(float) * Nc));
    m->rc = reinterpret_cast<float*>(take(sizeof(float) * Nc));
    m->zc = reinterpret_cast<float*>(take(sizeof(float) * Nc));
    m->pc = reinterpret_cast<float*>(take(sizeof(float) * Nc));
    m->qc = reinterpret_cast<float*>(take(sizeof(float) * Nc));
    m->dc = reinterpret_cast<float*>(take(sizeof(float) * Nc));
    m->scal = reinterpret_cast<double*>(take(sizeof(double) * P_COUNT));
    m->partials = reinterpret_cast<double*>(take(sizeof(double) * 2 * kMaxRedBlocks));
    m->ticket = reinterpret_cast<unsigned*>(take(64));
    TETMF_CK(cudaMallocHost(&m->host, 4 * sizeof(double)));
    if (int s = cg_diagonal(m->coarse->c, FEM_FP32, m->dc, nullptr, st)) return s;
  }
  m->degree = degree > 0 ? degree : 5;
  m->coarse_steps = coarse_steps > 0 ? coarse_steps : 20;
  if (m->prec != prec) {
    // largest eigenvalue of D^-1 A on the fine level, 12 power steps from a fixed vector, times 1.2
    const int64_t N = c.ndofs;
    std::vector<float> v0(N);
    for (int64_t i = 0; i < N; ++i) v0[i] = 1.0f + 0.5f * float((i * 7919) % 13) / 13.0f;
    TETMF_CK(cudaMemcpyAsync(m->zo, v0.data(), sizeof(float) * N, cudaMemcpyHostToDevice, st));
    double lam = 0.0;
    if (int s = lambda_max(c, prec, diag, m->zo, 12, m->cw, &lam, st)) return s;
    m->lam = 1.2 * lam;
    m->prec = prec;
  }
  return FEM_OK;
}

// flexible CG for A d = r (d = 0 on entry), preconditioned by V; r is overwritten by the residual
int pmg_inner_solve(Ctx& c, const float* diag, float* r, float* d, float* p, float* q, double rtol, int max_it,
                    int& iters, void* stream) {
  cudaStream_t st = as_stream(stream);
  Pmg& m = *static_cast<Pmg*>(c.pmg);
  const int64_t N = c.ndofs;
  const int rg = red_grid(N), eg = ew_grid(N);
  float* zo = m.zo;
  float* zn = m.zn;
  if (int e = vcycle(c, m, r, zo, diag, st)) return e;
  TETMF_CK(cudaMemcpyAsync(p, zo, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
  k_dot2<<<rg, kBlock, 0, st>>>(r, zo, r, r, N, m.partials, m.ticket, m.scal + P_A, m.scal + P_B);
  TETMF_LAUNCH_CK();
  double rz = 0.0, rr0 = 0.0;
  if (int e = read2(m, m.scal + P_A, rz, rr0, st)) return e;
  iters = 0;
  const double tol2 = rtol * rtol * rr0;
  while (iters < max_it) {
    if (int e = fine_apply(c, m.prec, p, q, st)) return e;
    k_dot<float><<<rg, kBlock, 0, st>>>(p, q, N, m.partials, m.ticket, m.scal + P_A);
    TETMF_LAUNCH_CK();
    double pq = 0.0, dummy = 0.0;
    if (int e = read2(m, m.scal + P_A, pq, dummy, st)) return e;
    const float alpha = pq != 0.0 ? float(rz / pq) : 0.0f;
    k_fcg_update<<<rg, kBlock, 0, st>>>(d, r, p, q, alpha, N, m.partials, m.ticket, m.scal + P_A);
    TETMF_LAUNCH_CK();
    double rr = 0.0;
    if (int e = read2(m, m.scal + P_A, rr, dummy, st)) return e;
    ++iters;
    if (!std::isfinite(rr)) {
      set_error("fem_solve: residual is not finite after %d p-multigrid iterations", iters);
      return FEM_ENOTCONV;
    }
    if (rr <= tol2) break;
    if (int e = vcycle(c, m, r, zn, diag, st)) return e;
    k_dot2<<<rg, kBlock, 0, st>>>(r, zn, r, zo, N, m.partials, m.ticket, m.scal + P_A, m.scal + P_B);
    TETMF_LAUNCH_CK();
    double rz_new = 0.0, rzo = 0.0;
    if (int e = read2(m, m.scal + P_A, rz_new, rzo, st)) return e;
    const float beta = rz != 0.0 ? float((rz_new - rzo) / rz) : 0.0f;
    k_xpby<<<eg, kBlock, 0, st>>>(p, zn, beta, N);
    TETMF_LAUNCH_CK();
    std::swap(zn, zo);
    rz = rz_new;
  }
  return FEM_OK;
}

}  // namespace tetmf
