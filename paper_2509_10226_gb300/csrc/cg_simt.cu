// Continuous-Galerkin cell kernels on the FP64 / FP32 FMA units (SIMT).
//
// One thread per cell, one 128-thread CTA per tile of 128 Morton-ordered
// cells: the "inter-element vectorisation" of Sec. 2.4 mapped onto the lanes
// of a warp.  The reference tables E (Eq. 4) and the quadrature weights live
// in shared memory and are read by broadcast (every lane reads the same
// entry: the "broadcast data structures" of Sec. 2.4).  Per quadrature point
// q a thread forms g = E_q u_e (3 nd FMAs), applies D_e as
// t = w_q k_q M_e g with the symmetric metric M_e = |det J| J^-1 J^-T, and
// accumulates y_e += E_q^T t (3 nd FMAs); the gather G_e skips constrained
// DoFs and the scatter G_e^T adds with atomics (Eq. 3).
#include <type_traits>

#include "common.cuh"

namespace tetmf {
namespace {

constexpr int kT = kTile;

__host__ __device__ constexpr int kstride(int nq) { return nq | 1; }  // odd stride: conflict-free rows

template <typename T>
struct Shared {
  T* E;
  T* w;
  T* V;
  T* k;   // [kT][kstride(nq)] coefficient tile (or null)
  T* dk;  // [kT][kstride(nq)] output tile of the coefficient gradient (or null)
};

template <int ND, int NQ, typename T>
__device__ inline Shared<T> load_tables(unsigned char* raw, const T* __restrict__ tabE, const T* __restrict__ tabW,
                                        const T* __restrict__ tabV, bool want_v, bool want_k, bool want_dk) {
  Shared<T> s;
  T* p = reinterpret_cast<T*>(raw);
  s.E = p;
  p += NQ * 3 * ND;
  s.w = p;
  p += NQ;
  s.V = want_v ? p : nullptr;
  if (want_v) p += NQ * ND;
  s.k = want_k ? p : nullptr;
  if (want_k) p += kT * kstride(NQ);
  s.dk = want_dk ? p : nullptr;
  for (int i = threadIdx.x; i < NQ * 3 * ND; i += blockDim.x) s.E[i] = tabE[i];
  for (int i = threadIdx.x; i < NQ; i += blockDim.x) s.w[i] = tabW[i];
  if (want_v)
    for (int i = threadIdx.x; i < NQ * ND; i += blockDim.x) s.V[i] = tabV[i];
  return s;
}

template <int NQ, typename T>
__device__ inline void load_coeff_tile(T* sk, const T* __restrict__ k, int64_t cell0, int64_t nc) {
  const int64_t ncell = nc - cell0 < kT ? nc - cell0 : kT;
  const int64_t n = ncell * NQ;
  const T* src = k + cell0 * NQ;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int c = int(i / NQ), q = int(i % NQ);
    sk[c * kstride(NQ) + q] = src[i];
  }
}

template <int ND, typename T>
__device__ inline void gather(const int32_t* __restrict__ idx, const T* __restrict__ u, int64_t tile, int lane,
                              int (&g)[ND], T (&ue)[ND]) {
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    g[j] = __ldg(idx + (tile * ND + j) * kT + lane);
    ue[j] = g[j] >= 0 ? __ldg(u + g[j]) : T(0);
  }
}

// y = A(k) u, Eq. 3.  The adjoint A(k)^T g is the same chain with D_e^T; the
// stored metric is symmetric, so D_e^T = D_e and the same kernel serves both.
// COLOUR: the launch covers the cells [lo, hi) of one colour (tiles from lo / 128 on), no two
// of which share a DoF, and adds to y without atomics.
// qmetric (curved cells, or null): [tiles][NQ][6][kT] metric per quadrature point instead of per cell.
// ncomp > 1: the components-batched vector Laplacian (Sec. 2.4, Sec. 3.1): ncomp independent
// components u + c * cstride share the indices, the metric and the tables of the cell, loaded once.
template <int ND, int NQ, typename T, bool COLOUR, bool VEC>
__global__ void __launch_bounds__(kT) k_cg_apply(const int32_t* __restrict__ idx, const T* __restrict__ metric,
                                                 const T* __restrict__ tabE, const T* __restrict__ tabW,
                                                 const T* __restrict__ u, T* __restrict__ y,
                                                 const T* __restrict__ kcoef, int64_t nc, int64_t lo, int64_t hi,
                                                 const T* __restrict__ qmetric, int ncomp, int64_t cstride) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Shared<T> s = load_tables<ND, NQ, T>(smem, tabE, tabW, nullptr, false, kcoef != nullptr, false);
  const int64_t tile = (COLOUR ? lo / kT : 0) + blockIdx.x;
  const int64_t cell0 = tile * kT;
  if (kcoef) load_coeff_tile<NQ, T>(s.k, kcoef, cell0, nc);
  __syncthreads();
  const int lane = threadIdx.x;
  if (cell0 + lane >= nc) return;
  if (COLOUR && (cell0 + lane < lo || cell0 + lane >= hi)) return;

  int g[ND];
  T ue[ND], ye[ND];
  gather<ND, T>(idx, u, tile, lane, g, ue);
  const T* mp = metric + tile * 6 * kT + lane;
  T m0 = mp[0], m1 = mp[kT], m2 = mp[2 * kT], m3 = mp[3 * kT], m4 = mp[4 * kT], m5 = mp[5 * kT];
  const T* qm = qmetric ? qmetric + tile * NQ * 6 * kT + lane : nullptr;

#pragma unroll 1
  for (int comp = 0; comp < (VEC ? ncomp : 1); ++comp) {
    T* yc = y + comp * cstride;
    if (VEC && comp > 0) {
      const T* uc = u + comp * cstride;
#pragma unroll
      for (int j = 0; j < ND; ++j) ue[j] = g[j] >= 0 ? __ldg(uc + g[j]) : T(0);
    }
#pragma unroll
    for (int j = 0; j < ND; ++j) ye[j] = T(0);
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
      if (qm) {
        const T* p = qm + q * 6 * kT;
        m0 = p[0], m1 = p[kT], m2 = p[2 * kT], m3 = p[3 * kT], m4 = p[4 * kT], m5 = p[5 * kT];
      }
      const T* Eq = s.E + q * 3 * ND;
      T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        gx = fma(Eq[j], ue[j], gx);
        gy = fma(Eq[ND + j], ue[j], gy);
        gz = fma(Eq[2 * ND + j], ue[j], gz);
      }
      T c = s.w[q];
      if (kcoef) c *= s.k[lane * kstride(NQ) + q];
      const T tx = c * fma(m0, gx, fma(m1, gy, m2 * gz));
      const T ty = c * fma(m1, gx, fma(m3, gy, m4 * gz));
      const T tz = c * fma(m2, gx, fma(m4, gy, m5 * gz));
#pragma unroll
      for (int j = 0; j < ND; ++j) ye[j] = fma(Eq[j], tx, fma(Eq[ND + j], ty, fma(Eq[2 * ND + j], tz, ye[j])));
    }
#pragma unroll
    for (int j = 0; j < ND; ++j)
      if (g[j] >= 0) {
        if constexpr (COLOUR) yc[g[j]] += ye[j];
        else atomicAdd(yc + g[j], ye[j]);
      }
  }  // components
}

// Backward of L = <g, A(k) u>: grad_u = A(k)^T g and dk_{e,q} = w_q gu^T M_e gg
// (= w_q |det J| grad u . grad g), one pass over the cells.
template <int ND, int NQ, typename T>
__global__ void __launch_bounds__(kT) k_cg_coeff_grad(const int32_t* __restrict__ idx, const T* __restrict__ metric,
                                                      const T* __restrict__ tabE, const T* __restrict__ tabW,
                                                      const T* __restrict__ u, const T* __restrict__ gv,
                                                      const T* __restrict__ kcoef, T* __restrict__ grad_u,
                                                      T* __restrict__ dk, int64_t nc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Shared<T> s = load_tables<ND, NQ, T>(smem, tabE, tabW, nullptr, false, kcoef != nullptr, true);
  const int64_t tile = blockIdx.x;
  const int64_t cell0 = tile * kT;
  if (kcoef) load_coeff_tile<NQ, T>(s.k, kcoef, cell0, nc);
  __syncthreads();
  const int lane = threadIdx.x;
  const bool active = cell0 + lane < nc;
  if (active) {
    int g[ND];
    T ue[ND], ge[ND], ye[ND];
    gather<ND, T>(idx, u, tile, lane, g, ue);
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      ge[j] = g[j] >= 0 ? __ldg(gv + g[j]) : T(0);
      ye[j] = T(0);
    }
    const T* mp = metric + tile * 6 * kT + lane;
    const T m0 = mp[0], m1 = mp[kT], m2 = mp[2 * kT], m3 = mp[3 * kT], m4 = mp[4 * kT], m5 = mp[5 * kT];
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
      const T* Eq = s.E + q * 3 * ND;
      T ax = T(0), ay = T(0), az = T(0), bx = T(0), by = T(0), bz = T(0);
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        ax = fma(Eq[j], ue[j], ax);
        ay = fma(Eq[ND + j], ue[j], ay);
        az = fma(Eq[2 * ND + j], ue[j], az);
        bx = fma(Eq[j], ge[j], bx);
        by = fma(Eq[ND + j], ge[j], by);
        bz = fma(Eq[2 * ND + j], ge[j], bz);
      }
      const T tx = fma(m0, bx, fma(m1, by, m2 * bz));
      const T ty = fma(m1, bx, fma(m3, by, m4 * bz));
      const T tz = fma(m2, bx, fma(m4, by, m5 * bz));
      const T wq = s.w[q];
      s.dk[lane * kstride(NQ) + q] = wq * fma(ax, tx, fma(ay, ty, az * tz));
      const T c = kcoef ? wq * s.k[lane * kstride(NQ) + q] : wq;
#pragma unroll
      for (int j = 0; j < ND; ++j)
        ye[j] = fma(Eq[j], c * tx, fma(Eq[ND + j], c * ty, fma(Eq[2 * ND + j], c * tz, ye[j])));
    }
#pragma unroll
    for (int j = 0; j < ND; ++j)
      if (g[j] >= 0) atomicAdd(grad_u + g[j], ye[j]);
  }
  __syncthreads();
  const int64_t ncell = nc - cell0 < kT ? nc - cell0 : kT;
  T* dst = dk + cell0 * NQ;
  for (int64_t i = threadIdx.x; i < ncell * NQ; i += blockDim.x) dst[i] = s.dk[(i / NQ) * kstride(NQ) + i % NQ];
}

// diag(A(k))_i = sum_e sum_q w_q k_q (E_q phi_i)^T M_e (E_q phi_i)
template <int ND, int NQ, typename T>
__global__ void __launch_bounds__(kT) k_cg_diag(const int32_t* __restrict__ idx, const T* __restrict__ metric,
                                                const T* __restrict__ tabE, const T* __restrict__ tabW,
                                                const T* __restrict__ kcoef, T* __restrict__ d, int64_t nc,
                                                const T* __restrict__ qmetric) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Shared<T> s = load_tables<ND, NQ, T>(smem, tabE, tabW, nullptr, false, kcoef != nullptr, false);
  const int64_t tile = blockIdx.x;
  const int64_t cell0 = tile * kT;
  if (kcoef) load_coeff_tile<NQ, T>(s.k, kcoef, cell0, nc);
  __syncthreads();
  const int lane = threadIdx.x;
  if (cell0 + lane >= nc) return;
  const T* mp = metric + tile * 6 * kT + lane;
  T m0 = mp[0], m1 = mp[kT], m2 = mp[2 * kT], m3 = mp[3 * kT], m4 = mp[4 * kT], m5 = mp[5 * kT];
  const T* qm = qmetric ? qmetric + tile * NQ * 6 * kT + lane : nullptr;
  T de[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) de[j] = T(0);
#pragma unroll 1
  for (int q = 0; q < NQ; ++q) {
    if (qm) {
      const T* p = qm + q * 6 * kT;
      m0 = p[0], m1 = p[kT], m2 = p[2 * kT], m3 = p[3 * kT], m4 = p[4 * kT], m5 = p[5 * kT];
    }
    const T* Eq = s.E + q * 3 * ND;
    T c = s.w[q];
    if (kcoef) c *= s.k[lane * kstride(NQ) + q];
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const T ex = Eq[j], ey = Eq[ND + j], ez = Eq[2 * ND + j];
      const T quad = ex * fma(m0, ex, fma(T(2) * m1, ey, T(2) * m2 * ez)) + ey * fma(m3, ey, T(2) * m4 * ez) +
                     m5 * ez * ez;
      de[j] = fma(c, quad, de[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const int gj = __ldg(idx + (tile * ND + j) * kT + lane);
    if (gj >= 0) atomicAdd(d + gj, de[j]);
  }
}

// b_i = f sum_e |det J_e| sum_q w_q phi_i(x_q); curved cells (qdet: [tiles][NQ][kT]):
// b_i = f sum_e sum_q w_q |det J_q| phi_i(x_q)
template <int ND, int NQ>
__global__ void __launch_bounds__(kT) k_cg_rhs(const int32_t* __restrict__ idx, const double* __restrict__ absdet,
                                               const double* __restrict__ tabV, const double* __restrict__ tabW,
                                               double f, double* __restrict__ b, int64_t nc,
                                               const double* __restrict__ qdet) {
  __shared__ double sv[ND];
  __shared__ double swv[NQ * ND];
  for (int j = threadIdx.x; j < ND; j += blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < NQ; ++q) acc = fma(tabW[q], tabV[q * ND + j], acc);
    sv[j] = acc;
  }
  for (int i = threadIdx.x; i < NQ * ND; i += blockDim.x) swv[i] = tabW[i / ND] * tabV[i];
  __syncthreads();
  const int64_t tile = blockIdx.x;
  const int lane = threadIdx.x;
  const int64_t cell = tile * kT + lane;
  if (cell >= nc) return;
  double be[ND];
  if (qdet) {
#pragma unroll
    for (int j = 0; j < ND; ++j) be[j] = 0.0;
    const double* dq = qdet + tile * NQ * kT + lane;
    for (int q = 0; q < NQ; ++q) {
      const double s = f * dq[q * kT];
#pragma unroll
      for (int j = 0; j < ND; ++j) be[j] = fma(s, swv[q * ND + j], be[j]);
    }
  } else {
    const double s = f * absdet[cell];
#pragma unroll
    for (int j = 0; j < ND; ++j) be[j] = s * sv[j];
  }
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const int gj = __ldg(idx + (tile * ND + j) * kT + lane);
    if (gj >= 0) atomicAdd(b + gj, be[j]);
  }
}

template <int ND, int NQ, typename T>
size_t smem_bytes(bool with_k, bool with_dk) {
  size_t n = size_t(NQ) * 3 * ND + NQ;
  if (with_k) n += size_t(kT) * kstride(NQ);
  if (with_dk) n += size_t(kT) * kstride(NQ);
  return n * sizeof(T);
}

template <int ND, int NQ, typename T>
int launch_apply(Ctx& c, const T* u, T* y, const T* k, const T* metric, const T* tab, cudaStream_t st,
                 int ncomp = 1) {
  const T* qmetric = std::is_same<T, double>::value ? reinterpret_cast<const T*>(c.d_qmetric64)
                                                     : reinterpret_cast<const T*>(c.d_qmetric32);
  const TableLayout L = tables_layout(c.tab);
  for (int comp = 0; comp < ncomp; ++comp)
    if (int e = init_rows<T>(y + comp * c.ndofs, u + comp * c.ndofs, c.d_mask, c.ndofs, T(0), st)) return e;
  const size_t sm = smem_bytes<ND, NQ, T>(k != nullptr, false);
  if (c.colour_start.empty()) {
    if (ncomp > 1) {
      if (int e = allow_smem(k_cg_apply<ND, NQ, T, false, true>, sm)) return e;
      k_cg_apply<ND, NQ, T, false, true><<<unsigned(c.ntiles), kT, sm, st>>>(
          c.d_idx, metric, tab + L.E, tab + L.w, u, y, k, c.nc, 0, c.nc, qmetric, ncomp, c.ndofs);
    } else {
      if (int e = allow_smem(k_cg_apply<ND, NQ, T, false, false>, sm)) return e;
      k_cg_apply<ND, NQ, T, false, false><<<unsigned(c.ntiles), kT, sm, st>>>(
          c.d_idx, metric, tab + L.E, tab + L.w, u, y, k, c.nc, 0, c.nc, qmetric, 1, c.ndofs);
    }
    TETMF_LAUNCH_CK();
    return FEM_OK;
  }
  // colour mode: one launch per colour, in colour order (components one after the other)
  if (int e = allow_smem(k_cg_apply<ND, NQ, T, true, false>, sm)) return e;
  for (int comp = 0; comp < ncomp; ++comp)
    for (size_t col = 0; col + 1 < c.colour_start.size(); ++col) {
      const int64_t lo = c.colour_start[col], hi = c.colour_start[col + 1];
      if (hi <= lo) continue;
      const int64_t tiles = (hi - 1) / kT - lo / kT + 1;
      k_cg_apply<ND, NQ, T, true, false><<<unsigned(tiles), kT, sm, st>>>(
          c.d_idx, metric, tab + L.E, tab + L.w, u + comp * c.ndofs, y + comp * c.ndofs, k, c.nc, lo, hi, qmetric, 1,
          c.ndofs);
      TETMF_LAUNCH_CK();
    }
  return FEM_OK;
}

template <int ND, int NQ, typename T>
int launch_coeff_grad(Ctx& c, const T* u, const T* g, const T* k, T* gu, T* dk, const T* metric, const T* tab,
                      cudaStream_t st) {
  const TableLayout L = tables_layout(c.tab);
  if (int e = init_rows<T>(gu, g, c.d_mask, c.ndofs, T(0), st)) return e;
  const size_t sm = smem_bytes<ND, NQ, T>(k != nullptr, true);
  if (int e = allow_smem(k_cg_coeff_grad<ND, NQ, T>, sm)) return e;
  k_cg_coeff_grad<ND, NQ, T><<<unsigned(c.ntiles), kT, sm, st>>>(c.d_idx, metric, tab + L.E, tab + L.w, u, g, k, gu,
                                                                  dk, c.nc);
  TETMF_LAUNCH_CK();
  return FEM_OK;
}

template <int ND, int NQ, typename T>
int launch_diag(Ctx& c, T* d, const T* k, const T* metric, const T* tab, cudaStream_t st) {
  const TableLayout L = tables_layout(c.tab);
  if (int e = init_rows<T>(d, nullptr, c.d_mask, c.ndofs, T(1), st)) return e;
  const size_t sm = smem_bytes<ND, NQ, T>(k != nullptr, false);
  if (int e = allow_smem(k_cg_diag<ND, NQ, T>, sm)) return e;
  const T* qmetric = std::is_same<T, double>::value ? reinterpret_cast<const T*>(c.d_qmetric64)
                                                     : reinterpret_cast<const T*>(c.d_qmetric32);
  k_cg_diag<ND, NQ, T><<<unsigned(c.ntiles), kT, sm, st>>>(c.d_idx, metric, tab + L.E, tab + L.w, k, d, c.nc,
                                                          qmetric);
  TETMF_LAUNCH_CK();
  return FEM_OK;
}

template <int ND, int NQ>
int launch_rhs(Ctx& c, double f, double* b, cudaStream_t st) {
  const TableLayout L = tables_layout(c.tab);
  if (int e = init_rows<double>(b, nullptr, c.d_mask, c.ndofs, 0.0, st)) return e;
  k_cg_rhs<ND, NQ><<<unsigned(c.ntiles), kT, 0, st>>>(c.d_idx, c.d_absdet, c.d_tab64 + L.V, c.d_tab64 + L.w, f, b,
                                                      c.nc, c.d_qdet64);
  TETMF_LAUNCH_CK();
  return FEM_OK;
}

}  // namespace

int cg_apply_simt(Ctx& c, int prec, const void* u, void* y, const void* k, bool /*transpose*/, void* stream) {
  cudaStream_t st = as_stream(stream);
  if (prec == FEM_FP64) {
    TETMF_DISPATCH_SPACE(c.p, c.nq, (launch_apply<ND, NQ, double>(c, static_cast<const double*>(u), static_cast<double*>(y),
                                                        static_cast<const double*>(k), c.d_metric64, c.d_tab64, st)))
  }
  TETMF_DISPATCH_SPACE(c.p, c.nq, (launch_apply<ND, NQ, float>(c, static_cast<const float*>(u), static_cast<float*>(y),
                                                     static_cast<const float*>(k), c.d_metric32, c.d_tab32, st)))
}

int cg_apply_vector_simt(Ctx& c, int prec, int ncomp, const void* u, void* y, void* stream) {
  cudaStream_t st = as_stream(stream);
  if (prec == FEM_FP64) {
    TETMF_DISPATCH_SPACE(c.p, c.nq, (launch_apply<ND, NQ, double>(c, static_cast<const double*>(u),
                                                                  static_cast<double*>(y), nullptr, c.d_metric64,
                                                                  c.d_tab64, st, ncomp)))
  }
  TETMF_DISPATCH_SPACE(c.p, c.nq, (launch_apply<ND, NQ, float>(c, static_cast<const float*>(u), static_cast<float*>(y),
                                                               nullptr, c.d_metric32, c.d_tab32, st, ncomp)))
}

int cg_coeff_grad(Ctx& c, int prec, const void* u, const void* g, const void* k, void* grad_u, void* dk,
                  void* stream) {
  if (c.curved) {
    set_error("fem_coeff_grad: curved cells are not offered");
    return FEM_EUNSUPPORTED;
  }
  cudaStream_t st = as_stream(stream);
  if (prec == FEM_FP64) {
    TETMF_DISPATCH_SPACE(c.p, c.nq, (launch_coeff_grad<ND, NQ, double>(
                              c, static_cast<const double*>(u), static_cast<const double*>(g),
                              static_cast<const double*>(k), static_cast<double*>(grad_u), static_cast<double*>(dk),
                              c.d_metric64, c.d_tab64, st)))
  }
  TETMF_DISPATCH_SPACE(c.p, c.nq, (launch_coeff_grad<ND, NQ, float>(
                            c, static_cast<const float*>(u), static_cast<const float*>(g),
                            static_cast<const float*>(k), static_cast<float*>(grad_u), static_cast<float*>(dk),
                            c.d_metric32, c.d_tab32, st)))
}

int cg_diagonal(Ctx& c, int prec, void* d, const void* k, void* stream) {
  cudaStream_t st = as_stream(stream);
  if (prec == FEM_FP64) {
    TETMF_DISPATCH_SPACE(c.p, c.nq, (launch_diag<ND, NQ, double>(c, static_cast<double*>(d), static_cast<const double*>(k),
                                                       c.d_metric64, c.d_tab64, st)))
  }
  TETMF_DISPATCH_SPACE(c.p, c.nq, (launch_diag<ND, NQ, float>(c, static_cast<float*>(d), static_cast<const float*>(k),
                                                    c.d_metric32, c.d_tab32, st)))
}

int cg_rhs_const(Ctx& c, double f, double* b, void* stream) {
  cudaStream_t st = as_stream(stream);
  TETMF_DISPATCH_SPACE(c.p, c.nq, (launch_rhs<ND, NQ>(c, f, b, st)))
}

}  // namespace tetmf
