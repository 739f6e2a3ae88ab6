// Transfer between the continuous spaces of two degrees on one mesh (the p-levels of the paper's
// hybrid multigrid, Sec. 4.1): prolongation evaluates the coarse function at the fine nodes,
// u_f = P u_c, with the cell table T[i][j] = phi^coarse_j(x_hat^fine_i); restriction applies P^T.
//
// One thread per cell, tiles of 128 cells in the library order shared by both spaces.  Each fine
// DoF is written by one owner cell (the first cell containing it), so the prolongation needs no
// atomics and is deterministic; the restriction weights each fine value by 1 / (number of cells
// containing the DoF) before the cell's T^T product and adds with atomics, which sums exactly
// the entries of P^T once.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace tetmf {

struct Transfer {
  Ctx* fine = nullptr;
  Ctx* coarse = nullptr;
  double* d_tab64 = nullptr;   // [ndf][ndc]
  float* d_tab32 = nullptr;
  uint8_t* d_owner = nullptr;  // [ntiles][ndf][kTile]
  double* d_w64 = nullptr;     // [Nf] 1 / multiplicity
  float* d_w32 = nullptr;
  std::vector<void*> allocations;
};

namespace {

constexpr int kT = kTile;

template <int NDF, int NDC, typename T>
__global__ void __launch_bounds__(kT) k_prolongate(const int32_t* __restrict__ idx_f, const int32_t* __restrict__ idx_c,
                                                   const uint8_t* __restrict__ owner, const T* __restrict__ tab,
                                                   const T* __restrict__ uc, T* __restrict__ uf, int64_t nc) {
  __shared__ T st[NDF * NDC];
  for (int i = threadIdx.x; i < NDF * NDC; i += kT) st[i] = tab[i];
  __syncthreads();
  const int64_t tile = blockIdx.x;
  const int lane = threadIdx.x;
  if (tile * kT + lane >= nc) return;
  T ul[NDC];
#pragma unroll
  for (int j = 0; j < NDC; ++j) {
    const int g = __ldg(idx_c + (tile * NDC + j) * kT + lane);
    ul[j] = g >= 0 ? __ldg(uc + g) : T(0);
  }
#pragma unroll
  for (int i = 0; i < NDF; ++i) {
    if (!owner[(tile * NDF + i) * kT + lane]) continue;
    const int g = __ldg(idx_f + (tile * NDF + i) * kT + lane);
    T v = T(0);
    if (g >= 0) {
#pragma unroll
      for (int j = 0; j < NDC; ++j) v = fma(st[i * NDC + j], ul[j], v);
    }
    uf[g >= 0 ? g : -1 - g] = v;  // constrained fine DoFs get 0
  }
}

template <int NDF, int NDC, typename T>
__global__ void __launch_bounds__(kT) k_restrict(const int32_t* __restrict__ idx_f, const int32_t* __restrict__ idx_c,
                                                 const T* __restrict__ wmul, const T* __restrict__ tab,
                                                 const T* __restrict__ rf, T* __restrict__ rc, int64_t nc) {
  __shared__ T st[NDF * NDC];
  for (int i = threadIdx.x; i < NDF * NDC; i += kT) st[i] = tab[i];
  __syncthreads();
  const int64_t tile = blockIdx.x;
  const int lane = threadIdx.x;
  if (tile * kT + lane >= nc) return;
  T rl[NDF];
#pragma unroll
  for (int i = 0; i < NDF; ++i) {
    const int g = __ldg(idx_f + (tile * NDF + i) * kT + lane);
    rl[i] = g >= 0 ? __ldg(rf + g) * __ldg(wmul + g) : T(0);
  }
#pragma unroll
  for (int j = 0; j < NDC; ++j) {
    const int g = __ldg(idx_c + (tile * NDC + j) * kT + lane);
    if (g < 0) continue;
    T s = T(0);
#pragma unroll
    for (int i = 0; i < NDF; ++i) s = fma(st[i * NDC + j], rl[i], s);
    atomicAdd(rc + g, s);
  }
}

template <int NDF, int NDC, typename T>
int run(Transfer& t, bool prolong, const T* in, T* out, const T* tab, const T* w, cudaStream_t st) {
  Ctx& f = *t.fine;
  if (prolong) {
    k_prolongate<NDF, NDC, T><<<unsigned(f.ntiles), kT, 0, st>>>(f.d_idx, t.coarse->d_idx, t.d_owner, tab, in, out,
                                                                 f.nc);
  } else {
    if (int e = init_rows<T>(out, nullptr, nullptr, t.coarse->ndofs, T(0), st)) return e;
    k_restrict<NDF, NDC, T><<<unsigned(f.ntiles), kT, 0, st>>>(f.d_idx, t.coarse->d_idx, w, tab, in, out, f.nc);
  }
  TETMF_LAUNCH_CK();
  return FEM_OK;
}

template <typename T>
int dispatch(Transfer& t, bool prolong, const T* in, T* out, const T* tab, const T* w, cudaStream_t st) {
  switch (t.fine->nd * 100 + t.coarse->nd) {
    case 1004: return run<10, 4, T>(t, prolong, in, out, tab, w, st);
    case 2004: return run<20, 4, T>(t, prolong, in, out, tab, w, st);
    case 2010: return run<20, 10, T>(t, prolong, in, out, tab, w, st);
    case 3504: return run<35, 4, T>(t, prolong, in, out, tab, w, st);
    case 3510: return run<35, 10, T>(t, prolong, in, out, tab, w, st);
    case 3520: return run<35, 20, T>(t, prolong, in, out, tab, w, st);
  }
  set_error("transfer between %d and %d DoFs per cell not supported", t.fine->nd, t.coarse->nd);
  return FEM_EUNSUPPORTED;
}

template <typename V>
int upload(Transfer& t, V** dst, const std::vector<V>& v) {
  void* p = nullptr;
  TETMF_CK(cudaMalloc(&p, std::max<size_t>(1, v.size()) * sizeof(V)));
  t.allocations.push_back(p);
  TETMF_CK(cudaMemcpy(p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice));
  *dst = static_cast<V*>(p);
  return FEM_OK;
}

}  // namespace

int transfer_create(Ctx& fine, Ctx& coarse, Transfer** out) {
  if (fine.kind != FEM_CG || coarse.kind != FEM_CG)
    return set_error("fem_transfer_create: CG spaces only"), FEM_EINVAL;
  if (fine.nc != coarse.nc || fine.cell_perm != coarse.cell_perm || fine.p <= coarse.p ||
      fine.dirichlet != coarse.dirichlet || fine.device != coarse.device || fine.device < 0)
    return set_error("fem_transfer_create: spaces must share the mesh, its cell order, the Dirichlet choice and "
                     "the device, with the fine degree above the coarse one"),
           FEM_EINVAL;
  Transfer* t = new (std::nothrow) Transfer;
  if (!t) return set_error("fem_transfer_create: out of host memory"), FEM_ENOMEM;
  t->fine = &fine;
  t->coarse = &coarse;
  const int ndf = fine.nd, ndc = coarse.nd;
  std::vector<double> tab;
  fine_nodes_coarse_values(fine.p, coarse.p, tab);  // [ndf][ndc]
  const int64_t T = kTile, nc = fine.nc;
  std::vector<uint8_t> owner(size_t(fine.ntiles) * ndf * T, 0);
  std::vector<int32_t> count(fine.ndofs, 0);
  for (int64_t e = 0; e < nc; ++e)
    for (int i = 0; i < ndf; ++i) {
      const int32_t d = fine.cell_dofs[size_t(e) * ndf + i];
      if (count[d]++ == 0) owner[(size_t(e / T) * ndf + i) * T + e % T] = 1;
    }
  std::vector<double> w(fine.ndofs);
  for (int64_t d = 0; d < fine.ndofs; ++d) w[d] = count[d] ? 1.0 / count[d] : 0.0;
  int s = FEM_OK;
  if (!s) s = upload(*t, &t->d_tab64, tab);
  if (!s) s = upload(*t, &t->d_tab32, std::vector<float>(tab.begin(), tab.end()));
  if (!s) s = upload(*t, &t->d_owner, owner);
  if (!s) s = upload(*t, &t->d_w64, w);
  if (!s) s = upload(*t, &t->d_w32, std::vector<float>(w.begin(), w.end()));
  if (s) {
    transfer_destroy(t);
    return s;
  }
  *out = t;
  return FEM_OK;
}

void transfer_destroy(Transfer* t) {
  if (!t) return;
  for (void* p : t->allocations) cudaFree(p);
  delete t;
}

int transfer_apply(Transfer& t, int prec, bool prolong, const void* in, void* out, void* stream) {
  cudaStream_t st = as_stream(stream);
  if (prec == FEM_FP64)
    return dispatch<double>(t, prolong, static_cast<const double*>(in), static_cast<double*>(out), t.d_tab64, t.d_w64,
                            st);
  return dispatch<float>(t, prolong, static_cast<const float*>(in), static_cast<float*>(out), t.d_tab32, t.d_w32, st);
}

}  // namespace tetmf
