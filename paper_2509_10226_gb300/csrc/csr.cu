// Assembled comparator (Sec. 3.2): the same continuous operator stored as a CSR
// matrix, and its SpMV.
//
// Pattern: built on the host from the cell -> DoF map (row i holds the DoFs of
// every cell that touches DoF i; Dirichlet rows keep only their diagonal and
// constrained columns are dropped, giving P A P + (I - P)).  Values: one thread
// per cell forms K_ij = sum_{a,b} M_ab S_ab[i][j], where
// S_ab[i][j] = sum_q w_q d_a phi_i(x_q) d_b phi_j(x_q) are reference-cell
// tables (the same quadrature as the matrix-free path), and adds it into the
// CSR values found by binary search in row i.
// SpMV: 4 (FP64) or 8 (FP32) lanes per row (rows average ~48 entries at p = 3), 64-bit row
// pointers, FP64 or FP32 values, FP64/FP32 accumulation as the vector type.
#include <algorithm>
#include <thread>
#include <vector>

#include "common.cuh"

namespace tetmf {
namespace {

constexpr int kT = kTile;

template <int ND>
__global__ void __launch_bounds__(kT) k_csr_values(const int32_t* __restrict__ idx, const double* __restrict__ metric,
                                                   const double* __restrict__ S, const int64_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ col, double* __restrict__ val,
                                                   int64_t nc) {
  extern __shared__ double sS[];  // [6][ND][ND]
  for (int i = threadIdx.x; i < 6 * ND * ND; i += kT) sS[i] = S[i];
  __syncthreads();
  const int64_t tile = blockIdx.x;
  const int lane = threadIdx.x;
  if (tile * kT + lane >= nc) return;
  const double* mp = metric + tile * 6 * kT + lane;
  double m[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) m[a] = mp[a * kT];
  int g[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) g[j] = idx[(tile * ND + j) * kT + lane];
  for (int i = 0; i < ND; ++i) {
    if (g[i] < 0) continue;
    const int64_t lo = rowptr[g[i]], hi = rowptr[g[i] + 1];
    for (int j = 0; j < ND; ++j) {
      if (g[j] < 0) continue;
      double v = 0.0;
#pragma unroll
      for (int a = 0; a < 6; ++a) v = fma(m[a], sS[(a * ND + i) * ND + j], v);
      int64_t l = lo, h = hi;
      while (l < h) {
        const int64_t mid = (l + h) >> 1;
        if (col[mid] < g[j])
          l = mid + 1;
        else
          h = mid;
      }
      atomicAdd(val + l, v);
    }
  }
}

__global__ void k_csr_dirichlet_diag(const int64_t* __restrict__ rowptr, const uint8_t* __restrict__ mask,
                                     double* __restrict__ val, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    if (mask[i]) val[rowptr[i]] = 1.0;
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = float(a[i]);
}

template <typename T, int G>
__global__ void __launch_bounds__(256) k_spmv(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                              const T* __restrict__ val, const T* __restrict__ u, T* __restrict__ y,
                                              int64_t n) {
  const int64_t row = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) / G;
  const int sub = threadIdx.x % G;
  T acc = T(0);
  if (row < n) {
    const int64_t lo = rowptr[row], hi = rowptr[row + 1];
    for (int64_t k = lo + sub; k < hi; k += G) acc = fma(__ldg(val + k), __ldg(u + __ldg(col + k)), acc);
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (row < n && sub == 0) y[row] = acc;
}

// host: CSR pattern from the cell -> DoF map
void build_pattern(const Ctx& c, std::vector<int64_t>& rowptr, std::vector<int32_t>& col) {
  const int64_t N = c.ndofs, nc = c.nc;
  const int nd = c.nd;
  std::vector<int64_t> cstart(N + 1, 0);
  for (int64_t p = 0; p < nc * nd; ++p) cstart[c.cell_dofs[p] + 1]++;
  for (int64_t i = 0; i < N; ++i) cstart[i + 1] += cstart[i];
  std::vector<int32_t> inc(nc * nd);
  {
    std::vector<int64_t> fill(cstart.begin(), cstart.end() - 1);
    for (int64_t p = 0; p < nc * nd; ++p) inc[fill[c.cell_dofs[p]]++] = int32_t(p / nd);
  }
  const bool dir = c.dirichlet != 0;
  auto row_cols = [&](int64_t i, std::vector<int32_t>& buf) {
    buf.clear();
    if (dir && c.mask[i]) {
      buf.push_back(int32_t(i));
      return;
    }
    for (int64_t t = cstart[i]; t < cstart[i + 1]; ++t) {
      const int32_t* cd = &c.cell_dofs[size_t(inc[t]) * nd];
      for (int j = 0; j < nd; ++j)
        if (!(dir && c.mask[cd[j]])) buf.push_back(cd[j]);
    }
    std::sort(buf.begin(), buf.end());
    buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
  };
  unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<int64_t> count(N, 0);
  auto pass = [&](bool write) {
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
      th.emplace_back([&, t, write]() {
        std::vector<int32_t> buf;
        for (int64_t i = t; i < N; i += nt) {
          row_cols(i, buf);
          if (!write)
            count[i] = int64_t(buf.size());
          else
            std::copy(buf.begin(), buf.end(), col.begin() + rowptr[i]);
        }
      });
    for (auto& x : th) x.join();
  };
  pass(false);
  rowptr.assign(N + 1, 0);
  for (int64_t i = 0; i < N; ++i) rowptr[i + 1] = rowptr[i] + count[i];
  col.resize(rowptr[N]);
  pass(true);
}

template <int ND>
int fill_values(Ctx& c, cudaStream_t st) {
  // reference tables S_ab, ab in (xx, xy, xz, yy, yz, zz); off-diagonal pairs
  // hold S_ab + S_ba so that K = sum_ab M_ab S_ab over the 6 stored entries
  const int pairs[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
  std::vector<double> S(6 * ND * ND, 0.0);
  for (int a = 0; a < 6; ++a) {
    const int x = pairs[a][0], z = pairs[a][1];
    for (int i = 0; i < ND; ++i)
      for (int j = 0; j < ND; ++j) {
        double s = 0.0;
        for (int q = 0; q < c.nq; ++q) {
          const double* Eq = &c.tab.E[size_t(q) * 3 * ND];
          double v = Eq[x * ND + i] * Eq[z * ND + j];
          if (x != z) v += Eq[z * ND + i] * Eq[x * ND + j];
          s += c.tab.wq[q] * v;
        }
        S[(a * ND + i) * ND + j] = s;
      }
  }
  double* dS = nullptr;
  TETMF_CK(cudaMalloc(&dS, S.size() * sizeof(double)));
  c.allocations.push_back(dS);
  TETMF_CK(cudaMemcpy(dS, S.data(), S.size() * sizeof(double), cudaMemcpyHostToDevice));
  TETMF_CK(cudaMemsetAsync(c.d_csr_val64, 0, c.csr_nnz * sizeof(double), st));
  const size_t sm = size_t(6) * ND * ND * sizeof(double);
  if (int e = allow_smem(k_csr_values<ND>, sm)) return e;
  k_csr_values<ND><<<unsigned(c.ntiles), kT, sm, st>>>(c.d_idx, c.d_metric64, dS, c.d_csr_rowptr, c.d_csr_col,
                                                      c.d_csr_val64, c.nc);
  TETMF_LAUNCH_CK();
  if (c.dirichlet) {
    k_csr_dirichlet_diag<<<unsigned(sm_count() * 4), 256, 0, st>>>(c.d_csr_rowptr, c.d_mask, c.d_csr_val64, c.ndofs);
    TETMF_LAUNCH_CK();
  }
  k_to_float<<<unsigned(sm_count() * 8), 256, 0, st>>>(c.d_csr_val64, c.d_csr_val32, c.csr_nnz);
  TETMF_LAUNCH_CK();
  return FEM_OK;
}

template <typename T>
int spmv(Ctx& c, const T* u, T* y, const T* val, cudaStream_t st) {
  // lanes per row: FP64 arithmetic is scarce on this GPU (the FP64 SpMV is FP64-pipe bound), so
  // the FP64 kernel uses 4 lanes per row (fewer shuffle-reduction adds); FP32 uses 8
  if constexpr (sizeof(T) == 8) {
    constexpr int G = 4;
    const int64_t threads = c.ndofs * G;
    k_spmv<T, G><<<unsigned((threads + 255) / 256), 256, 0, st>>>(c.d_csr_rowptr, c.d_csr_col, val, u, y, c.ndofs);
  } else {
    constexpr int G = 8;
    const int64_t threads = c.ndofs * G;
    k_spmv<T, G><<<unsigned((threads + 255) / 256), 256, 0, st>>>(c.d_csr_rowptr, c.d_csr_col, val, u, y, c.ndofs);
  }
  TETMF_LAUNCH_CK();
  return FEM_OK;
}

}  // namespace

int csr_build(Ctx& c, int64_t* nnz) {
  if (c.curved) {
    set_error("fem_csr_build: the assembled comparator is built for straight cells only");
    return FEM_EUNSUPPORTED;
  }
  if (c.d_csr_rowptr) {
    if (nnz) *nnz = c.csr_nnz;
    return FEM_OK;
  }
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  try {
    build_pattern(c, rowptr, col);
  } catch (const std::bad_alloc&) {
    set_error("fem_csr_build: out of host memory");
    return FEM_ENOMEM;
  }
  c.csr_nnz = rowptr.back();
  void* p = nullptr;
  TETMF_CK(cudaMalloc(&p, rowptr.size() * sizeof(int64_t)));
  c.allocations.push_back(p);
  c.d_csr_rowptr = static_cast<int64_t*>(p);
  TETMF_CK(cudaMalloc(&p, col.size() * sizeof(int32_t)));
  c.allocations.push_back(p);
  c.d_csr_col = static_cast<int32_t*>(p);
  TETMF_CK(cudaMalloc(&p, c.csr_nnz * sizeof(double)));
  c.allocations.push_back(p);
  c.d_csr_val64 = static_cast<double*>(p);
  TETMF_CK(cudaMalloc(&p, c.csr_nnz * sizeof(float)));
  c.allocations.push_back(p);
  c.d_csr_val32 = static_cast<float*>(p);
  TETMF_CK(cudaMemcpy(c.d_csr_rowptr, rowptr.data(), rowptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  TETMF_CK(cudaMemcpy(c.d_csr_col, col.data(), col.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  int st = FEM_OK;
  switch (c.p) {
    case 1: st = fill_values<4>(c, 0); break;
    case 2: st = fill_values<10>(c, 0); break;
    case 3: st = fill_values<20>(c, 0); break;
    case 4: st = fill_values<35>(c, 0); break;
  }
  if (st) return st;
  TETMF_CK(cudaDeviceSynchronize());
  if (nnz) *nnz = c.csr_nnz;
  return FEM_OK;
}

int csr_apply(Ctx& c, int prec, const void* u, void* y, void* stream) {
  cudaStream_t st = as_stream(stream);
  if (prec == FEM_FP64)
    return spmv<double>(c, static_cast<const double*>(u), static_cast<double*>(y), c.d_csr_val64, st);
  return spmv<float>(c, static_cast<const float*>(u), static_cast<float*>(y), c.d_csr_val32, st);
}

}  // namespace tetmf
