// Upload of a host plan to the device and release of every device buffer.
//
// Device layouts (all in library cell order, tiles of kTile = 128 cells; the
// last tile is padded):
//   idx       int32 [ntiles][nd][128]  global DoF of local node j of the tile's
//                                      lane-th cell; a constrained DoF d is
//                                      stored as -1-d (masked gather, Sec. 2.4)
//   metric    T [ntiles][6][128]       |det J| J^-1 J^-T (xx xy xz yy yz zz)
//   tables    T packed, see tables_layout: E [nq][3][nd], w [nq], V [nq][nd],
//             wf [nqf], Vf [4][nqf][nd], Ef [4][nqf][3][nd]
// Structure-of-arrays per tile makes every per-cell load of a warp one
// coalesced 128-byte (FP32) or 256-byte (FP64) transaction.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace tetmf {

int sm_count() {
  static int cached[16] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return 152;
  if (!cached[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cached[dev] = n;
  }
  return cached[dev];
}

namespace {

// Places a tile's groups in its shared-memory staging: group q of the sorted list goes to the
// 16-byte slot sig[q] (4 words, banks 4 (slot mod 8) .. 4 (slot mod 8) + 3), and the list is stored
// in slot order.  The row build reads node j of a warp's 32 cells with one instruction and the
// pre-reduction adds to them with one more; two distinct groups in the same bank group whose DoFs
// have the same remainder mod 4 fall in one bank and cost an extra shared-memory wavefront.  Slots
// stay inside windows of 8 consecutive groups of the sorted list, so a warp's 32 consecutive list
// entries are the same groups as before and touch the same memory sectors.  Inside a window the
// groups take the 8 bank groups greedily, the most-met group first, each the free bank group
// where it meets the fewest groups already placed.
const std::vector<int32_t>& bank_slots(const Ctx& c, int64_t e0, int64_t e1, const std::vector<int32_t>& buf,
                                       std::vector<std::vector<int32_t>>& adj, std::vector<int32_t>& order,
                                       std::vector<int32_t>& sig) {
  const int L = int(buf.size());
  if (int(adj.size()) < L) adj.resize(size_t(L));
  for (int q = 0; q < L; ++q) adj[size_t(q)].clear();
  // pairs of distinct groups met by one warp instruction in the same bank (DoF mod 4), once per
  // instruction
  int32_t seen[4][32];
  for (int64_t w0 = e0; w0 < e1; w0 += 32) {
    const int64_t w1 = std::min<int64_t>(e1, w0 + 32);
    for (int j = 0; j < c.nd; ++j) {
      int cnt[4] = {0, 0, 0, 0};
      for (int64_t e = w0; e < w1; ++e) {
        const int32_t d = c.cell_dofs[size_t(e) * c.nd + j];
        if (c.mask[d]) continue;
        const int32_t q = int32_t(std::lower_bound(buf.begin(), buf.end(), d / 4) - buf.begin());
        const int k = d & 3;
        bool dup = false;
        for (int i = 0; i < cnt[k]; ++i) dup |= seen[k][i] == q;
        if (dup) continue;
        for (int i = 0; i < cnt[k]; ++i) {
          adj[size_t(q)].push_back(seen[k][i]);
          adj[size_t(seen[k][i])].push_back(q);
        }
        seen[k][cnt[k]++] = q;
      }
    }
  }
  sig.assign(size_t(L), -1);
  for (int w = 0; w < L; w += 8) {
    const int n = std::min(8, L - w);
    order.clear();
    for (int q = w; q < w + n; ++q) order.push_back(q);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
      const size_t da = adj[size_t(a)].size(), db = adj[size_t(b)].size();
      return da > db || (da == db && a < b);
    });
    unsigned used = 0;
    for (const int q : order) {
      int cost[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (const int32_t o : adj[size_t(q)])
        if (sig[size_t(o)] >= 0) ++cost[sig[size_t(o)] & 7];
      int best = -1;
      for (int k = 0; k < n; ++k)
        if (!((used >> k) & 1u) && (best < 0 || cost[k] < cost[best])) best = k;
      used |= 1u << best;
      sig[size_t(q)] = w + best;
    }
  }
  return sig;
}

template <typename T>
int dalloc(Ctx& c, T** p, size_t n) {
  *p = nullptr;
  if (n == 0) return FEM_OK;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FEM_ENOMEM : FEM_ECUDA;
  }
  c.allocations.push_back(q);
  *p = static_cast<T*>(q);
  return FEM_OK;
}

template <typename T>
int put(Ctx& c, T** p, const std::vector<T>& h) {
  if (int s = dalloc(c, p, h.size())) return s;
  if (!h.empty()) TETMF_CK(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FEM_OK;
}

template <typename D, typename S>
std::vector<D> cast(const std::vector<S>& v) {
  std::vector<D> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = D(v[i]);
  return o;
}

}  // namespace

int upload(Ctx& c) {
  TETMF_CK(cudaSetDevice(c.device));
  const int64_t T = kTile;
  const size_t ncp = size_t(c.ntiles) * T;

  if (c.kind == FEM_CG) {
    std::vector<int32_t> idx(size_t(c.ntiles) * c.nd * T, 0);
    for (int64_t e = 0; e < c.nc; ++e) {
      const int64_t t = e / T, l = e % T;
      for (int j = 0; j < c.nd; ++j) {
        const int32_t d = c.cell_dofs[size_t(e) * c.nd + j];
        idx[(size_t(t) * c.nd + j) * T + l] = c.mask[d] ? -1 - d : d;
      }
    }
    if (int s = put(c, &c.d_idx, idx)) return s;
    // tile-local lists: the tensor-core kernels move each tile's values in whole 16-byte groups
    // of 4 consecutive DoFs (group g = DoFs 4g .. 4g+3).  Per tile: the distinct groups that hold
    // its unconstrained DoFs, in the order of their staging slots (sorted, then permuted inside
    // windows of 8 by bank_slots), and per (cell, local node) the node's position in the tile's
    // staging, 4 x (the group's slot) + (DoF mod 4).  The DoF numbering (by the set of
    // tiles sharing a DoF) makes these groups dense: about 4 of every 4.3 staged values are used.
    std::vector<int64_t> span(size_t(c.ntiles) * 2, 0);
    std::vector<int32_t> list;
    // node positions: per tile [ndp/2][128] pairs (node 2w in the low half, 2w+1 in the high half);
    // constrained nodes, the padding node and the lanes past the last cell point at 4 L (L = groups
    // in the list), a 4-value slot the kernel keeps at zero on gather and never flushes
    const int ndp = (c.nd + 1) / 2 * 2;
    std::vector<uint16_t> lidx(size_t(c.ntiles) * ndp * T, 0);
    std::vector<int32_t> buf, placed, order, sig;
    std::vector<std::vector<int32_t>> adj;
    list.reserve(size_t(c.nc) * 2);
    for (int64_t t = 0; t < c.ntiles; ++t) {
      buf.clear();
      const int64_t e1 = std::min<int64_t>(c.nc, (t + 1) * T);
      for (int64_t e = t * T; e < e1; ++e)
        for (int j = 0; j < c.nd; ++j) {
          const int32_t d = c.cell_dofs[size_t(e) * c.nd + j];
          if (!c.mask[d]) buf.push_back(d / 4);
        }
      std::sort(buf.begin(), buf.end());
      buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
      if (4 * buf.size() + 4 > 65535) {
        set_error("a 128-cell batch touches %zu groups of DoFs (at most %d)", buf.size(), 65535 / 4 - 1);
        return FEM_EUNSUPPORTED;
      }
      std::fill(lidx.begin() + size_t(t) * ndp * T, lidx.begin() + size_t(t + 1) * ndp * T,
                uint16_t(4 * buf.size()));
      const std::vector<int32_t>& slot = bank_slots(c, t * T, e1, buf, adj, order, sig);
      for (int64_t e = t * T; e < e1; ++e)
        for (int j = 0; j < c.nd; ++j) {
          const int32_t d = c.cell_dofs[size_t(e) * c.nd + j];
          if (c.mask[d]) continue;
          const size_t pos = std::lower_bound(buf.begin(), buf.end(), d / 4) - buf.begin();
          lidx[size_t(t) * ndp * T + ((size_t(j) / 2) * T + (e - t * T)) * 2 + (j & 1)] =
              uint16_t(4 * slot[pos] + (d & 3));
        }
      c.tl_max = std::max<int32_t>(c.tl_max, int32_t(buf.size()));
      span[2 * t] = int64_t(list.size());
      span[2 * t + 1] = int64_t(buf.size());
      placed.assign(buf.size(), 0);
      for (size_t q = 0; q < buf.size(); ++q) placed[size_t(slot[q])] = buf[q];
      list.insert(list.end(), placed.begin(), placed.end());
      while (list.size() % 4) list.push_back(buf.empty() ? 0 : buf.back());  // 16-byte aligned lists
    }
    if (int s = put(c, &c.d_tl_span, span)) return s;
    if (int s = put(c, &c.d_tl_list, list)) return s;
    if (int s = put(c, &c.d_tl_lidx, lidx)) return s;
    if (c.dirichlet)
      if (int s = put(c, &c.d_mask, c.mask)) return s;
  }
  std::vector<double> met(ncp * 6, 0.0);
  for (int64_t e = 0; e < c.nc; ++e) {
    const int64_t t = e / T, l = e % T;
    for (int a = 0; a < 6; ++a) met[(size_t(t) * 6 + a) * T + l] = c.metric[size_t(e) * 6 + a];
  }
  if (int s = put(c, &c.d_metric64, met)) return s;
  if (int s = put(c, &c.d_metric32, cast<float>(met))) return s;
  if (int s = put(c, &c.d_absdet, c.absdet)) return s;
  if (c.curved) {
    // [ntiles][nq][6][kTile] and [ntiles][nq][kTile]: coalesced per point inside a tile
    const int nq = c.nq;
    std::vector<double> qm(ncp * nq * 6, 0.0), qd(ncp * nq, 0.0);
    for (int64_t e = 0; e < c.nc; ++e) {
      const int64_t t = e / T, l = e % T;
      for (int q = 0; q < nq; ++q) {
        for (int a = 0; a < 6; ++a)
          qm[((size_t(t) * nq + q) * 6 + a) * T + l] = c.qmetric[(size_t(e) * nq + q) * 6 + a];
        qd[(size_t(t) * nq + q) * T + l] = c.qdet[size_t(e) * nq + q];
      }
    }
    if (int s = put(c, &c.d_qmetric64, qm)) return s;
    if (int s = put(c, &c.d_qmetric32, cast<float>(qm))) return s;
    if (int s = put(c, &c.d_qdet64, qd)) return s;
  }

  const TableLayout L = tables_layout(c.tab);
  std::vector<double> tab(L.total);
  std::memcpy(&tab[L.E], c.tab.E.data(), c.tab.E.size() * sizeof(double));
  std::memcpy(&tab[L.w], c.tab.wq.data(), c.tab.wq.size() * sizeof(double));
  std::memcpy(&tab[L.V], c.tab.V.data(), c.tab.V.size() * sizeof(double));
  std::memcpy(&tab[L.wf], c.tab.wqf.data(), c.tab.wqf.size() * sizeof(double));
  std::memcpy(&tab[L.Vf], c.tab.Vf.data(), c.tab.Vf.size() * sizeof(double));
  std::memcpy(&tab[L.Ef], c.tab.Ef.data(), c.tab.Ef.size() * sizeof(double));
  if (int s = put(c, &c.d_tab64, tab)) return s;
  if (int s = put(c, &c.d_tab32, cast<float>(tab))) return s;

  if (c.kind == FEM_DG) {
    if (int s = put(c, &c.d_fperm, c.tab.fperm)) return s;
    if (int s = put(c, &c.d_fi_cell, c.fi_cell)) return s;
    if (int s = put(c, &c.d_fi_code, c.fi_code)) return s;
    if (int s = put(c, &c.d_fi_geo64, c.fi_geo)) return s;
    if (int s = put(c, &c.d_fi_geo32, cast<float>(c.fi_geo))) return s;
    if (int s = put(c, &c.d_fb_cell, c.fb_cell)) return s;
    if (int s = put(c, &c.d_fb_code, c.fb_code)) return s;
    if (int s = put(c, &c.d_fb_geo64, c.fb_geo)) return s;
    if (int s = put(c, &c.d_fb_geo32, cast<float>(c.fb_geo))) return s;
  }
  if (int s = put(c, &c.d_status, std::vector<int32_t>(4, 0))) return s;
  if (int s = tc_prepare(c)) return s;  // E tables of the cell GEMMs (CG and DG)
  if (c.kind == FEM_DG)
    if (int s = dg_tc_prepare(c)) return s;
  TETMF_CK(cudaDeviceSynchronize());
  return FEM_OK;
}

int device_status(Ctx& c, int32_t* out) {
  TETMF_CK(cudaDeviceSynchronize());
  int32_t h = 0;
  TETMF_CK(cudaMemcpy(&h, c.d_status, sizeof(h), cudaMemcpyDeviceToHost));
  const int32_t zero = 0;
  TETMF_CK(cudaMemcpy(c.d_status, &zero, sizeof(zero), cudaMemcpyHostToDevice));
  *out = h;
  return FEM_OK;
}

void release(Ctx& c) {
  pmg_release(c);
  host_pipe_release(c);
  if (c.device >= 0 && !c.allocations.empty()) {
    cudaSetDevice(c.device);
    cudaDeviceSynchronize();
    for (void* p : c.allocations) cudaFree(p);
    cudaGetLastError();
  }
  c.allocations.clear();
}

}  // namespace tetmf
