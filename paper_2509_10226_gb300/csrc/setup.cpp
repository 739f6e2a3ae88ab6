// Host set-up of a context: mesh validation, cell reordering, DoF numbering,
// affine geometry, faces and the Dirichlet set, all in FP64.  Also the
// synchronous C entry points (create, destroy, queries) and argument checks
// of the hot calls, which dispatch to the CUDA launchers.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include <cuda_runtime.h>

#include "internal.h"

namespace tetmf {

namespace {
thread_local char g_err[1024] = "";
const int kFaceVerts[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
const int kPerms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
}  // namespace

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

namespace {

struct Key {
  int32_t v[4];
  bool operator<(const Key& o) const {
    for (int i = 0; i < 4; ++i)
      if (v[i] != o.v[i]) return v[i] < o.v[i];
    return false;
  }
  bool operator==(const Key& o) const {
    return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2] && v[3] == o.v[3];
  }
};

struct KeyPos {
  Key k;
  int64_t pos;
  bool operator<(const KeyPos& o) const {
    if (k < o.k) return true;
    if (o.k < k) return false;
    return pos < o.pos;
  }
};

uint64_t spread21(uint64_t x) {
  x &= 0x1fffffULL;
  x = (x | x << 32) & 0x1f00000000ffffULL;
  x = (x | x << 16) & 0x1f0000ff0000ffULL;
  x = (x | x << 8) & 0x100f00f00f00f00fULL;
  x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
  x = (x | x << 2) & 0x1249249249249249ULL;
  return x;
}

struct Geo {
  double J[3][3], Ji[3][3], det;
};

Geo cell_geometry(const double* xyz, const int32_t* cv) {
  Geo g;
  const double* X0 = xyz + 3 * int64_t(cv[0]);
  for (int a = 0; a < 3; ++a) {
    const double* Xa = xyz + 3 * int64_t(cv[a + 1]);
    for (int r = 0; r < 3; ++r) g.J[r][a] = Xa[r] - X0[r];
  }
  const double(&J)[3][3] = g.J;
  const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  g.det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  const double id = 1.0 / g.det;
  g.Ji[0][0] = c00 * id;
  g.Ji[1][0] = c01 * id;
  g.Ji[2][0] = c02 * id;
  g.Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
  g.Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
  g.Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
  g.Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
  g.Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
  g.Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  return g;
}

double longest_edge(const double* xyz, const int32_t* cv) {
  double L = 0.0;
  for (int a = 0; a < 4; ++a)
    for (int b = a + 1; b < 4; ++b) {
      double s = 0.0;
      for (int r = 0; r < 3; ++r) {
        const double d = xyz[3 * int64_t(cv[a]) + r] - xyz[3 * int64_t(cv[b]) + r];
        s += d * d;
      }
      L = std::max(L, std::sqrt(s));
    }
  return L;
}

// Colour the cells so that no two cells of one colour share a DoF (greedy, lowest free colour,
// cells visited in the current library order), then order the cells by colour, keeping the
// order inside each colour.  The scatter of one colour then needs no atomics, and colours are
// added one after the other: a deterministic summation order for every DoF.
void colour_cells(Ctx& c) {
  const int64_t nc = c.nc, N = c.ndofs;
  const int nd = c.nd;
  constexpr int kWords = 4;  // up to 256 colours
  std::vector<uint64_t> used(size_t(N) * kWords, 0);
  std::vector<int32_t> colour(nc);
  int ncol = 0;
  for (int64_t e = 0; e < nc; ++e) {
    uint64_t busy[kWords] = {0, 0, 0, 0};
    for (int j = 0; j < nd; ++j)
      for (int w = 0; w < kWords; ++w) busy[w] |= used[size_t(c.cell_dofs[size_t(e) * nd + j]) * kWords + w];
    int col = 0;
    while (col < 64 * kWords && ((busy[col / 64] >> (col % 64)) & 1u)) ++col;
    colour[e] = col;  // < 256: a cell shares DoFs with far fewer cells on any mesh this library accepts
    ncol = std::max(ncol, col + 1);
    for (int j = 0; j < nd; ++j) used[size_t(c.cell_dofs[size_t(e) * nd + j]) * kWords + col / 64] |= uint64_t(1) << (col % 64);
  }
  std::vector<int64_t> order(nc);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return colour[a] < colour[b]; });
  c.colour_start.assign(ncol + 1, 0);
  for (int64_t e = 0; e < nc; ++e) ++c.colour_start[colour[e] + 1];
  for (int k = 0; k < ncol; ++k) c.colour_start[k + 1] += c.colour_start[k];
  auto permute = [&](auto& v, int width) {
    auto old = v;
    for (int64_t i = 0; i < nc; ++i)
      for (int r = 0; r < width; ++r) v[size_t(i) * width + r] = old[size_t(order[i]) * width + r];
  };
  permute(c.cell_perm, 1);
  permute(c.cell_dofs, nd);
  permute(c.metric, 6);
  permute(c.absdet, 1);
  if (c.curved) {
    permute(c.qmetric, 6 * c.nq);
    permute(c.qdet, c.nq);
  }
}

int build_plan(Ctx& c, const fem_mesh_desc* m) {
  const double* xyz = m->xyz;
  const int32_t* ucells = m->cells;
  const int64_t nc = c.nc;
  c.xyz.assign(xyz, xyz + 3 * c.nv);
  c.ucells.assign(ucells, ucells + 4 * nc);

  // validation (vertex range, degenerate cells)
  for (int64_t e = 0; e < nc; ++e)
    for (int a = 0; a < 4; ++a)
      if (ucells[4 * e + a] < 0 || ucells[4 * e + a] >= c.nv) {
        set_error("cell %lld: vertex id %d out of range [0, %lld)", (long long)e, ucells[4 * e + a],
                  (long long)c.nv);
        return FEM_EMESH;
      }
  for (int64_t e = 0; e < nc; ++e) {
    const Geo g = cell_geometry(xyz, ucells + 4 * e);
    const double L = longest_edge(xyz, ucells + 4 * e);
    if (!(std::fabs(g.det) > 1e-12 * L * L * L)) {
      set_error("cell %lld is degenerate (|det J| = %g, longest edge %g)", (long long)e, g.det, L);
      return FEM_EMESH;
    }
  }

  // cell order: Morton code of the centroid (21 bits per axis over the
  // bounding box), ties by user id (Sec. 2.5, hierarchical locality ordering)
  c.cell_perm.resize(nc);
  std::iota(c.cell_perm.begin(), c.cell_perm.end(), 0);
  if (c.reorder == FEM_REORDER_MORTON) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t v = 0; v < c.nv; ++v)
      for (int r = 0; r < 3; ++r) {
        lo[r] = std::min(lo[r], xyz[3 * v + r]);
        hi[r] = std::max(hi[r], xyz[3 * v + r]);
      }
    std::vector<std::pair<uint64_t, int32_t>> key(nc);
    for (int64_t e = 0; e < nc; ++e) {
      uint64_t code = 0;
      for (int r = 0; r < 3; ++r) {
        double s = 0.0;
        for (int a = 0; a < 4; ++a) s += xyz[3 * int64_t(ucells[4 * e + a]) + r];
        s *= 0.25;
        const double ext = hi[r] - lo[r];
        double t = ext > 0 ? (s - lo[r]) / ext : 0.0;
        t = std::min(std::max(t, 0.0), 1.0);
        const uint64_t q = uint64_t(t * double((1u << 21) - 1));
        code |= spread21(q) << r;
      }
      key[e] = {code, int32_t(e)};
    }
    std::sort(key.begin(), key.end());
    // Inside each 128-cell batch, deal the Morton sequence round-robin over the
    // four warps (position i -> lane (i % 4) * 32 + i / 4): cells of one
    // neighbourhood share vertex and edge DoFs at the same local index, and
    // spreading them over warps keeps one warp's 32 scatter/gather addresses
    // for a local node mostly distinct.  The batch holds the same cells.
    for (int64_t t0 = 0; t0 < nc; t0 += kTile) {
      const int64_t n = std::min<int64_t>(kTile, nc - t0);
      const int64_t w = (n + 31) / 32;  // warps in this batch
      std::vector<int64_t> slot;
      slot.reserve(n);
      for (int64_t i = 0; i < n; ++i) slot.push_back((i % w) * 32 + i / w);
      // compact the lane numbers of a ragged batch to 0..n-1 in lane order
      std::vector<int64_t> order(n);
      std::iota(order.begin(), order.end(), 0);
      std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return slot[a] < slot[b]; });
      for (int64_t r = 0; r < n; ++r) c.cell_perm[t0 + r] = key[t0 + order[r]].second;
    }
  }
  auto lib_cell = [&](int64_t e) { return ucells + 4 * int64_t(c.cell_perm[e]); };

  // geometry: metric |det J| J^-1 J^-T (symmetric, 6 entries) per library cell
  c.metric.resize(size_t(nc) * 6);
  c.absdet.resize(nc);
  std::vector<Geo> geo(nc);
  for (int64_t e = 0; e < nc; ++e) {
    geo[e] = cell_geometry(xyz, lib_cell(e));
    const Geo& g = geo[e];
    const double ad = std::fabs(g.det);
    c.absdet[e] = ad;
    double M[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) s += g.Ji[a][k] * g.Ji[b][k];
        M[a][b] = ad * s;
      }
    double* out = &c.metric[size_t(e) * 6];
    out[0] = M[0][0];
    out[1] = M[0][1];
    out[2] = M[0][2];
    out[3] = M[1][1];
    out[4] = M[1][2];
    out[5] = M[2][2];
  }

  // curved cells: Jacobian of the second-order map at every quadrature point,
  // J[d][k] = sum_j X_j[d] d phi_j / d x_hat_k, then the same symmetric metric per point
  if (m->cell_nodes) {
    c.curved = true;
    const int nq = c.tab.nq;
    c.qmetric.assign(size_t(nc) * nq * 6, 0.0);
    c.qdet.assign(size_t(nc) * nq, 0.0);
    for (int64_t e = 0; e < nc; ++e) {
      const double* X = m->cell_nodes + size_t(c.cell_perm[e]) * 30;
      double sign = 0.0;
      for (int q = 0; q < nq; ++q) {
        double J[3][3];
        for (int d = 0; d < 3; ++d)
          for (int k = 0; k < 3; ++k) {
            double v = 0.0;
            for (int j = 0; j < 10; ++j) v += X[3 * j + d] * c.tab.G2[(size_t(q) * 3 + k) * 10 + j];
            J[d][k] = v;
          }
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        const double ad = std::fabs(det);
        if (q == 0) sign = det;
        if (!(ad > 1e-12 * std::fabs(geo[e].det)) || det * sign <= 0.0) {
          set_error("curved cell %lld folds or degenerates at quadrature point %d", (long long)c.cell_perm[e], q);
          return FEM_EMESH;
        }
        double Ji[3][3];
        Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        double M[3][3];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            double sm = 0.0;
            for (int k = 0; k < 3; ++k) sm += Ji[a][k] * Ji[b][k];
            M[a][b] = ad * sm;
          }
        double* out = &c.qmetric[(size_t(e) * nq + q) * 6];
        out[0] = M[0][0];
        out[1] = M[0][1];
        out[2] = M[0][2];
        out[3] = M[1][1];
        out[4] = M[1][2];
        out[5] = M[2][2];
        c.qdet[size_t(e) * nq + q] = ad;
      }
    }
  }

  // faces: sorted vertex triples, matched by sorting
  std::vector<KeyPos> fk(size_t(nc) * 4);
  for (int64_t e = 0; e < nc; ++e) {
    const int32_t* cv = lib_cell(e);
    for (int f = 0; f < 4; ++f) {
      Key k;
      for (int i = 0; i < 3; ++i) k.v[i] = cv[kFaceVerts[f][i]];
      std::sort(k.v, k.v + 3);
      k.v[3] = 0;
      fk[size_t(e) * 4 + f] = {k, e * 4 + f};
    }
  }
  std::sort(fk.begin(), fk.end());
  std::vector<std::array<int64_t, 2>> interior;  // packed cell*4+face of the two sides
  std::vector<int64_t> boundary;
  for (size_t i = 0; i < fk.size();) {
    size_t j = i + 1;
    while (j < fk.size() && fk[j].k == fk[i].k) ++j;
    if (j - i > 2) {
      set_error("face (%d, %d, %d) is shared by %zu cells", fk[i].k.v[0], fk[i].k.v[1], fk[i].k.v[2], j - i);
      return FEM_EMESH;
    }
    if (j - i == 1)
      boundary.push_back(fk[i].pos);
    else
      interior.push_back({fk[i].pos, fk[i + 1].pos});
    i = j;
  }

  if (c.kind == FEM_CG) {
    // DoF keys: node beta of a cell = sorted multiset of its vertices with
    // multiplicity beta_m; equal keys are the same global DoF
    std::vector<std::vector<int>> nodes;
    {
      std::vector<int> cur(4);
      for (int b0 = 0; b0 <= c.p; ++b0)
        for (int b1 = 0; b1 <= c.p - b0; ++b1)
          for (int b2 = 0; b2 <= c.p - b0 - b1; ++b2) nodes.push_back({b0, b1, b2, c.p - b0 - b1 - b2});
    }
    const int nd = c.nd;
    std::vector<KeyPos> dk(size_t(nc) * nd);
    for (int64_t e = 0; e < nc; ++e) {
      const int32_t* cv = lib_cell(e);
      for (int j = 0; j < nd; ++j) {
        Key k{{INT32_MAX, INT32_MAX, INT32_MAX, INT32_MAX}};
        int t = 0;
        for (int a = 0; a < 4; ++a)
          for (int r = 0; r < nodes[j][a]; ++r) k.v[t++] = cv[a];
        std::sort(k.v, k.v + t);
        dk[size_t(e) * nd + j] = {k, e * nd + j};
      }
    }
    std::sort(dk.begin(), dk.end());
    std::vector<int64_t> group_of(size_t(nc) * nd);
    std::vector<Key> group_key;
    for (size_t i = 0; i < dk.size();) {
      size_t j = i;
      while (j < dk.size() && dk[j].k == dk[i].k) {
        group_of[dk[j].pos] = int64_t(group_key.size());
        ++j;
      }
      group_key.push_back(dk[i].k);
      i = j;
    }
    dk.clear();
    dk.shrink_to_fit();
    const int64_t N = int64_t(group_key.size());
    c.ndofs = N;
    std::vector<int32_t> lib_of_group(N, -1);
    c.cell_dofs.resize(size_t(nc) * nd);
    c.dof_canon.resize(N);
    c.dof_keys.resize(size_t(N) * c.p);
    // DoF numbering by sharing class: every DoF is tagged with the increasing list of 128-cell
    // batches (tiles) whose cells touch it, and DoFs are numbered in lexicographic order of these
    // lists (a list sorts after the longer lists it is a prefix of), ties in first-touch order.  The
    // DoFs one tile touches then form a few contiguous runs (its own classes in one run, and one run
    // per class it shares with an earlier tile), which the tensor-core kernel moves with bulk copies
    // and bulk reductions instead of one access per DoF.
    {
      std::vector<int64_t> first(N, -1);
      std::vector<int32_t> cnt(N, 0), last(N, -1);
      for (int64_t pos = 0; pos < nc * nd; ++pos) {
        const int64_t g = group_of[pos];
        const int32_t t = int32_t(pos / nd / kTile);
        if (first[g] < 0) first[g] = pos;
        if (last[g] != t) {
          last[g] = t;
          ++cnt[g];
        }
      }
      std::vector<int64_t> off(N + 1, 0);
      for (int64_t g = 0; g < N; ++g) off[g + 1] = off[g] + cnt[g];
      std::vector<int32_t> tiles(static_cast<size_t>(off[N]));
      std::fill(last.begin(), last.end(), -1);
      std::vector<int64_t> fill(off.begin(), off.end() - 1);
      for (int64_t pos = 0; pos < nc * nd; ++pos) {
        const int64_t g = group_of[pos];
        const int32_t t = int32_t(pos / nd / kTile);
        if (last[g] != t) {
          last[g] = t;
          tiles[size_t(fill[g]++)] = t;
        }
      }
      std::vector<int64_t> order(N);
      std::iota(order.begin(), order.end(), int64_t(0));
      std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        const int64_t na = off[a + 1] - off[a], nb = off[b + 1] - off[b];
        for (int64_t i = 0;; ++i) {
          if (i == na || i == nb) {
            if (na != nb) return na > nb;  // a prefix sorts after the longer list
            return first[a] < first[b];
          }
          const int32_t ta = tiles[size_t(off[a] + i)], tb = tiles[size_t(off[b] + i)];
          if (ta != tb) return ta < tb;
        }
      });
      for (int64_t r = 0; r < N; ++r) {
        const int64_t g = order[r];
        lib_of_group[g] = int32_t(r);
        c.dof_canon[r] = g;
        for (int q = 0; q < c.p; ++q) c.dof_keys[size_t(r) * c.p + q] = group_key[g].v[q];
      }
      for (int64_t pos = 0; pos < nc * nd; ++pos) c.cell_dofs[pos] = lib_of_group[group_of[pos]];
    }

    c.mask.assign(N, 0);
    if (c.dirichlet) {
      std::vector<uint8_t> bvert(c.nv, 0);
      std::vector<std::pair<int32_t, int32_t>> bedge;
      std::vector<Key> bface;
      for (int64_t pos : boundary) {
        const int32_t* cv = lib_cell(pos / 4);
        const int f = int(pos % 4);
        int32_t t[3] = {cv[kFaceVerts[f][0]], cv[kFaceVerts[f][1]], cv[kFaceVerts[f][2]]};
        std::sort(t, t + 3);
        bface.push_back(Key{{t[0], t[1], t[2], 0}});
        for (int i = 0; i < 3; ++i) bvert[t[i]] = 1;
        bedge.push_back({t[0], t[1]});
        bedge.push_back({t[0], t[2]});
        bedge.push_back({t[1], t[2]});
      }
      std::sort(bedge.begin(), bedge.end());
      std::sort(bface.begin(), bface.end());
      for (int64_t i = 0; i < N; ++i) {
        int32_t d[4];
        int nd_ = 0;
        for (int r = 0; r < c.p; ++r) {
          const int32_t v = c.dof_keys[size_t(i) * c.p + r];
          if (nd_ == 0 || d[nd_ - 1] != v) d[nd_++] = v;
        }
        bool on = false;
        if (nd_ == 1)
          on = bvert[d[0]] != 0;
        else if (nd_ == 2)
          on = std::binary_search(bedge.begin(), bedge.end(), std::make_pair(d[0], d[1]));
        else if (nd_ == 3)
          on = std::binary_search(bface.begin(), bface.end(), Key{{d[0], d[1], d[2], 0}});
        c.mask[i] = on ? 1 : 0;
      }
    }
  } else {
    c.ndofs = nc * c.nd;
    c.dof_canon.resize(c.ndofs);
    for (int64_t e = 0; e < nc; ++e)
      for (int j = 0; j < c.nd; ++j) c.dof_canon[e * c.nd + j] = int64_t(c.cell_perm[e]) * c.nd + j;

    // faces of the SIPG operator (Eq. 5): owner = smaller user id, n out of the owner
    auto face_geo = [&](int64_t e, int f, double n[3], double& two_area) {
      const int32_t* cv = lib_cell(e);
      const double* A = xyz + 3 * int64_t(cv[kFaceVerts[f][0]]);
      const double* B = xyz + 3 * int64_t(cv[kFaceVerts[f][1]]);
      const double* C = xyz + 3 * int64_t(cv[kFaceVerts[f][2]]);
      const double* O = xyz + 3 * int64_t(cv[f]);
      const double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
      const double v[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
      double cr[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
      two_area = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
      double s = 0.0;
      for (int r = 0; r < 3; ++r) {
        n[r] = cr[r] / two_area;
        s += n[r] * (O[r] - A[r]);
      }
      if (s > 0)
        for (int r = 0; r < 3; ++r) n[r] = -n[r];
    };
    auto jinv_n = [&](int64_t e, const double n[3], double* a) {
      for (int k = 0; k < 3; ++k) a[k] = geo[e].Ji[k][0] * n[0] + geo[e].Ji[k][1] * n[1] + geo[e].Ji[k][2] * n[2];
    };
    // interior faces ordered by the owner's library position for locality
    struct F {
      int64_t cm, cp;
      int fm, fp, o;
    };
    std::vector<F> fl;
    fl.reserve(interior.size());
    for (auto& pr : interior) {
      int64_t e1 = pr[0] / 4, e2 = pr[1] / 4;
      int f1 = int(pr[0] % 4), f2 = int(pr[1] % 4);
      if (c.cell_perm[e2] < c.cell_perm[e1]) {
        std::swap(e1, e2);
        std::swap(f1, f2);
      }
      const int32_t* vm = lib_cell(e1);
      const int32_t* vp = lib_cell(e2);
      int o = -1;
      for (int k = 0; k < 6 && o < 0; ++k) {
        bool ok = true;
        for (int i = 0; i < 3; ++i)
          if (vp[kFaceVerts[f2][i]] != vm[kFaceVerts[f1][kPerms[k][i]]]) ok = false;
        if (ok) o = k;
      }
      if (o < 0) {
        set_error("internal: face orientation not found");
        return FEM_EMESH;
      }
      fl.push_back({e1, e2, f1, f2, o});
    }
    // faces in owner order, then inside windows of 4096 faces grouped by (local face of each side,
    // orientation): a warp of 32 consecutive faces then mostly reads the same reference-table rows
    // (broadcast) while the window keeps the owner locality
    std::sort(fl.begin(), fl.end(), [](const F& a, const F& b) { return a.cm < b.cm || (a.cm == b.cm && a.fm < b.fm); });
    for (size_t w0 = 0; w0 < fl.size(); w0 += 4096) {
      const size_t w1 = std::min(fl.size(), w0 + 4096);
      std::stable_sort(fl.begin() + w0, fl.begin() + w1, [](const F& a, const F& b) {
        const int ka = (a.fm * 4 + a.fp) * 6 + a.o, kb = (b.fm * 4 + b.fp) * 6 + b.o;
        return ka < kb;
      });
    }
    c.nfi = int64_t(fl.size());
    c.fi_cell.resize(size_t(2) * c.nfi);
    c.fi_code.resize(c.nfi);
    c.fi_geo.resize(size_t(8) * c.nfi);
    for (int64_t i = 0; i < c.nfi; ++i) {
      const F& f = fl[i];
      double n[3], two_area, am[3], ap[3];
      face_geo(f.cm, f.fm, n, two_area);
      jinv_n(f.cm, n, am);
      jinv_n(f.cp, n, ap);
      const double h = std::min(c.absdet[f.cm], c.absdet[f.cp]) / two_area;  // 3|K|/|F|
      c.fi_cell[i] = int32_t(f.cm);
      c.fi_cell[c.nfi + i] = int32_t(f.cp);
      c.fi_code[i] = f.fm | (f.fp << 2) | (f.o << 4);
      const double g8[8] = {am[0], am[1], am[2], ap[0], ap[1], ap[2], two_area, c.penalty / h};
      for (int r = 0; r < 8; ++r) c.fi_geo[size_t(r) * c.nfi + i] = g8[r];
    }
    std::sort(boundary.begin(), boundary.end());
    c.nfb = int64_t(boundary.size());
    c.fb_cell.resize(c.nfb);
    c.fb_code.resize(c.nfb);
    c.fb_geo.resize(size_t(5) * c.nfb);
    for (int64_t i = 0; i < c.nfb; ++i) {
      const int64_t e = boundary[i] / 4;
      const int f = int(boundary[i] % 4);
      double n[3], two_area, a[3];
      face_geo(e, f, n, two_area);
      jinv_n(e, n, a);
      const double h = c.absdet[e] / two_area;
      c.fb_cell[i] = int32_t(e);
      c.fb_code[i] = f;
      const double g5[5] = {a[0], a[1], a[2], two_area, c.penalty / h};
      for (int r = 0; r < 5; ++r) c.fb_geo[size_t(r) * c.nfb + i] = g5[r];
    }
  }
  if (c.kind == FEM_CG && c.scatter == FEM_SCATTER_COLOUR) colour_cells(c);
  c.ntiles = (nc + kTile - 1) / kTile;
  return FEM_OK;
}

int check_ctx(const fem_ctx* ctx) {
  if (!ctx) {
    set_error("null context");
    return FEM_EINVAL;
  }
  return FEM_OK;
}

}  // namespace

// device calls run on the calling thread's current device: it must be the context's device, since
// the context's buffers, the caller's stream and every launch have to live on one GPU
int check_device(const fem_ctx* ctx) {
  if (int s = check_ctx(ctx)) return s;
  if (ctx->c.device < 0) {
    set_error("host-only context (device = -1) cannot run device calls");
    return FEM_EINVAL;
  }
  int dev = -1;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaGetDevice failed: %s", cudaGetErrorString(e));
    return FEM_ECUDA;
  }
  if (dev != ctx->c.device) {
    set_error("the calling thread's current device %d is not the context's device %d", dev, ctx->c.device);
    return FEM_EINVAL;
  }
  return FEM_OK;
}

}  // namespace tetmf

namespace tetmf {
// y = A u without a coefficient, in any precision the space offers (shared by the smoother)
int apply_op(Ctx& c, int prec, const void* u, void* y, void* stream) {
  if (c.kind == FEM_DG) {
    if (prec == FEM_TF32 || prec == FEM_BF16) return dg_apply_tc(c, prec, u, y, stream);
    if (prec != FEM_FP64 && prec != FEM_FP32) return set_error("precision %d not offered for DG", prec), FEM_EUNSUPPORTED;
    return dg_apply(c, prec, u, y, stream);
  }
  switch (prec) {
    case FEM_FP64:
    case FEM_FP32:
      return cg_apply_simt(c, prec, u, y, nullptr, false, stream);
    case FEM_TF32:
    case FEM_BF16:
    case FEM_TF32X3:
      return cg_apply_tc(c, prec, u, y, nullptr, stream);
  }
  return set_error("unknown precision %d", prec), FEM_EUNSUPPORTED;
}
}  // namespace tetmf

using namespace tetmf;

struct fem_transfer {
  tetmf::Transfer* t = nullptr;
};

extern "C" {

const char* fem_last_error(void) { return g_err; }

int fem_create(const fem_mesh_desc* mesh, const fem_space_desc* space, fem_ctx** out) {
  g_err[0] = 0;
  if (!mesh || !space || !out || !mesh->xyz || !mesh->cells) {
    set_error("fem_create: null argument");
    return FEM_EINVAL;
  }
  *out = nullptr;
  if (mesh->n_cells < 1 || mesh->n_vertices < 4 || mesh->n_cells > INT32_MAX / 64 ||
      mesh->n_vertices > INT32_MAX) {
    set_error("fem_create: need n_cells in [1, %d] and n_vertices in [4, 2^31)", INT32_MAX / 64);
    return FEM_EINVAL;
  }
  if (space->kind != FEM_CG && space->kind != FEM_DG) {
    set_error("fem_create: kind must be FEM_CG or FEM_DG");
    return FEM_EINVAL;
  }
  if (space->degree < 1 || space->degree > 4) {
    set_error("fem_create: degree %d not supported (1..4)", space->degree);
    return FEM_EUNSUPPORTED;
  }
  if (space->reorder != FEM_REORDER_NONE && space->reorder != FEM_REORDER_MORTON) {
    set_error("fem_create: bad reorder value");
    return FEM_EINVAL;
  }
  if (space->dirichlet != 0 && space->dirichlet != 1) {
    set_error("fem_create: dirichlet must be 0 or 1");
    return FEM_EINVAL;
  }
  if (mesh->cell_nodes && space->kind != FEM_CG) {
    set_error("fem_create: curved cells (cell_nodes) are offered for CG spaces");
    return FEM_EINVAL;
  }
  if (space->scatter != FEM_SCATTER_ATOMIC && space->scatter != FEM_SCATTER_COLOUR) {
    set_error("fem_create: scatter must be FEM_SCATTER_ATOMIC or FEM_SCATTER_COLOUR");
    return FEM_EINVAL;
  }
  if (space->scatter == FEM_SCATTER_COLOUR && space->kind != FEM_CG) {
    set_error("fem_create: FEM_SCATTER_COLOUR is offered for CG spaces");
    return FEM_EINVAL;
  }
  if (space->cell_rule != FEM_RULE_STANDARD && space->cell_rule != FEM_RULE_MODIFIED) {
    set_error("fem_create: cell_rule must be FEM_RULE_STANDARD or FEM_RULE_MODIFIED");
    return FEM_EINVAL;
  }
  if (space->dirichlet && space->kind == FEM_DG) {
    set_error("fem_create: the DG space imposes Dirichlet data weakly; dirichlet must be 0");
    return FEM_EINVAL;
  }
  fem_ctx* ctx = new (std::nothrow) fem_ctx;
  if (!ctx) {
    set_error("fem_create: out of host memory");
    return FEM_ENOMEM;
  }
  Ctx& c = ctx->c;
  c.kind = space->kind;
  c.p = space->degree;
  c.dirichlet = space->dirichlet;
  c.reorder = space->reorder;
  c.scatter = space->scatter;
  c.device = space->device;
  c.penalty = space->dg_penalty_factor > 0 ? space->dg_penalty_factor : double((c.p + 1) * (c.p + 3));
  c.nv = mesh->n_vertices;
  c.nc = mesh->n_cells;
  int st = FEM_OK;
  try {
    build_tables(c.p, space->cell_rule == FEM_RULE_MODIFIED ? c.p - 1 : c.p, c.tab);
    c.nd = c.tab.nd;
    c.nq = c.tab.nq;
    c.nqf = c.tab.nqf;
    st = build_plan(c, mesh);
  } catch (const std::bad_alloc&) {
    set_error("fem_create: out of host memory");
    st = FEM_ENOMEM;
  }
  if (st == FEM_OK && c.device >= 0) st = upload(c);
  if (st != FEM_OK) {
    release(c);
    delete ctx;
    return st;
  }
  *out = ctx;
  return FEM_OK;
}

int fem_destroy(fem_ctx* ctx) {
  if (!ctx) return FEM_OK;
  release(ctx->c);
  delete ctx;
  return FEM_OK;
}

int fem_num_dofs(const fem_ctx* ctx, int64_t* n) {
  if (int s = check_ctx(ctx)) return s;
  if (!n) return set_error("null output"), FEM_EINVAL;
  *n = ctx->c.ndofs;
  return FEM_OK;
}

int fem_num_cells(const fem_ctx* ctx, int64_t* n) {
  if (int s = check_ctx(ctx)) return s;
  if (!n) return set_error("null output"), FEM_EINVAL;
  *n = ctx->c.nc;
  return FEM_OK;
}

int fem_dofs_per_cell(const fem_ctx* ctx, int32_t* nd) {
  if (int s = check_ctx(ctx)) return s;
  if (!nd) return set_error("null output"), FEM_EINVAL;
  *nd = ctx->c.nd;
  return FEM_OK;
}

int fem_num_qpoints(const fem_ctx* ctx, int32_t* nq) {
  if (int s = check_ctx(ctx)) return s;
  if (!nq) return set_error("null output"), FEM_EINVAL;
  *nq = ctx->c.nq;
  return FEM_OK;
}

int fem_num_faces(const fem_ctx* ctx, int64_t* interior, int64_t* boundary) {
  if (int s = check_ctx(ctx)) return s;
  if (!interior || !boundary) return set_error("null output"), FEM_EINVAL;
  *interior = ctx->c.nfi;
  *boundary = ctx->c.nfb;
  return FEM_OK;
}

int fem_cell_permutation(const fem_ctx* ctx, int32_t* lib_to_user) {
  if (int s = check_ctx(ctx)) return s;
  if (!lib_to_user) return set_error("null output"), FEM_EINVAL;
  std::memcpy(lib_to_user, ctx->c.cell_perm.data(), sizeof(int32_t) * ctx->c.nc);
  return FEM_OK;
}

int fem_dof_permutation(const fem_ctx* ctx, int64_t* lib_to_canonical) {
  if (int s = check_ctx(ctx)) return s;
  if (!lib_to_canonical) return set_error("null output"), FEM_EINVAL;
  std::memcpy(lib_to_canonical, ctx->c.dof_canon.data(), sizeof(int64_t) * ctx->c.ndofs);
  return FEM_OK;
}

int fem_dof_keys(const fem_ctx* ctx, int32_t* keys) {
  if (int s = check_ctx(ctx)) return s;
  if (!keys) return set_error("null output"), FEM_EINVAL;
  if (ctx->c.kind != FEM_CG) return set_error("fem_dof_keys: CG spaces only"), FEM_EINVAL;
  std::memcpy(keys, ctx->c.dof_keys.data(), sizeof(int32_t) * ctx->c.dof_keys.size());
  return FEM_OK;
}

int fem_colours(const fem_ctx* ctx, int32_t* n_colours, int64_t* starts) {
  if (int s = check_ctx(ctx)) return s;
  if (!n_colours) return set_error("null output"), FEM_EINVAL;
  const Ctx& c = ctx->c;
  *n_colours = c.colour_start.empty() ? 0 : int32_t(c.colour_start.size() - 1);
  if (starts && !c.colour_start.empty())
    std::memcpy(starts, c.colour_start.data(), sizeof(int64_t) * c.colour_start.size());
  return FEM_OK;
}

int fem_dof_coordinates(const fem_ctx* ctx, double* xyz) {
  if (int s = check_ctx(ctx)) return s;
  if (!xyz) return set_error("null output"), FEM_EINVAL;
  const Ctx& c = ctx->c;
  if (c.kind == FEM_CG) {
    // the node of a DoF is the mean of its key's vertices
    for (int64_t i = 0; i < c.ndofs; ++i)
      for (int d = 0; d < 3; ++d) {
        double s = 0.0;
        for (int r = 0; r < c.p; ++r) s += c.xyz[3 * size_t(c.dof_keys[size_t(i) * c.p + r]) + d];
        xyz[3 * i + d] = s / c.p;
      }
    return FEM_OK;
  }
  // DG: library DoF e * nd + j is node beta_j of library cell e: sum_a beta_j[a] x_a / p
  std::vector<std::array<int, 4>> betas;
  for (int b0 = 0; b0 <= c.p; ++b0)
    for (int b1 = 0; b1 <= c.p - b0; ++b1)
      for (int b2 = 0; b2 <= c.p - b0 - b1; ++b2) betas.push_back({b0, b1, b2, c.p - b0 - b1 - b2});
  for (int64_t e = 0; e < c.nc; ++e) {
    const int32_t* cv = c.ucells.data() + 4 * size_t(c.cell_perm[e]);
    for (int j = 0; j < c.nd; ++j)
      for (int d = 0; d < 3; ++d) {
        double s = 0.0;
        for (int a = 0; a < 4; ++a) s += betas[j][a] * c.xyz[3 * size_t(cv[a]) + d];
        xyz[3 * (e * c.nd + j) + d] = s / c.p;
      }
  }
  return FEM_OK;
}

int fem_dirichlet_mask(const fem_ctx* ctx, uint8_t* mask) {
  if (int s = check_ctx(ctx)) return s;
  if (!mask) return set_error("null output"), FEM_EINVAL;
  if (ctx->c.kind != FEM_CG) return set_error("fem_dirichlet_mask: CG spaces only"), FEM_EINVAL;
  std::memcpy(mask, ctx->c.mask.data(), ctx->c.mask.size());
  return FEM_OK;
}

int fem_device_status(fem_ctx* ctx, int32_t* status) {
  if (int s = check_device(ctx)) return s;
  if (!status) return set_error("null output"), FEM_EINVAL;
  return device_status(ctx->c, status);
}

int fem_chebyshev(fem_ctx* ctx, int32_t prec, const void* b, void* x, const void* diag, int32_t degree,
                  double lam_max, double ratio, void* work, void* stream) {
  if (int s = check_device(ctx)) return s;
  if (!b || !x || !diag || !work) return set_error("fem_chebyshev: null pointer"), FEM_EINVAL;
  if (degree < 1 || !(lam_max > 0.0) || !(ratio > 1.0))
    return set_error("fem_chebyshev: need degree >= 1, lam_max > 0, ratio > 1"), FEM_EINVAL;
  if (prec < FEM_FP64 || prec > FEM_TF32X3) return set_error("fem_chebyshev: unknown precision %d", prec), FEM_EUNSUPPORTED;
  return chebyshev(ctx->c, prec, b, x, diag, degree, lam_max, lam_max / ratio, work, stream);
}

int fem_lambda_max(fem_ctx* ctx, int32_t prec, const void* diag, const void* v0, int32_t iterations, void* work,
                   double* lam, void* stream) {
  if (int s = check_device(ctx)) return s;
  if (!diag || !v0 || !work || !lam) return set_error("fem_lambda_max: null pointer"), FEM_EINVAL;
  if (iterations < 1) return set_error("fem_lambda_max: iterations >= 1"), FEM_EINVAL;
  if (prec < FEM_FP64 || prec > FEM_TF32X3) return set_error("fem_lambda_max: unknown precision %d", prec), FEM_EUNSUPPORTED;
  return lambda_max(ctx->c, prec, diag, v0, iterations, work, lam, stream);
}

int fem_smoother_work_bytes(const fem_ctx* ctx, int32_t prec, int64_t* bytes) {
  if (int s = check_ctx(ctx)) return s;
  if (!bytes) return set_error("null output"), FEM_EINVAL;
  *bytes = int64_t(lambda_max_work_bytes(ctx->c, prec));
  return FEM_OK;
}

int fem_transfer_create(fem_ctx* fine, fem_ctx* coarse, fem_transfer** out) {
  if (int s = check_device(fine)) return s;
  if (int s = check_device(coarse)) return s;
  if (!out) return set_error("fem_transfer_create: null output"), FEM_EINVAL;
  fem_transfer* h = new (std::nothrow) fem_transfer;
  if (!h) return set_error("fem_transfer_create: out of host memory"), FEM_ENOMEM;
  if (int s = transfer_create(fine->c, coarse->c, &h->t)) {
    delete h;
    return s;
  }
  *out = h;
  return FEM_OK;
}

int fem_transfer_destroy(fem_transfer* t) {
  if (!t) return FEM_OK;
  transfer_destroy(t->t);
  delete t;
  return FEM_OK;
}

int fem_prolongate(fem_transfer* t, int32_t prec, const void* u_coarse, void* u_fine, void* stream) {
  if (!t || !u_coarse || !u_fine) return set_error("fem_prolongate: null pointer"), FEM_EINVAL;
  if (prec < FEM_FP64 || prec > FEM_TF32X3) return set_error("fem_prolongate: unknown precision %d", prec), FEM_EINVAL;
  return transfer_apply(*t->t, prec, true, u_coarse, u_fine, stream);
}

int fem_restrict(fem_transfer* t, int32_t prec, const void* r_fine, void* r_coarse, void* stream) {
  if (!t || !r_fine || !r_coarse) return set_error("fem_restrict: null pointer"), FEM_EINVAL;
  if (prec < FEM_FP64 || prec > FEM_TF32X3) return set_error("fem_restrict: unknown precision %d", prec), FEM_EINVAL;
  return transfer_apply(*t->t, prec, false, r_fine, r_coarse, stream);
}

int fem_apply_vector(fem_ctx* ctx, int32_t prec, int32_t ncomp, const void* u, void* y, void* stream) {
  if (int s = check_device(ctx)) return s;
  if (!u || !y || u == y) return set_error("fem_apply_vector: u and y must be distinct non-null"), FEM_EINVAL;
  if (ncomp < 1 || ncomp > 8) return set_error("fem_apply_vector: ncomp must be 1..8"), FEM_EINVAL;
  Ctx& c = ctx->c;
  if (c.kind != FEM_CG) return set_error("fem_apply_vector: CG spaces only"), FEM_EUNSUPPORTED;
  if (prec == FEM_FP64 || prec == FEM_FP32) return cg_apply_vector_simt(c, prec, ncomp, u, y, stream);
  if (prec != FEM_TF32 && prec != FEM_BF16 && prec != FEM_TF32X3)
    return set_error("fem_apply_vector: unknown precision %d", prec), FEM_EUNSUPPORTED;
  // tensor cores: one pass per component (the 128-cell tile is the GEMM's M dimension already)
  const size_t stride = size_t(c.ndofs) * sizeof(float);
  for (int comp = 0; comp < ncomp; ++comp)
    if (int s = cg_apply_tc(c, prec, static_cast<const char*>(u) + comp * stride, static_cast<char*>(y) + comp * stride,
                            nullptr, stream))
      return s;
  return FEM_OK;
}

int fem_apply(fem_ctx* ctx, int32_t prec, const void* u, void* y, const void* k, void* stream) {
  if (int s = check_device(ctx)) return s;
  if (!u || !y || u == y) return set_error("fem_apply: u and y must be distinct non-null"), FEM_EINVAL;
  Ctx& c = ctx->c;
  if (c.kind == FEM_DG) {
    if (k) return set_error("fem_apply: DG supports k = NULL only"), FEM_EUNSUPPORTED;
    if (prec == FEM_TF32 || prec == FEM_BF16) return dg_apply_tc(c, prec, u, y, stream);
    if (prec == FEM_TF32X3) return set_error("fem_apply: FEM_TF32X3 is offered for CG only"), FEM_EUNSUPPORTED;
    if (prec != FEM_FP64 && prec != FEM_FP32)
      return set_error("fem_apply: unknown precision %d", prec), FEM_EUNSUPPORTED;
    return dg_apply(c, prec, u, y, stream);
  }
  switch (prec) {
    case FEM_FP64:
    case FEM_FP32:
      return cg_apply_simt(c, prec, u, y, k, false, stream);
    case FEM_TF32:
    case FEM_BF16:
    case FEM_TF32X3:
      return cg_apply_tc(c, prec, u, y, k, stream);
    default:
      return set_error("fem_apply: unknown precision %d", prec), FEM_EUNSUPPORTED;
  }
}

int fem_selftest_wait(fem_ctx* ctx, int64_t limit_ns, int64_t* waited_ns) {
  if (int s = check_device(ctx)) return s;
  if (limit_ns < 1000 || limit_ns > 2000000000 || !waited_ns)
    return set_error("fem_selftest_wait: limit_ns in [1e3, 2e9] and an output array required"), FEM_EINVAL;
  return selftest_wait(ctx->c, limit_ns, waited_ns);
}

int fem_apply_host(fem_ctx* ctx, int32_t prec, int64_t nvec, const void* const* u_host, void* const* y_host) {
  if (int s = check_device(ctx)) return s;
  if (nvec < 1 || !u_host || !y_host) return set_error("fem_apply_host: nvec >= 1 and pointer arrays required"), FEM_EINVAL;
  for (int64_t b = 0; b < nvec; ++b)
    if (!u_host[b] || !y_host[b]) return set_error("fem_apply_host: null vector %lld", (long long)b), FEM_EINVAL;
  Ctx& c = ctx->c;
  if (c.kind == FEM_DG && prec == FEM_TF32X3)
    return set_error("fem_apply_host: FEM_TF32X3 is offered for CG only"), FEM_EUNSUPPORTED;
  if (prec < FEM_FP64 || prec > FEM_TF32X3) return set_error("fem_apply_host: unknown precision %d", prec), FEM_EUNSUPPORTED;
  return apply_host(c, prec, nvec, u_host, y_host);
}

int fem_apply_adjoint(fem_ctx* ctx, int32_t prec, const void* g, void* out, const void* k, void* stream) {
  if (int s = check_device(ctx)) return s;
  if (!g || !out || g == out) return set_error("fem_apply_adjoint: g and out must be distinct non-null"), FEM_EINVAL;
  Ctx& c = ctx->c;
  if (c.kind == FEM_DG) {
    // the SIPG form is symmetric: its adjoint is the same face/cell loop
    if (k) return set_error("fem_apply_adjoint: DG supports k = NULL only"), FEM_EUNSUPPORTED;
    if (prec == FEM_TF32 || prec == FEM_BF16) return dg_apply_tc(c, prec, g, out, stream);
    if (prec != FEM_FP64 && prec != FEM_FP32)
      return set_error("fem_apply_adjoint: unknown precision %d", prec), FEM_EUNSUPPORTED;
    return dg_apply(c, prec, g, out, stream);
  }
  if (prec != FEM_FP64 && prec != FEM_FP32)
    return set_error("fem_apply_adjoint: FEM_FP64 or FEM_FP32"), FEM_EUNSUPPORTED;
  return cg_apply_simt(c, prec, g, out, k, true, stream);
}

int fem_coeff_grad(fem_ctx* ctx, int32_t prec, const void* u, const void* g, const void* k, void* grad_u,
                   void* dk, void* stream) {
  if (int s = check_device(ctx)) return s;
  Ctx& c = ctx->c;
  if (c.kind != FEM_CG) return set_error("fem_coeff_grad: CG spaces only"), FEM_EINVAL;
  if (!u || !g || !grad_u || !dk || grad_u == u || grad_u == g || dk == u || dk == g || grad_u == dk)
    return set_error("fem_coeff_grad: null or aliased argument"), FEM_EINVAL;
  if (prec != FEM_FP64 && prec != FEM_FP32)
    return set_error("fem_coeff_grad: FEM_FP64 or FEM_FP32"), FEM_EUNSUPPORTED;
  return cg_coeff_grad(c, prec, u, g, k, grad_u, dk, stream);
}

int fem_diagonal(fem_ctx* ctx, int32_t prec, void* d, const void* k, void* stream) {
  if (int s = check_device(ctx)) return s;
  if (!d) return set_error("fem_diagonal: null output"), FEM_EINVAL;
  if (ctx->c.kind != FEM_CG) return set_error("fem_diagonal: CG spaces only"), FEM_EINVAL;
  if (prec != FEM_FP64 && prec != FEM_FP32)
    return set_error("fem_diagonal: FEM_FP64 or FEM_FP32"), FEM_EUNSUPPORTED;
  return cg_diagonal(ctx->c, prec, d, k, stream);
}

int fem_rhs_const(fem_ctx* ctx, double f, double* b, void* stream) {
  if (int s = check_device(ctx)) return s;
  if (!b) return set_error("fem_rhs_const: null output"), FEM_EINVAL;
  if (ctx->c.kind != FEM_CG) return set_error("fem_rhs_const: CG spaces only"), FEM_EINVAL;
  return cg_rhs_const(ctx->c, f, b, stream);
}

int fem_csr_build(fem_ctx* ctx, int64_t* nnz) {
  if (int s = check_device(ctx)) return s;
  if (ctx->c.kind != FEM_CG) return set_error("fem_csr_build: CG spaces only"), FEM_EINVAL;
  return csr_build(ctx->c, nnz);
}

int fem_csr_apply(fem_ctx* ctx, int32_t prec, const void* u, void* y, void* stream) {
  if (int s = check_device(ctx)) return s;
  if (!u || !y || u == y) return set_error("fem_csr_apply: u and y must be distinct non-null"), FEM_EINVAL;
  if (!ctx->c.d_csr_rowptr) return set_error("fem_csr_apply: call fem_csr_build first"), FEM_EINVAL;
  if (prec != FEM_FP64 && prec != FEM_FP32)
    return set_error("fem_csr_apply: FEM_FP64 or FEM_FP32"), FEM_EUNSUPPORTED;
  return csr_apply(ctx->c, prec, u, y, stream);
}

int fem_solve(fem_ctx* ctx, const fem_solve_opts* opts, const double* b, double* x, fem_solve_stats* stats,
              void* stream) {
  if (int s = check_device(ctx)) return s;
  if (!opts || !b || !x || !stats || (const void*)b == (const void*)x)
    return set_error("fem_solve: null or aliased argument"), FEM_EINVAL;
  if (ctx->c.kind != FEM_CG) return set_error("fem_solve: CG spaces only"), FEM_EINVAL;
  if (opts->mode != FEM_SOLVE_FP64_PCG && opts->mode != FEM_SOLVE_IR_MIXED && opts->mode != FEM_SOLVE_IR_PMG)
    return set_error("fem_solve: bad mode"), FEM_EINVAL;
  if (opts->mode != FEM_SOLVE_FP64_PCG && opts->inner_prec != FEM_FP32 && opts->inner_prec != FEM_TF32 &&
      opts->inner_prec != FEM_BF16 && opts->inner_prec != FEM_TF32X3)
    return set_error("fem_solve: inner_prec must be FEM_FP32, FEM_TF32, FEM_BF16 or FEM_TF32X3"), FEM_EUNSUPPORTED;
  if (!(opts->rtol > 0) || opts->max_inner < 1 || opts->max_outer < 1)
    return set_error("fem_solve: need rtol > 0, max_inner >= 1, max_outer >= 1"), FEM_EINVAL;
  return solve(ctx->c, opts, b, x, stats, stream);
}

}  // extern "C"
