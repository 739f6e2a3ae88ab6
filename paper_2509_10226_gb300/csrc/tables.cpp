// Reference-element tables: Grundmann-Moeller quadrature on the tetrahedron and the
// triangle, and Lagrange P_p shape functions in Silvester's product form.
//
// E (Eq. 4 of arxiv 2509.10226, Sec. 2.2) is the table of reference gradients of
// the shape functions at the quadrature points; V the table of values.  Face
// tables hold values and gradients at the face quadrature points of each of
// the four local faces (Eq. 7 counts their (1+3) n_qf x n_dof size).
#include <array>
#include <cmath>
#include <vector>

#include "internal.h"

namespace tetmf {
namespace {

// local face m is opposite local vertex m; vertices in increasing local order
const int kFaceVerts[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
const int kPerms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

void compose(int total, int parts, std::vector<int>& cur, std::vector<std::vector<int>>& out) {
  if (parts == 1) {
    cur.push_back(total);
    out.push_back(cur);
    cur.pop_back();
    return;
  }
  for (int first = 0; first <= total; ++first) {
    cur.push_back(first);
    compose(total - first, parts - 1, cur, out);
    cur.pop_back();
  }
}

std::vector<std::vector<int>> compositions(int total, int parts) {
  std::vector<std::vector<int>> out;
  std::vector<int> cur;
  compose(total, parts, cur, out);
  return out;
}

double factorial(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

// Grundmann-Moeller rule with parameter s on the unit n-simplex (degree 2s+1):
// weight (-1)^i (d+n-2i)^d / (2^{2s} i! (d+n-i)!), barycentric point
// lambda_j = (2 beta_j + 1)/(d+n-2i), |beta| = s-i; i ascending, beta
// lexicographic ascending.  Numerators and denominators are exact integers in
// double, so every weight is the correctly rounded value of the exact rational.
struct SimplexRule {
  std::vector<std::vector<double>> lambda;  // [nq][n+1]
  std::vector<std::vector<int>> beta;       // [nq][n+1]
  std::vector<int> group;                   // i of each point
  std::vector<double> w;
};

SimplexRule gm_rule(int s, int n) {
  SimplexRule r;
  const int d = 2 * s + 1;
  for (int i = 0; i <= s; ++i) {
    const double num = std::pow(double(d + n - 2 * i), d);
    const double den = std::ldexp(1.0, 2 * s) * factorial(i) * factorial(d + n - i);
    const double w = (i % 2 ? -1.0 : 1.0) * (num / den);
    const int dd = d + n - 2 * i;
    for (auto& b : compositions(s - i, n + 1)) {
      std::vector<double> lam(n + 1);
      for (int j = 0; j <= n; ++j) lam[j] = double(2 * b[j] + 1) / double(dd);
      r.lambda.push_back(lam);
      r.beta.push_back(b);
      r.group.push_back(i);
      r.w.push_back(w);
    }
  }
  return r;
}

// f(l) = prod_{m < b} (p l - m)/(m + 1) and its derivative
void silvester_factor(int p, int b, double l, double& f, double& df) {
  f = 1.0;
  df = 0.0;
  for (int m = 0; m < b; ++m) {
    const double a = (p * l - m) / (m + 1);
    df = df * a + f * (double(p) / (m + 1));
    f *= a;
  }
}

// values and reference gradients of all shape functions at reference point x
void eval_basis(int p, const std::vector<std::vector<int>>& nodes, const double x[3], double* val, double* grad,
                int nd) {
  const double lam[4] = {1.0 - x[0] - x[1] - x[2], x[0], x[1], x[2]};
  for (int j = 0; j < nd; ++j) {
    double f[4], df[4];
    for (int i = 0; i < 4; ++i) silvester_factor(p, nodes[j][i], lam[i], f[i], df[i]);
    double dl[4];
    for (int i = 0; i < 4; ++i) {
      double prod = df[i];
      for (int o = 0; o < 4; ++o)
        if (o != i) prod *= f[o];
      dl[i] = prod;
    }
    if (val) val[j] = f[0] * f[1] * f[2] * f[3];
    // d/dxhat_k = d/dlambda_k - d/dlambda_0
    if (grad)
      for (int k = 0; k < 3; ++k) grad[k * nd + j] = dl[k + 1] - dl[0];
  }
}

}  // namespace

void build_tables(int p, int s_cell, RefTables& t) {
  t.p = p;
  const auto nodes = compositions(p, 4);
  t.nd = int(nodes.size());
  const int nd = t.nd;

  const SimplexRule cell = gm_rule(s_cell, 3);
  t.nq = int(cell.w.size());
  t.xq.assign(size_t(t.nq) * 3, 0.0);
  t.wq = cell.w;
  t.E.assign(size_t(t.nq) * 3 * nd, 0.0);
  t.V.assign(size_t(t.nq) * nd, 0.0);
  for (int q = 0; q < t.nq; ++q) {
    double x[3] = {cell.lambda[q][1], cell.lambda[q][2], cell.lambda[q][3]};
    for (int k = 0; k < 3; ++k) t.xq[q * 3 + k] = x[k];
    eval_basis(p, nodes, x, &t.V[size_t(q) * nd], &t.E[size_t(q) * 3 * nd], nd);
  }

  // second-order geometry basis (curved cells) at the cell points
  {
    const auto nodes2 = compositions(2, 4);
    t.G2.assign(size_t(t.nq) * 3 * 10, 0.0);
    for (int q = 0; q < t.nq; ++q) eval_basis(2, nodes2, &t.xq[q * 3], nullptr, &t.G2[size_t(q) * 30], 10);
  }

  const SimplexRule tri = gm_rule(p, 2);
  t.nqf = int(tri.w.size());
  t.wqf = tri.w;
  t.Vf.assign(size_t(4) * t.nqf * nd, 0.0);
  t.Ef.assign(size_t(4) * t.nqf * 3 * nd, 0.0);
  const double ref[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int m = 0; m < 4; ++m)
    for (int q = 0; q < t.nqf; ++q) {
      double x[3] = {0, 0, 0};
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) x[k] += tri.lambda[q][i] * ref[kFaceVerts[m][i]][k];
      eval_basis(p, nodes, x, &t.Vf[(size_t(m) * t.nqf + q) * nd], &t.Ef[(size_t(m) * t.nqf + q) * 3 * nd], nd);
    }

  // the point with barycentrics mu w.r.t. the minus side's face vertices has
  // barycentrics mu'_i = mu_{pi(i)} w.r.t. the plus side's vertices when
  // V+[i] = V-[pi(i)]; GM triangle points are closed under such permutations
  t.fperm.assign(size_t(6) * t.nqf, -1);
  for (int o = 0; o < 6; ++o)
    for (int q = 0; q < t.nqf; ++q) {
      std::vector<int> b(3);
      for (int i = 0; i < 3; ++i) b[i] = tri.beta[q][kPerms[o][i]];
      for (int r = 0; r < t.nqf; ++r)
        if (tri.group[r] == tri.group[q] && tri.beta[r] == b) t.fperm[o * t.nqf + q] = r;
    }
}

void fine_nodes_coarse_values(int p_fine, int p_coarse, std::vector<double>& tab) {
  const auto fine = compositions(p_fine, 4), coarse = compositions(p_coarse, 4);
  const int ndf = int(fine.size()), ndc = int(coarse.size());
  tab.assign(size_t(ndf) * ndc, 0.0);
  for (int i = 0; i < ndf; ++i) {
    const double x[3] = {double(fine[i][1]) / p_fine, double(fine[i][2]) / p_fine, double(fine[i][3]) / p_fine};
    eval_basis(p_coarse, coarse, x, &tab[size_t(i) * ndc], nullptr, ndc);
  }
}

TableLayout tables_layout(const RefTables& t) {
  TableLayout L;
  int64_t off = 0;
  L.E = off;
  off += int64_t(t.nq) * 3 * t.nd;
  L.w = off;
  off += t.nq;
  L.V = off;
  off += int64_t(t.nq) * t.nd;
  L.wf = off;
  off += t.nqf;
  L.Vf = off;
  off += int64_t(4) * t.nqf * t.nd;
  L.Ef = off;
  off += int64_t(4) * t.nqf * 3 * t.nd;
  L.total = off;
  return L;
}

}  // namespace tetmf
