// Internal declarations shared by the host set-up and the CUDA translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "tetmf.h"

namespace tetmf {

constexpr int kTile = 128;  // cells per batch: one thread (or one TMEM lane) per cell

void set_error(const char* fmt, ...);

// Reference-element tables built by the library (Sec. 2.2, Eq. 4).
struct RefTables {
  int p = 0, nd = 0, nq = 0, nqf = 0;
  std::vector<double> xq;     // [nq][3] cell quadrature points (reference coords)
  std::vector<double> wq;     // [nq]
  std::vector<double> E;      // [nq][3][nd] d phi_j / d xhat_k at xq
  std::vector<double> V;      // [nq][nd] phi_j at xq
  std::vector<double> wqf;    // [nqf] triangle weights (sum 1/2)
  std::vector<double> Vf;     // [4][nqf][nd] values at face points of local face m
  std::vector<double> Ef;     // [4][nqf][3][nd] reference gradients there
  std::vector<int32_t> fperm; // [6][nqf] face point index seen from the other side
  std::vector<double> G2;     // [nq][3][10] reference gradients of the second-order geometry basis
};

// cell rule: Grundmann-Moeller with s = s_cell (p, or p - 1 for the modified integration of
// Sec. 3.3); face rule: s = p
void build_tables(int p, int s_cell, RefTables& t);

struct Ctx {
  // plan
  int kind = FEM_CG, p = 1, nd = 4, nq = 5, nqf = 4, dirichlet = 0, reorder = 1, device = -1;
  int scatter = 0;                  // FEM_SCATTER_ATOMIC / FEM_SCATTER_COLOUR
  std::vector<int64_t> colour_start;  // colour k = library cells [start[k], start[k+1]) (colour mode)
  double penalty = 0.0;
  int64_t nv = 0, nc = 0, ndofs = 0, ntiles = 0;
  RefTables tab;
  std::vector<int32_t> cell_perm;   // lib -> user
  std::vector<double> xyz;          // [nv][3] user vertex coordinates (copy)
  std::vector<int32_t> ucells;      // [nc][4] user cells (copy)
  std::vector<int32_t> cell_dofs;   // [nc][nd] lib DoF ids (CG; unmasked)
  std::vector<int32_t> dof_keys;    // [ndofs][p] (CG)
  std::vector<int64_t> dof_canon;   // lib DoF -> canonical DoF
  std::vector<uint8_t> mask;        // [ndofs] Dirichlet
  std::vector<double> metric;       // [nc][6] |det J| J^-1 J^-T (xx, xy, xz, yy, yz, zz)
  std::vector<double> absdet;       // [nc]
  bool curved = false;              // second-order cells: metric per quadrature point
  std::vector<double> qmetric;      // [nc][nq][6] |det J_q| J_q^-1 J_q^-T (curved)
  std::vector<double> qdet;         // [nc][nq] |det J_q| (curved)
  // DG faces (library cell ids)
  int64_t nfi = 0, nfb = 0;
  std::vector<int32_t> fi_cell;     // [2][nfi] minus, plus
  std::vector<int32_t> fi_code;     // [nfi] f- | f+ << 2 | o << 4
  std::vector<double> fi_geo;       // [8][nfi] a-(3) a+(3) 2|F| tau
  std::vector<int32_t> fb_cell;     // [nfb]
  std::vector<int32_t> fb_code;     // [nfb] f
  std::vector<double> fb_geo;       // [5][nfb] a(3) 2|F| tau

  // device buffers (owned)
  int32_t* d_idx = nullptr;         // [ntiles][nd][kTile], constrained DoF -> -1-id
  double* d_metric64 = nullptr;     // [ntiles][6][kTile]
  float* d_metric32 = nullptr;
  double* d_qmetric64 = nullptr;    // curved: [ntiles][nq][6][kTile]
  float* d_qmetric32 = nullptr;
  double* d_qdet64 = nullptr;       // curved: [ntiles][nq][kTile]
  double* d_absdet = nullptr;       // [nc]
  uint8_t* d_mask = nullptr;        // [ndofs] or null
  double* d_tab64 = nullptr;        // packed tables, see tables_layout
  float* d_tab32 = nullptr;
  int32_t* d_fperm = nullptr;
  int32_t* d_fi_cell = nullptr;
  int32_t* d_fi_code = nullptr;
  double* d_fi_geo64 = nullptr;
  float* d_fi_geo32 = nullptr;
  int32_t* d_fb_cell = nullptr;
  int32_t* d_fb_code = nullptr;
  double* d_fb_geo64 = nullptr;
  float* d_fb_geo32 = nullptr;
  // tile-local group lists (CG): the distinct 16-byte groups (DoFs 4g .. 4g+3) holding each tile's
  // unconstrained DoFs, and each (cell, local node) as its position in the tile's staging
  // (4 x the group's place in the list + DoF mod 4; constrained nodes use the zero slot 4 L)
  int64_t* d_tl_span = nullptr;     // [ntiles][2]: offset (a multiple of 4) and length of the list
  int32_t* d_tl_list = nullptr;     // group indices, each tile's list padded to a multiple of 4 entries
  uint16_t* d_tl_lidx = nullptr;    // [ntiles][ndp / 2][kTile] pairs of 16-bit positions
  int32_t tl_max = 0;               // longest list (groups)
  // tensor-core operand images (shared-memory byte images of E^T and E)
  void* d_tc_tf32 = nullptr;
  void* d_tc_bf16 = nullptr;
  void* d_tc_tf32x3 = nullptr;      // high then low TF32 parts (3xTF32)
  // DG tensor-core face loop: interior and boundary faces in tiles of 128 faces, in the order of
  // their minus cells; each side's cell relabelled so that the face is its local face 0 with the
  // face's vertices in increasing global order (one pair of tables for all); a boundary face has
  // the minus cell on both sides and its mirror flag set
  int64_t dg_ntiles = 0;
  int32_t* d_dgt_cell = nullptr;    // [dg_ntiles][2][128] minus, plus (padding faces: 0, 0)
  int32_t* d_dgt_perm = nullptr;    // [dg_ntiles][128] relabelling of each side: minus | plus << 8, 1 << 16 mirror
  float* d_dgt_geo = nullptr;       // [dg_ntiles][8][128] a-(3) a+(3) 2|F| tau, relabelled frames (padding: 0)
  int8_t* d_dg_dperm = nullptr;     // [24][nd rounded up to 16] old local DoF of each new local DoF, per relabelling
  void* d_dg_img_tf32 = nullptr;    // face-0 evaluation and integration tables (2 operand images)
  void* d_dg_img_bf16 = nullptr;
  // CSR comparator
  int64_t csr_nnz = 0;
  int64_t* d_csr_rowptr = nullptr;
  int32_t* d_csr_col = nullptr;
  double* d_csr_val64 = nullptr;
  float* d_csr_val32 = nullptr;
  int32_t* d_status = nullptr;      // device error word (bounded waits that gave up)
  // solver work space
  void* d_work = nullptr;
  size_t work_bytes = 0;

  void* pmg = nullptr;               // p-multigrid hierarchy of the solver (pmg.cu), built on first use
  void* host_pipe = nullptr;         // buffers and streams of fem_apply_host (host.cu), built on first use
  void* noalloc_work = nullptr;      // device address of the static work array of fem_solve_noalloc (solve.cu),
                                     // looked up by the first such call on this context
  std::vector<void*> allocations;   // every cudaMalloc, freed by destroy
};

// Offsets (in elements) of the packed reference tables on the device.
struct TableLayout {
  int64_t E, w, V, wf, Vf, Ef, total;
};
TableLayout tables_layout(const RefTables& t);

// argument check of every device entry point (setup.cpp): a context on a device, and that device
// current on the calling thread; FEM_EINVAL (or FEM_ECUDA) with the message set otherwise
int check_device(const fem_ctx* ctx);

// set-up steps implemented in .cu files
int upload(Ctx& c);
int device_status(Ctx& c, int32_t* out);
void release(Ctx& c);

// hot-call launchers (return FEM_* status)
int cg_apply_simt(Ctx& c, int prec, const void* u, void* y, const void* k, bool transpose, void* stream);
int cg_apply_tc(Ctx& c, int prec, const void* u, void* y, const void* k, void* stream);
int cg_coeff_grad(Ctx& c, int prec, const void* u, const void* g, const void* k, void* grad_u, void* dk,
                  void* stream);
int cg_diagonal(Ctx& c, int prec, void* d, const void* k, void* stream);
int cg_rhs_const(Ctx& c, double f, double* b, void* stream);
int dg_apply(Ctx& c, int prec, const void* u, void* y, void* stream);
int csr_build(Ctx& c, int64_t* nnz);
int csr_apply(Ctx& c, int prec, const void* u, void* y, void* stream);
int solve(Ctx& c, const fem_solve_opts* o, const double* b, double* x, fem_solve_stats* st, void* stream);
int tc_prepare(Ctx& c);
int dg_tc_prepare(Ctx& c);
int dg_apply_tc(Ctx& c, int prec, const void* u, void* y, void* stream);
int apply_op(Ctx& c, int prec, const void* u, void* y, void* stream);  // y = A u, no coefficient
int cg_apply_vector_simt(Ctx& c, int prec, int ncomp, const void* u, void* y, void* stream);
int chebyshev(Ctx& c, int prec, const void* b, void* x, const void* diag, int degree, double lam_max,
              double lam_min, void* work, void* stream);
int lambda_max(Ctx& c, int prec, const void* diag, const void* v0, int iterations, void* work, double* lam,
               void* stream);
size_t lambda_max_work_bytes(const Ctx& c, int prec);  // also enough for chebyshev
// p-multigrid (pmg.cu)
int pmg_setup(Ctx& c, int prec, const float* diag, int degree, int coarse_steps, void* stream);
int pmg_inner_solve(Ctx& c, const float* diag, float* r, float* d, float* p, float* q, double rtol, int max_it,
                    int& iters, void* stream);
void pmg_release(Ctx& c);
// host-buffer apply (host.cu): y_host[b] = A u_host[b], b < nvec, blocking
int apply_host(Ctx& c, int prec, int64_t nvec, const void* const* u_host, void* const* y_host);
void host_pipe_release(Ctx& c);
// bounded-wait diagnostics (selftest.cu): waits that nothing completes give up after limit_ns
int selftest_wait(Ctx& c, int64_t limit_ns, int64_t* waited_ns);
// p-transfer (transfer.cu)
struct Transfer;
int transfer_create(Ctx& fine, Ctx& coarse, Transfer** out);
void transfer_destroy(Transfer* t);
int transfer_apply(Transfer& t, int prec, bool prolong, const void* in, void* out, void* stream);
// tab[i][j] = phi_j of degree p_coarse at the reference node i of degree p_fine (beta order)
void fine_nodes_coarse_values(int p_fine, int p_coarse, std::vector<double>& tab);

}  // namespace tetmf

struct fem_ctx {
  tetmf::Ctx c;
};
