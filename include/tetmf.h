/*
 * tetmf — matrix-free Laplace/Poisson operators on affine tetrahedral meshes
 * (continuous P_p and SIPG discontinuous P_p), GB300 / sm_103a.
 *
 * C ABI.  Every entry point returns an int status (FEM_OK == 0 on success);
 * the text of the last error of the calling thread is available from
 * fem_last_error().  No C++ exception crosses this boundary.  Pointers are
 * plain host or device addresses as stated per argument; nothing here
 * refers to PyTorch.
 *
 * Operation (arxiv 2509.10226, Sec. 2.2, Eq. 3):
 *     y = A(u) = sum_e G_e^T E^T D_e E G_e u
 * G_e gathers the cell's DoF values, E (Eq. 4) holds the reference gradients
 * of the shape functions at the quadrature points, D_e applies J^-T, the
 * quadrature weight times |det J| (times the optional coefficient k_q) and
 * J^-1, E^T integrates back and G_e^T scatter-adds.  For the discontinuous
 * space (Eq. 2, Eq. 5) a face loop adds the SIPG flux terms.
 *
 * Conventions fixed by this library (the paper leaves them open):
 *   - quadrature: Grundmann-Moeller with s = p on cells (nq = 5/15/35/70 for
 *     p = 1..4; s = p - 1 with FEM_RULE_MODIFIED) and on faces (nqf =
 *     4/10/20/35); point order i ascending then beta lexicographic ascending;
 *     coefficient arrays k/dk use this order;
 *   - J = [x1-x0 | x2-x0 | x3-x0] from the user's vertex order of each cell;
 *     |det J| is used, so either orientation is accepted;
 *   - local shape-function order: beta in N^4, |beta| = p, lexicographic
 *     ascending, node (beta_1, beta_2, beta_3)/p on the reference cell;
 *   - SIPG: face owner K^- = adjacent cell with the smaller user id, n the unit
 *     normal out of K^-; tau_F = eta / h_F with h_F = min_K 3|K|/|F| and
 *     eta = (p+1)(p+3) unless given; boundary faces are homogeneous Dirichlet
 *     by the mirror principle (u+ = -u-, grad u+ = grad u-);
 *   - CG Dirichlet (optional): DoFs whose vertices lie on one boundary face
 *     are constrained; the operator is P A P + (I - P) (identity rows).
 *
 * Numbering.  The library renumbers cells (Morton order of centroids unless
 * reorder = FEM_REORDER_NONE) and DoFs (grouped by the set of 128-cell
 * batches of the library cell order that touch them, batches in order; within a
 * group, first touch in cell order).  Vectors
 * passed to the hot calls are in library order; fem_dof_permutation and
 * fem_cell_permutation translate.  Coefficients k and dk are [n_cells][nq]
 * row-major in library cell order.
 *
 * Streams.  Hot calls are asynchronous on the caller's CUDA stream, passed as
 * void* (a cudaStream_t; NULL = legacy default stream).  They allocate
 * nothing and never synchronise.  The calls documented as blocking
 * (fem_solve, fem_lambda_max, fem_apply_host, fem_selftest_wait) return
 * with their work complete.  Vector pointers of hot calls are caller-owned
 * device memory of the context's device; fem_apply_host takes host
 * pointers.  Every device call checks that the calling thread's current
 * device is the context's device and returns FEM_EINVAL before anything is
 * launched otherwise.  A context is not thread-safe; distinct contexts are
 * independent.
 */
#ifndef TETMF_H
#define TETMF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define FEM_OK 0
#define FEM_EINVAL 1        /* bad argument: null pointer, size, enum value  */
#define FEM_EMESH 2         /* degenerate cell, vertex id out of range,      */
                            /* face shared by more than two cells            */
#define FEM_EUNSUPPORTED 3  /* degree outside 1..4, precision not offered    */
#define FEM_ECUDA 4         /* a CUDA runtime call or kernel launch failed   */
#define FEM_ENOTCONV 5      /* solver hit its iteration cap                  */
#define FEM_ENOMEM 6        /* host or device allocation failed (set-up)     */

/* ---- enums ----------------------------------------------------------- */
#define FEM_CG 0
#define FEM_DG 1

/* arithmetic of the interpolation products; vectors are double for FEM_FP64
 * and float for every other value */
#define FEM_FP64 0   /* FP64 FMA units                                      */
#define FEM_FP32 1   /* FP32 FMA units                                      */
#define FEM_TF32 2   /* tcgen05 tensor cores, TF32 operands, FP32 accumulate */
#define FEM_BF16 3   /* tcgen05 tensor cores, BF16 operands, FP32 accumulate */
#define FEM_TF32X3 4 /* tcgen05 tensor cores, 3xTF32: every operand split into */
                     /* a TF32 high part and a TF32 low part, products       */
                     /* hi*hi + hi*lo + lo*hi accumulated in FP32 (CG,      */
                     /* degrees 1-3)                                        */

#define FEM_REORDER_NONE 0
#define FEM_REORDER_MORTON 1

/* scatter of the CG FP64/FP32 apply and adjoint */
#define FEM_SCATTER_ATOMIC 0  /* atomic adds (default)                           */
#define FEM_SCATTER_COLOUR 1  /* cells ordered by colour (no two cells of one    */
                              /* colour share a DoF), one launch per colour with */
                              /* plain adds: bitwise reproducible results        */

/* cell quadrature (face integrals always use the standard rule) */
#define FEM_RULE_STANDARD 0  /* Grundmann-Moeller s = p: exact to degree 2p+1      */
#define FEM_RULE_MODIFIED 1  /* s = p-1: exact to degree 2p-1 >= 2p-2, the degree */
                             /* of grad phi_i . grad phi_j on an affine cell      */
                             /* (Sec. 3.3); nq = 1/5/15/35 for p = 1..4          */

#define FEM_SOLVE_FP64_PCG 0   /* Jacobi-PCG, FP64 operator and vectors      */
#define FEM_SOLVE_IR_MIXED 1   /* FP64 iterative refinement around an inner  */
                               /* FP32-vector Jacobi-PCG (inner_prec apply)  */
#define FEM_SOLVE_IR_PMG 2     /* the same refinement around an inner flexible */
                               /* CG preconditioned by a two-level p-multigrid */
                               /* V-cycle (Chebyshev-Jacobi smoothing on the   */
                               /* space, fixed-step Jacobi-PCG on linear       */
                               /* elements of the same mesh; degree >= 2,      */
                               /* straight cells, atomic scatter)              */

typedef struct fem_ctx fem_ctx;

/* Mesh, host memory, copied by fem_create (the caller may free it after). */
typedef struct {
  int64_t n_vertices;
  const double* xyz;      /* [n_vertices][3]                                */
  int64_t n_cells;
  const int32_t* cells;   /* [n_cells][4] vertex ids, user vertex order     */
  const double* cell_nodes; /* NULL (straight cells) or [n_cells][10][3]:   */
                          /* second-order geometry nodes of each cell, the */
                          /* points sum_a beta_a x_a / 2 (|beta| = 2, beta */
                          /* lexicographic, user vertex order) moved onto  */
                          /* the curved cell; the map x(x_hat) is their P2 */
                          /* interpolant and J^-T, |det J| are taken at    */
                          /* every quadrature point (Sec. 3.2).  CG only;  */
                          /* nodes shared by cells must coincide.          */
} fem_mesh_desc;

typedef struct {
  int32_t kind;              /* FEM_CG or FEM_DG                             */
  int32_t degree;            /* p in 1..4                                    */
  int32_t dirichlet;         /* CG only: 0 none (pure Neumann), 1 homogeneous */
                             /* Dirichlet on the whole boundary              */
  int32_t reorder;           /* FEM_REORDER_MORTON (default) or _NONE        */
  double dg_penalty_factor;  /* eta; <= 0 selects (p+1)(p+3)                 */
  int32_t device;            /* CUDA device ordinal; -1 builds a host-only   */
                             /* plan: queries work, hot calls return EINVAL  */
  int32_t cell_rule;         /* FEM_RULE_STANDARD (0) or FEM_RULE_MODIFIED   */
  int32_t scatter;           /* FEM_SCATTER_ATOMIC (0) or FEM_SCATTER_COLOUR */
                             /* (CG only; tensor-core precisions and the     */
                             /* other hot calls keep atomic adds)            */
} fem_space_desc;

/* ---- set-up (synchronous) ------------------------------------------ */

/* Validate the mesh, build the plan (reordering, DoF numbering, geometry,
 * reference tables, faces) in FP64 on the host and upload it to `device`.
 * Sec. 2.3-2.5.  On success *out owns every internal buffer.
 * Errors: EINVAL (null pointers, n_cells outside [1, 2^25 - 1], n_vertices
 * outside [4, 2^31), bad enum), EUNSUPPORTED
 * (degree), EMESH (vertex id out of range, |det J| <= 1e-12 * (longest edge)^3,
 * non-manifold face), ENOMEM, ECUDA. */
int fem_create(const fem_mesh_desc* mesh, const fem_space_desc* space, fem_ctx** out);

/* Free the context and its device buffers (synchronises the device). NULL ok. */
int fem_destroy(fem_ctx* ctx);

/* Last error message of the calling thread ("" if none).  Static storage. */
const char* fem_last_error(void);

/* ---- queries (host, synchronous) ----------------------------------- */
int fem_num_dofs(const fem_ctx* ctx, int64_t* n);         /* global DoFs N   */
int fem_num_cells(const fem_ctx* ctx, int64_t* n);
int fem_dofs_per_cell(const fem_ctx* ctx, int32_t* nd);   /* (p+1)(p+2)(p+3)/6 */
int fem_num_qpoints(const fem_ctx* ctx, int32_t* nq);     /* cell rule size  */
int fem_num_faces(const fem_ctx* ctx, int64_t* interior, int64_t* boundary);

/* lib_to_user[c] = user id of library cell c; array of n_cells. */
int fem_cell_permutation(const fem_ctx* ctx, int32_t* lib_to_user);

/* lib_to_canonical[i] = canonical number of library DoF i; array of N.
 * CG canonical order: lexicographic order of the DoF keys (below).
 * DG canonical number: user_cell * nd + local index. */
int fem_dof_permutation(const fem_ctx* ctx, int64_t* lib_to_canonical);

/* CG only: keys[i][0..p-1] = sorted user vertex ids whose mean is the node of
 * library DoF i (vertex v_m of a cell repeated beta_m times).  Array N*p. */
int fem_dof_keys(const fem_ctx* ctx, int32_t* keys);

/* Colour mode: *n_colours = number of colours (0 in atomic mode) and, if
 * starts is not NULL, starts[0..n_colours] = first library cell of each
 * colour (colour k = cells [starts[k], starts[k+1])).  Host memory. */
int fem_colours(const fem_ctx* ctx, int32_t* n_colours, int64_t* starts);

/* xyz[i][0..2] = physical position of the node of library DoF i (the point
 * where its shape function is 1): sum_m beta_m x_m / p over the vertices x_m
 * of a cell containing it.  Array N*3 of double, host memory. */
int fem_dof_coordinates(const fem_ctx* ctx, double* xyz);

/* CG only: mask[i] = 1 if library DoF i is Dirichlet-constrained.  Array N. */
int fem_dirichlet_mask(const fem_ctx* ctx, uint8_t* mask);

/* Device error word of the context, then reset to 0 (synchronises the
 * device).  0 = no kernel reported a problem; bit 0 = a tensor-core kernel
 * gave up waiting for an MMA completion (bounded wait, about 1 s) and
 * returned without finishing its tiles.  Kernels never trap. */
int fem_device_status(fem_ctx* ctx, int32_t* status);

/* Diagnostics of the bounded waits (no GPU fault involved): runs one CTA of
 * two warpgroups that allocates TMEM and then waits, through the tensor-core
 * kernels' own wait helper, on two mbarriers that nothing completes.  The
 * first wait gives up after limit_ns (1e3..2e9) and raises the CTA's abort
 * flag, the other returns at once; the CTA frees its TMEM and sets bit 0 of the
 * device status word, exactly as an apply kernel that gave up would.
 * waited_ns[0..1] receive the two waits' durations.  Blocking (synchronises
 * the device); the context stays usable.  Read the word with
 * fem_device_status. */
int fem_selftest_wait(fem_ctx* ctx, int64_t limit_ns, int64_t* waited_ns);

/* Arithmetic-throughput probe (no counterpart in the paper; it measures the
 * denominators of the FP64 and FP32 rooflines the SIMT applies are reported
 * against).  Launches 4 x (SM count) blocks of 256 threads on the current
 * device, each thread running `iters` (a multiple of 8 in 8..2^30) iterations of eight
 * independent FMA chains: kind 0 = FP64 fma, 1 = FP32 fma, 2 = packed FP32x2
 * fma.  *flops (host) receives the floating-point operations launched (an FMA
 * counts 2).  sink: device double[1], written only in a case that cannot occur
 * (it keeps the compiler from removing the loop).  Asynchronous on `stream`;
 * time it with events.  Errors: EINVAL, ECUDA. */
int fem_fma_probe(int32_t kind, int64_t iters, double* sink, double* flops, void* stream);

/* ---- hot calls (asynchronous on `stream`, allocate nothing) -------- */

/* y = A(k) u.  u, y: device vectors of N values (double for FEM_FP64, float
 * otherwise), library order, must not alias.  k: NULL (k = 1) or device
 * [n_cells][nq] of the vector type.  Eq. 3 (CG), Eq. 5 (DG).  DG supports
 * k = NULL only; its FEM_TF32 / FEM_BF16 path (cell and face products on the
 * tensor cores, boundary faces with the mirror state in the same face tiles)
 * wants u and y 16-byte aligned (EINVAL otherwise).  Errors: EINVAL,
 * EUNSUPPORTED, ECUDA. */
int fem_apply(fem_ctx* ctx, int32_t prec, const void* u, void* y, const void* k, void* stream);

/* Vector Laplacian with ncomp (1..8) independent components, y_c = A u_c
 * (the vector-valued Poisson problem of Sec. 3.1): u, y are [ncomp][N]
 * component-major device arrays.  FEM_FP64 / FEM_FP32 run components-batched
 * (each cell's indices, metric and tables are loaded once and serve every
 * component); the tensor-core precisions run one pass per component.  CG
 * only, no coefficient.  Errors as fem_apply. */
int fem_apply_vector(fem_ctx* ctx, int32_t prec, int32_t ncomp, const void* u, void* y, void* stream);

/* out = A(k)^T g (the transposed chain G^T E^T D^T E G; D_e is symmetric).
 * Same arguments and layouts as fem_apply. */
int fem_apply_adjoint(fem_ctx* ctx, int32_t prec, const void* g, void* out, const void* k, void* stream);

/* Backward of L = <g, A(k) u> for CG, in one pass over the cells:
 * grad_u = A(k)^T g (N values) and dk[e][q] = w_q |det J_e| (grad u . grad g)
 * at quadrature point q of library cell e ([n_cells][nq]).  FEM_FP64 or
 * FEM_FP32.  grad_u and dk must not alias the inputs. */
int fem_coeff_grad(fem_ctx* ctx, int32_t prec, const void* u, const void* g, const void* k,
                   void* grad_u, void* dk, void* stream);

/* d = diag(A(k)) (Jacobi), N values; Dirichlet rows give 1.  FP64 or FP32. */
int fem_diagonal(fem_ctx* ctx, int32_t prec, void* d, const void* k, void* stream);

/* b_i = int f phi_i for a constant f (CG; FP64; Dirichlet entries 0). */
int fem_rhs_const(fem_ctx* ctx, double f, double* b, void* stream);

/* ---- host-buffer apply (blocking) ---------------------------------- */

/* y_host[b] = A u_host[b] for b = 0..nvec-1 with HOST vectors (a stream of
 * requests): u_host, y_host are arrays of nvec host pointers, each to N values
 * (double for FEM_FP64, float otherwise) in library order; no coefficient.
 * The same buffer may appear several times; page-locked (pinned) memory gives
 * the full link bandwidth.  The vectors pass through two device input and two
 * device output buffers owned by the context (allocated on the first call and
 * kept until fem_destroy): the copy of vector b+1 in, the apply of vector b
 * and the copy of vector b-1 out run concurrently on three streams of the
 * context.  The operator is fem_apply's (Eq. 3, Eq. 5).  Blocking: returns
 * when every y_host[b] is written; one call at a time per context (the slots
 * and streams are the context's).  Errors: EINVAL (nvec < 1, a null
 * pointer), EUNSUPPORTED, ENOMEM, ECUDA. */
int fem_apply_host(fem_ctx* ctx, int32_t prec, int64_t nvec, const void* const* u_host, void* const* y_host);

/* ---- smoother (Chebyshev-Jacobi, the smoother of Sec. 4.1's multigrid) */

/* `degree` steps of Chebyshev iteration for A x = b preconditioned by
 * D = diag(A), tuned to the interval [lam_max / ratio, lam_max] of the
 * spectrum of D^-1 A: with theta, delta the centre and half width,
 * sigma = theta / delta, d_0 = D^-1 r_0 / theta, rho_0 = 1 / sigma,
 * rho_k = 1 / (2 sigma - rho_{k-1}),
 * d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) D^-1 r_k,
 * x_{k+1} = x_k + d_k, r_k = b - A x_k.  x holds x_0 on entry and x_degree on
 * return.  b, x, diag: device vectors of N (double for FEM_FP64, float
 * otherwise; diag as fem_diagonal gives it, Dirichlet rows 1); the apply runs
 * in `prec` (no coefficient).  work: device scratch of
 * fem_smoother_work_bytes bytes.  Asynchronous, allocates nothing.  Errors:
 * EINVAL (null pointer, degree < 1, lam_max <= 0, ratio <= 1), EUNSUPPORTED,
 * ECUDA. */
int fem_chebyshev(fem_ctx* ctx, int32_t prec, const void* b, void* x, const void* diag, int32_t degree,
                  double lam_max, double ratio, void* work, void* stream);

/* Largest eigenvalue of D^-1 A by `iterations` steps of power iteration from
 * v0 (device, N values, not modified): v <- D^-1 A v / |D^-1 A v|_2, and
 * *lam = (v, A v) / (v, D v) of the last iterate before its update.  work as
 * for fem_chebyshev.  Blocking: reads three FP64 sums back every step
 * (deterministic two-pass reductions). */
int fem_lambda_max(fem_ctx* ctx, int32_t prec, const void* diag, const void* v0, int32_t iterations,
                   void* work, double* lam, void* stream);

/* Bytes of device scratch that fem_chebyshev and fem_lambda_max need. */
int fem_smoother_work_bytes(const fem_ctx* ctx, int32_t prec, int64_t* bytes);

/* ---- p-transfer (the p-levels of Sec. 4.1's hybrid multigrid) --------- */

typedef struct fem_transfer fem_transfer;

/* Transfer between two CG contexts on the same mesh (same cells, cell order,
 * Dirichlet choice and device; build both with the same reordering and
 * atomic scatter), fine degree above the coarse one.  Both contexts must
 * outlive the transfer.  Errors: EINVAL, ENOMEM, ECUDA, EUNSUPPORTED. */
int fem_transfer_create(fem_ctx* fine, fem_ctx* coarse, fem_transfer** out);
int fem_transfer_destroy(fem_transfer* t);

/* u_fine = P u_coarse: the coarse function evaluated at the fine nodes (exact:
 * the coarse space is contained in the fine one); constrained fine entries
 * are 0, constrained coarse entries of u_coarse are ignored.  Every fine
 * entry is written.  prec FEM_FP64: double vectors, otherwise float.
 * Asynchronous, allocates nothing. */
int fem_prolongate(fem_transfer* t, int32_t prec, const void* u_coarse, void* u_fine, void* stream);

/* r_coarse = P^T r_fine (constrained entries: 0 in, 0 out).  Asynchronous. */
int fem_restrict(fem_transfer* t, int32_t prec, const void* r_fine, void* r_coarse, void* stream);

/* ---- assembled comparator (Sec. 3.2) ------------------------------- */

/* Assemble the same operator as a CSR matrix on the device (CG only;
 * allocates, synchronous).  *nnz receives the number of stored entries. */
int fem_csr_build(fem_ctx* ctx, int64_t* nnz);

/* y = A u with the assembled CSR matrix (FEM_FP64 or FEM_FP32 values). */
int fem_csr_apply(fem_ctx* ctx, int32_t prec, const void* u, void* y, void* stream);

/* ---- solve (blocking) ---------------------------------------------- */
typedef struct {
  int32_t mode;          /* FEM_SOLVE_FP64_PCG, _IR_MIXED or _IR_PMG         */
  int32_t inner_prec;    /* IR: FEM_FP32, FEM_TF32, FEM_BF16 or FEM_TF32X3    */
  double rtol;           /* stop when ||b - A x|| / ||b|| <= rtol (FP64)     */
  double inner_rtol;     /* IR: relative reduction asked of each inner solve */
  int32_t max_outer;     /* IR outer iterations cap                          */
  int32_t max_inner;     /* PCG iterations cap (per inner solve for IR, in   */
                         /* total for FP64_PCG)                              */
  int32_t smoother_degree; /* IR_PMG: Chebyshev steps per smoothing (0: 5)   */
  int32_t coarse_steps;  /* IR_PMG: coarse Jacobi-PCG steps (0: 20)          */
} fem_solve_opts;

typedef struct {
  int32_t outer_iterations;  /* IR: refinement steps; FP64_PCG: PCG passes (a */
                             /* pass restarts from the true residual b - A x  */
                             /* when rounding left it above rtol)             */
  int32_t inner_iterations;  /* total PCG iterations                        */
  double rel_residual;       /* final ||b - A x|| / ||b|| computed in FP64   */
  double seconds;
} fem_solve_stats;

/* Solve A x = b (CG; Dirichlet spaces give an SPD operator).  b, x: device
 * double[N]; x holds the initial guess on entry and the last iterate on
 * return.  Work vectors are allocated by the context on the first call and
 * kept.  Runs on `stream` and synchronises it.  Returns FEM_ENOTCONV (x still
 * valid, stats filled) if a cap is hit.  The Jacobi-PCG iterations run in
 * blocks of eight recorded once per call into a CUDA graph (captured on a
 * private stream of the library, replayed on `stream`); where the capture
 * fails, the same iterations run as plain launches. */
int fem_solve(fem_ctx* ctx, const fem_solve_opts* opts, const double* b, double* x,
              fem_solve_stats* stats, void* stream);

/* ---- allocation-free solve ----------------------------------------- */

/* Largest problem fem_solve_noalloc accepts (global DoFs). */
#define FEM_SOLVE_NOALLOC_MAX_DOFS 262144

/* fem_solve without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not have a library allocate
 * device memory behind their back, e.g. an application whose memory manager
 * owns the whole device up front, or a code path that cannot afford the
 * device-wide synchronisation cudaMalloc/cudaFree may cause.
 * Same arguments, algorithm, results and errors as fem_solve, except:
 *   - the work space is a fixed 16 MiB (+64 KiB) device array inside this
 *     library, reserved on every GPU where the library's device code is
 *     loaded until the process exits; N > FEM_SOLVE_NOALLOC_MAX_DOFS is
 *     rejected with FEM_EINVAL before anything runs;
 *   - the first call on each context looks the array's address up
 *     (cudaGetSymbolAddress, with the context's device current) and keeps it
 *     in the context; make that first call before any stream capture on the
 *     device.  A device reset (cudaDeviceReset) frees the array together with
 *     every context's buffers: contexts created afterwards look the new
 *     address up, and contexts from before the reset must not be used again;
 *   - the calling thread's current device must be the context's device (as
 *     for every device call);
 *   - all calls share the one array and each call overwrites it: calls that
 *     overlap on the GPU (other streams, threads or contexts) race and must be
 *     serialised by the caller.
 * It calls no cudaMalloc, cudaFree, cudaMallocHost or other allocating
 * routine. */
int fem_solve_noalloc(fem_ctx* ctx, const fem_solve_opts* opts, const double* b, double* x,
                      fem_solve_stats* stats, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TETMF_H */
