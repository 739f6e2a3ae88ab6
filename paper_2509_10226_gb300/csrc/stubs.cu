// Entry points whose kernels are not built yet report FEM_EUNSUPPORTED.
#include "common.cuh"

namespace tetmf {
int csr_build(Ctx&, int64_t*) {
  set_error("CSR not available in this build");
  return FEM_EUNSUPPORTED;
}
int csr_apply(Ctx&, int, const void*, void*, void*) {
  set_error("CSR not available in this build");
  return FEM_EUNSUPPORTED;
}
int solve(Ctx&, const fem_solve_opts*, const double*, double*, fem_solve_stats*, void*) {
  set_error("solve not available in this build");
  return FEM_EUNSUPPORTED;
}
}  // namespace tetmf
