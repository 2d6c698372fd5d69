// Supernodal solves with FP64 factors (the kernels are in sn_impl.cuh).
#include "sn_impl.cuh"

namespace stmg {

cudaError_t sn_solve_real(const DevFactor<double>& F, double* Q, double* Z, double* U, double* P, int nrhs, int ld,
                          const SkSync& sy, cudaStream_t st) {
  return F.bm == kSnBmFP64 ? solve_real<PolNative<double>, kSnBmFP64>(F, Q, Z, U, P, nrhs, ld, sy, st)
                           : solve_real<PolNative<double>>(F, Q, Z, U, P, nrhs, ld, sy, st);
}
cudaError_t sn_solve_cplx(const DevFactor<double2>& F, double2* Q, double2* Z, double2* U, double2* P, int nrhs,
                          int ld, const SkSync& sy, cudaStream_t st) {
  return F.bm == kSnBmFP64 ? solve_cplx<PolC3M, kSnBmFP64>(F, Q, Z, U, P, nrhs, ld, sy, st)
                           : solve_cplx<PolC3M>(F, Q, Z, U, P, nrhs, ld, sy, st);
}

}  // namespace stmg
