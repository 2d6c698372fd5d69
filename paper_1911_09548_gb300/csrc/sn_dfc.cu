// Supernodal solve with the complex double-float factor (the kernels are in sn_impl.cuh).
#include "sn_impl.cuh"

namespace stmg {

cudaError_t sn_solve_cplx_df(const DevFactor<double2, float4>& F, double2* Q, double2* Z, double2* U, double2* P,
                             int nrhs, int ld, const SkSync& sy, cudaStream_t st) {
  return solve_cplx<PolDFC>(F, Q, Z, U, P, nrhs, ld, sy, st);
}

}  // namespace stmg
