// Supernodal solves with FP32 factors and the real double-float one (the kernels are in
// sn_impl.cuh).
#include "sn_impl.cuh"

namespace stmg {

cudaError_t sn_solve_realf(const DevFactor<float>& F, float* Q, float* Z, float* U, float* P, int nrhs, int ld,
                           const SkSync& sy, cudaStream_t st) {
  return solve_real<PolNative<float>>(F, Q, Z, U, P, nrhs, ld, sy, st);
}
cudaError_t sn_solve_cplxf(const DevFactor<float2>& F, float2* Q, float2* Z, float2* U, float2* P, int nrhs, int ld,
                           const SkSync& sy, cudaStream_t st) {
  return solve_cplx<PolNative<float2>>(F, Q, Z, U, P, nrhs, ld, sy, st);
}
cudaError_t sn_solve_real_df(const DevFactor<double, float2>& F, double* Q, double* Z, double* U, double* P, int nrhs,
                             int ld, const SkSync& sy, cudaStream_t st) {
  return solve_real<PolDF>(F, Q, Z, U, P, nrhs, ld, sy, st);
}

}  // namespace stmg
