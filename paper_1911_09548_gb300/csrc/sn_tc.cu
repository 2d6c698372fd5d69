// Supernodal solves with 16-bit factors: split-K on the CUDA cores for few right-hand
// sides, the tensor-core depths of tc_kernels.cu otherwise (the kernels are in sn_impl.cuh).
#include "sn_impl.cuh"

namespace stmg {

// 16-bit factor (BF16 or FP16) on the tensor cores: CUDA-core split-K for few
// right-hand sides, otherwise per depth the tcgen05 kernels (split-K for depths whose
// tiles fill fewer than sy.split_waves waves of the SMs).
template <typename PolC, typename WT>
cudaError_t solve_cplx_tc(const DevFactor<float2, WT>& F, float2* Q, float2* Z, float2* U, float2* P, float2* Ptc,
                          uint8_t* Bst, int nrhs, int ld, const SkSync& sy, cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  if (nrhs <= 2) return sn_solve_skinny<PolC, 2>(F, Q, Z, U, P, nrhs, ld, sy, st);
  if (nrhs <= 8) return sn_solve_skinny<PolC, 8>(F, Q, Z, U, P, nrhs, ld, sy, st);
  if (nrhs <= kSkMaxRhsC) return sn_solve_skinny<PolC, kSkMaxRhsC>(F, Q, Z, U, P, nrhs, ld, sy, st);
  const int64_t gy = (nrhs + kTcCols - 1) / kTcCols;
  const int64_t two_waves = (int64_t)sy.split_waves * F.n_sm;
  for (int d = F.max_depth; d >= 0; --d) {
    const int64_t tiles = F.h_fwd_off[d + 1] - F.h_fwd_off[d];
    if (tiles <= 0) continue;
    sn_tc2_depth(F, d, true, tiles * gy < two_waves, Q, Z, U, Ptc, Bst, nrhs, ld, sy, st);
  }
  for (int d = 0; d <= F.max_depth; ++d) {
    const int64_t tiles = F.h_bwd_off[d + 1] - F.h_bwd_off[d];
    if (tiles <= 0) continue;
    sn_tc2_depth(F, d, false, tiles * gy < two_waves, Q, Z, U, Ptc, Bst, nrhs, ld, sy, st);
  }
  return cudaGetLastError();
}

cudaError_t sn_solve_cplx_bf16(const DevFactor<float2, __nv_bfloat162>& F, float2* Q, float2* Z, float2* U,
                               float2* P, float2* Ptc, uint8_t* Bst, int nrhs, int ld, const SkSync& sy,
                               cudaStream_t st) {
  return solve_cplx_tc<PolBF16C>(F, Q, Z, U, P, Ptc, Bst, nrhs, ld, sy, st);
}
cudaError_t sn_solve_cplx_f16(const DevFactor<float2, __half2>& F, float2* Q, float2* Z, float2* U, float2* P,
                              float2* Ptc, uint8_t* Bst, int nrhs, int ld, const SkSync& sy, cudaStream_t st) {
  return solve_cplx_tc<PolF16C>(F, Q, Z, U, P, Ptc, Bst, nrhs, ld, sy, st);
}

cudaError_t sn_solve_cplx_bf16_cc(const DevFactor<float2, __nv_bfloat162>& F, float2* Q, float2* Z, float2* U,
                                  int nrhs, int ld, cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  SkSync none;
  return sn_solve_tiled<PolBF16CR, 32, kSkMaxRhsC, kSnBM>(F, Q, Z, U, nullptr, nrhs, ld, none, st);
}
cudaError_t sn_solve_cplx_f16_cc(const DevFactor<float2, __half2>& F, float2* Q, float2* Z, float2* U, int nrhs,
                                 int ld, cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  SkSync none;
  return sn_solve_tiled<PolF16CR, 32, kSkMaxRhsC, kSnBM>(F, Q, Z, U, nullptr, nrhs, ld, none, st);
}

}  // namespace stmg
