// Instantiates the forward and backward hot kernels for one slot count S
// (compiled once per S = 2..16 with -DPASFM_S=<S>) and exports their launchers.
#include "aux.cuh"
#include "kernels.cuh"

#ifndef PASFM_S
#error "compile with -DPASFM_S=<slots per pair>"
#endif
#define PASFM_CAT2(a, b) a##b
#define PASFM_CAT(a, b) PASFM_CAT2(a, b)

namespace pasfm {

template <int C>
static cudaError_t fwd_launch_c(const CUtensorMap& map, const FwdParams& P, dim3 grid, int threads, size_t smem,
                                cudaStream_t st) {
  auto k = fwd_cube_kernel<C, PASFM_S>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k<<<grid, threads, smem, st>>>(map, P);
  return cudaPeekAtLastError();
}

template <int C, bool ADJ, bool POSE>
static cudaError_t bwd_launch_c(const CUtensorMap& map, const BwdParams& P, dim3 grid, size_t smem,
                                cudaStream_t st) {
  auto k = bwd_cube_kernel<C, PASFM_S, ADJ, POSE>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k<<<grid, C * C, smem, st>>>(map, P);
  return cudaPeekAtLastError();
}

cudaError_t PASFM_CAT(fwd_launch_s, PASFM_S)(int C, const CUtensorMap& map, const FwdParams& P, dim3 grid,
                                             int threads, size_t smem, cudaStream_t st) {
  if (C == 16) return fwd_launch_c<16>(map, P, grid, threads, smem, st);
  if (C == 8) return fwd_launch_c<8>(map, P, grid, threads, smem, st);
  return cudaErrorInvalidValue;
}

// mode: 1 = adjoint, 2 = pose gradient, 3 = both
cudaError_t PASFM_CAT(bwd_launch_s, PASFM_S)(int C, int mode, const CUtensorMap& map, const BwdParams& P,
                                             dim3 grid, size_t smem, cudaStream_t st) {
  if (C == 16) {
    if (mode == 1) return bwd_launch_c<16, true, false>(map, P, grid, smem, st);
    if (mode == 2) return bwd_launch_c<16, false, true>(map, P, grid, smem, st);
    if (mode == 3) return bwd_launch_c<16, true, true>(map, P, grid, smem, st);
  } else if (C == 8) {
    if (mode == 1) return bwd_launch_c<8, true, false>(map, P, grid, smem, st);
    if (mode == 2) return bwd_launch_c<8, false, true>(map, P, grid, smem, st);
    if (mode == 3) return bwd_launch_c<8, true, true>(map, P, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace pasfm
