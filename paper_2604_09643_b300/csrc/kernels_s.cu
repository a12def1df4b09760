// Instantiates the forward and backward hot kernels for one pulse profile K and
// one slot count S (compiled once per pair with -DPASFM_K=<K> -DPASFM_S=<S>:
// the sphere for S = 2..16, the Gaussian for S = 2..32) and exports their
// launchers fwd_launch_k<K>_s<S> and bwd_launch_k<K>_s<S>.
#include "aux.cuh"
#include "kernels.cuh"

#if !defined(PASFM_S) || !defined(PASFM_K)
#error "compile with -DPASFM_K=<pulse profile> -DPASFM_S=<slots per pair>"
#endif
#define PASFM_CAT2(a, b) a##b
#define PASFM_CAT(a, b) PASFM_CAT2(a, b)
#define PASFM_NAME(what) PASFM_CAT(PASFM_CAT(PASFM_CAT(what, _k), PASFM_K), PASFM_CAT(_s, PASFM_S))

namespace pasfm {

template <int C>
static cudaError_t fwd_launch_c(const CUtensorMap& map, const FwdParams& P, dim3 grid, int threads, size_t smem,
                                cudaStream_t st) {
  auto k = fwd_cube_kernel<C, PASFM_S, PASFM_K>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k<<<grid, threads, smem, st>>>(map, P);
  return cudaPeekAtLastError();
}

template <int C, bool ADJ, bool POSE>
static cudaError_t bwd_launch_c(const CUtensorMap& map, const BwdParams& P, dim3 grid, size_t smem,
                                cudaStream_t st) {
  auto k = bwd_cube_kernel<C, PASFM_S, PASFM_K, ADJ, POSE>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k<<<grid, C * C, smem, st>>>(map, P);
  return cudaPeekAtLastError();
}

template <int C, bool ADJ, bool POSE>
static int bwd_occupancy_c(size_t smem) {
  auto k = bwd_cube_kernel<C, PASFM_S, PASFM_K, ADJ, POSE>;
  int n = 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, C * C, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <int C>
static cudaError_t fwd_batch_launch_c(const TmaBatch& maps, const FwdBatch& B, int ctas, int threads, size_t smem,
                                      cudaStream_t st) {
  auto k = fwd_batch_kernel<C, PASFM_S, PASFM_K>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k<<<ctas, threads, smem, st>>>(maps, B);
  return cudaPeekAtLastError();
}

template <int C>
static int fwd_batch_occupancy_c(int threads, size_t smem) {
  auto k = fwd_batch_kernel<C, PASFM_S, PASFM_K>;
  int n = 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <int C, bool ADJ, bool POSE>
static cudaError_t bwd_batch_launch_c(const TmaBatch& maps, const BwdBatch& B, int ctas, size_t smem,
                                      cudaStream_t st) {
  auto k = bwd_batch_kernel<C, PASFM_S, PASFM_K, ADJ, POSE>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k<<<ctas, C * C, smem, st>>>(maps, B);
  return cudaPeekAtLastError();
}

template <int C, bool ADJ, bool POSE>
static int bwd_batch_occupancy_c(size_t smem) {
  auto k = bwd_batch_kernel<C, PASFM_S, PASFM_K, ADJ, POSE>;
  int n = 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, C * C, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t PASFM_NAME(fwd_batch_launch)(int C, const TmaBatch& maps, const FwdBatch& B, int ctas, int threads,
                                         size_t smem, cudaStream_t st) {
  if (C == 16) return fwd_batch_launch_c<16>(maps, B, ctas, threads, smem, st);
  if (C == 8) return fwd_batch_launch_c<8>(maps, B, ctas, threads, smem, st);
  return cudaErrorInvalidValue;
}

int PASFM_NAME(fwd_batch_occupancy)(int C, int threads, size_t smem) {
  if (C == 16) return fwd_batch_occupancy_c<16>(threads, smem);
  if (C == 8) return fwd_batch_occupancy_c<8>(threads, smem);
  return 0;
}

cudaError_t PASFM_NAME(bwd_batch_launch)(int C, int mode, const TmaBatch& maps, const BwdBatch& B, int ctas,
                                         size_t smem, cudaStream_t st) {
  if (C == 16) {
    if (mode == 1) return bwd_batch_launch_c<16, true, false>(maps, B, ctas, smem, st);
    if (mode == 2) return bwd_batch_launch_c<16, false, true>(maps, B, ctas, smem, st);
    if (mode == 3) return bwd_batch_launch_c<16, true, true>(maps, B, ctas, smem, st);
  } else if (C == 8) {
    if (mode == 1) return bwd_batch_launch_c<8, true, false>(maps, B, ctas, smem, st);
    if (mode == 2) return bwd_batch_launch_c<8, false, true>(maps, B, ctas, smem, st);
    if (mode == 3) return bwd_batch_launch_c<8, true, true>(maps, B, ctas, smem, st);
  }
  return cudaErrorInvalidValue;
}

int PASFM_NAME(bwd_batch_occupancy)(int C, int mode, size_t smem) {
  if (C == 16) {
    if (mode == 1) return bwd_batch_occupancy_c<16, true, false>(smem);
    if (mode == 2) return bwd_batch_occupancy_c<16, false, true>(smem);
    if (mode == 3) return bwd_batch_occupancy_c<16, true, true>(smem);
  } else if (C == 8) {
    if (mode == 1) return bwd_batch_occupancy_c<8, true, false>(smem);
    if (mode == 2) return bwd_batch_occupancy_c<8, false, true>(smem);
    if (mode == 3) return bwd_batch_occupancy_c<8, true, true>(smem);
  }
  return 0;
}

cudaError_t PASFM_NAME(fwd_launch)(int C, const CUtensorMap& map, const FwdParams& P, dim3 grid,
                                             int threads, size_t smem, cudaStream_t st) {
  if (C == 16) return fwd_launch_c<16>(map, P, grid, threads, smem, st);
  if (C == 8) return fwd_launch_c<8>(map, P, grid, threads, smem, st);
  return cudaErrorInvalidValue;
}

// mode: 1 = adjoint, 2 = pose gradient, 3 = both
cudaError_t PASFM_NAME(bwd_launch)(int C, int mode, const CUtensorMap& map, const BwdParams& P,
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

// Resident CTAs per SM of the backward kernel (0 if the query fails).
int PASFM_NAME(bwd_occupancy)(int C, int mode, size_t smem) {
  if (C == 16) {
    if (mode == 1) return bwd_occupancy_c<16, true, false>(smem);
    if (mode == 2) return bwd_occupancy_c<16, false, true>(smem);
    if (mode == 3) return bwd_occupancy_c<16, true, true>(smem);
  } else if (C == 8) {
    if (mode == 1) return bwd_occupancy_c<8, true, false>(smem);
    if (mode == 2) return bwd_occupancy_c<8, false, true>(smem);
    if (mode == 3) return bwd_occupancy_c<8, true, true>(smem);
  }
  return 0;
}

}  // namespace pasfm
