// Lookup of the hot-kernel launchers compiled from kernels_s.cu, one pair per
// pulse profile K and slot count S.
#include "aux.cuh"

namespace pasfm {

#define PASFM_DECL_KS(K, S)                                                                                \
  cudaError_t fwd_launch_k##K##_s##S(int C, const CUtensorMap& map, const FwdParams& P, dim3 grid,         \
                                     int threads, size_t smem, cudaStream_t st);                           \
  cudaError_t bwd_launch_k##K##_s##S(int C, int mode, const CUtensorMap& map, const BwdParams& P, dim3 grid, \
                                     size_t smem, cudaStream_t st);                                         \
  int bwd_occupancy_k##K##_s##S(int C, int mode, size_t smem);                                               \
  cudaError_t fwd_batch_launch_k##K##_s##S(int C, const TmaBatch& maps, const FwdBatch& B, int ctas,          \
                                           int threads, size_t smem, cudaStream_t st);                        \
  int fwd_batch_occupancy_k##K##_s##S(int C, int threads, size_t smem);                                       \
  cudaError_t bwd_batch_launch_k##K##_s##S(int C, int mode, const TmaBatch& maps, const BwdBatch& B, int ctas, \
                                           size_t smem, cudaStream_t st);                                     \
  int bwd_batch_occupancy_k##K##_s##S(int C, int mode, size_t smem);
#define PASFM_DECL_K_2_16(K)                                                                            \
  PASFM_DECL_KS(K, 2) PASFM_DECL_KS(K, 3) PASFM_DECL_KS(K, 4) PASFM_DECL_KS(K, 5) PASFM_DECL_KS(K, 6)   \
  PASFM_DECL_KS(K, 7) PASFM_DECL_KS(K, 8) PASFM_DECL_KS(K, 9) PASFM_DECL_KS(K, 10) PASFM_DECL_KS(K, 11) \
  PASFM_DECL_KS(K, 12) PASFM_DECL_KS(K, 13) PASFM_DECL_KS(K, 14) PASFM_DECL_KS(K, 15) PASFM_DECL_KS(K, 16)
PASFM_DECL_K_2_16(0)
PASFM_DECL_K_2_16(1)
PASFM_DECL_KS(1, 17) PASFM_DECL_KS(1, 18) PASFM_DECL_KS(1, 19) PASFM_DECL_KS(1, 20) PASFM_DECL_KS(1, 21)
PASFM_DECL_KS(1, 22) PASFM_DECL_KS(1, 23) PASFM_DECL_KS(1, 24) PASFM_DECL_KS(1, 25) PASFM_DECL_KS(1, 26)
PASFM_DECL_KS(1, 27) PASFM_DECL_KS(1, 28) PASFM_DECL_KS(1, 29) PASFM_DECL_KS(1, 30) PASFM_DECL_KS(1, 31)
PASFM_DECL_KS(1, 32)

namespace {

#define PASFM_F(K, S) fwd_launch_k##K##_s##S
#define PASFM_B(K, S) bwd_launch_k##K##_s##S
const FwdLaunch kFwdSphere[kMaxSSphere + 1] = {
    nullptr,          nullptr,          PASFM_F(0, 2),  PASFM_F(0, 3),  PASFM_F(0, 4),  PASFM_F(0, 5),
    PASFM_F(0, 6),    PASFM_F(0, 7),    PASFM_F(0, 8),  PASFM_F(0, 9),  PASFM_F(0, 10), PASFM_F(0, 11),
    PASFM_F(0, 12),   PASFM_F(0, 13),   PASFM_F(0, 14), PASFM_F(0, 15), PASFM_F(0, 16)};
const BwdLaunch kBwdSphere[kMaxSSphere + 1] = {
    nullptr,          nullptr,          PASFM_B(0, 2),  PASFM_B(0, 3),  PASFM_B(0, 4),  PASFM_B(0, 5),
    PASFM_B(0, 6),    PASFM_B(0, 7),    PASFM_B(0, 8),  PASFM_B(0, 9),  PASFM_B(0, 10), PASFM_B(0, 11),
    PASFM_B(0, 12),   PASFM_B(0, 13),   PASFM_B(0, 14), PASFM_B(0, 15), PASFM_B(0, 16)};
const FwdLaunch kFwdGauss[kMaxSGauss + 1] = {
    nullptr,        nullptr,        PASFM_F(1, 2),  PASFM_F(1, 3),  PASFM_F(1, 4),  PASFM_F(1, 5),
    PASFM_F(1, 6),  PASFM_F(1, 7),  PASFM_F(1, 8),  PASFM_F(1, 9),  PASFM_F(1, 10), PASFM_F(1, 11),
    PASFM_F(1, 12), PASFM_F(1, 13), PASFM_F(1, 14), PASFM_F(1, 15), PASFM_F(1, 16), PASFM_F(1, 17),
    PASFM_F(1, 18), PASFM_F(1, 19), PASFM_F(1, 20), PASFM_F(1, 21), PASFM_F(1, 22), PASFM_F(1, 23),
    PASFM_F(1, 24), PASFM_F(1, 25), PASFM_F(1, 26), PASFM_F(1, 27), PASFM_F(1, 28), PASFM_F(1, 29),
    PASFM_F(1, 30), PASFM_F(1, 31), PASFM_F(1, 32)};
const BwdLaunch kBwdGauss[kMaxSGauss + 1] = {
    nullptr,        nullptr,        PASFM_B(1, 2),  PASFM_B(1, 3),  PASFM_B(1, 4),  PASFM_B(1, 5),
    PASFM_B(1, 6),  PASFM_B(1, 7),  PASFM_B(1, 8),  PASFM_B(1, 9),  PASFM_B(1, 10), PASFM_B(1, 11),
    PASFM_B(1, 12), PASFM_B(1, 13), PASFM_B(1, 14), PASFM_B(1, 15), PASFM_B(1, 16), PASFM_B(1, 17),
    PASFM_B(1, 18), PASFM_B(1, 19), PASFM_B(1, 20), PASFM_B(1, 21), PASFM_B(1, 22), PASFM_B(1, 23),
    PASFM_B(1, 24), PASFM_B(1, 25), PASFM_B(1, 26), PASFM_B(1, 27), PASFM_B(1, 28), PASFM_B(1, 29),
    PASFM_B(1, 30), PASFM_B(1, 31), PASFM_B(1, 32)};

#define PASFM_O(K, S) bwd_occupancy_k##K##_s##S
const BwdOccupancy kOccSphere[kMaxSSphere + 1] = {
    nullptr,          nullptr,          PASFM_O(0, 2),  PASFM_O(0, 3),  PASFM_O(0, 4),  PASFM_O(0, 5),
    PASFM_O(0, 6),    PASFM_O(0, 7),    PASFM_O(0, 8),  PASFM_O(0, 9),  PASFM_O(0, 10), PASFM_O(0, 11),
    PASFM_O(0, 12),   PASFM_O(0, 13),   PASFM_O(0, 14), PASFM_O(0, 15), PASFM_O(0, 16)};
const BwdOccupancy kOccGauss[kMaxSGauss + 1] = {
    nullptr,        nullptr,        PASFM_O(1, 2),  PASFM_O(1, 3),  PASFM_O(1, 4),  PASFM_O(1, 5),
    PASFM_O(1, 6),  PASFM_O(1, 7),  PASFM_O(1, 8),  PASFM_O(1, 9),  PASFM_O(1, 10), PASFM_O(1, 11),
    PASFM_O(1, 12), PASFM_O(1, 13), PASFM_O(1, 14), PASFM_O(1, 15), PASFM_O(1, 16), PASFM_O(1, 17),
    PASFM_O(1, 18), PASFM_O(1, 19), PASFM_O(1, 20), PASFM_O(1, 21), PASFM_O(1, 22), PASFM_O(1, 23),
    PASFM_O(1, 24), PASFM_O(1, 25), PASFM_O(1, 26), PASFM_O(1, 27), PASFM_O(1, 28), PASFM_O(1, 29),
    PASFM_O(1, 30), PASFM_O(1, 31), PASFM_O(1, 32)};

// Tables of the batched launchers, indexed like the single-scan ones (S = 0, 1 unused).
#define PASFM_ROW_2_16(X, K)                                                                                    \
  nullptr, nullptr, X(K, 2), X(K, 3), X(K, 4), X(K, 5), X(K, 6), X(K, 7), X(K, 8), X(K, 9), X(K, 10), X(K, 11), \
      X(K, 12), X(K, 13), X(K, 14), X(K, 15), X(K, 16)
#define PASFM_ROW_17_32(X, K)                                                                                   \
  X(K, 17), X(K, 18), X(K, 19), X(K, 20), X(K, 21), X(K, 22), X(K, 23), X(K, 24), X(K, 25), X(K, 26), X(K, 27), \
      X(K, 28), X(K, 29), X(K, 30), X(K, 31), X(K, 32)
#define PASFM_FB(K, S) fwd_batch_launch_k##K##_s##S
#define PASFM_FO(K, S) fwd_batch_occupancy_k##K##_s##S
#define PASFM_BB(K, S) bwd_batch_launch_k##K##_s##S
#define PASFM_BO(K, S) bwd_batch_occupancy_k##K##_s##S
const FwdBatchLaunch kFwdBatchSphere[kMaxSSphere + 1] = {PASFM_ROW_2_16(PASFM_FB, 0)};
const FwdBatchLaunch kFwdBatchGauss[kMaxSGauss + 1] = {PASFM_ROW_2_16(PASFM_FB, 1), PASFM_ROW_17_32(PASFM_FB, 1)};
const FwdBatchOccupancy kFwdBatchOccSphere[kMaxSSphere + 1] = {PASFM_ROW_2_16(PASFM_FO, 0)};
const FwdBatchOccupancy kFwdBatchOccGauss[kMaxSGauss + 1] = {PASFM_ROW_2_16(PASFM_FO, 1),
                                                               PASFM_ROW_17_32(PASFM_FO, 1)};
const BwdBatchLaunch kBwdBatchSphere[kMaxSSphere + 1] = {PASFM_ROW_2_16(PASFM_BB, 0)};
const BwdBatchLaunch kBwdBatchGauss[kMaxSGauss + 1] = {PASFM_ROW_2_16(PASFM_BB, 1), PASFM_ROW_17_32(PASFM_BB, 1)};
const BwdOccupancy kBwdBatchOccSphere[kMaxSSphere + 1] = {PASFM_ROW_2_16(PASFM_BO, 0)};
const BwdOccupancy kBwdBatchOccGauss[kMaxSGauss + 1] = {PASFM_ROW_2_16(PASFM_BO, 1), PASFM_ROW_17_32(PASFM_BO, 1)};

template <class T>
T pick(int K, int S, const T* sphere, const T* gauss) {
  if (S < kMinS) return nullptr;
  if (K == PASFM_KERNEL_SPHERE) return S <= kMaxSSphere ? sphere[S] : nullptr;
  if (K == PASFM_KERNEL_GAUSS) return S <= kMaxSGauss ? gauss[S] : nullptr;
  return nullptr;
}

}  // namespace

FwdBatchLaunch fwd_batch_launcher(int K, int S) { return pick(K, S, kFwdBatchSphere, kFwdBatchGauss); }
FwdBatchOccupancy fwd_batch_occupancy(int K, int S) { return pick(K, S, kFwdBatchOccSphere, kFwdBatchOccGauss); }
BwdBatchLaunch bwd_batch_launcher(int K, int S) { return pick(K, S, kBwdBatchSphere, kBwdBatchGauss); }
BwdOccupancy bwd_batch_occupancy(int K, int S) { return pick(K, S, kBwdBatchOccSphere, kBwdBatchOccGauss); }

BwdOccupancy bwd_occupancy(int K, int S) {
  if (S < kMinS) return nullptr;
  if (K == PASFM_KERNEL_SPHERE) return S <= kMaxSSphere ? kOccSphere[S] : nullptr;
  if (K == PASFM_KERNEL_GAUSS) return S <= kMaxSGauss ? kOccGauss[S] : nullptr;
  return nullptr;
}

FwdLaunch fwd_launcher(int K, int S) {
  if (S < kMinS) return nullptr;
  if (K == PASFM_KERNEL_SPHERE) return S <= kMaxSSphere ? kFwdSphere[S] : nullptr;
  if (K == PASFM_KERNEL_GAUSS) return S <= kMaxSGauss ? kFwdGauss[S] : nullptr;
  return nullptr;
}

BwdLaunch bwd_launcher(int K, int S) {
  if (S < kMinS) return nullptr;
  if (K == PASFM_KERNEL_SPHERE) return S <= kMaxSSphere ? kBwdSphere[S] : nullptr;
  if (K == PASFM_KERNEL_GAUSS) return S <= kMaxSGauss ? kBwdGauss[S] : nullptr;
  return nullptr;
}

}  // namespace pasfm
