// Declarations of the auxiliary kernels (aux.cu) and the per-S launchers of the
// hot kernels (kernels_s.cu, compiled once per slot count S).
#pragma once

#include "pasfm_dev.cuh"

namespace pasfm {

constexpr int kMinS = 2, kMaxSSphere = 16, kMaxSGauss = 32;

__global__ void elem_pos_kernel(const double* elem, const double* pose, double* xw, int F, int E, double lox,
                                double loy, double loz, double hix, double hiy, double hiz, double a0,
                                unsigned* status);
// fwd_reduce_kernel<LANES> for LANES = ceil(W / 32), launched with 8 warps and
// fwd_reduce_smem() bytes of dynamic shared memory
cudaError_t fwd_reduce_launch(const RedParams& P, int blocks, cudaStream_t st);
// the same over several scans' chunks in one launch (window length W shared)
cudaError_t fwd_reduce_batch_launch(const RedBatch& B, int W, cudaStream_t st);
__global__ void trace_init_kernel(unsigned long long* trace, int n);
size_t fwd_reduce_smem();
__global__ void loss_rows_kernel(const float* sig, const void* meas, int dtype, const uint8_t* mask, float* g,
                                 double* loss_part, int n_rows, int Nt);
__global__ void sum_kernel(const double* part, int n, double* out);
__global__ void pose_rows_kernel(const double* gpart, int ncubes, int n_rows, int64_t row0, double* G);
__global__ void grad6_kernel(const double* xw, const double* G, int E, double* grad6);
__global__ void adam_vol_kernel(void* p0, int dtype, const float* grad, float* m, float* v, int64_t n, float b1,
                                float b2, float lr_t, float inv_sqrt_bc2, float eps, int nonneg);
__global__ void adam_pose_kernel(double* pose, const double* grad6, double* m, double* v, int F, double b1,
                                 double b2, double bc1, double bc2, double lr_rot, double lr_trans, double eps,
                                 int fix0, int freeze);

__global__ void apply_twist_kernel(const double* pose, const double* xi, double* out, int F);
__global__ void twist_grad_kernel(const double* xi, const double* g6, double* out, int F);

__global__ void resample_kernel(const float* src, int sx, int sy, int sz, double sox, double soy, double soz,
                                double sdx, double sdy, double sdz, float* dst, int nx, int ny, int nz, double ox,
                                double oy, double oz, double dx, double dy, double dz);

__global__ void lowpass_kernel(const float* src, float* dst, int Nt, int r, int decim, int Nout, const float* w);

__global__ void nc_grad_kernel(const float* sim, const void* meas, int dtype, const uint8_t* mask, int64_t n_rows,
                               int Nt, int meas_repeat, float scale, float* g, double* nc_out);
__global__ void scale_kernel(float* x, int64_t n, float alpha);
// first difference of every trace: D[r][n] = g[r][n] - g[r][n-1], n in [0, Ntd), g = 0
// outside [0, Nt)
__global__ void diff_rows_kernel(const void* g, int dtype, int64_t rows, int Nt, int Ntd, float* D);
// FP32 throughput probe (fp32_probe_kernel): flops per launch and the launch itself
double fp32_probe_flops(int blocks, int iters, int mode);
cudaError_t fp32_probe_launch(int mode, int blocks, int iters, float* out, cudaStream_t st);
// shared-memory read-modify-write probe (smem_probe_kernel): bytes per launch and the launch
double smem_probe_bytes(int blocks, int iters);
cudaError_t smem_probe_launch(int blocks, int iters, float* out, cudaStream_t st);
__global__ void nc_scores_kernel(const float* sim, const void* meas, int dtype, const uint8_t* mask, int E, int Nt,
                                 double* out);

using FwdLaunch = cudaError_t (*)(int C, const CUtensorMap& map, const FwdParams& P, dim3 grid, int threads,
                                  size_t smem, cudaStream_t st);
using BwdLaunch = cudaError_t (*)(int C, int mode, const CUtensorMap& map, const BwdParams& P, dim3 grid,
                                  size_t smem, cudaStream_t st);
// persistent batched launches over several scans (grid = CTAs to keep resident)
using FwdBatchLaunch = cudaError_t (*)(int C, const TmaBatch& maps, const FwdBatch& B, int ctas, int threads,
                                       size_t smem, cudaStream_t st);
using BwdBatchLaunch = cudaError_t (*)(int C, int mode, const TmaBatch& maps, const BwdBatch& B, int ctas,
                                       size_t smem, cudaStream_t st);
// resident CTAs per SM of the batched kernels (0 if the query fails)
using FwdBatchOccupancy = int (*)(int C, int threads, size_t smem);

// Launchers of the hot kernels for pulse profile K and slot count S; null when
// (K, S) is not compiled (sphere: S = 2..16, Gaussian: S = 2..32).
// TGV regulariser (tgv.cu): kernel, its shared-memory size, tile count and grid,
// block size and TMA boxes (u region, w region, volume-gradient tile).
__global__ void tgv_kernel(const __grid_constant__ CUtensorMap umap, const __grid_constant__ CUtensorMap wmap,
                           const __grid_constant__ CUtensorMap gmap, const TgvParams P);
size_t tgv_smem_bytes();
int tgv_tiles(int nx, int ny, int nz);
dim3 tgv_grid(int nx, int ny, int nz);
int tgv_threads();
void tgv_boxes(unsigned* box3, unsigned* box4, unsigned* boxg);

using BwdOccupancy = int (*)(int C, int mode, size_t smem);

FwdLaunch fwd_launcher(int K, int S);
BwdLaunch bwd_launcher(int K, int S);
BwdOccupancy bwd_occupancy(int K, int S);
FwdBatchLaunch fwd_batch_launcher(int K, int S);
BwdBatchLaunch bwd_batch_launcher(int K, int S);
FwdBatchOccupancy fwd_batch_occupancy(int K, int S);
BwdOccupancy bwd_batch_occupancy(int K, int S);

// Adds the n_parts per-part adjoint sums in part order into vol (or overwrites it).
__global__ void sum_parts_kernel(const float* parts, int n_parts, int64_t nvox, float* vol, int accumulate);

}  // namespace pasfm
