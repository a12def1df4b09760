// Auxiliary sm_103a kernels: element positions (A1), the fixed-order reduction
// of per-cube forward partials with the fused loss head (A2/A3), the pose-
// gradient reductions (A5), and Adam on the volume and on the frame twists (A6).
// All reductions visit their terms in a fixed order, so repeated calls give
// bit-identical results.
#include <climits>

#include "aux.cuh"
#include "pasfm_dev.cuh"

namespace pasfm {

// fwd_reduce_kernel: samples per warp accumulator, and cubes whose windows a warp loads
// per step (4 measured fastest on the full scan: 0.67 ms against 0.75 at 8 and 0.83 at 2;
// at 8 the loads' registers spill and fewer blocks fit an SM)
constexpr int kRedChunk = 1024;
constexpr int kRedUnroll = 4;

// x_fj = R_f e_j + t_f in FP64; flag elements closer than a0 to the grid box.
__global__ void elem_pos_kernel(const double* __restrict__ elem, const double* __restrict__ pose,
                                double* __restrict__ xw, int F, int E, double lox, double loy, double loz,
                                double hix, double hiy, double hiz, double a0, unsigned* status) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= static_cast<int64_t>(F) * E) return;
  const int f = static_cast<int>(k / E), j = static_cast<int>(k % E);
  const double* P = pose + 12 * static_cast<int64_t>(f);
  const double e0 = elem[3 * j], e1 = elem[3 * j + 1], e2 = elem[3 * j + 2];
  double x[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) x[a] = fma(P[4 * a], e0, fma(P[4 * a + 1], e1, fma(P[4 * a + 2], e2, P[4 * a + 3])));
  xw[3 * k] = x[0];
  xw[3 * k + 1] = x[1];
  xw[3 * k + 2] = x[2];
  const double bx = fmax(fmax(lox - x[0], x[0] - hix), 0.0);
  const double by = fmax(fmax(loy - x[1], x[1] - hiy), 0.0);
  const double bz = fmax(fmax(loz - x[2], x[2] - hiz), 0.0);
  if (bx * bx + by * by + bz * bz <= a0 * a0) atomicOr(status, PASFM_STATUS_ELEMENT_INSIDE);
}

// Emit sample n of a trace: signal and/or masked residual with its square.
struct Emitter {
  float* sig;
  float* g;
  const void* meas;
  int dtype;
  bool keep;
  double lsum;
  __device__ __forceinline__ void operator()(int64_t off, float s) {
    if (sig) sig[off] = s;
    if (g) {
      const float r = keep ? s - load_elem(meas, off, dtype) : 0.f;
      g[off] = r;
      lsum = fma(static_cast<double>(r), static_cast<double>(r), lsum);
    }
  }
};

__device__ __forceinline__ void block_loss(double lsum, double* out, int warp, int lane) {
  __shared__ double wsum[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) wsum[warp] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (blockDim.x >> 5); ++w) t += wsum[w];
    *out = 0.5 * t;
  }
}

// One warp per trace: sum the per-cube partial windows in cube order.  LANES =
// ceil(W / 32) words per lane and cube, so that only the window's own words are
// loaded and kRedUnroll cubes' loads are in flight at once.
template <int LANES>
__device__ __forceinline__ void fwd_reduce_block(const RedParams& P, int block) {
  extern __shared__ float racc[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = block * 8 + warp;
  float* acc = racc + warp * kRedChunk;
  Emitter em{P.sig_out, P.g_out, P.meas, P.dtype_sig, true, 0.0};
  if (row < P.n_rows) {
    const int* n0 = P.n0tab + static_cast<int64_t>(row) * P.ncubes;
    const float* part = P.part + static_cast<int64_t>(row) * P.ncubes * P.W;
    int nmin = INT_MAX, nmax = INT_MIN;
    for (int cc = lane; cc < P.ncubes; cc += 32) {
      const int v = n0[cc];
      nmin = min(nmin, v);
      nmax = max(nmax, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nmin = min(nmin, __shfl_xor_sync(0xffffffffu, nmin, o));
      nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    }
    // 64-bit sums: a cube whose window base was never written (a timed-out forward CTA)
    // may hold any value, and every access below stays in bounds whatever it is
    const int lo = max(nmin, 0);
    const int hi = static_cast<int>(min(static_cast<int64_t>(nmax) + P.W, static_cast<int64_t>(P.Nt)));
    const int64_t grow = static_cast<int64_t>(P.f_begin) * P.E + row;
    em.keep = P.mask ? (P.mask[grow] != 0) : true;
    const int64_t base = grow * P.Nt;
    for (int n = lane; n < P.Nt; n += 32)
      if (n < lo || n >= hi) em(base + n, 0.f);
    for (int cs = lo; cs < hi; cs += kRedChunk) {
      const int len = min(kRedChunk, hi - cs);
      for (int k = lane; k < len; k += 32) acc[k] = 0.f;
      __syncwarp();
      for (int cc = 0; cc < P.ncubes; cc += kRedUnroll) {
        int o[kRedUnroll];
        float v[kRedUnroll][LANES];
#pragma unroll
        for (int u = 0; u < kRedUnroll; ++u) {
          const int64_t ou = cc + u < P.ncubes ? static_cast<int64_t>(n0[cc + u]) - cs : INT_MIN / 2;
          const bool okc = ou < len && ou + P.W > 0;  // the cube's window meets this chunk
          o[u] = okc ? static_cast<int>(ou) : INT_MIN / 2;
          const float* src = part + static_cast<int64_t>(cc + u) * P.W;
#pragma unroll
          for (int m = 0; m < LANES; ++m) {
            const int k = lane + 32 * m;
            v[u][m] = (okc && k < P.W) ? src[k] : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < kRedUnroll; ++u) {
#pragma unroll
          for (int m = 0; m < LANES; ++m) {
            const int k = lane + 32 * m;
            const int pos = o[u] + k;
            if (k < P.W && pos >= 0 && pos < len) acc[pos] += v[u][m];
          }
          __syncwarp();
        }
      }
      for (int k = lane; k < len; k += 32) em(base + cs + k, acc[k]);
      __syncwarp();
    }
  }
  if (P.loss_part) block_loss(em.lsum, P.loss_part + P.loss_offset + block, warp, lane);
}

template <int LANES>
__global__ void __launch_bounds__(256) fwd_reduce_kernel(const RedParams P) {
  fwd_reduce_block<LANES>(P, blockIdx.x);
}

// The reductions of several scans' chunks (same window length) in one launch: scan s
// owns blocks [blocks[s], blocks[s + 1]), each summing 8 of its traces as above.
template <int LANES>
__global__ void __launch_bounds__(256) fwd_reduce_batch_kernel(const __grid_constant__ RedBatch B) {
  const int b = blockIdx.x;
  int s = 0;
  while (b >= B.blocks[s + 1]) ++s;
  fwd_reduce_block<LANES>(B.R[s], b - B.blocks[s]);
}

size_t fwd_reduce_smem() { return size_t(8) * kRedChunk * 4; }

namespace {
template <int LANES>
cudaError_t reduce_launch_l(const RedParams& P, int blocks, cudaStream_t st) {
  const size_t smem = fwd_reduce_smem();
  cudaError_t e = cudaFuncSetAttribute(fwd_reduce_kernel<LANES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  fwd_reduce_kernel<LANES><<<blocks, 256, smem, st>>>(P);
  return cudaGetLastError();
}
}  // namespace

template <int LANES>
cudaError_t reduce_batch_launch_l(const RedBatch& B, cudaStream_t st) {
  const size_t smem = fwd_reduce_smem();
  cudaError_t e = cudaFuncSetAttribute(fwd_reduce_batch_kernel<LANES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  fwd_reduce_batch_kernel<LANES><<<B.blocks[B.n], 256, smem, st>>>(B);
  return cudaGetLastError();
}

cudaError_t fwd_reduce_batch_launch(const RedBatch& B, int W, cudaStream_t st) {
  if (B.n <= 0 || B.blocks[B.n] == 0) return cudaSuccess;
  switch ((W + 31) / 32) {
    case 1: return reduce_batch_launch_l<1>(B, st);
    case 2: return reduce_batch_launch_l<2>(B, st);
    case 3: return reduce_batch_launch_l<3>(B, st);
    case 4: return reduce_batch_launch_l<4>(B, st);
    case 5: return reduce_batch_launch_l<5>(B, st);
    case 6: return reduce_batch_launch_l<6>(B, st);
    case 7: return reduce_batch_launch_l<7>(B, st);
    case 8: return reduce_batch_launch_l<8>(B, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t fwd_reduce_launch(const RedParams& P, int blocks, cudaStream_t st) {
  switch ((P.W + 31) / 32) {
    case 1: return reduce_launch_l<1>(P, blocks, st);
    case 2: return reduce_launch_l<2>(P, blocks, st);
    case 3: return reduce_launch_l<3>(P, blocks, st);
    case 4: return reduce_launch_l<4>(P, blocks, st);
    case 5: return reduce_launch_l<5>(P, blocks, st);
    case 6: return reduce_launch_l<6>(P, blocks, st);
    case 7: return reduce_launch_l<7>(P, blocks, st);
    case 8: return reduce_launch_l<8>(P, blocks, st);
    default: return cudaErrorInvalidValue;
  }
}

// trace[s] = (max, 0) for the batched launches' per-scan tile intervals.
__global__ void trace_init_kernel(unsigned long long* trace, int n) {
  const int i = threadIdx.x;
  if (i < n) {
    trace[2 * i] = ~0ull;
    trace[2 * i + 1] = 0ull;
  }
}

// Standalone loss head: one warp per trace.
__global__ void __launch_bounds__(256) loss_rows_kernel(const float* __restrict__ sig, const void* meas,
                                                        int dtype, const uint8_t* __restrict__ mask,
                                                        float* g, double* loss_part, int n_rows, int Nt) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + warp;
  Emitter em{nullptr, g, meas, dtype, true, 0.0};
  if (row < n_rows) {
    em.keep = mask ? (mask[row] != 0) : true;
    const int64_t base = static_cast<int64_t>(row) * Nt;
    for (int n = lane; n < Nt; n += 32) em(base + n, sig[base + n]);
  }
  block_loss(em.lsum, loss_part + blockIdx.x, warp, lane);
}

// Sum block partials in a fixed order (one block).
__global__ void __launch_bounds__(256) sum_kernel(const double* __restrict__ part, int n, double* out) {
  __shared__ double s[256];
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) t += part[i];
  s[threadIdx.x] = t;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// Element gradients: one warp per trace sums its per-cube partials (cube order).
__global__ void __launch_bounds__(256) pose_rows_kernel(const double* __restrict__ gpart, int ncubes,
                                                        int n_rows, int64_t row0, double* __restrict__ G) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + warp;
  if (row >= n_rows) return;
  const double* src = gpart + static_cast<int64_t>(row) * ncubes * 3;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int k = lane; k < ncubes; k += 32) {
    a += src[3 * k];
    b += src[3 * k + 1];
    c += src[3 * k + 2];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if (lane == 0) {
    double* dst = G + (row0 + row) * 3;
    dst[0] = a;
    dst[1] = b;
    dst[2] = c;
  }
}

// grad6[f] = (sum_j x_fj x G_fj, sum_j G_fj): one block per frame.
__global__ void __launch_bounds__(256) grad6_kernel(const double* __restrict__ xw, const double* __restrict__ G,
                                                    int E, double* __restrict__ grad6) {
  __shared__ double s[6][256];
  const int f = blockIdx.x;
  double w0 = 0, w1 = 0, w2 = 0, v0 = 0, v1 = 0, v2 = 0;
  for (int j = threadIdx.x; j < E; j += 256) {
    const double* x = xw + (static_cast<int64_t>(f) * E + j) * 3;
    const double* g = G + (static_cast<int64_t>(f) * E + j) * 3;
    w0 += x[1] * g[2] - x[2] * g[1];
    w1 += x[2] * g[0] - x[0] * g[2];
    w2 += x[0] * g[1] - x[1] * g[0];
    v0 += g[0];
    v1 += g[1];
    v2 += g[2];
  }
  const int t = threadIdx.x;
  s[0][t] = w0;
  s[1][t] = w1;
  s[2][t] = w2;
  s[3][t] = v0;
  s[4][t] = v1;
  s[5][t] = v2;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w)
      for (int q = 0; q < 6; ++q) s[q][t] += s[q][t + w];
    __syncthreads();
  }
  if (t < 6) grad6[6 * f + t] = s[t][0];
}

// Adam on the volume in its storage type; moments in FP32.
__global__ void adam_vol_kernel(void* p0, int dtype, const float* __restrict__ grad, float* __restrict__ m,
                                float* __restrict__ v, int64_t n, float b1, float b2, float lr_t,
                                float inv_sqrt_bc2, float eps, int nonneg) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = grad[i];
  const float mi = fmaf(b1, m[i], (1.f - b1) * g);
  const float vi = fmaf(b2, v[i], (1.f - b2) * g * g);
  m[i] = mi;
  v[i] = vi;
  float p = load_elem(p0, i, dtype);
  p -= lr_t * mi / (sqrtf(vi) * inv_sqrt_bc2 + eps);
  if (nonneg) p = fmaxf(p, 0.f);
  if (dtype == PASFM_BF16) {
    static_cast<__nv_bfloat16*>(p0)[i] = __float2bfloat16_rn(p);
  } else if (dtype == PASFM_F16) {
    static_cast<__half*>(p0)[i] = __float2half_rn(p);
  } else {
    static_cast<float*>(p0)[i] = p;
  }
}

// Adam on the frame twists (FP64), then the left retraction
// R <- Exp(dw) R, t <- Exp(dw) t + dv (Rodrigues).
__global__ void adam_pose_kernel(double* __restrict__ pose, const double* __restrict__ grad6,
                                 double* __restrict__ m, double* __restrict__ v, int F, double b1, double b2,
                                 double bc1, double bc2, double lr_rot, double lr_trans, double eps, int fix0,
                                 int freeze) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  double dxi[6];
  for (int k = 0; k < 6; ++k) {
    const double g = grad6[6 * f + k];
    const double mk = b1 * m[6 * f + k] + (1.0 - b1) * g;
    const double vk = b2 * v[6 * f + k] + (1.0 - b2) * g * g;
    m[6 * f + k] = mk;
    v[6 * f + k] = vk;
    const double lr = k < 3 ? lr_rot : lr_trans;
    dxi[k] = -lr * (mk / bc1) / (sqrt(vk / bc2) + eps);
  }
  if (freeze || (fix0 && f == 0)) return;
  const double w0 = dxi[0], w1 = dxi[1], w2 = dxi[2];
  const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
  const double th = sqrt(th2);
  double A, B;
  if (th < 1e-12) {
    A = 1.0;
    B = 0.5;
  } else {
    A = sin(th) / th;
    B = (1.0 - cos(th)) / th2;
  }
  // Exp = I + A K + B K^2 with K = skew(w)
  const double K[3][3] = {{0, -w2, w1}, {w2, 0, -w0}, {-w1, w0, 0}};
  double Ex[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double k2 = 0.0;
      for (int q = 0; q < 3; ++q) k2 += K[r][q] * K[q][c];
      Ex[r][c] = (r == c ? 1.0 : 0.0) + A * K[r][c] + B * k2;
    }
  double* P = pose + 12 * static_cast<int64_t>(f);
  double out[12];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int q = 0; q < 3; ++q) s += Ex[r][q] * P[4 * q + c];
      out[4 * r + c] = s;
    }
    out[4 * r + 3] += dxi[3 + r];
  }
  for (int k = 0; k < 12; ++k) P[k] = out[k];
}

}  // namespace pasfm

namespace pasfm {

// Rodrigues pieces of the SO(3) exponential and its left Jacobian:
// Exp(w) = I + A K + B K^2, J_l(w) = I + B K + C K^2, K = skew(w),
// A = sin t / t, B = (1 - cos t) / t^2, C = (t - sin t) / t^3.
__device__ void so3_coeffs(double w0, double w1, double w2, double* A, double* B, double* C) {
  const double t2 = w0 * w0 + w1 * w1 + w2 * w2;
  if (t2 < 1e-12) {  // series to O(t^4)
    *A = 1.0 - t2 / 6.0;
    *B = 0.5 - t2 / 24.0;
    *C = 1.0 / 6.0 - t2 / 120.0;
    return;
  }
  const double t = sqrt(t2);
  *A = sin(t) / t;
  *B = (1.0 - cos(t)) / t2;
  *C = (t - sin(t)) / (t2 * t);
}

__device__ void so3_matrix(double w0, double w1, double w2, double a, double b, double M[3][3]) {
  const double K[3][3] = {{0, -w2, w1}, {w2, 0, -w0}, {-w1, w0, 0}};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double k2 = 0.0;
      for (int q = 0; q < 3; ++q) k2 += K[r][q] * K[q][c];
      M[r][c] = (r == c ? 1.0 : 0.0) + a * K[r][c] + b * k2;
    }
}

// pose_out[f] = left twist xi_f applied to pose[f]: R' = Exp(w) R, t' = Exp(w) t + v.
__global__ void apply_twist_kernel(const double* __restrict__ pose, const double* __restrict__ xi,
                                   double* __restrict__ out, int F) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const double* x = xi + 6 * static_cast<int64_t>(f);
  double A, B, C;
  so3_coeffs(x[0], x[1], x[2], &A, &B, &C);
  double E[3][3];
  so3_matrix(x[0], x[1], x[2], A, B, E);
  const double* P = pose + 12 * static_cast<int64_t>(f);
  double o[12];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int q = 0; q < 3; ++q) s += E[r][q] * P[4 * q + c];
      o[4 * r + c] = s;
    }
    o[4 * r + 3] += x[3 + r];
  }
  double* Q = out + 12 * static_cast<int64_t>(f);
  for (int k = 0; k < 12; ++k) Q[k] = o[k];
}

// Gradient in the twist coordinates from the gradient at the twisted pose:
// dL/dv = g_v, dL/dw = J_l(w)^T (g_w - v x g_v).
__global__ void twist_grad_kernel(const double* __restrict__ xi, const double* __restrict__ g6,
                                  double* __restrict__ out, int F) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const double* x = xi + 6 * static_cast<int64_t>(f);
  const double* g = g6 + 6 * static_cast<int64_t>(f);
  double A, B, C;
  so3_coeffs(x[0], x[1], x[2], &A, &B, &C);
  double J[3][3];
  so3_matrix(x[0], x[1], x[2], B, C, J);
  const double r[3] = {g[0] - (x[4] * g[5] - x[5] * g[4]), g[1] - (x[5] * g[3] - x[3] * g[5]),
                       g[2] - (x[3] * g[4] - x[4] * g[3])};
  double* o = out + 6 * static_cast<int64_t>(f);
  for (int c = 0; c < 3; ++c) o[c] = J[0][c] * r[0] + J[1][c] * r[1] + J[2][c] * r[2];
  for (int c = 0; c < 3; ++c) o[3 + c] = g[3 + c];
}

}  // namespace pasfm

namespace pasfm {

// Trilinear resampling between voxel-centred grids covering the same world
// region (coarse-to-fine level change): dst(r) = src interpolated at r, with
// coordinates clamped to the source's outermost voxel centres.
__global__ void resample_kernel(const float* __restrict__ src, int sx, int sy, int sz, double sox, double soy,
                                double soz, double sdx, double sdy, double sdz, float* __restrict__ dst, int nx,
                                int ny, int nz, double ox, double oy, double oz, double dx, double dy, double dz) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t n = static_cast<int64_t>(nx) * ny * nz;
  if (i >= n) return;
  const int ix = static_cast<int>(i % nx), iy = static_cast<int>((i / nx) % ny), iz = static_cast<int>(i / (int64_t(nx) * ny));
  const double u[3] = {(ox + dx * ix - sox) / sdx, (oy + dy * iy - soy) / sdy, (oz + dz * iz - soz) / sdz};
  const int lim[3] = {sx, sy, sz};
  int i0[3];
  double w[3];
  for (int a = 0; a < 3; ++a) {
    const double c = fmin(fmax(u[a], 0.0), static_cast<double>(lim[a] - 1));
    int k = static_cast<int>(floor(c));
    if (k > lim[a] - 2) k = max(lim[a] - 2, 0);
    i0[a] = k;
    w[a] = lim[a] > 1 ? c - k : 0.0;
  }
  double acc = 0.0;
  for (int cz = 0; cz < 2; ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        const int jx = min(i0[0] + cx, sx - 1), jy = min(i0[1] + cy, sy - 1), jz = min(i0[2] + cz, sz - 1);
        const double wt = (cx ? w[0] : 1.0 - w[0]) * (cy ? w[1] : 1.0 - w[1]) * (cz ? w[2] : 1.0 - w[2]);
        acc += wt * src[(static_cast<int64_t>(jz) * sy + jy) * sx + jx];
      }
  dst[i] = static_cast<float>(acc);
}

}  // namespace pasfm

namespace pasfm {

// Gaussian low-pass along the time axis of every trace (coarse levels of the
// coarse-to-fine optimiser compare their wider pulses with band-limited data):
// dst[n] = sum_k w_k src[n + k], |k| <= r, w_k ~ exp(-k^2 / (2 sigma^2)) summing
// to 1, samples outside the record taken as zero.  One block per trace; the
// trace is staged in shared memory, so dst may alias src.
__global__ void __launch_bounds__(256) scale_kernel(float* __restrict__ x, int64_t n, float alpha) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    x[i] *= alpha;
}

__global__ void __launch_bounds__(256) diff_rows_kernel(const void* __restrict__ g, int dtype, int64_t rows,
                                                        int Nt, int Ntd, float* __restrict__ D) {
  const int64_t total = rows * Ntd;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = i / Ntd;
    const int n = static_cast<int>(i - r * Ntd);
    const int64_t base = r * Nt;
    const float cur = n < Nt ? load_elem(g, base + n, dtype) : 0.f;
    const float prev = (n >= 1 && n - 1 < Nt) ? load_elem(g, base + n - 1, dtype) : 0.f;
    D[i] = cur - prev;
  }
}

// FP32 throughput probe: kProbeChains independent FMA chains per thread for `iters`
// rounds (a multiple of 16; PACKED: two-wide packed FMAs on float2 chains).  The chains converge to
// c / (1 - m); their sum is stored only if it equals an impossible value, so no chain
// can be dropped and the kernel touches no memory.
// Independent FMA chains on every lane.  MODE 0: scalar FP32 (fmaf); 1: packed FP32
// (two FMAs per lane per instruction, __ffma2_rn on float2); 2: packed FP16 (__hfma2 on
// half2); 3: packed BF16 (__hfma2 on bfloat162).
template <int MODE>
__global__ void __launch_bounds__(256) fp32_probe_kernel(float* out, int iters, float m, float c) {
  constexpr int kProbeChains = 8;
  const float seed = 1e-3f * static_cast<float>(threadIdx.x);
  float s = 0.f;
  if constexpr (MODE == 1) {
    float2 a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = make_float2(seed + k, seed - k);
    const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) a[k] = __ffma2_rn(a[k], m2, c2);
    }
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += a[k].x + a[k].y;
  } else if constexpr (MODE == 2) {
    __half2 a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = __floats2half2_rn(seed + 0.01f * k, seed - 0.01f * k);
    const __half2 m2 = __float2half2_rn(m), c2 = __float2half2_rn(c);
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) a[k] = __hfma2(a[k], m2, c2);
    }
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += __low2float(a[k]) + __high2float(a[k]);
  } else if constexpr (MODE == 3) {
    __nv_bfloat162 a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = __floats2bfloat162_rn(seed + 0.01f * k, seed - 0.01f * k);
    const __nv_bfloat162 m2 = __float2bfloat162_rn(m), c2 = __float2bfloat162_rn(c);
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) a[k] = __hfma2(a[k], m2, c2);
    }
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += __low2float(a[k]) + __high2float(a[k]);
  } else {
    float a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = seed + k;
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) a[k] = fmaf(a[k], m, c);
    }
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += a[k];
  }
  if (s == -1.2345e30f) out[0] = s;
}

// Shared-memory read-modify-write probe, the access pattern of the forward's window:
// each thread owns a column of a [64 slots][256 threads] float array (a warp's access
// is one conflict-free 128-byte wavefront) and adds to 4 slot streams per round, 16
// rounds unrolled with compile-time slots, so every update is a load, an add and a
// store with no address arithmetic.
__global__ void __launch_bounds__(256) smem_probe_kernel(float* out, int iters, float v) {
  extern __shared__ float sp_win[];
  // volatile: every update is a real load and store (a private column could otherwise
  // live in registers), as in the forward, whose lanes' columns are indexed at run time
  volatile float* col = sp_win + threadIdx.x;
#pragma unroll
  for (int k = 0; k < 64; ++k) col[k * 256] = 0.f;
  for (int i = 0; i < iters; i += 16) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int s = (16 * j + 5 * r) & 63;
        col[s * 256] += v;
      }
    }
  }
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < 64; ++k) sum += col[k * 256];
  if (sum == -1.2345e30f) out[0] = sum;
}

double smem_probe_bytes(int blocks, int iters) {
  // per update: one 128-byte load and one 128-byte store wavefront per warp
  return double(blocks) * (256 / 32) * iters * 4 * 2 * 128.0;
}

cudaError_t smem_probe_launch(int blocks, int iters, float* out, cudaStream_t st) {
  const int smem = 64 * 256 * 4;
  cudaError_t e = cudaFuncSetAttribute(smem_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  smem_probe_kernel<<<blocks, 256, smem, st>>>(out, iters, 1e-3f);
  return cudaGetLastError();
}

double fp32_probe_flops(int blocks, int iters, int mode) {
  return double(blocks) * 256.0 * iters * 8 * 2 * (mode == 0 ? 1 : 2);
}

cudaError_t fp32_probe_launch(int mode, int blocks, int iters, float* out, cudaStream_t st) {
  switch (mode) {
    case 0: fp32_probe_kernel<0><<<blocks, 256, 0, st>>>(out, iters, 0.9999f, 1e-4f); break;
    case 1: fp32_probe_kernel<1><<<blocks, 256, 0, st>>>(out, iters, 0.9999f, 1e-4f); break;
    case 2: fp32_probe_kernel<2><<<blocks, 256, 0, st>>>(out, iters, 0.9999f, 1e-4f); break;
    case 3: fp32_probe_kernel<3><<<blocks, 256, 0, st>>>(out, iters, 0.9999f, 1e-4f); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) sum_parts_kernel(const float* __restrict__ parts, int n_parts, int64_t nvox,
                                                        float* __restrict__ vol, int accumulate) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nvox;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float acc = parts[i];
    for (int p = 1; p < n_parts; ++p) acc += parts[p * nvox + i];
    vol[i] = accumulate ? vol[i] + acc : acc;
  }
}

__global__ void __launch_bounds__(256) lowpass_kernel(const float* src, float* dst, int Nt, int r, int decim,
                                                      int Nout, const float* __restrict__ w) {
  extern __shared__ float row[];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * Nt;
  for (int n = threadIdx.x; n < Nt; n += blockDim.x) row[n] = src[base + n];
  __syncthreads();
  const int64_t obase = static_cast<int64_t>(blockIdx.x) * Nout;
  for (int m = threadIdx.x; m < Nout; m += blockDim.x) {
    const int n = m * decim;
    float acc = 0.f;
    const int k0 = max(-r, -n), k1 = min(r, Nt - 1 - n);
    for (int k = k0; k <= k1; ++k) acc = fmaf(w[k + r], row[n + k], acc);
    dst[obase + m] = acc;
  }
}

}  // namespace pasfm

namespace pasfm {

// Negative-correlation scores (Eq. 3) of K candidate trace sets against one
// frame's measured traces: score[k] = mean over kept elements j of
//   -Cov(sim_kj, meas_j) / (sigma(sim_kj) sigma(meas_j)).
// One block per candidate, one warp per element at a time; per-lane FP32 runs
// of at most ceil(Nt / 32) terms, carried to FP64 for the moments.
__global__ void __launch_bounds__(256) nc_scores_kernel(const float* __restrict__ sim, const void* meas,
                                                        int dtype, const uint8_t* __restrict__ mask, int E,
                                                        int Nt, double* __restrict__ out) {
  __shared__ double wsum[8];
  __shared__ int wcnt[8];
  const int k = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double acc = 0.0;
  int cnt = 0;
  for (int j = warp; j < E; j += nw) {
    if (mask && !mask[j]) continue;
    const float* s = sim + (static_cast<int64_t>(k) * E + j) * Nt;
    const int64_t mb = static_cast<int64_t>(j) * Nt;
    float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
    for (int n = lane; n < Nt; n += 32) {
      const float x = s[n], y = load_elem(meas, mb + n, dtype);
      a += x;
      b += y;
      aa = fmaf(x, x, aa);
      bb = fmaf(y, y, bb);
      ab = fmaf(x, y, ab);
    }
    double m[5] = {a, b, aa, bb, ab};
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m[q] += __shfl_xor_sync(0xffffffffu, m[q], o);
    const double cov = m[4] - m[0] * m[1] / Nt;
    const double vx = m[2] - m[0] * m[0] / Nt, vy = m[3] - m[1] * m[1] / Nt;
    const double den = sqrt(fmax(vx, 0.0) * fmax(vy, 0.0));
    acc += den > 0.0 ? -cov / den : 0.0;
    ++cnt;
  }
  if (lane == 0) {
    wsum[warp] = acc;
    wcnt[warp] = cnt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    int c = 0;
    for (int w = 0; w < nw; ++w) {
      t += wsum[w];
      c += wcnt[w];
    }
    out[k] = c ? t / c : 0.0;
  }
}

// Gradient of the NC loss (Eq. 3) summed over the kept traces: one warp per
// trace; centred sums in two passes (means, then centred moments: FP32 runs of at
// most ceil(Nt / 32) terms per lane, carried to FP64), then
//   g_n = -scale (m~_n / |m~| - rho s~_n / |s~|) / |s~|,  rho = <s~, m~> / (|s~| |m~|).
// g may alias sim: each lane reads s_n before writing g_n at the same n.
__global__ void __launch_bounds__(256) nc_grad_kernel(const float* sim, const void* meas, int dtype,
                                                      const uint8_t* __restrict__ mask, int64_t n_rows, int Nt,
                                                      int meas_repeat, float scale, float* g,
                                                      double* __restrict__ nc_out) {
  const int lane = threadIdx.x & 31;
  const int64_t row = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n_rows) return;
  const int64_t base = row * Nt;
  const int64_t mrow = row / meas_repeat;  // measured trace paired with this simulated one
  const int64_t mbase = mrow * Nt;
  const bool keep = !mask || mask[row];
  auto warp_sum = [](double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };
  double s_mean = 0.0, m_mean = 0.0, ns = 0.0, nm = 0.0, rho = 0.0;
  if (keep) {
    float a = 0.f, b = 0.f;
    for (int n = lane; n < Nt; n += 32) {
      a += sim[base + n];
      b += load_elem(meas, mbase + n, dtype);
    }
    s_mean = warp_sum(a) / Nt;
    m_mean = warp_sum(b) / Nt;
    const float sm = static_cast<float>(s_mean), mm = static_cast<float>(m_mean);
    float ss = 0.f, qq = 0.f, sq = 0.f;
    for (int n = lane; n < Nt; n += 32) {
      const float x = sim[base + n] - sm, y = load_elem(meas, mbase + n, dtype) - mm;
      ss = fmaf(x, x, ss);
      qq = fmaf(y, y, qq);
      sq = fmaf(x, y, sq);
    }
    ns = sqrt(warp_sum(ss));
    nm = sqrt(warp_sum(qq));
    const double c = warp_sum(sq);
    rho = (ns > 0.0 && nm > 0.0) ? c / (ns * nm) : 0.0;
  }
  const bool live = keep && ns > 0.0 && nm > 0.0;
  const float sm = static_cast<float>(s_mean), mm = static_cast<float>(m_mean);
  const float cm = live ? static_cast<float>(-scale / (nm * ns)) : 0.f;
  const float cs = live ? static_cast<float>(scale * rho / (ns * ns)) : 0.f;
  for (int n = lane; n < Nt; n += 32) {
    const float x = sim[base + n] - sm, y = load_elem(meas, mbase + n, dtype) - mm;
    g[base + n] = fmaf(cm, y, cs * x);
  }
  if (lane == 0 && nc_out) nc_out[row] = live ? -rho : 0.0;
}

}  // namespace pasfm
