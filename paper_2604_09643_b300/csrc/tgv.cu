// Smoothed second-order total generalized variation (TGV) of the volume, the
// regulariser of Stages 1 and 5 (Eq. 2, L_TGV):
//
//   J(u, w) = sum_i alpha1 sqrt(|D u - w|^2 + eps^2) + alpha0 sqrt(|E(w)|_F^2 + eps^2),
//   E(w)_ab = (D_a w_b + D_b w_a) / 2,
//
// D_a the forward difference along axis a over the spacing, zero on the last
// index.  With q = alpha1 (D u - w) / phi1 and P = alpha0 E / phi2 the gradients
// are dJ/du = sum_a D_a^T q_a and dJ/dw_b = -q_b + sum_a D_a^T P_ab, where
// (D_a^T y)[j] = ([j_a >= 1] y[j - e_a] - [j_a <= n_a - 2] y[j]) / d_a.
//
// One CTA per 32 x 4 x 4 tile, one voxel per thread, four CTAs per SM.  The
// tile's u and w with a one-voxel halo below and above (x widened to a 4-voxel
// boundary) and its slice of the accumulated volume gradient are staged in
// shared memory by TMA (zero fill outside the grid; plain loads when rows are
// not 16-byte aligned or p0 is 16-bit), so no thread waits on a dependent global
// load.  q and P are formed once for the tile plus its lower halo, so each output
// reads its neighbours' q and P from shared memory: u and w come from HBM once
// per tile (halos from L2) and the gradients are written once.  The norms use one
// rsqrt each (phi = f rsqrt(f), alpha / phi = alpha rsqrt(f)).  The energy is
// reduced per CTA in FP64 and summed in a fixed order.
#include "aux.cuh"

namespace pasfm {

namespace {

constexpr int TX = 32, TY = 4, TZ = 4;                // tile
constexpr int TN = TX * TY * TZ;
constexpr int RX = TX + 8, RY = TY + 2, RZ = TZ + 2;  // staged region: x in [x0-4, x0+36), y, z in [-1, +5)
constexpr int RN = RX * RY * RZ;
constexpr int QX = TX + 1, QY = TY + 1, QZ = TZ + 1;  // q, P at tile offsets -1..T-1
constexpr int QN = QX * QY * QZ;

struct TgvBuf {
  float u[RN];
  float w[3][RN];
  float gu[TN];  // the tile's accumulated volume gradient (when accumulating)
};

struct TgvSmem {
  TgvBuf buf;
  float qp[9][QN];  // q_x, q_y, q_z, P_xx, P_yy, P_zz, P_xy, P_xz, P_yz
  double red[TN / 32];
  uint64_t bar;
};

__device__ __forceinline__ int ridx(int x, int y, int z) { return (z * RY + y) * RX + x; }
__device__ __forceinline__ int qidx(int x, int y, int z) { return (z * QY + y) * QX + x; }

}  // namespace

__global__ void __launch_bounds__(TN, 4)
    tgv_kernel(const __grid_constant__ CUtensorMap umap, const __grid_constant__ CUtensorMap wmap,
               const __grid_constant__ CUtensorMap gmap, const TgvParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TgvSmem& S = *reinterpret_cast<TgvSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const int64_t nvox = static_cast<int64_t>(P.nx) * P.ny * P.nz;
  const float inv_d[3] = {P.inv_dx, P.inv_dy, P.inv_dz};
  const int nn[3] = {P.nx, P.ny, P.nz};
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  TgvBuf& B = S.buf;

  // stage u, w (region) and the tile's accumulated volume gradient
  bool ok = true;
  if (P.use_tma) {
    if (tid == 0) {
      mbar_init(&S.bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
      mbar_arrive_expect_tx(&S.bar, static_cast<uint32_t>(4 * RN * 4 + (P.accumulate ? TN * 4 : 0)));
      tma_load_3d(B.u, &umap, &S.bar, x0 - 4, y0 - 1, z0 - 1);
      tma_load_4d(B.w[0], &wmap, &S.bar, x0 - 4, y0 - 1, z0 - 1, 0);
      if (P.accumulate) tma_load_3d(B.gu, &gmap, &S.bar, x0, y0, z0);
    }
    // one thread polls the barrier; the others sleep in the block barrier below rather than
    // spend issue slots that the co-resident tiles' arithmetic needs (the barrier orders the
    // copies' completion, observed by thread 0, before every thread's reads)
    if (tid == 0) ok = mbar_wait_limited(&S.bar, 0, P.status, P.wait_cycles);
  } else {
    for (int k = tid; k < RN; k += blockDim.x) {
      const int rx = k % RX, ry = (k / RX) % RY, rz = k / (RX * RY);
      const int gx = x0 - 4 + rx, gy = y0 - 1 + ry, gz = z0 - 1 + rz;
      const bool in = gx >= 0 && gx < P.nx && gy >= 0 && gy < P.ny && gz >= 0 && gz < P.nz;
      const int64_t g = (static_cast<int64_t>(gz) * P.ny + gy) * P.nx + gx;
      B.u[k] = in ? load_elem(P.u, g, P.dtype_u) : 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) B.w[c][k] = in ? P.w[c * nvox + g] : 0.f;
    }
    const int gx = x0 + tid % TX, gy = y0 + (tid / TX) % TY, gz = z0 + tid / (TX * TY);
    const bool in = gx < P.nx && gy < P.ny && gz < P.nz;
    B.gu[tid] = (in && P.accumulate) ? P.grad_u[(static_cast<int64_t>(gz) * P.ny + gy) * P.nx + gx] : 0.f;
  }
  if (__syncthreads_or(!ok)) {
    if (tid == 0 && P.use_tma) mbar_wait_bounded(&S.bar, 0, P.status);  // let the copies land before exit
    return;
  }

  float e_loc = 0.f;
  {
    // q and P at tile offsets (-1..TX-1, -1..TY-1, -1..TZ-1); the energy over the tile
    for (int k = tid; k < QN; k += blockDim.x) {
      const int qz = k / (QX * QY), rem = k - qz * (QX * QY);
      const int qy = rem / QX, qx = rem - qy * QX;
      const int g[3] = {x0 - 1 + qx, y0 - 1 + qy, z0 - 1 + qz};
      const bool in = g[0] >= 0 && g[0] < P.nx && g[1] >= 0 && g[1] < P.ny && g[2] >= 0 && g[2] < P.nz;
      float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (in) {
        const int r = ridx(qx + 3, qy, qz);  // region offset of this point
        const int step[3] = {1, RX, RX * RY};
        float du[3], dw[3][3];  // dw[a][c] = D_a w_c
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const bool fwd = g[a] + 1 < nn[a];
          du[a] = fwd ? (B.u[r + step[a]] - B.u[r]) * inv_d[a] : 0.f;
#pragma unroll
          for (int c = 0; c < 3; ++c) dw[a][c] = fwd ? (B.w[c][r + step[a]] - B.w[c][r]) * inv_d[a] : 0.f;
        }
        const float rx_ = du[0] - B.w[0][r], ry_ = du[1] - B.w[1][r], rz_ = du[2] - B.w[2][r];
        const float f1 = fmaf(rx_, rx_, fmaf(ry_, ry_, fmaf(rz_, rz_, P.eps2)));
        const float r1 = rsqrtf(f1), phi1 = f1 * r1;
        const float exx = dw[0][0], eyy = dw[1][1], ezz = dw[2][2];
        const float exy = 0.5f * (dw[0][1] + dw[1][0]), exz = 0.5f * (dw[0][2] + dw[2][0]),
                    eyz = 0.5f * (dw[1][2] + dw[2][1]);
        const float f2 = fmaf(exx, exx, fmaf(eyy, eyy, fmaf(ezz, ezz, P.eps2))) +
                         2.f * fmaf(exy, exy, fmaf(exz, exz, eyz * eyz));
        const float r2 = rsqrtf(f2), phi2 = f2 * r2;
        const float c1 = P.alpha1 * r1, c0 = P.alpha0 * r2;
        v[0] = c1 * rx_;
        v[1] = c1 * ry_;
        v[2] = c1 * rz_;
        v[3] = c0 * exx;
        v[4] = c0 * eyy;
        v[5] = c0 * ezz;
        v[6] = c0 * exy;
        v[7] = c0 * exz;
        v[8] = c0 * eyz;
        if (qx >= 1 && qy >= 1 && qz >= 1) e_loc += fmaf(P.alpha1, phi1, P.alpha0 * phi2);
      }
#pragma unroll
      for (int c = 0; c < 9; ++c) S.qp[c][k] = v[c];
    }
    __syncthreads();

    // gradients at this thread's voxel
    const int tx = tid % TX, ty = (tid / TX) % TY, tz = tid / (TX * TY);
    const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
    if (gx < P.nx && gy < P.ny && gz < P.nz) {
      const int gj[3] = {gx, gy, gz};
      const int c = qidx(tx + 1, ty + 1, tz + 1);
      const int back[3] = {c - 1, c - QX, c - QX * QY};
      // transpose of D_a applied to a component field at this voxel
      auto dT = [&](int comp, int a) {
        const float prev = gj[a] >= 1 ? S.qp[comp][back[a]] : 0.f;
        const float here = gj[a] <= nn[a] - 2 ? S.qp[comp][c] : 0.f;
        return (prev - here) * inv_d[a];
      };
      // P_ab as a component of qp: diagonal 3 + a, off-diagonal xy 6, xz 7, yz 8
      auto pc = [](int a, int b2) { return a == b2 ? 3 + a : (a + b2 == 1 ? 6 : (a + b2 == 2 ? 7 : 8)); };
      const float gu = dT(0, 0) + dT(1, 1) + dT(2, 2);
      const int64_t g = (static_cast<int64_t>(gz) * P.ny + gy) * P.nx + gx;
      P.grad_u[g] = P.accumulate ? B.gu[tid] + gu : gu;
#pragma unroll
      for (int cb = 0; cb < 3; ++cb) {
        const float gw = -S.qp[cb][c] + dT(pc(0, cb), 0) + dT(pc(1, cb), 1) + dT(pc(2, cb), 2);
        P.grad_w[cb * nvox + g] = gw;
      }
    }
  }

  // the tile's energy in FP64, fixed order
  double e = e_loc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((tid & 31) == 0) S.red[tid >> 5] = e;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int k = 0; k < TN / 32; ++k) t += S.red[k];
    P.energy_part[(static_cast<int64_t>(blockIdx.z) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
  }
}

size_t tgv_smem_bytes() { return sizeof(TgvSmem); }

int tgv_tiles(int nx, int ny, int nz) {
  return ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY) * ((nz + TZ - 1) / TZ);
}

dim3 tgv_grid(int nx, int ny, int nz) { return dim3((nx + TX - 1) / TX, (ny + TY - 1) / TY, (nz + TZ - 1) / TZ); }

int tgv_threads() { return TN; }

void tgv_boxes(unsigned* box3, unsigned* box4, unsigned* boxg) {
  box3[0] = RX;
  box3[1] = RY;
  box3[2] = RZ;
  box4[0] = RX;
  box4[1] = RY;
  box4[2] = RZ;
  box4[3] = 3;
  boxg[0] = TX;
  boxg[1] = TY;
  boxg[2] = TZ;
}

}  // namespace pasfm
