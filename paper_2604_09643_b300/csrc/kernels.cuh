// Hot kernels of the radiation operator (sm_103a, FP32 pair arithmetic).
//
//   fwd_cube_kernel  -- forward s = A(p0; poses).  Element-stationary: lane =
//                       element, a warp owns 32 elements, a CTA owns one cube of
//                       C^3 voxels (staged by a 3-D TMA load) for one frame.
//                       Each lane scatters its pulse samples into a private
//                       column of a shared-memory time window laid out
//                       [slot][32 lanes], so any per-lane offset is
//                       bank-conflict free and no atomics are needed.  The
//                       window (the cube's distance range for that element)
//                       holds the running sum of the slot weights, so a pair
//                       writes S - 1 slots (its weights sum to zero; S >= 3); the
//                       flush differences it into a per-cube partial trace and
//                       fwd_reduce_kernel sums the partials in a fixed order.
//   bwd_cube_kernel  -- adjoint v = A^T g and/or pose gradient.  Voxel-
//                       stationary: a thread owns a row of C voxels along x; the
//                       CTA walks all (frame, element) traces in batches of 32
//                       whose sample windows are staged by 2-D TMA loads into a
//                       double buffer.  The adjoint is an atomic-free gather; the
//                       pose gradient is reduced per element with warp shuffles
//                       and a fixed-order block reduction, then carried to FP64.
//
// Sample slots: a voxel-element pair touches at most S = floor(2 a0 / h) + 2
// consecutive samples.  With psi = (d - a0 - tau0) / h + 1/2 and first slot
// n_s = floor(psi), the slot boundaries beta_k = (n_s - psi) h - a0 + k h satisfy
// beta_0 <= -a0 and beta_S > a0, boundaries 1..S-2 lie inside [-a0, a0] and only
// boundary S-1 needs a clamp.  Sample n_s + k then gets
//     W = (b_k - b_{k+1}) / (4 d h),  b_k = clamp(beta_k)^2,  b_0 = b_S = a0^2,
// which is the interval average of the uniform-sphere pulse (Appendix A).
//
// The Gaussian kernel (Eq. 1, K_G) has the same slot structure with a0 replaced
// by the support half-width sup = 4 sigma: sample n_s + k gets
//     W = sigma^2 (E_{k+1} - E_k) / (2 d h),  E_k = exp(-clamp(beta_k)^2 / (2 sigma^2)),
// E_0 = E_S = exp(-8).  In the code a0 below stands for sup; template parameter K
// selects the profile (PASFM_KERNEL_SPHERE or PASFM_KERNEL_GAUSS).
#pragma once

#include "pasfm_dev.cuh"

namespace pasfm {

// ------------------------------------------------------------------------
// per-pair slot math
// ------------------------------------------------------------------------
struct PairMath {
  float rs;       // 1 / d
  unsigned idx;   // first slot's index in the window (before clamping)
  float beta1;    // boundary between slots 0 and 1 (mm); boundary 0 is <= -a0 and never used
};

// idx_bias = kMagicBits + (window slot 0 relative to N_c), so that
// idx = n_s - (slot 0) comes out of the rounding trick with one integer op.
__device__ __forceinline__ PairMath pair_math(float A, float dc2, float dcf, float phim, float inv_h, float h,
                                              float cb1, int idx_bias) {
  PairMath m;
  const float D2 = dc2 + A;
  m.rs = rsqrtf(D2);
  const float del = __fdividef(A, fmaf(D2, m.rs, dcf));  // d - d_c = A / (d + d_c), no cancellation
  const float psi = fmaf(del, inv_h, phim);               // psi_c - N_c - 1/2 + delta / h
  const float t = psi + kMagic;                           // round to nearest = floor(psi + 1/2)
  m.idx = static_cast<unsigned>(__float_as_int(t) - idx_bias);
  m.beta1 = fmaf((t - kMagic) - psi, h, cb1);             // (n_s - psi_full) h - a0 + h
  return m;
}

// ------------------------------------------------------------------------
// Gaussian boundary values
// ------------------------------------------------------------------------
// Index of the boundary the recurrences start from: the one nearest the pulse
// centre (beta_k = beta1 + (k - 1) h with beta1 in (-sup, -sup + h] and
// sup ~ (S - 1) h / 2).
template <int S>
__host__ __device__ constexpr int gauss_centre() { return S / 2 < 1 ? 1 : S / 2; }

// E[k] = exp(-beta_k^2 / (2 sigma^2)) for the boundaries k = 1..S-1 (E[0] is
// not set).  Three exp2f per pair; the other values come from the ratio
// recurrence of a Gaussian on an equispaced grid, E_{k+1} = E_k r_k with
// r_{k+1} = r_k q (the device of "fast Gaussian gridding", Greengard & Lee,
// SIAM Rev. 2004), run outward both ways from the centre boundary so that
// rounding grows only toward the tails, where E is small.  Boundary S-1 can
// lie past the support edge; E decreases for beta > 0, so the max with the
// edge value is its clamp.
template <int S>
__device__ __forceinline__ void gauss_boundaries(float beta1, float h, const GaussConst& G, float (&E)[S]) {
  constexpr int kc = gauss_centre<S>();
  const float bc = fmaf(static_cast<float>(kc - 1), h, beta1);
  E[kc] = exp2f(G.c1 * (bc * bc));
  float up = exp2f(fmaf(bc, G.c2, G.c3));   // E_{kc+1} / E_kc
  float dn = exp2f(fmaf(-bc, G.c2, G.c3));  // E_{kc-1} / E_kc
#pragma unroll
  for (int k = kc + 1; k < S; ++k) {
    E[k] = E[k - 1] * up;
    up *= G.q;
  }
#pragma unroll
  for (int k = kc - 1; k >= 1; --k) {
    E[k] = E[k + 1] * dn;
    dn *= G.q;
  }
  E[S - 1] = fmaxf(E[S - 1], G.e_clamp);
}

// ------------------------------------------------------------------------
// forward
// ------------------------------------------------------------------------
template <int C>
__host__ __device__ constexpr int fwd_tile_bytes() { return C * C * C * 4; }
template <int C>
__host__ __device__ constexpr int fwd_win_offset() {
  return ((fwd_tile_bytes<C>() + C * C + 16 + 127) / 128) * 128;
}

template <int C, int S, int K>
__global__ void __launch_bounds__(256, 2)
    fwd_cube_kernel(const __grid_constant__ CUtensorMap p0map, const FwdParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  float* tile = reinterpret_cast<float*>(smem);
  uint8_t* rowflag = smem + fwd_tile_bytes<C>();
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + ((fwd_tile_bytes<C>() + C * C + 7) / 8) * 8);
  float* win = reinterpret_cast<float*>(smem + fwd_win_offset<C>());

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nwarps = blockDim.x >> 5;
  const int c = blockIdx.x;
  const int ncubes = gridDim.x;
  const int cx = c % P.ncx, cy = (c / P.ncx) % P.ncy, cz = c / (P.ncx * P.ncy);
  const int fl = blockIdx.y, f = P.f_begin + fl;
  const int j = (blockIdx.z * nwarps + warp) * kWarp + lane;
  const bool valid = j < P.E;
  const int jj = valid ? j : P.E - 1;

  // 1. stage the p0 cube (zero outside the grid)
  if (P.use_tma) {
    if (tid == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
      mbar_arrive_expect_tx(bar, fwd_tile_bytes<C>());
      tma_load_3d(tile, &p0map, bar, cx * C, cy * C, cz * C);
    }
  } else {
    for (int k = tid; k < C * C * C; k += blockDim.x) {
      const int lx = k % C, ly = (k / C) % C, lz = k / (C * C);
      const int ix = cx * C + lx, iy = cy * C + ly, iz = cz * C + lz;
      float v = 0.f;
      if (ix < P.nx && iy < P.ny && iz < P.nz)
        v = load_elem(P.p0, (static_cast<int64_t>(iz) * P.ny + iy) * P.nx + ix, P.dtype_vol);
      tile[k] = v;
    }
  }

  // 2. zero this lane's window column
  float* col = win + warp * P.W * kWarp + lane;
  for (int k = 0; k < P.W; ++k) col[k * kWarp] = 0.f;

  // 3. per-(cube, element) reference in FP64
  const double* xp = P.xw + (static_cast<int64_t>(f) * P.E + jj) * 3;
  const double hc = 0.5 * (C - 1);
  const PairRef R = make_ref(xp[0], xp[1], xp[2], P.ox + P.dx * (cx * C + hc), P.oy + P.dy * (cy * C + hc),
                             P.oz + P.dz * (cz * C + hc), P.sup, P.tau0, P.inv_h);
  const int nb_rel = static_cast<int>(floorf(R.phim - P.nb_shift)) - 1;
  const float dxf = static_cast<float>(P.dx), dyf = static_cast<float>(P.dy), dzf = static_cast<float>(P.dz);
  float Pix[C];
#pragma unroll
  for (int ix = 0; ix < C; ++ix) {
    const float qx = (ix - 0.5f * (C - 1)) * dxf;
    Pix[ix] = qx * (qx + R.m2ux);
  }

  // 4. wait for the tile; flag rows that hold any nonzero voxel
  bool ok = true;
  if (P.use_tma) ok = mbar_wait_bounded(bar, 0, P.status);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) mbar_wait_bounded(bar, 0, P.status);  // let the copy land before exit
    return;
  }
  for (int r = tid; r < C * C; r += blockDim.x) {
    bool nz = false;
#pragma unroll
    for (int ix = 0; ix < C; ++ix) nz |= tile[r * C + ix] != 0.f;
    rowflag[r] = nz ? 1 : 0;
  }
  __syncthreads();

  // 5. pair loop: every voxel of the cube against this lane's element
  const unsigned max_idx = static_cast<unsigned>(P.W - S);
  const int idx_bias = kMagicBits + nb_rel;
  // Clamp detection.  A voxel's distance to the element is convex along a row, and the
  // first slot index grows with the distance, so a row's largest index is at one of its
  // two ends: those are the only pairs checked.  (The window covers the cube's
  // distance range with half a sample to spare, so no index is clamped unless the
  // geometry is degenerate; the clamp itself is applied to every pair.)
  unsigned seen = 0;  // largest raw index at the row ends (a negative one wraps to a huge value)
  for (int lz = 0; lz < C; ++lz) {
    const float qz = (lz - 0.5f * (C - 1)) * dzf;
    const float Cz = qz * (qz + R.m2uz);
    for (int ly = 0; ly < C; ++ly) {
      if (!rowflag[lz * C + ly]) continue;
      const float qy = (ly - 0.5f * (C - 1)) * dyf;
      const float Crow = fmaf(qy, qy + R.m2uy, Cz);
      const float* prow = tile + (lz * C + ly) * C;
#pragma unroll
      for (int i4 = 0; i4 < C; i4 += 4) {
        const float4 pv4 = *reinterpret_cast<const float4*>(prow + i4);
        const float pv[4] = {pv4.x, pv4.y, pv4.z, pv4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const PairMath m = pair_math(Pix[i4 + u] + Crow, R.dc2, R.dcf, R.phim, P.inv_hf, P.h, P.cb1, idx_bias);
          if (i4 + u == 0 || i4 + u == C - 1) seen = max(seen, m.idx);
          float* slot = col + min(m.idx, max_idx) * kWarp;
          const float s = pv[u] * m.rs;
          // The pair's slot weights b_k - b_{k+1} (k = 0..S-1) sum to b_0 - b_S = 0, so
          // for S >= 3 the window holds their running sum: slot k gets b_0 - b_{k+1} for
          // k = 0..S-2 and slot S-1 gets nothing.  That is S - 1 read-modify-writes
          // instead of S through shared memory, which bounds this loop; the flush takes
          // the first difference.  Sphere: b_0 = a0^2, b_k = beta_k^2 inside, the last
          // boundary clamped.  Gaussian: b = -E, b_0 = -E(edge).  At S = 2 (a pulse
          // narrower than a sample) every pair is a +-w dipole on two slots; the running
          // sum would then hold two separately accumulated sums per sample whose
          // difference cancels in homogeneous regions, so the weights go in directly.
          if constexpr (S == 2) {
            float w;
            if constexpr (K == PASFM_KERNEL_GAUSS) {
              float E[S];
              gauss_boundaries<S>(m.beta1, P.h, P.gs, E);
              w = E[1] - P.gs.e_clamp;
            } else {
              const float bc = fminf(m.beta1, P.supf);
              w = fmaf(-bc, bc, P.sup2);
            }
            slot[0] = fmaf(s, w, slot[0]);
            slot[kWarp] = fmaf(-s, w, slot[kWarp]);
          } else if constexpr (K == PASFM_KERNEL_GAUSS) {
            float E[S];
            gauss_boundaries<S>(m.beta1, P.h, P.gs, E);
#pragma unroll
            for (int k = 0; k <= S - 2; ++k) slot[k * kWarp] = fmaf(s, E[k + 1] - P.gs.e_clamp, slot[k * kWarp]);
          } else {
            float beta = m.beta1;
#pragma unroll
            for (int k = 0; k <= S - 2; ++k) {
              if (k > 0) beta += P.h;
              const float bc = (k == S - 2) ? fminf(beta, P.supf) : beta;
              slot[k * kWarp] = fmaf(s, fmaf(-bc, bc, P.sup2), slot[k * kWarp]);
            }
          }
        }
      }
    }
  }
  if (seen > max_idx) atomicOr(P.status, PASFM_STATUS_INDEX_CLAMPED);

  // 6. flush the window (its first difference for S >= 3) as this cube's partial trace
  //    (scaled by 1 / (4 h), or sigma^2 / (2 h))
  __syncwarp();
  if (valid) {
    const int64_t row = static_cast<int64_t>(fl) * P.E + j;
    float* dst = P.part + (row * ncubes + c) * P.W;
    float prev = 0.f;
    for (int k = 0; k < P.W; k += 4) {
      const float c0 = col[(k + 0) * kWarp], c1 = col[(k + 1) * kWarp], c2 = col[(k + 2) * kWarp],
                  c3 = col[(k + 3) * kWarp];
      float4 v;
      if constexpr (S >= 3) {
        v.x = (c0 - prev) * P.p0_scale;
        v.y = (c1 - c0) * P.p0_scale;
        v.z = (c2 - c1) * P.p0_scale;
        v.w = (c3 - c2) * P.p0_scale;
        prev = c3;
      } else {
        v = make_float4(c0 * P.p0_scale, c1 * P.p0_scale, c2 * P.p0_scale, c3 * P.p0_scale);
      }
      *reinterpret_cast<float4*>(dst + k) = v;
    }
    P.n0tab[row * ncubes + c] = R.Nc + nb_rel;
  }
}

// ------------------------------------------------------------------------
// backward (adjoint gather + pose-gradient reduction)
// ------------------------------------------------------------------------
constexpr int kBatch = 32;  // traces staged per batch

template <int C>
struct BwdLayout {
  static constexpr int NT = C * C;
  static constexpr int NW = NT / kWarp;
  // offsets in bytes, given the staged window length WP (floats)
  __host__ __device__ static int win_bytes(int WP) { return 2 * kBatch * WP * 4; }
  __host__ __device__ static int refa_off(int WP) { return win_bytes(WP); }
  __host__ __device__ static int refb_off(int WP) { return refa_off(WP) + 2 * kBatch * 16; }
  __host__ __device__ static int refu_off(int WP) { return refb_off(WP) + 2 * kBatch * 16; }
  __host__ __device__ static int red_off(int WP) { return refu_off(WP) + 2 * kBatch * 24; }
  __host__ __device__ static int bar_off(int WP) { return red_off(WP) + 2 * NW * kBatch * 16; }
  __host__ __device__ static int total(int WP) { return bar_off(WP) + 16; }
};

template <int C>
__device__ __forceinline__ void bwd_thread_row(int tid, int& ty, int& tz) {
  const int w = tid >> 5, l = tid & 31;
  if (C == 16) {  // a warp covers 4 (y) x 8 (z) rows
    ty = 4 * (w & 3) + (l & 3);
    tz = 8 * (w >> 2) + (l >> 2);
  } else {        // C == 8: a warp covers 8 (y) x 4 (z) rows
    ty = l & 7;
    tz = 4 * w + (l >> 3);
  }
}

template <int C, int S, int K, bool ADJ, bool POSE>
__global__ void __launch_bounds__(C* C, (C == 16 ? 2 : 8))
    bwd_cube_kernel(const __grid_constant__ CUtensorMap gmap, const BwdParams P) {
  using L = BwdLayout<C>;
  extern __shared__ __align__(128) unsigned char smem[];
  const int WP = P.WP;
  float* win = reinterpret_cast<float*>(smem);
  float4* refa = reinterpret_cast<float4*>(smem + L::refa_off(WP));
  float4* refb = reinterpret_cast<float4*>(smem + L::refb_off(WP));
  double* refu = reinterpret_cast<double*>(smem + L::refu_off(WP));
  float4* red = reinterpret_cast<float4*>(smem + L::red_off(WP));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::bar_off(WP));

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = blockIdx.x, ncubes = gridDim.x;
  const int cx = c % P.ncx, cy = (c / P.ncx) % P.ncy, cz = c / (P.ncx * P.ncy);
  int ty, tz;
  bwd_thread_row<C>(tid, ty, tz);
  const int iy = cy * C + ty, iz = cz * C + tz;
  const bool row_in = iy < P.ny && iz < P.nz;

  const float dxf = static_cast<float>(P.dx);
  const float qy = (ty - 0.5f * (C - 1)) * static_cast<float>(P.dy);
  const float qz = (tz - 0.5f * (C - 1)) * static_cast<float>(P.dz);
  float qx[C];
#pragma unroll
  for (int k = 0; k < C; ++k) qx[k] = (k - 0.5f * (C - 1)) * dxf;

  float p0s[POSE ? C : 1];
  if (POSE) {
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const int ix = cx * C + k;
      p0s[k] = (row_in && ix < P.nx)
                   ? load_elem(P.p0, (static_cast<int64_t>(iz) * P.ny + iy) * P.nx + ix, P.dtype_vol) * P.scale
                   : 0.f;
    }
  }
  // adjoint: per-batch partial sums (<= 32 traces x S terms) folded once per batch
  float acc[ADJ ? C : 1], bacc[ADJ ? C : 1];
  if (ADJ) {
#pragma unroll
    for (int k = 0; k < C; ++k) acc[k] = bacc[k] = 0.f;
  }

  const double hc = 0.5 * (C - 1);
  const double rcx = P.ox + P.dx * (cx * C + hc), rcy = P.oy + P.dy * (cy * C + hc),
               rcz = P.oz + P.dz * (cz * C + hc);
  // this CTA's share of the (frame, element) items: [ib, ib + nl)
  const int ib = blockIdx.y * P.part_items;
  const int nl = max(0, min(P.n_items - ib, P.part_items));
  const int nb = (nl + kBatch - 1) / kBatch;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // producer: one warp stages batch b into buffer buf (lane l handles trace l)
  auto issue = [&](int b, int buf) {
    const int it = ib + b * kBatch + lane;
    const int cnt = min(kBatch, nl - b * kBatch);
    float* wdst = win + (buf * kBatch + lane) * WP;
    int x0 = 0, row = 0;
    if (it < ib + nl) {
      const int fl = it / P.E, j = it % P.E;
      const int f = P.f_begin + fl;
      row = f * P.E + j;
      const double* xp = P.xw + static_cast<int64_t>(row) * 3;
      const PairRef R = make_ref(xp[0], xp[1], xp[2], rcx, rcy, rcz, P.sup, P.tau0, P.inv_h);
      const int n0 = R.Nc + static_cast<int>(floorf(R.phim - P.nb_shift)) - 1;
      x0 = n0 & ~3;
      const float mk = (POSE && P.mask) ? (P.mask[row] ? 1.f : 0.f) : 1.f;
      refa[buf * kBatch + lane] = make_float4(R.m2ux, R.m2uy, R.m2uz, R.dc2);
      refb[buf * kBatch + lane] = make_float4(R.dcf, R.phim, __int_as_float(R.Nc - x0), mk);
      if (POSE) {
        refu[(buf * kBatch + lane) * 3 + 0] = R.ux;
        refu[(buf * kBatch + lane) * 3 + 1] = R.uy;
        refu[(buf * kBatch + lane) * 3 + 2] = R.uz;
      }
      if (!P.use_tma) {  // plain loads with zero fill outside [0, Nt)
        const int64_t base = static_cast<int64_t>(row) * P.Nt;
        for (int k = 0; k < WP; ++k) {
          const int n = x0 + k;
          wdst[k] = (n >= 0 && n < P.Nt) ? load_elem(P.g, base + n, P.dtype_sig) : 0.f;
        }
      }
    }
    if (P.use_tma) {
      __syncwarp();  // the warp's reference writes happen before lane 0's (releasing) arrival
      if (lane == 0) mbar_arrive_expect_tx(&bar[buf], static_cast<uint32_t>(cnt * WP * 4));
      __syncwarp();
      if (it < ib + nl) tma_load_2d(wdst, &gmap, &bar[buf], x0, row);
    } else {
      __threadfence_block();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar[buf]);
    }
  };

  if (warp == 0 && nb > 0) {
    issue(0, 0);
    if (nb > 1) issue(1, 1);
  }

  // One block barrier per batch.  After the barrier of batch b, warp b % NW
  // (rotating, so the extra work is spread over the warps) reduces batch b's
  // pose partials and restages buffer b & 1 with batch b + 2, while the other
  // warps already compute batch b + 1.  The warp-reduction slots are
  // double-buffered; the reducing warp's program order keeps its reads of
  // refs[buf] ahead of its producer writes.  A timed-out wait makes every
  // thread skip the compute, and the barrier (an OR vote) ends the CTA.
  const unsigned max_idx = static_cast<unsigned>(WP - S);
  unsigned seen = 0;  // largest raw window index at the row ends (see fwd_cube_kernel)
  for (int b = 0; b < nb; ++b) {
    const int buf = b & 1;
    const bool ok = mbar_wait_bounded(&bar[buf], (b >> 1) & 1, P.status);
    const int cnt = min(kBatch, nl - b * kBatch);
    const float* wb = win + buf * kBatch * WP;
    for (int e = 0; ok && e < cnt; ++e) {
      const float4 ra = refa[buf * kBatch + e];
      const float4 rb = refb[buf * kBatch + e];
      const int idx_bias = kMagicBits - __float_as_int(rb.z);
      const float* wv = wb + e * WP;
      const float Crow = fmaf(qy, qy + ra.y, qz * (qz + ra.z));
      float R0 = 0.f, R1 = 0.f;
#pragma unroll
      for (int k = 0; k < C; ++k) {
        const float A = fmaf(qx[k], qx[k] + ra.x, Crow);
        const PairMath m = pair_math(A, ra.w, rb.x, rb.y, P.inv_hf, P.h, P.cb1, idx_bias);
        if (k == 0 || k == C - 1) seen = max(seen, m.idx);
        const float* gw = wv + min(m.idx, max_idx);
        // S1 = sum_k g_k (b_k - b_{k+1}) by parts; S2 = the boundary-motion term of dW/dd
        float S1, S2 = 0.f, lam;
        if constexpr (K == PASFM_KERNEL_GAUSS) {
          // b_s = -E_s (sign folded into P.scale < 0); visited outward from the centre
          // boundary as in gauss_boundaries, without an array of values
          constexpr int kc = gauss_centre<S>();
          const float bc = fmaf(static_cast<float>(kc - 1), P.h, m.beta1);
          const float Ec = exp2f(P.gs.c1 * (bc * bc));
          float up = exp2f(fmaf(bc, P.gs.c2, P.gs.c3));
          float dn = exp2f(fmaf(-bc, P.gs.c2, P.gs.c3));
          // With u_s = E_s dg_s and beta_s = bc + (s - kc) h, the boundary-motion sum
          // S2 = sum_s beta_s u_s over the boundaries inside the support is
          // bc U + h T with U = sum_s u_s and T = sum_s (s - kc) u_s; boundary S-1
          // (possibly past the edge, where it does not move with d) is added on its own.
          // Each sweep keeps the running sum P_j of u over its first j boundaries and the
          // sum Q of those running sums: sum_{j=0..J} j u_j = J P_J - (P_0 + ... + P_{J-1}),
          // two operations per boundary instead of three.
          float E = Ec, gp = gw[kc - 1];
          float Pu = 0.f, Qu = 0.f, Pd = 0.f, Qd = 0.f, last = 0.f;
          S1 = 0.f;
#pragma unroll
          for (int s = kc; s < S; ++s) {
            if (s > kc) {
              E *= up;
              up *= P.gs.q;
            }
            const float gs = gw[s];
            const float dg = gs - gp;
            gp = gs;
            if (s == S - 1) {
              const float Es = fmaxf(E, P.gs.e_clamp);
              S1 = fmaf(Es, dg, S1);
              if (POSE) {
                const float beta = fmaf(static_cast<float>(s - 1), P.h, m.beta1);
                last = beta < P.supf ? beta * Es * dg : 0.f;
              }
            } else if (POSE) {
              Pu = fmaf(E, dg, Pu);
              if (s < S - 2) Qu += Pu;
            } else {
              S1 = fmaf(E, dg, S1);
            }
          }
          const float g_last = gp;
          E = Ec;
          float gn = gw[kc - 1];
#pragma unroll
          for (int s = kc - 1; s >= 1; --s) {
            E *= dn;
            dn *= P.gs.q;
            const float gs = gw[s - 1];
            const float dg = gn - gs;
            gn = gs;
            if (POSE) {
              Pd = fmaf(E, dg, Pd);
              if (s >= 2) Qd += Pd;
            } else {
              S1 = fmaf(E, dg, S1);
            }
          }
          if (POSE) {
            // upward sweep: j = s - kc in 0..S-2-kc; downward: j = kc - s in 1..kc-1, weight -j
            const float U = Pu + Pd;
            const float T = fmaf(static_cast<float>(S - 2 - kc), Pu, -Qu) - fmaf(static_cast<float>(kc - 1), Pd, -Qd);
            S1 += U;
            S2 = fmaf(bc, U, fmaf(P.h, T, last));
          }
          S1 = fmaf(P.gs.e_clamp, gn - g_last, S1);
          lam = P.lam;
        } else if constexpr (S >= 3) {
          // Sphere, b_s = beta_s^2 on the interior boundaries s = 1..n (n = S - 2,
          // beta_s = beta1 + (s - 1) h), b_{S-1} = min(beta_{S-1}, a0)^2, b_0 = b_S = a0^2.
          // Summation by parts turns the interior sums into three fixed combinations of
          // the window values, M_p = sum_s (s - 1)^p dg_s (p = 0, 1, 2):
          //   S1 = a0^2 (g_0 - g_{S-1}) + beta1^2 M0 + 2 h beta1 M1 + h^2 M2 + b_{S-1} dg_{S-1},
          //   S2 = -(beta1 M0 + h M1) - D dg_{S-1},  D = beta_{S-1} inside the support, else 0,
          // which costs about a third fewer instructions than a boundary-by-boundary sum.
          float g[S];
#pragma unroll
          for (int s = 0; s < S; ++s) g[s] = gw[s];
          constexpr int n = S - 2;
          const float M0 = g[n] - g[0];
          float M1 = static_cast<float>(n - 1) * g[n], M2 = static_cast<float>((n - 1) * (n - 1)) * g[n];
#pragma unroll
          for (int s = 1; s <= n - 1; ++s) {
            M1 -= g[s];
            M2 = fmaf(-static_cast<float>(2 * s - 1), g[s], M2);
          }
          const float dgl = g[S - 1] - g[n];
          const float b1 = m.beta1;
          const float bl = fmaf(static_cast<float>(S - 2), P.h, b1);  // beta_{S-1}
          const float tl = fminf(bl, P.supf);
          const float X = fmaf(P.h, M1, b1 * M0);  // sum of beta_s dg_s over the interior
          if (POSE) S2 = -fmaf(bl < P.supf ? bl : 0.f, dgl, X);
          const float Y = fmaf(P.h, M1, X);        // beta1 M0 + 2 h M1
          S1 = fmaf(b1, Y, fmaf(P.h * P.h, M2, fmaf(fmaf(tl, tl, -P.sup2), dgl, -P.sup2 * M0)));
          lam = 2.f;
        } else {  // S = 2: boundary 1 is the clamped one
          float g[S];
#pragma unroll
          for (int s = 0; s < S; ++s) g[s] = gw[s];
          float beta = m.beta1;
          S1 = P.sup2 * (g[0] - g[S - 1]);
#pragma unroll
          for (int s = 1; s < S; ++s) {
            if (s > 1) beta += P.h;
            const float dg = g[s] - g[s - 1];
            const float bc = (s == S - 1) ? fminf(beta, P.supf) : beta;
            S1 = fmaf(bc * bc, dg, S1);
            if (POSE) {
              const float D = (s == S - 1) ? (beta < P.supf ? beta : 0.f) : beta;
              S2 = fmaf(-D, dg, S2);
            }
          }
          lam = 2.f;
        }
        const float t1 = m.rs * S1;
        if (ADJ) bacc[k] += t1;
        if (POSE) {
          const float coef = p0s[k] * (m.rs * m.rs) * fmaf(lam, S2, -t1);
          R0 += coef;
          R1 = fmaf(coef, qx[k], R1);
        }
      }
      if (POSE) {
        // reduce-scatter: lanes 0-7 end with sum(R0), 8-15 sum(R1), 16-23 sum(qy R0), 24-31 sum(qz R0)
        const float R2 = qy * R0, R3 = qz * R0;
        const bool hi16 = lane & 16, hi8 = lane & 8;
        const float ka = hi16 ? R2 : R0, kb = hi16 ? R3 : R1;
        const float sa = hi16 ? R0 : R2, sb = hi16 ? R1 : R3;
        const float A2 = ka + __shfl_xor_sync(0xffffffffu, sa, 16);
        const float B2 = kb + __shfl_xor_sync(0xffffffffu, sb, 16);
        float Cv = (hi8 ? B2 : A2) + __shfl_xor_sync(0xffffffffu, hi8 ? A2 : B2, 8);
        Cv += __shfl_xor_sync(0xffffffffu, Cv, 4);
        Cv += __shfl_xor_sync(0xffffffffu, Cv, 2);
        Cv += __shfl_xor_sync(0xffffffffu, Cv, 1);
        if ((lane & 7) == 0) reinterpret_cast<float*>(&red[(buf * L::NW + warp) * kBatch + e])[lane >> 3] = Cv;
      }
    }
    if (ADJ) {  // fold the batch partial (<= 32 traces x S terms) into the voxel sum
#pragma unroll
      for (int k = 0; k < C; ++k) {
        acc[k] += bacc[k];
        bacc[k] = 0.f;
      }
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {  // let copies in flight land before the CTA exits
        mbar_wait_bounded(&bar[buf], (b >> 1) & 1, P.status);
        if (b + 1 < nb) mbar_wait_bounded(&bar[buf ^ 1], ((b + 1) >> 1) & 1, P.status);
      }
      return;
    }
    if (warp == b % L::NW) {
      if (POSE && lane < cnt) {
        double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
        for (int w = 0; w < L::NW; ++w) {
          const float4 v = red[(buf * L::NW + w) * kBatch + lane];
          r0 += v.x;
          r1 += v.y;
          r2 += v.z;
          r3 += v.w;
        }
        const float mk = refb[buf * kBatch + lane].w;
        const double* u = refu + (buf * kBatch + lane) * 3;
        double* gp = P.gpart + (static_cast<int64_t>(ib + b * kBatch + lane) * ncubes + c) * 3;
        gp[0] = mk * (u[0] * r0 - r1);
        gp[1] = mk * (u[1] * r0 - r2);
        gp[2] = mk * (u[2] * r0 - r3);
      }
      __syncwarp();
      if (b + 2 < nb) issue(b + 2, buf);
    }
  }
  if (seen > max_idx) atomicOr(P.status, PASFM_STATUS_INDEX_CLAMPED);

  if (ADJ && row_in) {
    // one part: straight into the volume; several: into this part's slice of vol_parts,
    // summed in part order by sum_parts_kernel
    const int64_t nvox = static_cast<int64_t>(P.nx) * P.ny * P.nz;
    float* out = (P.n_parts > 1 ? P.vol_parts + blockIdx.y * nvox : P.vol) +
                 (static_cast<int64_t>(iz) * P.ny + iy) * P.nx;
    const bool add = P.n_parts == 1 && P.accumulate;
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const int ix = cx * C + k;
      if (ix < P.nx) {
        const float v = acc[k] * P.scale;
        out[ix] = add ? out[ix] + v : v;
      }
    }
  }
}

}  // namespace pasfm
