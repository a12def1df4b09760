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
//                       writes S - 1 slots (its weights sum to zero; 3 <= S <= 8);
//                       the flush differences it into a per-cube partial trace and
//                       fwd_reduce_kernel sums the partials in a fixed order.
//                       Voxels go in pairs along a row, in packed FP32.
//   bwd_cube_kernel  -- adjoint v = A^T g and/or pose gradient.  Voxel-
//                       stationary: a thread owns a row of C voxels along x; the
//                       CTA walks all (frame, element) traces in batches of 32
//                       whose sample windows (for the sphere, of the traces'
//                       first differences) are staged by 2-D TMA loads into a
//                       double buffer.  The adjoint is an atomic-free gather; the
//                       pose gradient is reduced per element with warp shuffles
//                       and a fixed-order block reduction, then carried to FP64.
//                       The row's voxels go in pairs, in packed FP32.
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
// The callers pass A in units of the sample spacing, Ah = A / h (their per-row and
// per-trace terms are formed scaled), so that D2 = d_c^2 + h Ah and
// psi = phi_c + Ah / (d + d_c) each take one FMA: d - d_c = A / (d + d_c) without
// cancellation, and no separate division by h.
__device__ __forceinline__ PairMath pair_math(float Ah, float dc2, float dcf, float phim, float h, float cb1,
                                              int idx_bias) {
  PairMath m;
  const float D2 = fmaf(h, Ah, dc2);
  m.rs = rsqrtf(D2);
  const float psi = fmaf(Ah, __fdividef(1.f, fmaf(D2, m.rs, dcf)), phim);  // psi_c - N_c - 1/2 + delta / h
  const float t = psi + kMagic;                                             // round to nearest = floor(psi + 1/2)
  m.idx = static_cast<unsigned>(__float_as_int(t) - idx_bias);
  m.beta1 = fmaf((t - kMagic) - psi, h, cb1);                               // (n_s - psi_full) h - a0 + h
  return m;
}

// Two pairs at once (the same element against two neighbouring voxels of a row):
// Blackwell's packed FP32 instructions do two FMAs, adds or multiplies per lane in
// one issue slot, with the rounding of the scalar instruction.  The hot loops are
// bound by instruction issue, so every operation the two pairs share in form runs
// packed; the reciprocal square root, the reciprocal and the integer index stay
// scalar.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 min2(float2 a, float b) { return make_float2(fminf(a.x, b), fminf(a.y, b)); }

struct PairMath2 {
  float2 rs;
  unsigned idx0, idx1;
  float2 beta1;
};

__device__ __forceinline__ PairMath2 pair_math2(float2 Ah, float dc2, float dcf, float phim, float h, float cb1,
                                                int idx_bias) {
  PairMath2 m;
  const float2 D2 = fma2(f2(h), Ah, f2(dc2));
  m.rs = make_float2(rsqrtf(D2.x), rsqrtf(D2.y));
  const float2 den = fma2(D2, m.rs, f2(dcf));
  const float2 psi = fma2(Ah, make_float2(__fdividef(1.f, den.x), __fdividef(1.f, den.y)), f2(phim));
  const float2 t = add2(psi, f2(kMagic));
  m.idx0 = static_cast<unsigned>(__float_as_int(t.x) - idx_bias);
  m.idx1 = static_cast<unsigned>(__float_as_int(t.y) - idx_bias);
  m.beta1 = fma2(fma2(psi, f2(-1.f), add2(t, f2(-kMagic))), f2(h), f2(cb1));
  return m;
}

// The same with A itself (the backward): delta = A / (d + d_c) formed first, then
// psi = phi_c + delta / h.
__device__ __forceinline__ PairMath2 pair_math2_del(float2 A, float dc2, float dcf, float phim, float inv_h, float h,
                                                    float cb1, int idx_bias) {
  PairMath2 m;
  const float2 D2 = add2(f2(dc2), A);
  m.rs = make_float2(rsqrtf(D2.x), rsqrtf(D2.y));
  const float2 den = fma2(D2, m.rs, f2(dcf));
  const float2 del = mul2(A, make_float2(__fdividef(1.f, den.x), __fdividef(1.f, den.y)));
  const float2 psi = fma2(del, f2(inv_h), f2(phim));
  const float2 t = add2(psi, f2(kMagic));
  m.idx0 = static_cast<unsigned>(__float_as_int(t.x) - idx_bias);
  m.idx1 = static_cast<unsigned>(__float_as_int(t.y) - idx_bias);
  m.beta1 = fma2(fma2(psi, f2(-1.f), add2(t, f2(-kMagic))), f2(h), f2(cb1));
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

// gauss_boundaries for two pairs, packed
template <int S>
__device__ __forceinline__ void gauss_boundaries2(float2 beta1, float h, const GaussConst& G, float2 (&E)[S]) {
  constexpr int kc = gauss_centre<S>();
  const float2 bc = fma2(f2(static_cast<float>(kc - 1)), f2(h), beta1);
  const float2 eb = mul2(f2(G.c1), mul2(bc, bc));
  E[kc] = make_float2(exp2f(eb.x), exp2f(eb.y));
  const float2 ua = fma2(bc, f2(G.c2), f2(G.c3)), da = fma2(bc, f2(-G.c2), f2(G.c3));
  float2 up = make_float2(exp2f(ua.x), exp2f(ua.y));
  float2 dn = make_float2(exp2f(da.x), exp2f(da.y));
#pragma unroll
  for (int k = kc + 1; k < S; ++k) {
    E[k] = mul2(E[k - 1], up);
    up = mul2(up, f2(G.q));
  }
#pragma unroll
  for (int k = kc - 1; k >= 1; --k) {
    E[k] = mul2(E[k + 1], dn);
    dn = mul2(dn, f2(G.q));
  }
  E[S - 1] = make_float2(fmaxf(E[S - 1].x, G.e_clamp), fmaxf(E[S - 1].y, G.e_clamp));
}

// ------------------------------------------------------------------------
// forward
// ------------------------------------------------------------------------
// The forward window holds the running sum of the slot weights for 3 <= S <= 8 (one
// read-modify-write fewer per pair) and the weights themselves otherwise: at S = 2 the
// running sum would cancel worst, and for wider pulses the running sums (one-signed, so
// they add up over a dense volume while the trace they difference to cancels) carry a
// rounding error that grows with S: on 16^3 cubes of a dense volume 3.0e-6 relative L2
// at S = 4, 6.8e-6 at S = 11, 7.0-8.0e-6 at S = 12, 8.5e-6 at S = 16 and 1.2e-5 at
// S = 32 (the bound is 1e-5), against 0.7-0.9e-6 with the weights written directly.
__host__ __device__ constexpr bool fwd_running_sum(int S) { return S >= 3 && S <= 8; }

template <int C>
__host__ __device__ constexpr int fwd_tile_bytes() { return C * C * C * 4; }
template <int C>
__host__ __device__ constexpr int fwd_win_offset() {
  return ((fwd_tile_bytes<C>() + C * C + 16 + 127) / 128) * 128;
}

// Shared-memory layout of a forward CTA: the p0 tile, row flags, the staging barrier and
// the per-warp windows.
template <int C>
struct FwdSmem {
  float* tile;
  uint8_t* rowflag;
  uint64_t* bar;
  float* win;
  __device__ explicit FwdSmem(unsigned char* smem)
      : tile(reinterpret_cast<float*>(smem)),
        rowflag(smem + fwd_tile_bytes<C>()),
        bar(reinterpret_cast<uint64_t*>(smem + ((fwd_tile_bytes<C>() + C * C + 7) / 8) * 8)),
        win(reinterpret_cast<float*>(smem + fwd_win_offset<C>())) {}
};

// One forward tile: cube c (of ncubes) of frame fl of the launch's frame chunk against
// element group eg.  Q holds what every scan of a launch shares (pulse profile, sample
// slots, window length, wait bound); G the scan's own fields (grid, frames, arrays,
// status).  A single-scan launch passes its one parameter block for both.  The caller
// has initialised the staging barrier; `parity` is the phase this tile's copy completes.
// Returns false when that copy's wait ran out: the copy has landed and the CTA must exit.
template <int C, int S, int K>
__device__ __forceinline__ bool fwd_tile(const CUtensorMap* p0map, const FwdParams& Q, const FwdParams& G,
                                         const FwdSmem<C>& sm, int c, int ncubes, int fl, int eg, uint32_t parity) {
  float* tile = sm.tile;
  uint8_t* rowflag = sm.rowflag;
  uint64_t* bar = sm.bar;
  float* win = sm.win;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nwarps = blockDim.x >> 5;
  const int cx = c % G.ncx, cy = (c / G.ncx) % G.ncy, cz = c / (G.ncx * G.ncy);
  const int f = G.f_begin + fl;
  const int j = (eg * nwarps + warp) * kWarp + lane;
  const bool valid = j < G.E;
  const int jj = valid ? j : G.E - 1;

  // 1. stage the p0 cube (zero outside the grid)
  if (G.use_tma) {
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier tiles' reads of `tile`
      mbar_arrive_expect_tx(bar, fwd_tile_bytes<C>());
      tma_load_3d(tile, p0map, bar, cx * C, cy * C, cz * C);
    }
  } else {
    for (int k = tid; k < C * C * C; k += blockDim.x) {
      const int lx = k % C, ly = (k / C) % C, lz = k / (C * C);
      const int ix = cx * C + lx, iy = cy * C + ly, iz = cz * C + lz;
      float v = 0.f;
      if (ix < G.nx && iy < G.ny && iz < G.nz)
        v = load_elem(G.p0, (static_cast<int64_t>(iz) * G.ny + iy) * G.nx + ix, G.dtype_vol);
      tile[k] = v;
    }
  }

  // 2. zero this lane's window column
  float* col = win + warp * Q.W * kWarp + lane;
  for (int k = 0; k < Q.W; ++k) col[k * kWarp] = 0.f;

  // 3. per-(cube, element) reference in FP64
  const double* xp = G.xw + (static_cast<int64_t>(f) * G.E + jj) * 3;
  const double hc = 0.5 * (C - 1);
  const PairRef R = make_ref(xp[0], xp[1], xp[2], G.ox + G.dx * (cx * C + hc), G.oy + G.dy * (cy * C + hc),
                             G.oz + G.dz * (cz * C + hc), Q.sup, Q.tau0, Q.inv_h);
  const int nb_rel = static_cast<int>(floorf(R.phim - Q.nb_shift)) - 1;
  const float dxf = static_cast<float>(G.dx), dyf = static_cast<float>(G.dy), dzf = static_cast<float>(G.dz);
  // the x, y and z parts of A = |q|^2 - 2 q.u, in units of h
  float Pix[C];
#pragma unroll
  for (int ix = 0; ix < C; ++ix) {
    const float qx = (ix - 0.5f * (C - 1)) * dxf;
    Pix[ix] = (qx * Q.inv_hf) * (qx + R.m2ux);
  }
  float2 Pix2[C / 2];
#pragma unroll
  for (int i = 0; i < C / 2; ++i) Pix2[i] = make_float2(Pix[2 * i], Pix[2 * i + 1]);

  // 4. wait for the tile; flag rows that hold any nonzero voxel
  bool ok = true;
  if (G.use_tma) ok = mbar_wait_limited(bar, parity, G.status, Q.wait_cycles);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) mbar_wait_bounded(bar, parity, G.status);  // let the copy land before exit
    return false;
  }
  for (int r = tid; r < C * C; r += blockDim.x) {
    bool nz = false;
#pragma unroll
    for (int ix = 0; ix < C; ++ix) nz |= tile[r * C + ix] != 0.f;
    rowflag[r] = nz ? 1 : 0;
  }
  __syncthreads();

  // 5. pair loop: every voxel of the cube against this lane's element
  const unsigned max_idx = static_cast<unsigned>(Q.W - S);
  const int idx_bias = kMagicBits + nb_rel;
  // Clamp detection.  A voxel's distance to the element is convex along a row, and the
  // first slot index grows with the distance, so a row's largest index is at one of its
  // two ends: those are the only pairs checked.  (The window covers the cube's
  // distance range with half a sample to spare, so no index is clamped unless the
  // geometry is degenerate; the clamp itself is applied to every pair.)
  unsigned seen = 0;  // largest raw index at the row ends (a negative one wraps to a huge value)
  for (int lz = 0; lz < C; ++lz) {
    const float qz = (lz - 0.5f * (C - 1)) * dzf;
    const float Cz = (qz * Q.inv_hf) * (qz + R.m2uz);
    for (int ly = 0; ly < C; ++ly) {
      if (!rowflag[lz * C + ly]) continue;
      const float qy = (ly - 0.5f * (C - 1)) * dyf;
      const float Crow = fmaf(qy * Q.inv_hf, qy + R.m2uy, Cz);
      const float* prow = tile + (lz * C + ly) * C;
      // The pair's slot weights b_k - b_{k+1} (k = 0..S-1) sum to b_0 - b_S = 0, so for
      // 3 <= S <= 8 the window holds their running sum, negated: slot k gets
      // b_{k+1} - b_0 for k = 0..S-2 and slot S-1 gets nothing.  That is S - 1
      // read-modify-writes instead of S through shared memory, which bounds this loop;
      // the flush takes the first difference (wider pulses write the weights).  Sphere: b_0 = a0^2, b_k = beta_k^2 inside, the last boundary
      // clamped.  Gaussian: b = -E, b_0 = -E(edge).  Voxels go in pairs along the row
      // (packed arithmetic); their read-modify-writes stay in voxel order, since the two
      // windows may overlap.
      if constexpr (S >= 3) {
#pragma unroll
        for (int i4 = 0; i4 < C; i4 += 4) {
          const float4 pv4 = *reinterpret_cast<const float4*>(prow + i4);
#pragma unroll
          for (int u = 0; u < 4; u += 2) {
            const int i = i4 + u;
            const float2 pv = u == 0 ? make_float2(pv4.x, pv4.y) : make_float2(pv4.z, pv4.w);
            const PairMath2 m = pair_math2(add2(Pix2[i / 2], f2(Crow)), R.dc2, R.dcf, R.phim, Q.h, Q.cb1, idx_bias);
            if (i == 0) seen = max(seen, m.idx0);
            if (i + 1 == C - 1) seen = max(seen, m.idx1);
            float* sa = col + min(m.idx0, max_idx) * kWarp;
            float* sb = col + min(m.idx1, max_idx) * kWarp;
            const float2 s = mul2(pv, m.rs);
            if constexpr (!fwd_running_sum(S) && K == PASFM_KERNEL_GAUSS) {
              // the slot weights themselves, b_k - b_{k+1} = E_{k+1} - E_k (E_0 = E_S = edge)
              float2 E[S];
              gauss_boundaries2<S>(m.beta1, Q.h, Q.gs, E);
              float2 w[S];
              w[0] = add2(E[1], f2(-Q.gs.e_clamp));
#pragma unroll
              for (int k = 1; k <= S - 2; ++k) w[k] = fma2(E[k], f2(-1.f), E[k + 1]);
              w[S - 1] = fma2(E[S - 1], f2(-1.f), f2(Q.gs.e_clamp));
#pragma unroll
              for (int k = 0; k < S; ++k) sa[k * kWarp] = fmaf(s.x, w[k].x, sa[k * kWarp]);
#pragma unroll
              for (int k = 0; k < S; ++k) sb[k * kWarp] = fmaf(s.y, w[k].y, sb[k * kWarp]);
            } else {
              float2 c[S - 1];  // b_{k+1} - b_0
              if constexpr (K == PASFM_KERNEL_GAUSS) {
                float2 E[S];
                gauss_boundaries2<S>(m.beta1, Q.h, Q.gs, E);
#pragma unroll
                for (int k = 0; k <= S - 2; ++k) c[k] = fma2(E[k + 1], f2(-1.f), f2(Q.gs.e_clamp));
              } else {
                float2 beta = m.beta1;
#pragma unroll
                for (int k = 0; k <= S - 2; ++k) {
                  if (k > 0) beta = add2(beta, f2(Q.h));
                  const float2 bc = (k == S - 2) ? min2(beta, Q.supf) : beta;
                  c[k] = fma2(bc, bc, f2(-Q.sup2));
                }
              }
              if constexpr (fwd_running_sum(S)) {
#pragma unroll
                for (int k = 0; k <= S - 2; ++k) sa[k * kWarp] = fmaf(s.x, c[k].x, sa[k * kWarp]);
#pragma unroll
                for (int k = 0; k <= S - 2; ++k) sb[k * kWarp] = fmaf(s.y, c[k].y, sb[k * kWarp]);
              } else {
                // the slot weights themselves, b_k - b_{k+1}: -c_0, c_{k-1} - c_k, c_{S-2}
                float2 w[S];
                w[0] = fma2(c[0], f2(-1.f), f2(0.f));
#pragma unroll
                for (int k = 1; k <= S - 2; ++k) w[k] = fma2(c[k], f2(-1.f), c[k - 1]);
                w[S - 1] = c[S - 2];
#pragma unroll
                for (int k = 0; k < S; ++k) sa[k * kWarp] = fmaf(s.x, w[k].x, sa[k * kWarp]);
#pragma unroll
                for (int k = 0; k < S; ++k) sb[k * kWarp] = fmaf(s.y, w[k].y, sb[k * kWarp]);
              }
            }
          }
        }
      } else {
        // S = 2 (a pulse narrower than a sample): every pair is a +-w dipole on two
        // slots.  A running sum would hold two separately accumulated sums per sample
        // whose difference cancels in homogeneous regions, so the weights go in directly.
#pragma unroll
        for (int i = 0; i < C; ++i) {
          const PairMath m = pair_math(Pix[i] + Crow, R.dc2, R.dcf, R.phim, Q.h, Q.cb1, idx_bias);
          if (i == 0 || i == C - 1) seen = max(seen, m.idx);
          float* slot = col + min(m.idx, max_idx) * kWarp;
          const float s = prow[i] * m.rs;
          float w;
          if constexpr (K == PASFM_KERNEL_GAUSS) {
            float E[S];
            gauss_boundaries<S>(m.beta1, Q.h, Q.gs, E);
            w = E[1] - Q.gs.e_clamp;
          } else {
            const float bc = fminf(m.beta1, Q.supf);
            w = fmaf(-bc, bc, Q.sup2);
          }
          slot[0] = fmaf(s, w, slot[0]);
          slot[kWarp] = fmaf(-s, w, slot[kWarp]);
        }
      }
    }
  }
  if (seen > max_idx) atomicOr(G.status, PASFM_STATUS_INDEX_CLAMPED);

  // 6. flush the window (its first difference for S >= 3) as this cube's partial trace
  //    (scaled by 1 / (4 h), or sigma^2 / (2 h))
  __syncwarp();
  if (valid) {
    const int64_t row = static_cast<int64_t>(fl) * G.E + j;
    float* dst = G.part + (row * ncubes + c) * Q.W;
    float prev = 0.f;
    for (int k = 0; k < Q.W; k += 4) {
      const float c0 = col[(k + 0) * kWarp], c1 = col[(k + 1) * kWarp], c2 = col[(k + 2) * kWarp],
                  c3 = col[(k + 3) * kWarp];
      float4 v;
      if constexpr (fwd_running_sum(S)) {  // minus the running sum: T_k = W_{k-1} - W_k
        v.x = (prev - c0) * Q.p0_scale;
        v.y = (c0 - c1) * Q.p0_scale;
        v.z = (c1 - c2) * Q.p0_scale;
        v.w = (c2 - c3) * Q.p0_scale;
        prev = c3;
      } else {
        v = make_float4(c0 * Q.p0_scale, c1 * Q.p0_scale, c2 * Q.p0_scale, c3 * Q.p0_scale);
      }
      *reinterpret_cast<float4*>(dst + k) = v;
    }
    G.n0tab[row * ncubes + c] = R.Nc + nb_rel;
  }
  return true;
}


template <int C, int S, int K>
__global__ void __launch_bounds__(256, 2)
    fwd_cube_kernel(const __grid_constant__ CUtensorMap p0map, const FwdParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  const FwdSmem<C> sm(smem);
  if (threadIdx.x == 0) {
    mbar_init(sm.bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  fwd_tile<C, S, K>(&p0map, P, P, sm, blockIdx.x, gridDim.x, blockIdx.y, blockIdx.z, 0);
}

// Persistent forward over the tiles of several scans that share one instantiation and
// profile (one launch per serving iteration and group): CTAs take tiles from a global
// counter until the list is exhausted.  Scan s owns tiles [tiles[s], tiles[s + 1]), a
// tile being (cube, frame of the chunk, element group) with the cube fastest, exactly
// the block coordinates of its single-scan launch, so a scan's results do not depend on
// the other scans of the batch.
template <int C, int S, int K>
__global__ void __launch_bounds__(256, 2)
    fwd_batch_kernel(const __grid_constant__ TmaBatch maps, const __grid_constant__ FwdBatch B) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_tile;
  const FwdSmem<C> sm(smem);
  if (threadIdx.x == 0) {
    mbar_init(sm.bar, 1);
    fence_mbar_init();
  }
  uint32_t phase = 0;  // completed phases of the staging barrier
  const int total = B.tiles[B.n];
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(B.counter, 1);
    __syncthreads();  // also: the previous tile's shared memory is free
    const int t = s_tile;
    if (t >= total) break;
    int s = 0;
    while (t >= B.tiles[s + 1]) ++s;
    const FwdParams& G = B.G[s];
    const int local = t - B.tiles[s], nc = B.ncubes[s];
    const int c = local % nc, rest = local / nc;
    const unsigned long long t0 = B.trace ? globaltimer() : 0ull;
    if (!fwd_tile<C, S, K>(&maps.m[s], B.Q, G, sm, c, nc, rest % B.fc[s], rest / B.fc[s], phase & 1)) return;
    if (G.use_tma) ++phase;
    if (B.trace && threadIdx.x == 0) trace_tile(B.trace, s, t0);
    __syncthreads();  // every thread is past s_tile before thread 0 takes the next tile
  }
}

// ------------------------------------------------------------------------
// backward (adjoint gather + pose-gradient reduction)
// ------------------------------------------------------------------------

// The backward's slot sums for two voxels of a row against one trace window (ga, gb:
// each voxel's first slot), packed.  S1 = sum_s g_s (b_s - b_{s+1}) is the adjoint's;
// lam S2 is minus the boundary-motion term of dW/dd (lam turns the boundary offsets
// into derivatives of b and carries the sign, so that no operand needs negating).
// GWIN: the window may hold the traces themselves (P.diff == 0: the pose-gradient-only
// kernel of the allocation-free entry point); otherwise the sphere's windows always hold
// the first differences.
template <int S, int K, bool POSE, bool GWIN>
__device__ __forceinline__ void slot_sums2(const float* ga, const float* gb, float2 beta1, const BwdParams& P,
                                           float2& S1, float2& S2, float& lam) {
  if constexpr (K == PASFM_KERNEL_GAUSS) {
    constexpr int kc = gauss_centre<S>();
    const float2 bc = fma2(f2(static_cast<float>(kc - 1)), f2(P.h), beta1);
    const float2 eb = mul2(f2(P.gs.c1), mul2(bc, bc));
    const float2 Ec = make_float2(exp2f(eb.x), exp2f(eb.y));
    const float2 ua = fma2(bc, f2(P.gs.c2), f2(P.gs.c3)), da = fma2(bc, f2(-P.gs.c2), f2(P.gs.c3));
    float2 up = make_float2(exp2f(ua.x), exp2f(ua.y));
    float2 dn = make_float2(exp2f(da.x), exp2f(da.y));
    float2 E = Ec, gp = make_float2(ga[kc - 1], gb[kc - 1]);
    float2 Pu = f2(0.f), Qu = f2(0.f), Pd = f2(0.f), Qd = f2(0.f), last = f2(0.f);
    S1 = f2(0.f);
#pragma unroll
    for (int s = kc; s < S; ++s) {
      if (s > kc) {
        E = mul2(E, up);
        up = mul2(up, f2(P.gs.q));
      }
      const float2 gs = make_float2(ga[s], gb[s]);
      const float2 dg = fma2(gp, f2(-1.f), gs);
      gp = gs;
      if (s == S - 1) {
        const float2 Es = make_float2(fmaxf(E.x, P.gs.e_clamp), fmaxf(E.y, P.gs.e_clamp));
        S1 = fma2(Es, dg, S1);
        if (POSE) {
          const float2 beta = fma2(f2(static_cast<float>(s - 1)), f2(P.h), beta1);
          const float2 bed = mul2(mul2(beta, Es), dg);
          last = make_float2(beta.x < P.supf ? bed.x : 0.f, beta.y < P.supf ? bed.y : 0.f);
        }
      } else if (POSE) {
        Pu = fma2(E, dg, Pu);
        if (s < S - 2) Qu = add2(Qu, Pu);
      } else {
        S1 = fma2(E, dg, S1);
      }
    }
    const float2 g_last = gp;
    E = Ec;
    float2 gn = make_float2(ga[kc - 1], gb[kc - 1]);
#pragma unroll
    for (int s = kc - 1; s >= 1; --s) {
      E = mul2(E, dn);
      dn = mul2(dn, f2(P.gs.q));
      const float2 gs = make_float2(ga[s - 1], gb[s - 1]);
      const float2 dg = fma2(gs, f2(-1.f), gn);
      gn = gs;
      if (POSE) {
        Pd = fma2(E, dg, Pd);
        if (s >= 2) Qd = add2(Qd, Pd);
      } else {
        S1 = fma2(E, dg, S1);
      }
    }
    if (POSE) {
      const float2 U = add2(Pu, Pd);
      // T = (Ju Pu - Qu) - (Jd Pd - Qd)
      const float2 T = fma2(f2(static_cast<float>(S - 2 - kc)), Pu,
                            fma2(f2(-static_cast<float>(kc - 1)), Pd, fma2(Qu, f2(-1.f), Qd)));
      S1 = add2(S1, U);
      S2 = fma2(bc, U, fma2(f2(P.h), T, last));
    }
    S1 = fma2(f2(P.gs.e_clamp), fma2(g_last, f2(-1.f), gn), S1);
    lam = -P.lam;  // S2 carries its own sign
  } else if constexpr (S >= 3) {
    constexpr int n = S - 2;
    float2 M0, M1, M2, dgl;
    if (!GWIN || P.diff) {  // the window holds d_s = g_s - g_(s-1): M_p = sum_s (s - 1)^p d_s directly
      float2 d[S];
#pragma unroll
      for (int s = 1; s < S; ++s) d[s] = make_float2(ga[s], gb[s]);
      M0 = d[1];
      M1 = M2 = f2(0.f);
#pragma unroll
      for (int s = 2; s <= n; ++s) {
        M0 = add2(M0, d[s]);
        M1 = s == 2 ? d[2] : fma2(f2(static_cast<float>(s - 1)), d[s], M1);
        M2 = s == 2 ? d[2] : fma2(f2(static_cast<float>((s - 1) * (s - 1))), d[s], M2);
      }
      dgl = d[S - 1];
    } else {
      float2 g[S];
#pragma unroll
      for (int s = 0; s < S; ++s) g[s] = make_float2(ga[s], gb[s]);
      M0 = fma2(g[0], f2(-1.f), g[n]);
      M1 = g[n];
      M2 = g[n];
      if constexpr (n != 2) {
        M1 = mul2(f2(static_cast<float>(n - 1)), g[n]);
        M2 = mul2(f2(static_cast<float>((n - 1) * (n - 1))), g[n]);
      }
#pragma unroll
      for (int s = 1; s <= n - 1; ++s) {
        M1 = fma2(g[s], f2(-1.f), M1);
        M2 = fma2(f2(-static_cast<float>(2 * s - 1)), g[s], M2);
      }
      dgl = fma2(g[n], f2(-1.f), g[S - 1]);
    }
    const float2 bl = fma2(f2(static_cast<float>(S - 2)), f2(P.h), beta1);
    const float2 tl = min2(bl, P.supf);
    const float2 X = fma2(f2(P.h), M1, mul2(beta1, M0));
    if (POSE) {
      const float2 D = make_float2(bl.x < P.supf ? bl.x : 0.f, bl.y < P.supf ? bl.y : 0.f);
      S2 = fma2(D, dgl, X);  // minus the boundary-motion sum; lam carries the sign
    }
    const float2 Y = fma2(f2(P.h), M1, X);
    S1 = fma2(beta1, Y, fma2(f2(P.h * P.h), M2, fma2(fma2(tl, tl, f2(-P.sup2)), dgl, mul2(f2(-P.sup2), M0))));
    lam = 2.f;
  } else {  // S = 2, per voxel
    const float* gv[2] = {ga, gb};
    const float b1[2] = {beta1.x, beta1.y};
    float s1[2], s2[2];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const float d1 = (!GWIN || P.diff) ? gv[v][1] : gv[v][1] - gv[v][0];  // g_1 - g_0
      const float bc = fminf(b1[v], P.supf);
      s1[v] = fmaf(bc, bc, -P.sup2) * d1;
      s2[v] = POSE ? (b1[v] < P.supf ? b1[v] : 0.f) * d1 : 0.f;  // minus the sum
    }
    S1 = make_float2(s1[0], s1[1]);
    S2 = make_float2(s2[0], s2[1]);
    lam = 2.f;
  }
}

constexpr int kBatch = 32;  // traces staged per batch

// hi + lo += v with the rounding error of the addition kept (TwoSum: exact for any order of
// magnitudes, six FP32 additions)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (v - bp);
  hi = s;
  lo += err;
}

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
  __host__ __device__ static int pix_off(int WP) { return red_off(WP) + 2 * NW * kBatch * 16; }
  __host__ __device__ static int acc_off(int WP) { return pix_off(WP) + 2 * kBatch * C * 4; }
  __host__ __device__ static int bar_off(int WP) { return acc_off(WP) + NT * C * 4; }
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

// Resident CTAs per SM: three 16^3 CTAs (80 registers a thread; the adjoint's voxel sums
// live in shared memory), whose 24 warps hide the dependent chains better than two CTAs
// at 128 registers, at the price of a few spilled registers (measured 2% faster on the
// sphere, 4% on the Gaussian at S = 12); eight 8^3 CTAs.
// One backward tile: cube c (of ncubes) against part `part` of the (frame, element) items
// of the launch's frame chunk.  Q holds what every scan of a launch shares (pulse profile,
// slot count, staged window length, wait bound), G the scan's own fields; a single-scan
// launch passes its one parameter block for both.  The caller has initialised the two
// staging barriers; par0 / par1 are the phases their next completions carry.  Returns
// false when a staged-copy wait ran out: the copies in flight have landed and the CTA must
// exit.  On return every batch this tile staged has been waited for; *nbatches receives
// their count (batch b used buffer b & 1).
template <int C, int S, int K, bool ADJ, bool POSE>
__device__ __forceinline__ bool bwd_tile(const CUtensorMap* gmap, const BwdParams& Q, const BwdParams& G,
                                         unsigned char* smem, int c, int ncubes, int part, uint32_t par0,
                                         uint32_t par1, int* nbatches) {
  using L = BwdLayout<C>;
  const int WP = Q.WP;
  float* win = reinterpret_cast<float*>(smem);
  float4* refa = reinterpret_cast<float4*>(smem + L::refa_off(WP));
  float4* refb = reinterpret_cast<float4*>(smem + L::refb_off(WP));
  double* refu = reinterpret_cast<double*>(smem + L::refu_off(WP));
  float4* red = reinterpret_cast<float4*>(smem + L::red_off(WP));
  float2* pix = reinterpret_cast<float2*>(smem + L::pix_off(WP));
  float* accs = reinterpret_cast<float*>(smem + L::acc_off(WP));  // [voxel k][thread]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::bar_off(WP));

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cx = c % G.ncx, cy = (c / G.ncx) % G.ncy, cz = c / (G.ncx * G.ncy);
  int ty, tz;
  bwd_thread_row<C>(tid, ty, tz);
  const int iy = cy * C + ty, iz = cz * C + tz;
  const bool row_in = iy < G.ny && iz < G.nz;

  const float dxf = static_cast<float>(G.dx);
  const float qy = (ty - 0.5f * (C - 1)) * static_cast<float>(G.dy);
  const float qz = (tz - 0.5f * (C - 1)) * static_cast<float>(G.dz);

  // p0 along this thread's row, voxels (2k, 2k + 1)
  float2 p0s2[POSE ? C / 2 : 1];
  if (POSE) {
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const int ix = cx * C + k;
      const float v = (row_in && ix < G.nx)
                          ? load_elem(G.p0, (static_cast<int64_t>(iz) * G.ny + iy) * G.nx + ix, G.dtype_vol) * Q.scale
                          : 0.f;
      if (k % 2) {
        p0s2[k / 2].y = v;
      } else {
        p0s2[k / 2].x = v;
      }
    }
  }
  // adjoint: per-batch partial sums (<= 32 traces x S terms) folded once per batch
  float2 bacc[ADJ ? C / 2 : 1];
  if (ADJ) {
#pragma unroll
    for (int k = 0; k < C / 2; ++k) bacc[k] = f2(0.f);
#pragma unroll
    for (int k = 0; k < C; ++k) accs[k * L::NT + tid] = 0.f;
  }

  const double hc = 0.5 * (C - 1);
  const double rcx = G.ox + G.dx * (cx * C + hc), rcy = G.oy + G.dy * (cy * C + hc),
               rcz = G.oz + G.dz * (cz * C + hc);
  // this CTA's share of the (frame, element) items: [ib, ib + nl)
  const int ib = part * G.part_items;
  const int nl = max(0, min(G.n_items - ib, G.part_items));
  const int nb = (nl + kBatch - 1) / kBatch;
  *nbatches = nb;
  // phase of batch b's completion on its buffer b & 1
  auto parity = [&](int b) -> uint32_t { return ((b & 1 ? par1 : par0) + (b >> 1)) & 1u; };

  // producer: one warp stages batch b into buffer buf (lane l handles trace l)
  auto issue = [&](int b, int buf) {
    const int it = ib + b * kBatch + lane;
    const int cnt = min(kBatch, nl - b * kBatch);
    float* wdst = win + (buf * kBatch + lane) * WP;
    int x0 = 0, row = 0;
    if (it < ib + nl) {
      const int fl = it / G.E, j = it % G.E;
      const int f = G.f_begin + fl;
      row = f * G.E + j;
      const double* xp = G.xw + static_cast<int64_t>(row) * 3;
      const PairRef R = make_ref(xp[0], xp[1], xp[2], rcx, rcy, rcz, Q.sup, Q.tau0, Q.inv_h);
      const int n0 = R.Nc + static_cast<int>(floorf(R.phim - Q.nb_shift)) - 1;
      x0 = n0 & ~3;
      const float mk = (POSE && G.mask) ? (G.mask[row] ? 1.f : 0.f) : 1.f;
      refa[buf * kBatch + lane] = make_float4(R.m2ux, R.m2uy, R.m2uz, R.dc2);
      // the x part of A, q_x (q_x - 2 u_x), for the C voxels of a row: the same for every
      // row of the cube, so formed once per trace
      float2* pd = pix + (buf * kBatch + lane) * (C / 2);
#pragma unroll
      for (int k = 0; k < C / 2; ++k) {
        const float qa = (2 * k - 0.5f * (C - 1)) * dxf, qb = (2 * k + 1 - 0.5f * (C - 1)) * dxf;
        pd[k] = make_float2(qa * (qa + R.m2ux), qb * (qb + R.m2ux));
      }
      refb[buf * kBatch + lane] = make_float4(R.dcf, R.phim, __int_as_float(R.Nc - x0), mk);
      if (POSE) {
        refu[(buf * kBatch + lane) * 3 + 0] = R.ux;
        refu[(buf * kBatch + lane) * 3 + 1] = R.uy;
        refu[(buf * kBatch + lane) * 3 + 2] = R.uz;
      }
      if (!G.use_tma) {  // plain loads with zero fill outside [0, Nt)
        const int64_t base = static_cast<int64_t>(row) * G.Nt;
        for (int k = 0; k < WP; ++k) {
          const int n = x0 + k;
          wdst[k] = (n >= 0 && n < G.Nt) ? load_elem(G.g, base + n, G.dtype_sig) : 0.f;
        }
      }
    }
    if (G.use_tma) {
      __syncwarp();  // the warp's reference writes happen before lane 0's (releasing) arrival
      if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads of the buffer
        mbar_arrive_expect_tx(&bar[buf], static_cast<uint32_t>(cnt * WP * 4));
      }
      __syncwarp();
      if (it < ib + nl) tma_load_2d(wdst, gmap, &bar[buf], x0, row);
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
    const bool ok = mbar_wait_limited(&bar[buf], parity(b), G.status, Q.wait_cycles);
    const int cnt = min(kBatch, nl - b * kBatch);
    const float* wb = win + buf * kBatch * WP;
    for (int e = 0; ok && e < cnt; ++e) {
      const float4 ra = refa[buf * kBatch + e];
      const float4 rb = refb[buf * kBatch + e];
      const int idx_bias = kMagicBits - __float_as_int(rb.z);
      const float* wv = wb + e * WP;
      const float Crow = fmaf(qy, qy + ra.y, qz * (qz + ra.z));
      const float2* pe = pix + (buf * kBatch + e) * (C / 2);
      float2 R0v = f2(0.f), R1v = f2(0.f);
#pragma unroll
      for (int k2 = 0; k2 < C / 2; ++k2) {
        const int k = 2 * k2;
        const float2 A = add2(pe[k2], f2(Crow));
        const PairMath2 m = pair_math2_del(A, ra.w, rb.x, rb.y, Q.inv_hf, Q.h, Q.cb1, idx_bias);
        if (k == 0) seen = max(seen, m.idx0);
        if (k + 1 == C - 1) seen = max(seen, m.idx1);
        float2 S1, S2 = f2(0.f);
        float lam;
        slot_sums2<S, K, POSE, !ADJ>(wv + min(m.idx0, max_idx), wv + min(m.idx1, max_idx), m.beta1, Q, S1, S2, lam);
        const float2 t1 = mul2(m.rs, S1);
        if (ADJ) bacc[k2] = add2(bacc[k2], t1);
        if (POSE) {  // minus the coefficient: p0 (1/d^2) (t1 - dW/dd boundary term)
          const float2 cf = mul2(mul2(m.rs, m.rs), fma2(f2(lam), S2, t1));
          // sum p0 cf and sum p0 cf q_x; q_x = (voxel index - (C - 1) / 2) dx, so the second
          // takes compile-time offsets here and dx once per trace (no per-voxel p0 q_x array:
          // 16 registers fewer, spills down, -3% on the sphere backward)
          const float2 pc = mul2(p0s2[k2], cf);
          R0v = add2(R0v, pc);
          R1v = fma2(pc, make_float2(2 * k2 - 0.5f * (C - 1), 2 * k2 + 1 - 0.5f * (C - 1)), R1v);
        }
      }
      const float R0 = -(R0v.x + R0v.y), R1 = -(R1v.x + R1v.y) * dxf;
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
      for (int k = 0; k < C / 2; ++k) {
        accs[(2 * k) * L::NT + tid] += bacc[k].x;
        accs[(2 * k + 1) * L::NT + tid] += bacc[k].y;
        bacc[k] = f2(0.f);
      }
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {  // let copies in flight land before the CTA exits
        mbar_wait_bounded(&bar[buf], parity(b), G.status);
        if (b + 1 < nb) mbar_wait_bounded(&bar[buf ^ 1], parity(b + 1), G.status);
      }
      return false;
    }
    if (warp == b % L::NW) {
      if (POSE && lane < cnt) {
        // the warps' partial sums, added in warp order in compensated FP32 (Knuth's TwoSum
        // keeps each addition's rounding error in a second word): as exact as FP64 here and
        // far cheaper than B300's FP64 adds, which kept this rotating warp behind the others
        float4 hi = red[(buf * L::NW) * kBatch + lane], lo = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int w = 1; w < L::NW; ++w) {
          const float4 v = red[(buf * L::NW + w) * kBatch + lane];
          two_sum_acc(hi.x, lo.x, v.x);
          two_sum_acc(hi.y, lo.y, v.y);
          two_sum_acc(hi.z, lo.z, v.z);
          two_sum_acc(hi.w, lo.w, v.w);
        }
        const double r0 = double(hi.x) + lo.x, r1 = double(hi.y) + lo.y, r2 = double(hi.z) + lo.z,
                     r3 = double(hi.w) + lo.w;
        const float mk = refb[buf * kBatch + lane].w;
        const double* u = refu + (buf * kBatch + lane) * 3;
        double* gp = G.gpart + (static_cast<int64_t>(ib + b * kBatch + lane) * ncubes + c) * 3;
        gp[0] = mk * (u[0] * r0 - r1);
        gp[1] = mk * (u[1] * r0 - r2);
        gp[2] = mk * (u[2] * r0 - r3);
      }
      __syncwarp();
      if (b + 2 < nb) issue(b + 2, buf);
    }
  }
  if (seen > max_idx) atomicOr(G.status, PASFM_STATUS_INDEX_CLAMPED);

  if (ADJ && row_in) {
    // one part: straight into the volume; several: into this part's slice of vol_parts,
    // summed in part order by sum_parts_kernel
    const int64_t nvox = static_cast<int64_t>(G.nx) * G.ny * G.nz;
    float* out = (G.n_parts > 1 ? G.vol_parts + part * nvox : G.vol) +
                 (static_cast<int64_t>(iz) * G.ny + iy) * G.nx;
    const bool add = G.n_parts == 1 && G.accumulate;
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const int ix = cx * C + k;
      if (ix < G.nx) {
        const float v = accs[k * L::NT + tid] * Q.scale;
        out[ix] = add ? out[ix] + v : v;
      }
    }
  }
  return true;
}


template <int C, int S, int K, bool ADJ, bool POSE>
__global__ void __launch_bounds__(C* C, (C == 16 ? 3 : 8))
    bwd_cube_kernel(const __grid_constant__ CUtensorMap gmap, const BwdParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + BwdLayout<C>::bar_off(P.WP));
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  int nb;
  bwd_tile<C, S, K, ADJ, POSE>(&gmap, P, P, smem, blockIdx.x, gridDim.x, blockIdx.y, 0, 0, &nb);
}

// Persistent backward over the tiles of several scans sharing one instantiation and
// profile: a tile is (cube, part), the cube fastest, as the block coordinates of the
// scan's single-scan launch (the same part split), so its results do not depend on the
// batch.  The two staging barriers keep their phases across tiles.
template <int C, int S, int K, bool ADJ, bool POSE>
__global__ void __launch_bounds__(C* C, (C == 16 ? 3 : 8))
    bwd_batch_kernel(const __grid_constant__ TmaBatch maps, const __grid_constant__ BwdBatch B) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_tile;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + BwdLayout<C>::bar_off(B.Q.WP));
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  uint32_t par0 = 0, par1 = 0;
  const int total = B.tiles[B.n];
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(B.counter, 1);
    __syncthreads();  // also: the previous tile's shared memory is free
    const int t = s_tile;
    if (t >= total) break;
    int s = 0;
    while (t >= B.tiles[s + 1]) ++s;
    const int local = t - B.tiles[s], nc = B.ncubes[s];
    const unsigned long long t0 = B.trace ? globaltimer() : 0ull;
    int nb = 0;
    if (!bwd_tile<C, S, K, ADJ, POSE>(&maps.m[s], B.Q, B.G[s], smem, local % nc, nc, local / nc, par0, par1, &nb))
      return;
    par0 ^= ((nb + 1) >> 1) & 1u;  // batches 0, 2, 4, ... completed on buffer 0
    par1 ^= (nb >> 1) & 1u;
    if (B.trace && threadIdx.x == 0) trace_tile(B.trace, s, t0);
    __syncthreads();  // every thread is past s_tile before thread 0 takes the next tile
  }
}

}  // namespace pasfm
