// Device-side building blocks shared by the sm_103a kernels of the radiation
// operator: launch parameter blocks, mbarrier / TMA (cp.async.bulk.tensor)
// wrappers in inline PTX, bounded waits, and the per-(cube, element) reference
// quantities of the time-of-flight math.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pasfm.h"

namespace pasfm {

constexpr int kWarp = 32;
constexpr float kMagic = 12582912.0f;            // 1.5 * 2^23: x + kMagic rounds x to an integer
constexpr int kMagicBits = 0x4B400000;           // bit pattern of kMagic
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz: bound of every device wait

// ---------------------------------------------------------------------------
// Plan: how a geometry maps onto cubes of voxels and time windows (host-built).
// ---------------------------------------------------------------------------
struct Plan {
  int K;          // voxel pulse: PASFM_KERNEL_SPHERE or PASFM_KERNEL_GAUSS
  double sup;     // pulse support half-width in distance (mm): a0, or 4 sigma
  double sigma;   // Gaussian width (mm); 0 for the sphere
  int C;          // cube side in voxels (8 or 16)
  int S;          // sample slots per voxel-element pair: floor(2 sup / h) + 2
  int W;          // forward window length per element and cube (multiple of 4)
  int WP;         // backward staged window length (W + 4, a multiple of 32: 128-byte TMA rows)
  int ncx, ncy, ncz, ncubes;
  int fwd_warps;  // warps (32 elements each) per forward CTA
  int n_egroups;  // element groups of 32 * fwd_warps
  double h, inv_h, tau0, rho;
  float nb_shift; // rho / h: window base offset in samples
};

// Per-(cube, element) reference quantities, computed in FP64 and rounded.
//   u = x - r_c (element relative to the cube centre), d_c = |u|,
//   psi_c = (d_c - sup - tau0) / h + 1/2 = N_c + phi_c  (N_c integer; sup = the
//   pulse support half-width, a0 for the sphere and 4 sigma for the Gaussian).
// A voxel at r_c + q then has  A = |q|^2 - 2 q.u,  d = sqrt(d_c^2 + A),
// delta = d - d_c = A / (d + d_c), and its first touched sample is
// N_c + floor(phi_c + delta / h).  Only small quantities are kept in FP32.

// Constants of the Gaussian boundary values E(beta) = exp(-beta^2 / (2 sigma^2)),
// in base 2 for exp2f, and of their ratio recurrence on the sample grid.
struct GaussConst {
  float c1;       // -log2(e) / (2 sigma^2):        E(beta)           = 2^(c1 beta^2)
  float c2, c3;   // -log2(e) h / sigma^2, c1 h^2:  E(beta+h)/E(beta) = 2^(c2 beta + c3)
  float q;        // exp(-h^2 / sigma^2): ratio of consecutive such ratios
  float e_clamp;  // E at the support edge, exp(-8)
};

struct FwdParams {
  const double* xw;     // [F][E][3]
  const void* p0;       // [nz][ny][nx] of dtype_vol (fallback loads)
  float* part;          // [Fc][E][ncubes][W]
  int* n0tab;           // [Fc][E][ncubes] absolute sample index of window slot 0
  int dtype_vol;
  int nx, ny, nz;
  int ncx, ncy;
  int E, f_begin;
  int W;
  double ox, oy, oz, dx, dy, dz;
  double tau0, inv_h, sup;
  float h, supf, sup2, nb_shift, p0_scale, inv_hf, cb1;
  GaussConst gs;
  int use_tma;
  long long wait_cycles;  // bound of the first wait for each staged copy (SM clock cycles)
  unsigned* status;
};

struct TgvParams {
  const void* u;        // volume [nz][ny][nx] of dtype_u
  int dtype_u;
  const float* w;       // auxiliary field [3][nz][ny][nx]
  float* grad_u;        // [nz][ny][nx], overwritten or accumulated into
  int accumulate;
  float* grad_w;        // [3][nz][ny][nx], overwritten
  double* energy_part;  // one per CTA
  int nx, ny, nz;
  float inv_dx, inv_dy, inv_dz, alpha1, alpha0, eps2;
  int use_tma;
  long long wait_cycles;  // bound of the first wait for each staged copy (SM clock cycles)
  unsigned* status;
};

struct RedParams {
  const float* part;    // [Fc][E][ncubes][W]
  const int* n0tab;     // [Fc][E][ncubes]
  int E, f_begin, n_rows, ncubes, W, Nt;
  float* sig_out;       // [F][E][Nt] or null
  float* g_out;         // [F][E][Nt] residual or null
  const void* meas;     // [F][E][Nt] of dtype_sig or null
  int dtype_sig;
  const uint8_t* mask;  // [F][E] or null
  double* loss_part;    // per block, or null
  int loss_offset;      // block offset into loss_part (frame chunks)
};

struct BwdParams {
  const double* xw;     // [F][E][3]
  const void* p0;       // volume (POSE)
  const void* g;        // [F][E][Nt] of dtype_sig (fallback loads)
  const uint8_t* mask;  // [F][E] or null (POSE)
  float* vol;           // [nz][ny][nx] adjoint output (ADJ)
  float* vol_parts;     // [n_parts][nz][ny][nx] per-part adjoint sums when n_parts > 1 (ADJ)
  int n_parts;          // CTAs per cube (grid.y); each takes part_items consecutive items
  int part_items;       // multiple of the 32-item batch
  double* gpart;        // [Fc * E][ncubes][3] per-cube element gradients (POSE)
  int dtype_vol, dtype_sig;
  int nx, ny, nz, ncx, ncy;
  int E, f_begin, n_items, Nt;
  int WP, accumulate;   // accumulate: add into vol instead of overwriting
  double ox, oy, oz, dx, dy, dz;
  double tau0, inv_h, sup;
  float h, supf, sup2, nb_shift, scale, inv_hf, cb1;
  float lam;            // pose-coefficient weight of the boundary term: 2 (sphere), 1 / sigma^2 (Gaussian)
  GaussConst gs;
  int use_tma;
  int diff;             // sphere: the staged trace is the difference g_n - g_(n-1)
  long long wait_cycles;  // bound of the first wait for each staged copy (SM clock cycles)
  unsigned* status;
};

// ---------------------------------------------------------------------------
// Batched launches: several scans that share one kernel instantiation and pulse
// profile in one persistent launch (the serving loop's step over resident scans).
// The per-scan blocks travel as kernel parameters (constant bank, at most 32 KB).
// ---------------------------------------------------------------------------
constexpr int kMaxBatch = 16;  // scans per batched launch

struct TmaBatch {
  CUtensorMap m[kMaxBatch];  // each scan's staging map (p0 cubes, or trace windows)
};

struct FwdBatch {
  FwdParams Q;               // what the scans share: W, the pulse profile, sampling, wait bound
  FwdParams G[kMaxBatch];    // each scan's own grid, frames, arrays and status word
  int tiles[kMaxBatch + 1];  // scan s owns tiles [tiles[s], tiles[s + 1])
  int ncubes[kMaxBatch];     // cubes of scan s
  int fc[kMaxBatch];         // frames of scan s in this launch's chunk
  int n;                     // scans in the launch
  int* counter;              // next tile to take (zero before the launch)
  unsigned long long* trace; // [scan][2]: first tile start, last tile end (globaltimer ns), or null
};

struct BwdBatch {
  BwdParams Q;               // what the scans share: WP, the pulse profile, sampling, wait bound
  BwdParams G[kMaxBatch];    // each scan's own grid, items, arrays, part split and status word
  int tiles[kMaxBatch + 1];
  int ncubes[kMaxBatch];
  int n;
  int* counter;
  unsigned long long* trace;
};

// kernel parameters are limited to 32764 bytes
static_assert(sizeof(TmaBatch) + sizeof(FwdBatch) <= 32764, "batched forward parameters too large");
static_assert(sizeof(TmaBatch) + sizeof(BwdBatch) <= 32764, "batched backward parameters too large");

struct RedBatch {
  RedParams R[kMaxBatch];    // each scan's rows of this chunk (W shared)
  int blocks[kMaxBatch + 1]; // scan s owns row blocks [blocks[s], blocks[s + 1])
  int n;
};

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Widen scan s's [first start, last end] interval by one tile that started at t0.
__device__ __forceinline__ void trace_tile(unsigned long long* trace, int s, unsigned long long t0) {
  atomicMin(&trace[2 * s], t0);
  atomicMax(&trace[2 * s + 1], globaltimer());
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of `bar` for at most `limit` SM clock cycles; on expiry set
// the TIMEOUT status bit and return false (callers then skip the compute, let their
// copies in flight land with mbar_wait_bounded and exit).  A limit <= 0 reports the
// expiry at once without looking at the barrier: the host's wait-limit setting uses it
// to exercise that error path deterministically.
__device__ __forceinline__ bool mbar_wait_limited(uint64_t* bar, uint32_t parity, unsigned* status,
                                                  long long limit) {
  if (limit <= 0) {
    atomicOr(status, PASFM_STATUS_TIMEOUT);
    return false;
  }
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > limit) {
      atomicOr(status, PASFM_STATUS_TIMEOUT);
      return false;
    }
  }
}

// The same with the full bound kWaitCycles (~1 s): the drain of copies in flight
// before a CTA exits.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned* status) {
  return mbar_wait_limited(bar, parity, status, kWaitCycles);
}

// 2-D tiled TMA load (coordinates in elements, x innermost) completing on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y)
      : "memory");
}

// 3-D tiled TMA load.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                            int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// 4-D tiled TMA load.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                            int c) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z), "r"(c)
      : "memory");
}

__device__ __forceinline__ float load_elem(const void* p, int64_t i, int dtype) {
  if (dtype == PASFM_BF16) {
    const uint16_t v = static_cast<const uint16_t*>(p)[i];
    return __uint_as_float(static_cast<uint32_t>(v) << 16);
  }
  if (dtype == PASFM_F16) return __half2float(static_cast<const __half*>(p)[i]);
  return static_cast<const float*>(p)[i];
}

// Per-(cube, element) FP64 reference quantities, rounded to what the pair loop needs.
struct PairRef {
  float m2ux, m2uy, m2uz;  // -2 u
  float dc2;               // d_c^2
  float dcf;               // d_c
  float phim;              // phi_c - 1/2
  int Nc;                  // integer part of psi_c
  double ux, uy, uz;       // u in FP64 (pose-gradient epilogue)
};

__device__ __forceinline__ PairRef make_ref(double x0, double x1, double x2, double rcx, double rcy, double rcz,
                                            double sup, double tau0, double inv_h) {
  PairRef r;
  r.ux = x0 - rcx;
  r.uy = x1 - rcy;
  r.uz = x2 - rcz;
  const double dc2 = r.ux * r.ux + r.uy * r.uy + r.uz * r.uz;
  const double dc = sqrt(dc2);
  const double psi = (dc - sup - tau0) * inv_h + 0.5;
  const double N = floor(psi);
  r.Nc = static_cast<int>(N);
  r.phim = static_cast<float>(psi - N) - 0.5f;
  r.m2ux = static_cast<float>(-2.0 * r.ux);
  r.m2uy = static_cast<float>(-2.0 * r.uy);
  r.m2uz = static_cast<float>(-2.0 * r.uz);
  r.dc2 = static_cast<float>(dc2);
  r.dcf = static_cast<float>(dc);
  return r;
}

}  // namespace pasfm
