// Host side of libpasfm: the C ABI declared in include/pasfm.h.
//
// Planning (cube size, sample slots, window lengths, frame chunks), workspace
// ownership, TMA descriptor encoding, launch sequencing on the caller's stream,
// argument validation and per-launch CUDA-event timing.  Every compute step of
// the operator runs in the kernels of kernels.cuh / aux.cu; nothing here
// touches array contents on the host.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "aux.cuh"
#include "kernels.cuh"

using namespace pasfm;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) return fail(PASFM_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

#define TRY(expr)                  \
  do {                             \
    int r_ = (expr);               \
    if (r_ != PASFM_OK) return r_; \
  } while (0)

struct Buf {
  void* p = nullptr;
  size_t n = 0;
};

struct Rec {
  const char* name;
  cudaEvent_t a, b;
};

constexpr size_t kDefaultPartialBudget = size_t(4) << 30;
constexpr int kMaxParts = 8;  // backward CTAs per cube (item parts); bounds the per-part adjoint buffer
// length of a difference trace: samples 0..Nt (the last is minus g[Nt-1]), padded to 4 floats
inline int diff_len(int Nt) { return (Nt + 1 + 3) & ~3; }
constexpr int kFwdWmax16 = 128;  // forward window cap for 16^3 cubes (8 warps x W x 128 B)
constexpr int kFwdWmax8 = 200;   // forward window cap for 8^3 cubes

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

struct Geo {  // validated geometry with defaults applied
  pasfm_geom g;
  double a0;
  double sup;      // pulse support half-width (mm): a0, or 4 sigma for the Gaussian
  int64_t nvox;
  int64_t n_rows;  // F * E
};

constexpr double kGaussSupport = 4.0;  // Gaussian support half-width in sigmas (reading: unstated)

int check_geom(const pasfm_geom* g, Geo* out) {
  if (!g) return fail(PASFM_EINVAL, "geom is NULL");
  if (g->nx < 0 || g->ny < 0 || g->nz < 0 || g->n_elem < 0 || g->n_frames < 0 || g->n_samples < 0)
    return fail(PASFM_EINVAL, "negative size in geom");
  if (!(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0)) return fail(PASFM_EINVAL, "voxel spacing must be > 0");
  if (!(g->fs_mhz > 0) || !(g->c_mm_per_us > 0)) return fail(PASFM_EINVAL, "fs and c must be > 0");
  if (!std::isfinite(g->t0_us) || !std::isfinite(g->ox) || !std::isfinite(g->oy) || !std::isfinite(g->oz))
    return fail(PASFM_EINVAL, "non-finite origin or t0");
  for (int d : {g->dtype_vol, g->dtype_sig})
    if (d != PASFM_F32 && d != PASFM_BF16 && d != PASFM_F16) return fail(PASFM_EINVAL, "unknown dtype %d", d);
  if (g->kernel != PASFM_KERNEL_SPHERE && g->kernel != PASFM_KERNEL_GAUSS)
    return fail(PASFM_EINVAL, "unknown kernel %d", g->kernel);
  if (g->reserved != 0) return fail(PASFM_EINVAL, "geom.reserved must be 0");
  if (g->kernel == PASFM_KERNEL_GAUSS && !(g->sigma_mm > 0 && std::isfinite(g->sigma_mm)))
    return fail(PASFM_EINVAL, "the Gaussian kernel needs a finite sigma_mm > 0");
  out->g = *g;
  out->a0 = g->a0_mm > 0 ? g->a0_mm : 0.5 * std::min(g->dx, std::min(g->dy, g->dz));
  out->sup = g->kernel == PASFM_KERNEL_GAUSS ? kGaussSupport * g->sigma_mm : out->a0;
  out->nvox = int64_t(g->nx) * g->ny * g->nz;
  out->n_rows = int64_t(g->n_frames) * g->n_elem;
  if (out->n_rows > INT32_MAX / 2) return fail(PASFM_EUNSUPPORTED, "F * E too large");
  return PASFM_OK;
}

int make_plan(const Geo& G, Plan* pl) {
  const pasfm_geom& g = G.g;
  pl->h = g.c_mm_per_us / g.fs_mhz;
  pl->inv_h = 1.0 / pl->h;
  pl->tau0 = g.c_mm_per_us * g.t0_us;
  pl->K = g.kernel;
  pl->sup = G.sup;
  pl->sigma = g.kernel == PASFM_KERNEL_GAUSS ? g.sigma_mm : 0.0;
  const double L = 2.0 * G.sup / pl->h;
  pl->S = static_cast<int>(std::floor(L)) + 2;
  const int smax = g.kernel == PASFM_KERNEL_GAUSS ? kMaxSGauss : kMaxSSphere;
  if (pl->S > smax)
    return fail(PASFM_EUNSUPPORTED, "support / h = %.3f: a pair spans %d samples, more than the %d compiled",
                L / 2, pl->S, smax);
  const double diag = std::sqrt(g.dx * g.dx + g.dy * g.dy + g.dz * g.dz);
  auto window = [&](int C) {
    const double rho = 0.5 * (C - 1) * diag;
    int W = static_cast<int>(std::ceil(2.0 * rho / pl->h)) + pl->S + 3;
    return (W + 3) & ~3;
  };
  int C = 16, W = window(16);
  if (W > kFwdWmax16) {
    C = 8;
    W = window(8);
    if (W > kFwdWmax8)
      return fail(PASFM_EUNSUPPORTED, "voxel spacing %.3g mm spans too many samples (window %d)", diag, W);
  }
  pl->C = C;
  pl->W = W;
  pl->rho = 0.5 * (C - 1) * diag;
  pl->nb_shift = static_cast<float>(pl->rho / pl->h);
  // Each staged trace row is a TMA destination, which must start on a 128-byte boundary:
  // WP stays a multiple of 32 floats (W + 4 covers the window and its 4-aligned start).
  pl->WP = ((W + 4) + 31) & ~31;
  pl->ncx = (g.nx + C - 1) / C;
  pl->ncy = (g.ny + C - 1) / C;
  pl->ncz = (g.nz + C - 1) / C;
  pl->ncubes = pl->ncx * pl->ncy * pl->ncz;
  pl->fwd_warps = std::max(1, std::min(8, (g.n_elem + 31) / 32));
  pl->n_egroups = std::max(1, (g.n_elem + 32 * pl->fwd_warps - 1) / (32 * pl->fwd_warps));
  return PASFM_OK;
}

size_t fwd_per_frame(const Geo& G, const Plan& pl) {
  return size_t(G.g.n_elem) * pl.ncubes * (size_t(pl.W) * 4 + 4);
}
size_t bwd_per_frame(const Geo& G, const Plan& pl) { return size_t(G.g.n_elem) * pl.ncubes * 24; }

int frames_per_chunk(size_t per_frame, size_t budget, int F) {
  if (per_frame == 0) return std::max(F, 1);
  size_t k = budget / per_frame;
  if (k < 1) k = 1;
  return static_cast<int>(std::min<size_t>(k, std::max(F, 1)));
}

}  // namespace

struct pasfm_ctx {
  int device = 0;
  unsigned* status = nullptr;
  Buf xw, part, n0, gres, vgrad, gpart, G, grad6, lpart, lscalar, taps, vparts, gw, tpart, gdiff, bcount;
  int sms = 0;  // streaming multiprocessors of the device
  size_t budget = kDefaultPartialBudget;
  long long wait_cycles = kWaitCycles;  // bound of the kernels' first wait for each staged copy
  bool timing = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  int64_t launches = 0;

  int ensure(Buf& b, size_t bytes) {
    if (b.n >= bytes) return PASFM_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
    if (bytes == 0) return PASFM_OK;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return fail(PASFM_ENOMEM, "workspace allocation of %zu bytes failed", bytes);
    }
    b.n = bytes;
    return PASFM_OK;
  }
  cudaEvent_t event() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // begin/end bracket one kernel launch for timing and launch counting
  cudaEvent_t begin(cudaStream_t st) {
    ++launches;
    if (!timing) return nullptr;
    cudaEvent_t a = event();
    cudaEventRecord(a, st);
    return a;
  }
  void end(const char* name, cudaEvent_t a, cudaStream_t st) {
    if (!a) return;
    cudaEvent_t b = event();
    cudaEventRecord(b, st);
    recs.push_back({name, a, b});
  }
};

namespace {

int check_launch(const char* what) {
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(PASFM_ECUDA, "%s launch failed: %s", what, cudaGetErrorString(e));
  }
  return PASFM_OK;
}

int set_device(pasfm_ctx* ctx) {
  int cur = -1;
  CUDA_TRY(cudaGetDevice(&cur));
  if (cur != ctx->device) CUDA_TRY(cudaSetDevice(ctx->device));
  return PASFM_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Factor of the slot sums: W = kappa (b_k - b_{k+1}) / d with kappa = 1 / (4 h) for
// the sphere (b = beta^2) and sigma^2 / (2 h) for the Gaussian (b = -E).
double pulse_scale(const Plan& pl) {
  return pl.K == PASFM_KERNEL_GAUSS ? pl.sigma * pl.sigma / (2.0 * pl.h) : 0.25 / pl.h;
}

}  // namespace

namespace pasfm {

// Time-of-flight and pulse-profile fields shared by the forward and backward parameters.
template <class Params>
void set_profile(const Plan& pl, Params& P) {
  P.tau0 = pl.tau0;
  P.inv_h = pl.inv_h;
  P.sup = pl.sup;
  P.h = static_cast<float>(pl.h);
  P.supf = static_cast<float>(pl.sup);
  P.sup2 = P.supf * P.supf;
  P.nb_shift = pl.nb_shift;
  P.inv_hf = static_cast<float>(pl.inv_h);
  P.cb1 = static_cast<float>(-pl.sup + 0.5 * pl.h);
  P.gs = GaussConst{};
  if (pl.K == PASFM_KERNEL_GAUSS) {
    const double s2 = pl.sigma * pl.sigma, log2e = 1.4426950408889634;
    P.gs.c1 = static_cast<float>(-log2e / (2.0 * s2));
    P.gs.c2 = static_cast<float>(-log2e * pl.h / s2);
    P.gs.c3 = static_cast<float>(-log2e * pl.h * pl.h / (2.0 * s2));
    P.gs.q = static_cast<float>(std::exp(-pl.h * pl.h / s2));
    P.gs.e_clamp = static_cast<float>(std::exp(-pl.sup * pl.sup / (2.0 * s2)));
  }
}

// Profile fields of the backward parameters, including the sign-folded scale
// (the Gaussian slot sums run over +E, i.e. -b) and the pose-term weight.
void set_bwd_profile(const Plan& pl, BwdParams* P) {
  set_profile(pl, *P);
  const double k = pulse_scale(pl);
  P->scale = static_cast<float>(pl.K == PASFM_KERNEL_GAUSS ? -k : k);
  P->lam = static_cast<float>(pl.K == PASFM_KERNEL_GAUSS ? 1.0 / (pl.sigma * pl.sigma) : 2.0);
}

}  // namespace pasfm

namespace {

// CTAs per cube for the backward: the item list of every cube is split into
// `parts` runs (whole 32-item batches) so that ncubes * parts CTAs fill the
// resident slots in whole waves.  A last partial wave leaves SMs idle (512
// cubes on 296 slots use 86% of them); the split is taken when it gains more
// than 1% and every part keeps at least 4 batches.
int choose_parts(int ncubes, int n_items, int slots) {
  if (slots <= 0 || ncubes <= 0) return 1;
  auto eff = [&](int p) {
    const int64_t ctas = int64_t(ncubes) * p;
    const int64_t waves = (ctas + slots - 1) / slots;
    return double(ctas) / double(waves * slots);
  };
  int best = 1;
  double best_eff = eff(1);
  for (int p = 2; p <= kMaxParts; ++p) {
    const int per = ((n_items + p - 1) / p + 31) / 32 * 32;
    if (per < 4 * 32 || int64_t(per) * (p - 1) >= n_items) break;
    const double e = eff(p);
    if (e > best_eff + 0.01) {
      best = p;
      best_eff = e;
    }
  }
  return best;
}

// A1: element positions into `out`.
int run_elem_pos(pasfm_ctx* ctx, const Geo& G, const double* elem, const double* pose, double* out,
                 cudaStream_t st) {
  const pasfm_geom& g = G.g;
  const int64_t n = G.n_rows;
  if (n == 0) return PASFM_OK;
  const double lox = g.ox, loy = g.oy, loz = g.oz;
  const double hix = g.ox + g.dx * std::max(g.nx - 1, 0), hiy = g.oy + g.dy * std::max(g.ny - 1, 0),
               hiz = g.oz + g.dz * std::max(g.nz - 1, 0);
  // an empty grid has no voxel an element could be inside
  const double supchk = G.nvox > 0 ? G.sup : -1.0;
  cudaEvent_t t = ctx->begin(st);
  elem_pos_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(
      elem, pose, out, g.n_frames, g.n_elem, lox, loy, loz, hix, hiy, hiz, supchk, ctx->status);
  ctx->end("elem_pos", t, st);
  return check_launch("elem_pos");
}

// Forward parameter block and p0 staging map of one scan (every field but f_begin), and
// its partial-result workspace for frame chunks of Fc frames.
int fwd_setup(pasfm_ctx* ctx, const Geo& G, const Plan& pl, const void* p0, const double* xw, int Fc, FwdParams* out,
              CUtensorMap* map) {
  const pasfm_geom& g = G.g;
  TRY(ctx->ensure(ctx->part, size_t(Fc) * g.n_elem * pl.ncubes * pl.W * 4));
  TRY(ctx->ensure(ctx->n0, size_t(Fc) * g.n_elem * pl.ncubes * 4));
  std::memset(map, 0, sizeof *map);
  int use_tma = 0;
  auto enc = encode_fn();
  if (enc && g.dtype_vol == PASFM_F32 && g.nx % 4 == 0 && aligned16(p0)) {
    cuuint64_t dims[3] = {cuuint64_t(g.nx), cuuint64_t(g.ny), cuuint64_t(g.nz)};
    cuuint64_t strides[2] = {cuuint64_t(g.nx) * 4, cuuint64_t(g.nx) * g.ny * 4};
    cuuint32_t box[3] = {cuuint32_t(pl.C), cuuint32_t(pl.C), cuuint32_t(pl.C)};
    cuuint32_t es[3] = {1, 1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(p0), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
      use_tma = 1;
  }
  FwdParams P{};
  P.xw = xw;
  P.p0 = p0;
  P.part = static_cast<float*>(ctx->part.p);
  P.n0tab = static_cast<int*>(ctx->n0.p);
  P.dtype_vol = g.dtype_vol;
  P.nx = g.nx;
  P.ny = g.ny;
  P.nz = g.nz;
  P.ncx = pl.ncx;
  P.ncy = pl.ncy;
  P.E = g.n_elem;
  P.W = pl.W;
  P.ox = g.ox;
  P.oy = g.oy;
  P.oz = g.oz;
  P.dx = g.dx;
  P.dy = g.dy;
  P.dz = g.dz;
  set_profile(pl, P);
  P.p0_scale = static_cast<float>(pulse_scale(pl));
  P.use_tma = use_tma;
  P.wait_cycles = ctx->wait_cycles;
  P.status = ctx->status;
  *out = P;
  return PASFM_OK;
}

size_t fwd_smem(const Plan& pl) {
  return size_t(pl.C == 16 ? fwd_win_offset<16>() : fwd_win_offset<8>()) + size_t(pl.fwd_warps) * pl.W * 32 * 4;
}

// Reduction of one frame chunk [fb, fb + fc) of a scan's forward partials.
RedParams red_params(const FwdParams& P, const Geo& G, const Plan& pl, int fb, int fc, float* sig_out, float* g_out,
                     const void* meas, const uint8_t* mask, double* loss_part, int loss_off) {
  RedParams R{};
  R.part = P.part;
  R.n0tab = P.n0tab;
  R.E = G.g.n_elem;
  R.f_begin = fb;
  R.n_rows = fc * G.g.n_elem;
  R.ncubes = pl.ncubes;
  R.W = pl.W;
  R.Nt = G.g.n_samples;
  R.sig_out = sig_out;
  R.g_out = g_out;
  R.meas = meas;
  R.dtype_sig = G.g.dtype_sig;
  R.mask = mask;
  R.loss_part = loss_part;
  R.loss_offset = loss_off;
  return R;
}

// Forward over all frames: per-cube kernels then the ordered reduction.
// Writes sig_out (may be null) and/or the masked residual g_out with loss.
int run_forward(pasfm_ctx* ctx, const Geo& G, const Plan& pl, const void* p0, const double* xw, float* sig_out,
                float* g_out, const void* meas, const uint8_t* mask, double* loss_out, cudaStream_t st) {
  const pasfm_geom& g = G.g;
  const int F = g.n_frames;
  const int Fc = frames_per_chunk(fwd_per_frame(G, pl), ctx->budget, F);
  const int n_chunks = (F + Fc - 1) / Fc;
  const int blocks_total = static_cast<int>((G.n_rows + 7) / 8) + n_chunks;
  if (g_out) {
    TRY(ctx->ensure(ctx->lpart, size_t(blocks_total) * 8));
    TRY(ctx->ensure(ctx->lscalar, 8));
  }
  FwdParams P;
  CUtensorMap map;
  TRY(fwd_setup(ctx, G, pl, p0, xw, Fc, &P, &map));

  const int threads = 32 * pl.fwd_warps;
  const size_t smem = fwd_smem(pl);
  int loss_off = 0;
  for (int fb = 0; fb < F; fb += Fc) {
    const int fc = std::min(Fc, F - fb);
    P.f_begin = fb;
    dim3 grid(pl.ncubes, fc, pl.n_egroups);
    cudaEvent_t t = ctx->begin(st);
    cudaError_t e = fwd_launcher(pl.K, pl.S)(pl.C, map, P, grid, threads, smem, st);
    ctx->end("fwd_cube", t, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PASFM_ECUDA, "fwd_cube launch: %s", cudaGetErrorString(e));
    }

    const RedParams R = red_params(P, G, pl, fb, fc, sig_out, g_out, meas, mask,
                                   g_out ? static_cast<double*>(ctx->lpart.p) : nullptr, loss_off);
    const int rblocks = (R.n_rows + 7) / 8;
    t = ctx->begin(st);
    const cudaError_t re = fwd_reduce_launch(R, rblocks, st);
    ctx->end("fwd_reduce", t, st);
    if (re != cudaSuccess) return fail(PASFM_ECUDA, "fwd_reduce launch: %s", cudaGetErrorString(re));
    loss_off += rblocks;
  }
  if (g_out) {
    double* dst = loss_out ? loss_out : static_cast<double*>(ctx->lscalar.p);
    cudaEvent_t t = ctx->begin(st);
    sum_kernel<<<1, 256, 0, st>>>(static_cast<double*>(ctx->lpart.p), loss_off, dst);
    ctx->end("loss_sum", t, st);
    TRY(check_launch("loss_sum"));
  }
  return PASFM_OK;
}

// Backward parameter block and trace staging map of one scan (every field but the frame
// chunk's f_begin, n_items, accumulate and part split), with the workspace it needs for
// frame chunks of Fc frames.  For the sphere the kernel reads the traces' first
// differences (its slot sums need only those), formed here into the workspace.
int bwd_setup(pasfm_ctx* ctx, const Geo& G, const Plan& pl, int mode, const void* p0, const double* xw,
              const void* gsig_in, int dtype_in, const uint8_t* mask, float* vol, int Fc, BwdParams* out,
              CUtensorMap* map, cudaStream_t st) {
  const pasfm_geom& g = G.g;
  const bool diff = pl.K == PASFM_KERNEL_SPHERE;
  const void* gsig = gsig_in;
  int dtype_sig = dtype_in, Nt = g.n_samples;
  if (diff && G.n_rows > 0) {
    const int Ntd = diff_len(g.n_samples);
    TRY(ctx->ensure(ctx->gdiff, size_t(G.n_rows) * Ntd * 4));
    const int64_t total = G.n_rows * int64_t(Ntd);
    cudaEvent_t t = ctx->begin(st);
    diff_rows_kernel<<<static_cast<unsigned>(std::min<int64_t>((total + 255) / 256, 148 * 32)), 256, 0, st>>>(
        gsig_in, dtype_in, G.n_rows, g.n_samples, Ntd, static_cast<float*>(ctx->gdiff.p));
    ctx->end("diff_rows", t, st);
    TRY(check_launch("diff_rows"));
    gsig = ctx->gdiff.p;
    dtype_sig = PASFM_F32;
    Nt = Ntd;
  }
  if (mode & 2) TRY(ctx->ensure(ctx->gpart, size_t(Fc) * g.n_elem * pl.ncubes * 24));
  if (mode & 1) TRY(ctx->ensure(ctx->vparts, size_t(G.nvox) * 4 * kMaxParts));

  std::memset(map, 0, sizeof *map);
  int use_tma = 0;
  auto enc = encode_fn();
  if (enc && dtype_sig == PASFM_F32 && Nt % 4 == 0 && aligned16(gsig) && pl.WP <= 256) {
    cuuint64_t dims[2] = {cuuint64_t(Nt), cuuint64_t(G.n_rows)};
    cuuint64_t strides[1] = {cuuint64_t(Nt) * 4};
    cuuint32_t box[2] = {cuuint32_t(pl.WP), 1};
    cuuint32_t es[2] = {1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(gsig), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
      use_tma = 1;
  }

  BwdParams P{};
  P.xw = xw;
  P.p0 = p0;
  P.g = gsig;
  P.mask = mask;
  P.vol = vol;
  P.vol_parts = static_cast<float*>(ctx->vparts.p);
  P.gpart = static_cast<double*>(ctx->gpart.p);
  P.dtype_vol = g.dtype_vol;
  P.dtype_sig = dtype_sig;
  P.nx = g.nx;
  P.ny = g.ny;
  P.nz = g.nz;
  P.ncx = pl.ncx;
  P.ncy = pl.ncy;
  P.E = g.n_elem;
  P.Nt = Nt;
  P.WP = pl.WP;
  P.ox = g.ox;
  P.oy = g.oy;
  P.oz = g.oz;
  P.dx = g.dx;
  P.dy = g.dy;
  P.dz = g.dz;
  set_bwd_profile(pl, &P);
  P.use_tma = use_tma;
  P.diff = diff ? 1 : 0;
  P.wait_cycles = ctx->wait_cycles;
  P.status = ctx->status;
  *out = P;
  return PASFM_OK;
}

size_t bwd_smem(const Plan& pl) { return pl.C == 16 ? BwdLayout<16>::total(pl.WP) : BwdLayout<8>::total(pl.WP); }

// Frame chunk [fb, fb + fc) of a backward: items, accumulation and the split of every
// cube's items into parts (per_sm: resident CTAs of the single-scan kernel per SM).
void bwd_chunk(pasfm_ctx* ctx, const Plan& pl, int E, int fb, int fc, int per_sm, BwdParams* P) {
  P->f_begin = fb;
  P->n_items = fc * E;
  P->accumulate = fb > 0;
  P->n_parts = choose_parts(pl.ncubes, P->n_items, per_sm * ctx->sms);
  P->part_items = P->n_parts > 1 ? ((P->n_items + P->n_parts - 1) / P->n_parts + 31) / 32 * 32 : P->n_items;
}

// Backward: mode 1 adjoint into vol, 2 pose gradient into G rows, 3 both.
int run_backward(pasfm_ctx* ctx, const Geo& G, const Plan& pl, int mode, const void* p0, const double* xw,
                 const void* gsig_in, int dtype_in, const uint8_t* mask, float* vol, double* Gout,
                 cudaStream_t st) {
  const pasfm_geom& g = G.g;
  const int F = g.n_frames, E = g.n_elem;
  const bool pose = mode & 2;
  const int Fc = pose ? frames_per_chunk(bwd_per_frame(G, pl), ctx->budget, F) : std::max(F, 1);
  BwdParams P;
  CUtensorMap map;
  TRY(bwd_setup(ctx, G, pl, mode, p0, xw, gsig_in, dtype_in, mask, vol, Fc, &P, &map, st));
  const size_t smem = bwd_smem(pl);
  const int per_sm = bwd_occupancy(pl.K, pl.S)(pl.C, mode, smem);
  const bool adj = mode & 1;

  for (int fb = 0; fb < F; fb += Fc) {
    const int fc = std::min(Fc, F - fb);
    bwd_chunk(ctx, pl, E, fb, fc, per_sm, &P);
    cudaEvent_t t = ctx->begin(st);
    cudaError_t e = bwd_launcher(pl.K, pl.S)(pl.C, mode, map, P, dim3(pl.ncubes, P.n_parts), smem, st);
    ctx->end("bwd_cube", t, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PASFM_ECUDA, "bwd_cube launch: %s", cudaGetErrorString(e));
    }
    if (adj && P.n_parts > 1) {
      const int64_t nv = G.nvox;
      const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((nv + 255) / 256, 148 * 16));
      t = ctx->begin(st);
      sum_parts_kernel<<<blocks, 256, 0, st>>>(P.vol_parts, P.n_parts, nv, vol, P.accumulate);
      ctx->end("sum_parts", t, st);
      TRY(check_launch("sum_parts"));
    }
    if (pose) {
      const int rows = fc * E;
      t = ctx->begin(st);
      pose_rows_kernel<<<(rows + 7) / 8, 256, 0, st>>>(P.gpart, pl.ncubes, rows, int64_t(fb) * E, Gout);
      ctx->end("pose_rows", t, st);
      TRY(check_launch("pose_rows"));
    }
  }
  return PASFM_OK;
}

// F3: TGV energy and gradients (tgv.cu).  energy_out may be null.
int run_tgv(pasfm_ctx* ctx, const Geo& G, const void* p0, const float* w, double alpha1, double alpha0, double eps,
            float* grad_u, int accumulate, float* grad_w, double* energy_out, cudaStream_t st) {
  const pasfm_geom& g = G.g;
  const int tiles = tgv_tiles(g.nx, g.ny, g.nz);
  const dim3 grid = tgv_grid(g.nx, g.ny, g.nz);
  const size_t smem = tgv_smem_bytes();
  CUDA_TRY(cudaFuncSetAttribute(tgv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  TRY(ctx->ensure(ctx->tpart, size_t(tiles) * 8));
  CUtensorMap umap, wmap, gmap;
  std::memset(&umap, 0, sizeof umap);
  std::memset(&wmap, 0, sizeof wmap);
  std::memset(&gmap, 0, sizeof gmap);
  int use_tma = 0;
  auto enc = encode_fn();
  if (enc && g.dtype_vol == PASFM_F32 && g.nx % 4 == 0 && aligned16(p0) && aligned16(w) && aligned16(grad_u)) {
    unsigned b3[3], b4[4], bg[3];
    tgv_boxes(b3, b4, bg);
    cuuint64_t d3[3] = {cuuint64_t(g.nx), cuuint64_t(g.ny), cuuint64_t(g.nz)};
    cuuint64_t s3[2] = {cuuint64_t(g.nx) * 4, cuuint64_t(g.nx) * g.ny * 4};
    cuuint32_t bx3[3] = {b3[0], b3[1], b3[2]};
    cuuint32_t bxg[3] = {bg[0], bg[1], bg[2]};
    cuuint64_t d4[4] = {cuuint64_t(g.nx), cuuint64_t(g.ny), cuuint64_t(g.nz), 3};
    cuuint64_t s4[3] = {cuuint64_t(g.nx) * 4, cuuint64_t(g.nx) * g.ny * 4, cuuint64_t(G.nvox) * 4};
    cuuint32_t bx4[4] = {b4[0], b4[1], b4[2], b4[3]};
    cuuint32_t es[4] = {1, 1, 1, 1};
    auto mk = [&](CUtensorMap* m, int rank, void* base, cuuint64_t* dims, cuuint64_t* strides, cuuint32_t* box) {
      return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, base, dims, strides, box, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    if (mk(&umap, 3, const_cast<void*>(p0), d3, s3, bx3) && mk(&wmap, 4, const_cast<float*>(w), d4, s4, bx4) &&
        mk(&gmap, 3, grad_u, d3, s3, bxg))
      use_tma = 1;
  }
  TgvParams P{};
  P.u = p0;
  P.dtype_u = g.dtype_vol;
  P.w = w;
  P.grad_u = grad_u;
  P.accumulate = accumulate;
  P.grad_w = grad_w;
  P.energy_part = static_cast<double*>(ctx->tpart.p);
  P.nx = g.nx;
  P.ny = g.ny;
  P.nz = g.nz;
  P.inv_dx = static_cast<float>(1.0 / g.dx);
  P.inv_dy = static_cast<float>(1.0 / g.dy);
  P.inv_dz = static_cast<float>(1.0 / g.dz);
  P.alpha1 = static_cast<float>(alpha1);
  P.alpha0 = static_cast<float>(alpha0);
  P.eps2 = static_cast<float>(eps * eps);
  P.use_tma = use_tma;
  P.wait_cycles = ctx->wait_cycles;
  P.status = ctx->status;
  cudaEvent_t t = ctx->begin(st);
  tgv_kernel<<<grid, tgv_threads(), smem, st>>>(umap, wmap, gmap, P);
  ctx->end("tgv", t, st);
  TRY(check_launch("tgv"));
  if (energy_out) {
    t = ctx->begin(st);
    sum_kernel<<<1, 256, 0, st>>>(P.energy_part, tiles, energy_out);
    ctx->end("tgv_sum", t, st);
    TRY(check_launch("tgv_sum"));
  }
  return PASFM_OK;
}

int run_grad6(pasfm_ctx* ctx, const Geo& G, const double* xw, const double* Gm, double* grad6, cudaStream_t st) {
  if (G.g.n_frames == 0) return PASFM_OK;
  cudaEvent_t t = ctx->begin(st);
  grad6_kernel<<<G.g.n_frames, 256, 0, st>>>(xw, Gm, G.g.n_elem, grad6);
  ctx->end("grad6", t, st);
  return check_launch("grad6");
}

// ---------------------------------------------------------------------------
// Batched gradient step over several scans (pasfm_step_batch)
// ---------------------------------------------------------------------------
int prepare(pasfm_ctx* ctx, const pasfm_geom* geom, Geo* G, Plan* pl);

// Fields of the forward parameters that every scan of one batched launch must share.
bool same_fwd_profile(const FwdParams& a, const FwdParams& b) {
  return a.W == b.W && a.tau0 == b.tau0 && a.inv_h == b.inv_h && a.sup == b.sup && a.h == b.h &&
         a.supf == b.supf && a.sup2 == b.sup2 && a.nb_shift == b.nb_shift && a.p0_scale == b.p0_scale &&
         a.inv_hf == b.inv_hf && a.cb1 == b.cb1 && std::memcmp(&a.gs, &b.gs, sizeof a.gs) == 0 &&
         a.wait_cycles == b.wait_cycles;
}

bool same_bwd_profile(const BwdParams& a, const BwdParams& b) {
  return a.WP == b.WP && a.tau0 == b.tau0 && a.inv_h == b.inv_h && a.sup == b.sup && a.h == b.h &&
         a.supf == b.supf && a.sup2 == b.sup2 && a.nb_shift == b.nb_shift && a.scale == b.scale &&
         a.inv_hf == b.inv_hf && a.cb1 == b.cb1 && a.lam == b.lam && a.diff == b.diff &&
         std::memcmp(&a.gs, &b.gs, sizeof a.gs) == 0 && a.wait_cycles == b.wait_cycles;
}

struct BatchScan {  // one scan of a batched step
  pasfm_ctx* ctx;
  Geo G;
  Plan pl;
  pasfm_adam* state;
  void* p0;
  double* pose;
  double* loss_out;
  int mode;             // backward: 1 volume, 2 poses, 3 both, 0 none
  int Fc, nfc;          // forward frames per chunk, chunks
  int Fb, nbc;          // backward frames per chunk, chunks
  int loss_off;         // loss partial blocks so far
  int per_sm;           // resident single-scan backward CTAs per SM (part split)
  FwdParams fp;
  BwdParams bp;
  CUtensorMap fmap, bmap;
};

// Scans grouped by what one batched launch needs them to share; groups of at most
// kMaxBatch.  key(a, b) says whether scans a and b may share a launch.
template <class Key>
std::vector<std::vector<int>> group_scans(const std::vector<int>& idx, Key key) {
  std::vector<std::vector<int>> groups;
  for (int i : idx) {
    bool placed = false;
    for (auto& g : groups)
      if (int(g.size()) < kMaxBatch && key(g.front(), i)) {
        g.push_back(i);
        placed = true;
        break;
      }
    if (!placed) groups.push_back({i});
  }
  return groups;
}

int step_batch(int n, pasfm_ctx* const* ctxs, const pasfm_geom* geoms, void* const* p0s, double* const* poses,
               const double* const* elems, const void* const* meas, const uint8_t* const* masks,
               pasfm_adam* states, double* const* loss_outs, unsigned long long* trace, cudaStream_t st) {
  if (n < 0) return fail(PASFM_EINVAL, "negative scan count");
  if (n == 0) return PASFM_OK;
  if (trace && n > 1024) return fail(PASFM_EINVAL, "trace_ns: at most 1024 scans");
  if (!ctxs || !geoms || !p0s || !poses || !elems || !meas || !states)
    return fail(PASFM_EINVAL, "NULL array argument");
  std::vector<BatchScan> sc(n);
  for (int i = 0; i < n; ++i) {
    BatchScan& b = sc[i];
    b.ctx = ctxs[i];
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == b.ctx) return fail(PASFM_EINVAL, "scans %d and %d share a context", k, i);
    TRY(prepare(b.ctx, &geoms[i], &b.G, &b.pl));
    if (b.ctx->device != ctxs[0]->device) return fail(PASFM_EINVAL, "scan %d is on another device", i);
    b.state = &states[i];
    b.p0 = p0s[i];
    b.pose = poses[i];
    b.loss_out = loss_outs ? loss_outs[i] : nullptr;
    const pasfm_adam* a = b.state;
    if (b.G.nvox == 0 || b.G.n_rows == 0 || b.G.g.n_samples == 0)
      return fail(PASFM_EINVAL, "scan %d: a step needs a non-empty volume, array and record", i);
    if (!b.p0 || !b.pose || !elems[i] || !meas[i]) return fail(PASFM_EINVAL, "scan %d: NULL array argument", i);
    const bool uv = !(a->flags & PASFM_ADAM_FREEZE_VOLUME), up = !(a->flags & PASFM_ADAM_FREEZE_POSES);
    if ((uv && (!a->m_vol || !a->v_vol)) || (up && (!a->m_pose || !a->v_pose)))
      return fail(PASFM_EINVAL, "scan %d: Adam moment array is NULL", i);
    if (!(a->beta1 >= 0 && a->beta1 < 1 && a->beta2 >= 0 && a->beta2 < 1 && a->eps >= 0))
      return fail(PASFM_EINVAL, "scan %d: Adam betas must lie in [0, 1) and eps >= 0", i);
    b.mode = (uv ? 1 : 0) | (up ? 2 : 0);
  }
  TRY(set_device(ctxs[0]));
  pasfm_ctx* lead = ctxs[0];

  // workspaces, element positions, forward parameters
  int n_counters = 0;
  for (int i = 0; i < n; ++i) {
    BatchScan& b = sc[i];
    pasfm_ctx* c = b.ctx;
    const Geo& G = b.G;
    const int F = G.g.n_frames;
    TRY(c->ensure(c->xw, size_t(G.n_rows) * 24));
    TRY(c->ensure(c->gres, size_t(G.n_rows) * G.g.n_samples * 4));
    TRY(c->ensure(c->vgrad, size_t(G.nvox) * 4));
    TRY(c->ensure(c->G, size_t(G.n_rows) * 24));
    TRY(c->ensure(c->grad6, size_t(F) * 48));
    b.Fc = frames_per_chunk(fwd_per_frame(G, b.pl), c->budget, F);
    b.nfc = (F + b.Fc - 1) / b.Fc;
    TRY(c->ensure(c->lpart, (size_t(G.n_rows + 7) / 8 + b.nfc) * 8));
    TRY(c->ensure(c->lscalar, 8));
    b.Fb = (b.mode & 2) ? frames_per_chunk(bwd_per_frame(G, b.pl), c->budget, F) : std::max(F, 1);
    b.nbc = b.mode ? (F + b.Fb - 1) / b.Fb : 0;
    b.loss_off = 0;
    n_counters += b.nfc + b.nbc;
    TRY(run_elem_pos(c, G, elems[i], b.pose, static_cast<double*>(c->xw.p), st));
    TRY(fwd_setup(c, G, b.pl, b.p0, static_cast<double*>(c->xw.p), b.Fc, &b.fp, &b.fmap));
  }
  // tile counters; sized generously so that later batches do not regrow the buffer
  // (a reallocation's cudaFree would synchronise the device)
  TRY(lead->ensure(lead->bcount, std::max<size_t>(size_t(n_counters), 4096) * sizeof(int)));
  int* counters = static_cast<int*>(lead->bcount.p);
  int next_counter = 0;
  CUDA_TRY(cudaMemsetAsync(counters, 0, size_t(n_counters) * sizeof(int), st));
  if (trace) {
    trace_init_kernel<<<1, std::max(32, ((n + 31) / 32) * 32), 0, st>>>(trace, n);
    TRY(check_launch("trace_init"));
  }

  std::vector<int> all(n);
  for (int i = 0; i < n; ++i) all[i] = i;

  // forward, one launch per group and frame-chunk round, then the groups' reductions
  const auto fwd_groups = group_scans(all, [&](int a, int b) {
    const Plan &p = sc[a].pl, &q = sc[b].pl;
    return p.K == q.K && p.S == q.S && p.C == q.C && p.fwd_warps == q.fwd_warps &&
           same_fwd_profile(sc[a].fp, sc[b].fp);
  });
  int max_fc = 0;
  for (auto& b : sc) max_fc = std::max(max_fc, b.nfc);
  for (int r = 0; r < max_fc; ++r) {
    for (const auto& grp : fwd_groups) {
      TmaBatch maps;
      FwdBatch B;
      std::memset(&maps, 0, sizeof maps);
      std::memset(&B, 0, sizeof B);
      RedBatch RB;
      std::memset(&RB, 0, sizeof RB);
      std::vector<int> members;
      for (int i : grp) {
        BatchScan& b = sc[i];
        if (r >= b.nfc) continue;
        const int k = B.n++;
        const int fb = r * b.Fc, fc = std::min(b.Fc, b.G.g.n_frames - fb);
        B.G[k] = b.fp;
        B.G[k].f_begin = fb;
        B.ncubes[k] = b.pl.ncubes;
        B.fc[k] = fc;
        B.tiles[k + 1] = B.tiles[k] + b.pl.ncubes * fc * b.pl.n_egroups;
        maps.m[k] = b.fmap;
        RB.R[k] = red_params(B.G[k], b.G, b.pl, fb, fc, nullptr, static_cast<float*>(b.ctx->gres.p), meas[i],
                             masks ? masks[i] : nullptr, static_cast<double*>(b.ctx->lpart.p), b.loss_off);
        RB.blocks[k + 1] = RB.blocks[k] + (RB.R[k].n_rows + 7) / 8;
        RB.n = B.n;
        b.loss_off += (RB.R[k].n_rows + 7) / 8;
        members.push_back(i);
      }
      if (B.n == 0) continue;
      const Plan& pl = sc[members[0]].pl;
      B.Q = sc[members[0]].fp;
      B.counter = counters + next_counter++;
      B.trace = trace;
      const int threads = 32 * pl.fwd_warps;
      const size_t smem = fwd_smem(pl);
      const int per_sm = std::max(1, fwd_batch_occupancy(pl.K, pl.S)(pl.C, threads, smem));
      const int ctas = std::min(B.tiles[B.n], per_sm * std::max(lead->sms, 1));
      cudaEvent_t t = lead->begin(st);
      cudaError_t e = fwd_batch_launcher(pl.K, pl.S)(pl.C, maps, B, ctas, threads, smem, st);
      lead->end("fwd_cube_batch", t, st);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PASFM_ECUDA, "fwd_cube batch launch: %s", cudaGetErrorString(e));
      }
      t = lead->begin(st);
      e = fwd_reduce_batch_launch(RB, pl.W, st);
      lead->end("fwd_reduce_batch", t, st);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PASFM_ECUDA, "fwd_reduce batch launch: %s", cudaGetErrorString(e));
      }
    }
  }
  for (auto& b : sc) {
    double* dst = b.loss_out ? b.loss_out : static_cast<double*>(b.ctx->lscalar.p);
    cudaEvent_t t = b.ctx->begin(st);
    sum_kernel<<<1, 256, 0, st>>>(static_cast<double*>(b.ctx->lpart.p), b.loss_off, dst);
    b.ctx->end("loss_sum", t, st);
    TRY(check_launch("loss_sum"));
  }

  // backward (adjoint and / or pose gradient), one launch per group and frame-chunk round
  std::vector<int> bwd_idx;
  for (int i = 0; i < n; ++i) {
    BatchScan& b = sc[i];
    if (!b.mode) continue;
    pasfm_ctx* c = b.ctx;
    TRY(bwd_setup(c, b.G, b.pl, b.mode, b.p0, static_cast<double*>(c->xw.p), c->gres.p, PASFM_F32, nullptr,
                  static_cast<float*>(c->vgrad.p), b.Fb, &b.bp, &b.bmap, st));
    b.per_sm = bwd_occupancy(b.pl.K, b.pl.S)(b.pl.C, b.mode, bwd_smem(b.pl));
    bwd_idx.push_back(i);
  }
  const auto bwd_groups = group_scans(bwd_idx, [&](int a, int b) {
    const Plan &p = sc[a].pl, &q = sc[b].pl;
    return p.K == q.K && p.S == q.S && p.C == q.C && sc[a].mode == sc[b].mode &&
           same_bwd_profile(sc[a].bp, sc[b].bp);
  });
  int max_bc = 0;
  for (auto& b : sc) max_bc = std::max(max_bc, b.nbc);
  for (int r = 0; r < max_bc; ++r) {
    for (const auto& grp : bwd_groups) {
      TmaBatch maps;
      BwdBatch B;
      std::memset(&maps, 0, sizeof maps);
      std::memset(&B, 0, sizeof B);
      std::vector<int> members;
      for (int i : grp) {
        BatchScan& b = sc[i];
        if (r >= b.nbc) continue;
        const int k = B.n++;
        const int fb = r * b.Fb, fc = std::min(b.Fb, b.G.g.n_frames - fb);
        bwd_chunk(b.ctx, b.pl, b.G.g.n_elem, fb, fc, b.per_sm, &b.bp);
        B.G[k] = b.bp;
        B.ncubes[k] = b.pl.ncubes;
        B.tiles[k + 1] = B.tiles[k] + b.pl.ncubes * b.bp.n_parts;
        maps.m[k] = b.bmap;
        members.push_back(i);
      }
      if (B.n == 0) continue;
      const BatchScan& lead_scan = sc[members[0]];
      const Plan& pl = lead_scan.pl;
      B.Q = lead_scan.bp;
      B.counter = counters + next_counter++;
      B.trace = trace;
      const size_t smem = bwd_smem(pl);
      const int per_sm = std::max(1, bwd_batch_occupancy(pl.K, pl.S)(pl.C, lead_scan.mode, smem));
      const int ctas = std::min(B.tiles[B.n], per_sm * std::max(lead->sms, 1));
      cudaEvent_t t = lead->begin(st);
      cudaError_t e = bwd_batch_launcher(pl.K, pl.S)(pl.C, lead_scan.mode, maps, B, ctas, smem, st);
      lead->end("bwd_cube_batch", t, st);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PASFM_ECUDA, "bwd_cube batch launch: %s", cudaGetErrorString(e));
      }
      for (int i : members) {  // per scan: part sums into the volume gradient, element gradients
        BatchScan& b = sc[i];
        pasfm_ctx* c = b.ctx;
        const BwdParams& P = b.bp;
        const int fc = P.n_items / b.G.g.n_elem;
        if ((b.mode & 1) && P.n_parts > 1) {
          const int64_t nv = b.G.nvox;
          const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((nv + 255) / 256, 148 * 16));
          t = c->begin(st);
          sum_parts_kernel<<<blocks, 256, 0, st>>>(P.vol_parts, P.n_parts, nv, P.vol, P.accumulate);
          c->end("sum_parts", t, st);
          TRY(check_launch("sum_parts"));
        }
        if (b.mode & 2) {
          const int rows = fc * b.G.g.n_elem;
          t = c->begin(st);
          pose_rows_kernel<<<(rows + 7) / 8, 256, 0, st>>>(P.gpart, b.pl.ncubes, rows,
                                                           int64_t(P.f_begin) * b.G.g.n_elem,
                                                           static_cast<double*>(c->G.p));
          c->end("pose_rows", t, st);
          TRY(check_launch("pose_rows"));
        }
      }
    }
  }

  // Adam on each scan's poses and volume
  for (auto& b : sc) {
    pasfm_ctx* c = b.ctx;
    pasfm_adam* a = b.state;
    const int64_t k = a->step + 1;
    if (b.mode) {
      const double bc1 = 1.0 - std::pow(a->beta1, double(k));
      const double bc2 = 1.0 - std::pow(a->beta2, double(k));
      if (b.mode & 2) {
        TRY(run_grad6(c, b.G, static_cast<double*>(c->xw.p), static_cast<double*>(c->G.p),
                      static_cast<double*>(c->grad6.p), st));
        cudaEvent_t t = c->begin(st);
        adam_pose_kernel<<<(b.G.g.n_frames + 63) / 64, 64, 0, st>>>(
            b.pose, static_cast<double*>(c->grad6.p), a->m_pose, a->v_pose, b.G.g.n_frames, a->beta1, a->beta2,
            bc1, bc2, a->lr_rot, a->lr_trans, a->eps, (a->flags & PASFM_ADAM_FIX_FRAME0) ? 1 : 0, 0);
        c->end("adam_pose", t, st);
        TRY(check_launch("adam_pose"));
      }
      if (b.mode & 1) {
        cudaEvent_t t = c->begin(st);
        adam_vol_kernel<<<static_cast<unsigned>((b.G.nvox + 255) / 256), 256, 0, st>>>(
            b.p0, b.G.g.dtype_vol, static_cast<float*>(c->vgrad.p), a->m_vol, a->v_vol, b.G.nvox,
            static_cast<float>(a->beta1), static_cast<float>(a->beta2), static_cast<float>(a->lr_vol / bc1),
            static_cast<float>(1.0 / std::sqrt(bc2)), static_cast<float>(a->eps),
            (a->flags & PASFM_ADAM_NONNEG) ? 1 : 0);
        c->end("adam_vol", t, st);
        TRY(check_launch("adam_vol"));
      }
    }
    a->step = k;
  }
  return PASFM_OK;
}

int prepare(pasfm_ctx* ctx, const pasfm_geom* geom, Geo* G, Plan* pl) {
  if (!ctx) return fail(PASFM_EINVAL, "ctx is NULL");
  TRY(check_geom(geom, G));
  TRY(make_plan(*G, pl));
  TRY(set_device(ctx));
  return PASFM_OK;
}

}  // namespace

extern "C" {

int pasfm_abi_version(void) { return 3; }

const char* pasfm_last_error(void) { return g_err.c_str(); }

int pasfm_create(pasfm_ctx** out, int device) {
  if (!out) return fail(PASFM_EINVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return fail(PASFM_ECUDA, "CUDA device %d is not available (%d visible)", device, n);
  }
  CUDA_TRY(cudaSetDevice(device));
  pasfm_ctx* ctx = new pasfm_ctx();
  ctx->device = device;
  if (cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    ctx->sms = 0;
  }
  if (cudaMalloc(&ctx->status, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(ctx->status, 0, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return fail(PASFM_ECUDA, "status word allocation failed");
  }
  *out = ctx;
  return PASFM_OK;
}

int pasfm_destroy(pasfm_ctx* ctx) {
  if (!ctx) return PASFM_OK;
  cudaSetDevice(ctx->device);
  for (Buf* b : {&ctx->xw, &ctx->part, &ctx->n0, &ctx->gres, &ctx->vgrad, &ctx->gpart, &ctx->G, &ctx->grad6,
                 &ctx->lpart, &ctx->lscalar, &ctx->taps, &ctx->vparts, &ctx->gw, &ctx->tpart, &ctx->gdiff,
                 &ctx->bcount})
    if (b->p) cudaFree(b->p);
  for (auto& r : ctx->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ctx->pool) cudaEventDestroy(e);
  if (ctx->status) cudaFree(ctx->status);
  delete ctx;
  return PASFM_OK;
}

int pasfm_set_partial_budget(pasfm_ctx* ctx, size_t bytes) {
  if (!ctx) return fail(PASFM_EINVAL, "ctx is NULL");
  ctx->budget = bytes ? bytes : kDefaultPartialBudget;
  return PASFM_OK;
}

int pasfm_set_wait_limit(pasfm_ctx* ctx, int64_t cycles) {
  if (!ctx) return fail(PASFM_EINVAL, "ctx is NULL");
  ctx->wait_cycles = cycles < 0 ? kWaitCycles : static_cast<long long>(cycles);
  return PASFM_OK;
}

int pasfm_workspace_size(const pasfm_geom* geom, size_t* bytes) {
  if (!bytes) return fail(PASFM_EINVAL, "bytes is NULL");
  Geo G;
  Plan pl;
  TRY(check_geom(geom, &G));
  TRY(make_plan(G, &pl));
  const int F = G.g.n_frames;
  const size_t budget = kDefaultPartialBudget;
  const int Ff = frames_per_chunk(fwd_per_frame(G, pl), budget, F);
  const int Fb = frames_per_chunk(bwd_per_frame(G, pl), budget, F);
  size_t b = size_t(G.n_rows) * 24;                                         // xw
  b += size_t(Ff) * fwd_per_frame(G, pl);                                   // part + n0
  b += size_t(Fb) * bwd_per_frame(G, pl);                                   // gpart
  b += size_t(G.n_rows) * G.g.n_samples * 4;                                // residual (step)
  if (G.g.kernel == PASFM_KERNEL_SPHERE) b += size_t(G.n_rows) * diff_len(G.g.n_samples) * 4;  // its difference
  b += size_t(G.nvox) * 4;                                                  // volume gradient (step)
  b += size_t(G.nvox) * 4 * kMaxParts;                                      // per-part adjoint sums
  b += size_t(G.nvox) * 12 + size_t(tgv_tiles(G.g.nx, G.g.ny, G.g.nz)) * 8;  // TGV grad_w, energy partials
  b += size_t(G.n_rows) * 24 + size_t(F) * 48;                              // G, grad6
  b += (size_t(G.n_rows + 7) / 8 + (F + Ff - 1) / std::max(Ff, 1) + 2) * 8;  // loss partials
  *bytes = b;
  return PASFM_OK;
}

int pasfm_reserve(pasfm_ctx* ctx, const pasfm_geom* geom) {
  Geo G;
  Plan pl;
  TRY(prepare(ctx, geom, &G, &pl));
  const int F = G.g.n_frames;
  const int Ff = frames_per_chunk(fwd_per_frame(G, pl), ctx->budget, F);
  const int Fb = frames_per_chunk(bwd_per_frame(G, pl), ctx->budget, F);
  TRY(ctx->ensure(ctx->xw, size_t(G.n_rows) * 24));
  TRY(ctx->ensure(ctx->part, size_t(Ff) * G.g.n_elem * pl.ncubes * pl.W * 4));
  TRY(ctx->ensure(ctx->n0, size_t(Ff) * G.g.n_elem * pl.ncubes * 4));
  TRY(ctx->ensure(ctx->gpart, size_t(Fb) * G.g.n_elem * pl.ncubes * 24));
  TRY(ctx->ensure(ctx->gres, size_t(G.n_rows) * G.g.n_samples * 4));
  if (G.g.kernel == PASFM_KERNEL_SPHERE) TRY(ctx->ensure(ctx->gdiff, size_t(G.n_rows) * diff_len(G.g.n_samples) * 4));
  TRY(ctx->ensure(ctx->vgrad, size_t(G.nvox) * 4));
  TRY(ctx->ensure(ctx->vparts, size_t(G.nvox) * 4 * kMaxParts));
  TRY(ctx->ensure(ctx->G, size_t(G.n_rows) * 24));
  TRY(ctx->ensure(ctx->grad6, size_t(F) * 48));
  TRY(ctx->ensure(ctx->gw, size_t(G.nvox) * 12));
  TRY(ctx->ensure(ctx->tpart, size_t(tgv_tiles(G.g.nx, G.g.ny, G.g.nz)) * 8));
  TRY(ctx->ensure(ctx->lpart, (size_t(G.n_rows + 7) / 8 + (F + Ff - 1) / std::max(Ff, 1) + 2) * 8));
  TRY(ctx->ensure(ctx->lscalar, 8));
  return PASFM_OK;
}

int pasfm_element_positions(pasfm_ctx* ctx, const pasfm_geom* geom, const double* elem, const double* pose,
                            double* xw_out, void* stream) {
  Geo G;
  Plan pl;
  TRY(prepare(ctx, geom, &G, &pl));
  if (G.n_rows > 0 && (!elem || !pose || !xw_out)) return fail(PASFM_EINVAL, "NULL array argument");
  return run_elem_pos(ctx, G, elem, pose, xw_out, static_cast<cudaStream_t>(stream));
}

int pasfm_forward(pasfm_ctx* ctx, const pasfm_geom* geom, const void* p0, const double* elem, const double* pose,
                  float* sig_out, void* stream) {
  Geo G;
  Plan pl;
  TRY(prepare(ctx, geom, &G, &pl));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t sig_bytes = size_t(G.n_rows) * G.g.n_samples * 4;
  if (sig_bytes == 0) return PASFM_OK;
  if (!sig_out || !elem || !pose || (G.nvox > 0 && !p0)) return fail(PASFM_EINVAL, "NULL array argument");
  if (G.nvox == 0) {
    CUDA_TRY(cudaMemsetAsync(sig_out, 0, sig_bytes, st));
    return PASFM_OK;
  }
  TRY(ctx->ensure(ctx->xw, size_t(G.n_rows) * 24));
  double* xw = static_cast<double*>(ctx->xw.p);
  TRY(run_elem_pos(ctx, G, elem, pose, xw, st));
  return run_forward(ctx, G, pl, p0, xw, sig_out, nullptr, nullptr, nullptr, nullptr, st);
}

int pasfm_adjoint(pasfm_ctx* ctx, const pasfm_geom* geom, const double* elem, const double* pose, const void* g,
                  float* vol_out, void* stream) {
  Geo G;
  Plan pl;
  TRY(prepare(ctx, geom, &G, &pl));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (G.nvox == 0) return PASFM_OK;
  if (!vol_out) return fail(PASFM_EINVAL, "vol_out is NULL");
  if (G.n_rows == 0 || G.g.n_samples == 0) {
    CUDA_TRY(cudaMemsetAsync(vol_out, 0, size_t(G.nvox) * 4, st));
    return PASFM_OK;
  }
  if (!elem || !pose || !g) return fail(PASFM_EINVAL, "NULL array argument");
  TRY(ctx->ensure(ctx->xw, size_t(G.n_rows) * 24));
  double* xw = static_cast<double*>(ctx->xw.p);
  TRY(run_elem_pos(ctx, G, elem, pose, xw, st));
  return run_backward(ctx, G, pl, 1, nullptr, xw, g, G.g.dtype_sig, nullptr, vol_out, nullptr, st);
}

int pasfm_pose_grad(pasfm_ctx* ctx, const pasfm_geom* geom, const void* p0, const double* elem,
                    const double* pose, const void* g, const uint8_t* mask, double* grad6_out,
                    double* gelem_out, void* stream) {
  Geo G;
  Plan pl;
  TRY(prepare(ctx, geom, &G, &pl));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (G.g.n_frames == 0) return PASFM_OK;
  if (!grad6_out) return fail(PASFM_EINVAL, "grad6_out is NULL");
  if (G.n_rows == 0 || G.nvox == 0 || G.g.n_samples == 0) {
    CUDA_TRY(cudaMemsetAsync(grad6_out, 0, size_t(G.g.n_frames) * 48, st));
    if (gelem_out && G.n_rows) CUDA_TRY(cudaMemsetAsync(gelem_out, 0, size_t(G.n_rows) * 24, st));
    return PASFM_OK;
  }
  if (!elem || !pose || !g || !p0) return fail(PASFM_EINVAL, "NULL array argument");
  TRY(ctx->ensure(ctx->xw, size_t(G.n_rows) * 24));
  double* xw = static_cast<double*>(ctx->xw.p);
  double* Gm = gelem_out;
  if (!Gm) {
    TRY(ctx->ensure(ctx->G, size_t(G.n_rows) * 24));
    Gm = static_cast<double*>(ctx->G.p);
  }
  TRY(run_elem_pos(ctx, G, elem, pose, xw, st));
  TRY(run_backward(ctx, G, pl, 2, p0, xw, g, G.g.dtype_sig, mask, nullptr, Gm, st));
  return run_grad6(ctx, G, xw, Gm, grad6_out, st);
}

int pasfm_loss(pasfm_ctx* ctx, const pasfm_geom* geom, const float* sig, const void* meas, const uint8_t* mask,
               float* g_out, double* loss_out, void* stream) {
  Geo G;
  if (!ctx) return fail(PASFM_EINVAL, "ctx is NULL");
  TRY(check_geom(geom, &G));
  TRY(set_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t rows = G.n_rows;
  if (!loss_out) return fail(PASFM_EINVAL, "loss_out is NULL");
  if (rows == 0 || G.g.n_samples == 0) {
    CUDA_TRY(cudaMemsetAsync(loss_out, 0, 8, st));
    return PASFM_OK;
  }
  if (!sig || !meas || !g_out) return fail(PASFM_EINVAL, "NULL array argument");
  const int blocks = static_cast<int>((rows + 7) / 8);
  TRY(ctx->ensure(ctx->lpart, size_t(blocks) * 8));
  cudaEvent_t t = ctx->begin(st);
  loss_rows_kernel<<<blocks, 256, 0, st>>>(sig, meas, G.g.dtype_sig, mask, g_out,
                                           static_cast<double*>(ctx->lpart.p), static_cast<int>(rows),
                                           G.g.n_samples);
  ctx->end("loss_rows", t, st);
  TRY(check_launch("loss_rows"));
  t = ctx->begin(st);
  sum_kernel<<<1, 256, 0, st>>>(static_cast<double*>(ctx->lpart.p), blocks, loss_out);
  ctx->end("loss_sum", t, st);
  return check_launch("loss_sum");
}

int pasfm_step(pasfm_ctx* ctx, const pasfm_geom* geom, void* p0, double* pose, const double* elem,
               const void* meas, const uint8_t* mask, pasfm_adam* state, double* loss_out, void* stream) {
  return pasfm_step_tgv(ctx, geom, p0, pose, elem, meas, mask, state, nullptr, loss_out, nullptr, stream);
}

int pasfm_tgv_grad(pasfm_ctx* ctx, const pasfm_geom* geom, const void* p0, const float* w, double alpha1,
                   double alpha0, double eps, float* grad_u, int accumulate, float* grad_w, double* energy_out,
                   void* stream) {
  Geo G;
  Plan pl;
  TRY(prepare(ctx, geom, &G, &pl));
  if (!(alpha1 >= 0) || !(alpha0 >= 0) || !(eps > 0) || !std::isfinite(alpha1) || !std::isfinite(alpha0) ||
      !std::isfinite(eps))
    return fail(PASFM_EINVAL, "TGV weights must be finite, alpha >= 0 and eps > 0");
  if (G.nvox == 0) return PASFM_OK;
  if (!p0 || !w || !grad_u || !grad_w) return fail(PASFM_EINVAL, "NULL array argument");
  if (G.nvox > (int64_t(1) << 31) / 3) return fail(PASFM_EUNSUPPORTED, "volume too large for the TGV kernel");
  return run_tgv(ctx, G, p0, w, alpha1, alpha0, eps, grad_u, accumulate, grad_w, energy_out,
                 static_cast<cudaStream_t>(stream));
}

int pasfm_step_tgv(pasfm_ctx* ctx, const pasfm_geom* geom, void* p0, double* pose, const double* elem,
                   const void* meas, const uint8_t* mask, pasfm_adam* state, const pasfm_tgv* tgv,
                   double* loss_out, double* tgv_out, void* stream) {
  Geo G;
  Plan pl;
  TRY(prepare(ctx, geom, &G, &pl));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!state) return fail(PASFM_EINVAL, "state is NULL");
  if (tgv) {
    if (state->flags & PASFM_ADAM_FREEZE_VOLUME) return fail(PASFM_EINVAL, "a TGV step needs volume updates");
    if (!tgv->w || !tgv->m_w || !tgv->v_w) return fail(PASFM_EINVAL, "TGV array is NULL");
    if (!(tgv->alpha1 >= 0) || !(tgv->alpha0 >= 0) || !(tgv->eps > 0) || !std::isfinite(tgv->lr_w))
      return fail(PASFM_EINVAL, "TGV weights must be finite, alpha >= 0 and eps > 0");
    if (G.nvox > (int64_t(1) << 31) / 3) return fail(PASFM_EUNSUPPORTED, "volume too large for the TGV kernel");
  }
  if (G.nvox == 0 || G.n_rows == 0 || G.g.n_samples == 0)
    return fail(PASFM_EINVAL, "pasfm_step needs a non-empty volume, array and record");
  if (!p0 || !pose || !elem || !meas) return fail(PASFM_EINVAL, "NULL array argument");
  const bool upd_vol = !(state->flags & PASFM_ADAM_FREEZE_VOLUME);
  const bool upd_pose = !(state->flags & PASFM_ADAM_FREEZE_POSES);
  if ((upd_vol && (!state->m_vol || !state->v_vol)) || (upd_pose && (!state->m_pose || !state->v_pose)))
    return fail(PASFM_EINVAL, "Adam moment array is NULL");
  if (!(state->beta1 >= 0 && state->beta1 < 1 && state->beta2 >= 0 && state->beta2 < 1 && state->eps >= 0))
    return fail(PASFM_EINVAL, "Adam betas must lie in [0, 1) and eps >= 0");

  TRY(ctx->ensure(ctx->xw, size_t(G.n_rows) * 24));
  TRY(ctx->ensure(ctx->gres, size_t(G.n_rows) * G.g.n_samples * 4));
  if (G.g.kernel == PASFM_KERNEL_SPHERE) TRY(ctx->ensure(ctx->gdiff, size_t(G.n_rows) * diff_len(G.g.n_samples) * 4));
  TRY(ctx->ensure(ctx->vgrad, size_t(G.nvox) * 4));
  TRY(ctx->ensure(ctx->vparts, size_t(G.nvox) * 4 * kMaxParts));
  TRY(ctx->ensure(ctx->G, size_t(G.n_rows) * 24));
  TRY(ctx->ensure(ctx->grad6, size_t(G.g.n_frames) * 48));
  double* xw = static_cast<double*>(ctx->xw.p);
  float* gres = static_cast<float*>(ctx->gres.p);

  TRY(run_elem_pos(ctx, G, elem, pose, xw, st));
  TRY(run_forward(ctx, G, pl, p0, xw, nullptr, gres, meas, mask, loss_out, st));
  const int mode = (upd_vol ? 1 : 0) | (upd_pose ? 2 : 0);
  const int64_t k = state->step + 1;
  if (mode == 0) {
    state->step = k;
    return PASFM_OK;
  }
  TRY(run_backward(ctx, G, pl, mode, p0, xw, gres, PASFM_F32, nullptr, static_cast<float*>(ctx->vgrad.p),
                   static_cast<double*>(ctx->G.p), st));
  const double bc1 = 1.0 - std::pow(state->beta1, double(k));
  const double bc2 = 1.0 - std::pow(state->beta2, double(k));
  if (tgv) {
    // regulariser: its volume gradient joins the data gradient, then w takes its own Adam step
    TRY(ctx->ensure(ctx->gw, size_t(G.nvox) * 12));
    float* gw = static_cast<float*>(ctx->gw.p);
    TRY(run_tgv(ctx, G, p0, tgv->w, tgv->alpha1, tgv->alpha0, tgv->eps, static_cast<float*>(ctx->vgrad.p), 1, gw,
                tgv_out, st));
    cudaEvent_t t = ctx->begin(st);
    adam_vol_kernel<<<static_cast<unsigned>((3 * G.nvox + 255) / 256), 256, 0, st>>>(
        tgv->w, PASFM_F32, gw, tgv->m_w, tgv->v_w, 3 * G.nvox, static_cast<float>(state->beta1),
        static_cast<float>(state->beta2), static_cast<float>(tgv->lr_w / bc1), static_cast<float>(1.0 / std::sqrt(bc2)),
        static_cast<float>(state->eps), 0);
    ctx->end("adam_w", t, st);
    TRY(check_launch("adam_w"));
  }
  if (upd_pose) {
    TRY(run_grad6(ctx, G, xw, static_cast<double*>(ctx->G.p), static_cast<double*>(ctx->grad6.p), st));
    cudaEvent_t t = ctx->begin(st);
    adam_pose_kernel<<<(G.g.n_frames + 63) / 64, 64, 0, st>>>(
        pose, static_cast<double*>(ctx->grad6.p), state->m_pose, state->v_pose, G.g.n_frames, state->beta1,
        state->beta2, bc1, bc2, state->lr_rot, state->lr_trans, state->eps,
        (state->flags & PASFM_ADAM_FIX_FRAME0) ? 1 : 0, 0);
    ctx->end("adam_pose", t, st);
    TRY(check_launch("adam_pose"));
  }
  if (upd_vol) {
    cudaEvent_t t = ctx->begin(st);
    adam_vol_kernel<<<static_cast<unsigned>((G.nvox + 255) / 256), 256, 0, st>>>(
        p0, G.g.dtype_vol, static_cast<float*>(ctx->vgrad.p), state->m_vol, state->v_vol, G.nvox,
        static_cast<float>(state->beta1), static_cast<float>(state->beta2),
        static_cast<float>(state->lr_vol / bc1), static_cast<float>(1.0 / std::sqrt(bc2)),
        static_cast<float>(state->eps), (state->flags & PASFM_ADAM_NONNEG) ? 1 : 0);
    ctx->end("adam_vol", t, st);
    TRY(check_launch("adam_vol"));
  }
  state->step = k;
  return PASFM_OK;
}

int pasfm_step_batch(int n, pasfm_ctx* const* ctxs, const pasfm_geom* geoms, void* const* p0, double* const* pose,
                     const double* const* elem, const void* const* meas, const uint8_t* const* mask,
                     pasfm_adam* states, double* const* loss_out, uint64_t* trace_ns, void* stream) {
  return step_batch(n, ctxs, geoms, p0, pose, elem, meas, mask, states, loss_out,
                    reinterpret_cast<unsigned long long*>(trace_ns), static_cast<cudaStream_t>(stream));
}

int pasfm_apply_twists(pasfm_ctx* ctx, int n_frames, const double* pose, const double* xi, double* pose_out,
                       void* stream) {
  if (!ctx) return fail(PASFM_EINVAL, "ctx is NULL");
  if (n_frames < 0) return fail(PASFM_EINVAL, "negative frame count");
  if (n_frames == 0) return PASFM_OK;
  if (!pose || !xi || !pose_out) return fail(PASFM_EINVAL, "NULL array argument");
  TRY(set_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t t = ctx->begin(st);
  apply_twist_kernel<<<(n_frames + 127) / 128, 128, 0, st>>>(pose, xi, pose_out, n_frames);
  ctx->end("apply_twist", t, st);
  return check_launch("apply_twist");
}

int pasfm_twist_grad(pasfm_ctx* ctx, int n_frames, const double* xi, const double* grad6, double* grad_xi_out,
                     void* stream) {
  if (!ctx) return fail(PASFM_EINVAL, "ctx is NULL");
  if (n_frames < 0) return fail(PASFM_EINVAL, "negative frame count");
  if (n_frames == 0) return PASFM_OK;
  if (!xi || !grad6 || !grad_xi_out) return fail(PASFM_EINVAL, "NULL array argument");
  TRY(set_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t t = ctx->begin(st);
  twist_grad_kernel<<<(n_frames + 127) / 128, 128, 0, st>>>(xi, grad6, grad_xi_out, n_frames);
  ctx->end("twist_grad", t, st);
  return check_launch("twist_grad");
}

int pasfm_resample(pasfm_ctx* ctx, const pasfm_geom* src_geom, const float* src, const pasfm_geom* dst_geom,
                   float* dst, void* stream) {
  if (!ctx || !src_geom || !dst_geom) return fail(PASFM_EINVAL, "NULL argument");
  Geo S, D;
  TRY(check_geom(src_geom, &S));
  TRY(check_geom(dst_geom, &D));
  if (D.nvox == 0) return PASFM_OK;
  if (S.nvox == 0) return fail(PASFM_EINVAL, "empty source grid");
  if (!src || !dst) return fail(PASFM_EINVAL, "NULL array argument");
  TRY(set_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const pasfm_geom& a = *src_geom;
  const pasfm_geom& b = *dst_geom;
  cudaEvent_t t = ctx->begin(st);
  resample_kernel<<<static_cast<unsigned>((D.nvox + 255) / 256), 256, 0, st>>>(
      src, a.nx, a.ny, a.nz, a.ox, a.oy, a.oz, a.dx, a.dy, a.dz, dst, b.nx, b.ny, b.nz, b.ox, b.oy, b.oz, b.dx,
      b.dy, b.dz);
  ctx->end("resample", t, st);
  return check_launch("resample");
}

int pasfm_lowpass(pasfm_ctx* ctx, int64_t n_rows, int n_samples, double sigma, int decim, const float* src,
                  float* dst, void* stream) {
  if (!ctx) return fail(PASFM_EINVAL, "ctx is NULL");
  if (n_rows < 0 || n_samples < 0 || !std::isfinite(sigma)) return fail(PASFM_EINVAL, "bad size or sigma");
  if (decim < 1) return fail(PASFM_EINVAL, "decim must be >= 1");
  if (n_rows == 0 || n_samples == 0) return PASFM_OK;
  if (!src || !dst) return fail(PASFM_EINVAL, "NULL array argument");
  if (decim > 1 && src == dst) return fail(PASFM_EINVAL, "dst may alias src only without decimation");
  if (n_rows > INT32_MAX) return fail(PASFM_EUNSUPPORTED, "too many traces");
  if (size_t(n_samples) * 4 > 200 * 1024) return fail(PASFM_EUNSUPPORTED, "trace longer than 51200 samples");
  TRY(set_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Gaussian taps, radius int(4 sigma + 0.5), normalised to sum 1 (sigma <= 0: identity)
  const int r = sigma > 0 ? static_cast<int>(4.0 * sigma + 0.5) : 0;
  if (r > 4096) return fail(PASFM_EUNSUPPORTED, "sigma too large");
  std::vector<float> w(2 * r + 1);
  double tot = 0.0;
  for (int k = -r; k <= r; ++k) tot += r ? std::exp(-0.5 * k * k / (sigma * sigma)) : 1.0;
  for (int k = -r; k <= r; ++k)
    w[k + r] = static_cast<float>((r ? std::exp(-0.5 * k * k / (sigma * sigma)) : 1.0) / tot);
  TRY(ctx->ensure(ctx->taps, w.size() * sizeof(float)));
  CUDA_TRY(cudaMemcpyAsync(ctx->taps.p, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  const size_t smem = size_t(n_samples) * 4;
  CUDA_TRY(cudaFuncSetAttribute(lowpass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  cudaEvent_t t = ctx->begin(st);
  const int n_out = (n_samples + decim - 1) / decim;
  lowpass_kernel<<<static_cast<unsigned>(n_rows), 256, smem, st>>>(src, dst, n_samples, r, decim, n_out,
                                                                   static_cast<float*>(ctx->taps.p));
  ctx->end("lowpass", t, st);
  TRY(check_launch("lowpass"));
  // the host tap buffer must outlive the asynchronous copy
  CUDA_TRY(cudaStreamSynchronize(st));
  return PASFM_OK;
}

int pasfm_nc_scores(pasfm_ctx* ctx, int n_cand, int n_elem, int n_samples, const float* sim, const void* meas,
                    int dtype_meas, const uint8_t* mask, double* scores_out, void* stream) {
  if (!ctx) return fail(PASFM_EINVAL, "ctx is NULL");
  if (n_cand < 0 || n_elem < 0 || n_samples < 0) return fail(PASFM_EINVAL, "negative size");
  if (dtype_meas != PASFM_F32 && dtype_meas != PASFM_BF16 && dtype_meas != PASFM_F16)
    return fail(PASFM_EINVAL, "unknown dtype %d", dtype_meas);
  if (n_cand == 0) return PASFM_OK;
  if (!sim || !meas || !scores_out) return fail(PASFM_EINVAL, "NULL array argument");
  TRY(set_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t t = ctx->begin(st);
  nc_scores_kernel<<<n_cand, 256, 0, st>>>(sim, meas, dtype_meas, mask, n_elem, n_samples, scores_out);
  ctx->end("nc_scores", t, st);
  return check_launch("nc_scores");
}

int pasfm_nc_grad(pasfm_ctx* ctx, int64_t n_rows, int n_samples, const float* sim, const void* meas, int dtype_meas,
                  int meas_repeat, const uint8_t* mask, double scale, float* g_out, double* nc_out, void* stream) {
  if (!ctx) return fail(PASFM_EINVAL, "ctx is NULL");
  if (n_rows < 0 || n_samples < 0 || !std::isfinite(scale)) return fail(PASFM_EINVAL, "bad size or scale");
  if (meas_repeat < 1) return fail(PASFM_EINVAL, "meas_repeat must be >= 1");
  if (dtype_meas != PASFM_F32 && dtype_meas != PASFM_BF16 && dtype_meas != PASFM_F16)
    return fail(PASFM_EINVAL, "unknown dtype %d", dtype_meas);
  if (n_rows == 0 || n_samples == 0) return PASFM_OK;
  if (!sim || !meas || !g_out) return fail(PASFM_EINVAL, "NULL array argument");
  if ((n_rows + 7) / 8 > INT32_MAX) return fail(PASFM_EUNSUPPORTED, "too many traces");
  TRY(set_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t t = ctx->begin(st);
  nc_grad_kernel<<<static_cast<unsigned>((n_rows + 7) / 8), 256, 0, st>>>(
      sim, meas, dtype_meas, mask, n_rows, n_samples, meas_repeat, static_cast<float>(scale), g_out, nc_out);
  ctx->end("nc_grad", t, st);
  return check_launch("nc_grad");
}

int pasfm_scale(pasfm_ctx* ctx, int64_t n, double alpha, float* x, void* stream) {
  if (!ctx) return fail(PASFM_EINVAL, "ctx is NULL");
  if (n < 0 || !std::isfinite(alpha)) return fail(PASFM_EINVAL, "bad size or factor");
  if (n == 0) return PASFM_OK;
  if (!x) return fail(PASFM_EINVAL, "NULL array argument");
  TRY(set_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t t = ctx->begin(st);
  scale_kernel<<<static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 148 * 32)), 256, 0, st>>>(
      x, n, static_cast<float>(alpha));
  ctx->end("scale", t, st);
  return check_launch("scale");
}

int pasfm_fp32_probe(int device, int packed, double* tflops_out) {
  if (!tflops_out) return fail(PASFM_EINVAL, "NULL output");
  if (packed < 0 || packed > 3) return fail(PASFM_EINVAL, "probe mode %d is not 0..3", packed);
  CUDA_TRY(cudaSetDevice(device));
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  float* out = nullptr;
  CUDA_TRY(cudaMalloc(&out, sizeof(float)));
  const int blocks = sms * 8, iters = 1 << 14, reps = 5;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = fp32_probe_launch(packed, blocks, iters, out, nullptr);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(a, nullptr);
  for (int r = 0; e == cudaSuccess && r < reps; ++r) e = fp32_probe_launch(packed, blocks, iters, out, nullptr);
  if (e == cudaSuccess) e = cudaEventRecord(b, nullptr);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) return fail(PASFM_ECUDA, "fp32 probe: %s", cudaGetErrorString(e));
  *tflops_out = reps * fp32_probe_flops(blocks, iters, packed) / (ms * 1e-3) / 1e12;
  return PASFM_OK;
}

int pasfm_smem_probe(int device, double* tbs_out) {
  if (!tbs_out) return fail(PASFM_EINVAL, "NULL output");
  CUDA_TRY(cudaSetDevice(device));
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  float* out = nullptr;
  CUDA_TRY(cudaMalloc(&out, sizeof(float)));
  const int blocks = sms * 3, iters = 1 << 14, reps = 5;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = smem_probe_launch(blocks, iters, out, nullptr);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(a, nullptr);
  for (int r = 0; e == cudaSuccess && r < reps; ++r) e = smem_probe_launch(blocks, iters, out, nullptr);
  if (e == cudaSuccess) e = cudaEventRecord(b, nullptr);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) return fail(PASFM_ECUDA, "shared-memory probe: %s", cudaGetErrorString(e));
  *tbs_out = reps * smem_probe_bytes(blocks, iters) / (ms * 1e-3) / 1e12;
  return PASFM_OK;
}

int pasfm_status(pasfm_ctx* ctx, void* stream, uint32_t* bits) {
  if (!ctx) return fail(PASFM_EINVAL, "ctx is NULL");
  TRY(set_device(ctx));
  CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  unsigned v = 0;
  CUDA_TRY(cudaMemcpy(&v, ctx->status, sizeof v, cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(ctx->status, 0, sizeof v));
  if (bits) *bits = v;
  if (v & PASFM_STATUS_TIMEOUT) return fail(PASFM_ETIMEOUT, "a bounded device wait expired (status 0x%x)", v);
  if (v) return fail(PASFM_EDEVICE, "device status 0x%x (element inside the grid or index clamped)", v);
  return PASFM_OK;
}

int pasfm_timing_enable(pasfm_ctx* ctx, int enable) {
  if (!ctx) return fail(PASFM_EINVAL, "ctx is NULL");
  ctx->timing = enable != 0;
  return PASFM_OK;
}

int pasfm_timing_reset(pasfm_ctx* ctx) {
  if (!ctx) return fail(PASFM_EINVAL, "ctx is NULL");
  for (auto& r : ctx->recs) {
    cudaEventSynchronize(r.b);
    ctx->pool.push_back(r.a);
    ctx->pool.push_back(r.b);
  }
  ctx->recs.clear();
  return PASFM_OK;
}

int pasfm_timing_read(pasfm_ctx* ctx, const char* kernel, double* ms_total, int64_t* launches) {
  if (!ctx || !kernel) return fail(PASFM_EINVAL, "NULL argument");
  double ms = 0.0;
  int64_t n = 0;
  for (auto& r : ctx->recs) {
    if (std::strcmp(kernel, "*") != 0 && std::strcmp(kernel, r.name) != 0) continue;
    CUDA_TRY(cudaEventSynchronize(r.b));
    float t = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
    ms += t;
    ++n;
  }
  if (ms_total) *ms_total = ms;
  if (launches) *launches = n;
  return PASFM_OK;
}

int64_t pasfm_launch_count(pasfm_ctx* ctx) { return ctx ? ctx->launches : -1; }

}  // extern "C"

namespace pasfm {

// Geometry validation and planning for entry points defined in other
// translation units (the allocation-free pose gradient in noalloc.cu).
int plan_geometry(const pasfm_geom* geom, Plan* pl) {
  Geo G;
  TRY(check_geom(geom, &G));
  TRY(make_plan(G, pl));
  return PASFM_OK;
}

// Record an error message for pasfm_last_error() from another translation unit.
int report_error(int code, const char* msg) { return fail(code, "%s", msg); }

}  // namespace pasfm
