// Allocation-free pose gradient: pasfm_pose_grad_noalloc.
//
// Some callers cannot ask the CUDA runtime for device memory while they run:
// code embedded in a host application whose device memory is owned by a
// fixed pool that forbids allocations outside it, or a real-time loop where the
// latency and implicit device synchronisation of cudaMalloc / cudaFree are not
// acceptable.  This entry point serves them: it computes exactly what
// pasfm_pose_grad computes, with the same kernels, but its scratch (element
// positions, per-cube partial element gradients, element gradients when the
// caller does not want them, and a status word) lives in one file-scope
// __device__ array of PASFM_NOALLOC_SCRATCH_BYTES that every GPU loading the
// library holds until the process exits.  No context is needed and nothing
// is allocated.
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "aux.cuh"
#include "kernels.cuh"

namespace pasfm {
int plan_geometry(const pasfm_geom* geom, Plan* pl);
void set_bwd_profile(const Plan& pl, BwdParams* P);
int report_error(int code, const char* msg);
}  // namespace pasfm

using namespace pasfm;

namespace {

constexpr size_t kStatusBytes = 256;  // status word, padded to keep the rest 256-byte aligned

// The shared scratch.  Host code sees only a stand-in symbol; the device
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PASFM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once per device).
int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return report_error(PASFM_ECUDA, "pasfm_pose_grad_noalloc: no usable current CUDA device");
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return report_error(PASFM_ECUDA, "pasfm_pose_grad_noalloc: cudaGetSymbolAddress of the scratch failed");
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PASFM_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
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

// This entry point has no context status word to report through, so a device-side
// failure recorded in the scratch status word (a staged-copy wait that ran out, which
// leaves per-cube partials unwritten; an element inside the pulse support of the grid;
// a clamped sample index) turns the outputs into NaN, which the caller can test.
__global__ void noalloc_report_kernel(const unsigned* __restrict__ status, double* __restrict__ grad6, int64_t n6,
                                      double* __restrict__ gelem, int64_t nelem) {
  if (*status == 0u) return;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int64_t i = threadIdx.x; i < n6; i += blockDim.x) grad6[i] = nan;
  if (gelem)
    for (int64_t i = threadIdx.x; i < nelem; i += blockDim.x) gelem[i] = nan;
}

int launch_ok(const char* what) {
  const cudaError_t e = cudaPeekAtLastError();
  if (e == cudaSuccess) return PASFM_OK;
  cudaGetLastError();
  return report_error(PASFM_ECUDA, what);
}

}  // namespace

extern "C" int pasfm_pose_grad_noalloc(const pasfm_geom* geom, const void* p0, const double* elem,
                                       const double* pose, const void* g, const uint8_t* mask, double* grad6_out,
                                       double* gelem_out, void* stream) {
  Plan pl;
  int rc = plan_geometry(geom, &pl);
  if (rc != PASFM_OK) return rc;
  const int F = geom->n_frames, E = geom->n_elem, Nt = geom->n_samples;
  const int64_t rows = int64_t(F) * E;
  const int64_t nvox = int64_t(geom->nx) * geom->ny * geom->nz;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (F == 0) return PASFM_OK;
  if (!grad6_out) return report_error(PASFM_EINVAL, "pasfm_pose_grad_noalloc: grad6_out is NULL");
  if (rows == 0 || nvox == 0 || Nt == 0) {
    if (cudaMemsetAsync(grad6_out, 0, size_t(F) * 48, st) != cudaSuccess ||
        (gelem_out && rows && cudaMemsetAsync(gelem_out, 0, size_t(rows) * 24, st) != cudaSuccess)) {
      cudaGetLastError();
      return report_error(PASFM_ECUDA, "pasfm_pose_grad_noalloc: cudaMemsetAsync failed");
    }
    return PASFM_OK;
  }
  if (!p0 || !elem || !pose || !g) return report_error(PASFM_EINVAL, "pasfm_pose_grad_noalloc: NULL array");

  // scratch layout: [status | xw F*E*3 | gpart F*E*ncubes*3 | G F*E*3 (only without gelem_out)]
  const size_t xw_bytes = size_t(rows) * 24;
  const size_t gpart_bytes = size_t(rows) * pl.ncubes * 24;
  const size_t G_bytes = gelem_out ? 0 : size_t(rows) * 24;
  const size_t need = kStatusBytes + xw_bytes + gpart_bytes + G_bytes;
  if (need > size_t(PASFM_NOALLOC_SCRATCH_BYTES)) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "pasfm_pose_grad_noalloc: this geometry needs %zu bytes of scratch, more than the fixed %zu; "
             "use pasfm_pose_grad or fewer frames per call",
             need, size_t(PASFM_NOALLOC_SCRATCH_BYTES));
    return report_error(PASFM_EUNSUPPORTED, msg);
  }
  void* base = nullptr;
  rc = scratch_address(&base);
  if (rc != PASFM_OK) return rc;
  unsigned char* sb = static_cast<unsigned char*>(base);
  unsigned* status = reinterpret_cast<unsigned*>(sb);
  double* xw = reinterpret_cast<double*>(sb + kStatusBytes);
  double* gpart = reinterpret_cast<double*>(sb + kStatusBytes + xw_bytes);
  double* Gm = gelem_out ? gelem_out : reinterpret_cast<double*>(sb + kStatusBytes + xw_bytes + gpart_bytes);

  // only the status word must start at zero; every other scratch byte used is written before it is
  // read, unless a kernel records a failure there, in which case the outputs become NaN (below)
  if (cudaMemsetAsync(status, 0, sizeof(unsigned), st) != cudaSuccess) {
    cudaGetLastError();
    return report_error(PASFM_ECUDA, "pasfm_pose_grad_noalloc: cudaMemsetAsync failed");
  }

  const double hix = geom->ox + geom->dx * (geom->nx - 1), hiy = geom->oy + geom->dy * (geom->ny - 1),
               hiz = geom->oz + geom->dz * (geom->nz - 1);
  elem_pos_kernel<<<static_cast<unsigned>((rows + 255) / 256), 256, 0, st>>>(
      elem, pose, xw, F, E, geom->ox, geom->oy, geom->oz, hix, hiy, hiz, pl.sup, status);
  rc = launch_ok("pasfm_pose_grad_noalloc: elem_pos launch failed");
  if (rc != PASFM_OK) return rc;

  CUtensorMap map;
  std::memset(&map, 0, sizeof map);
  int use_tma = 0;
  auto enc = encoder();
  if (enc && geom->dtype_sig == PASFM_F32 && Nt % 4 == 0 && (reinterpret_cast<uintptr_t>(g) & 15u) == 0 &&
      pl.WP <= 256) {
    cuuint64_t dims[2] = {cuuint64_t(Nt), cuuint64_t(rows)};
    cuuint64_t strides[1] = {cuuint64_t(Nt) * 4};
    cuuint32_t box[2] = {cuuint32_t(pl.WP), 1};
    cuuint32_t es[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(g), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
      use_tma = 1;
  }
  BwdParams P{};
  P.xw = xw;
  P.p0 = p0;
  P.g = g;
  P.mask = mask;
  P.vol = nullptr;
  P.gpart = gpart;
  P.dtype_vol = geom->dtype_vol;
  P.dtype_sig = geom->dtype_sig;
  P.nx = geom->nx;
  P.ny = geom->ny;
  P.nz = geom->nz;
  P.ncx = pl.ncx;
  P.ncy = pl.ncy;
  P.E = E;
  P.f_begin = 0;
  P.n_items = static_cast<int>(rows);
  P.n_parts = 1;  // one CTA per cube: no per-part adjoint buffer is needed (pose gradient only)
  P.part_items = static_cast<int>(rows);
  P.vol_parts = nullptr;
  P.Nt = Nt;
  P.WP = pl.WP;
  P.accumulate = 0;
  P.ox = geom->ox;
  P.oy = geom->oy;
  P.oz = geom->oz;
  P.dx = geom->dx;
  P.dy = geom->dy;
  P.dz = geom->dz;
  set_bwd_profile(pl, &P);
  P.use_tma = use_tma;
  P.wait_cycles = kWaitCycles;
  P.status = status;
  const size_t smem = pl.C == 16 ? BwdLayout<16>::total(pl.WP) : BwdLayout<8>::total(pl.WP);
  const cudaError_t e = bwd_launcher(pl.K, pl.S)(pl.C, 2, map, P, dim3(pl.ncubes), smem, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return report_error(PASFM_ECUDA, "pasfm_pose_grad_noalloc: bwd_cube launch failed");
  }
  pose_rows_kernel<<<static_cast<unsigned>((rows + 7) / 8), 256, 0, st>>>(gpart, pl.ncubes, static_cast<int>(rows),
                                                                          0, Gm);
  rc = launch_ok("pasfm_pose_grad_noalloc: pose_rows launch failed");
  if (rc != PASFM_OK) return rc;
  grad6_kernel<<<F, 256, 0, st>>>(xw, Gm, E, grad6_out);
  rc = launch_ok("pasfm_pose_grad_noalloc: grad6 launch failed");
  if (rc != PASFM_OK) return rc;
  noalloc_report_kernel<<<1, 256, 0, st>>>(status, grad6_out, int64_t(F) * 6, gelem_out, rows * 3);
  return launch_ok("pasfm_pose_grad_noalloc: status report launch failed");
}
