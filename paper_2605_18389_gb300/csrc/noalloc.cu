// shot_heat_apply_noalloc: the heat convolution without any device allocation.
//
// Some callers cannot call cudaMalloc at the point where they need a heat convolution:
// code running while another component owns the allocator (a memory pool that must not
// grow, a framework that forbids allocation inside its step, or a section being
// captured into a CUDA graph by someone else), or processes that run under a hard
// device-memory budget fixed at start-up.  For them this entry point runs the same
// kernels as shot_heat_apply but keeps its scratch (the folded ring spectra and the
// Legendre coefficients) in one file-scope __device__ array instead of the grid's
// workspace, which shot_heat_apply may have to grow with cudaMalloc.
//
// The array is SHOT_NOALLOC_SCRATCH_BYTES (8 MiB) and, like every __device__ variable,
// exists on every GPU that loads this library until the process exits.  Host code must
// not use the symbol itself as a device address: on the first call on a device (with
// that device current) cudaGetSymbolAddress resolves the device address, which is then
// cached per device and passed to the kernels.  That first call should therefore come
// before any stream capture that includes this entry point.
//
// All calls share the one array: two calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on it and must be serialised by the caller.  A call
// also writes the grid's heat multipliers h_l for its t (launch_heat_mult), so it races as well
// with any overlapping call on the same grid (shot_heat_apply, a solve), which reads them.
// Every call writes the scratch it reads before reading it (the padding columns of the
// spectra are never read into a stored output), so nothing needs clearing between calls.
#include <mutex>

#include "shot_internal.cuh"

namespace shot {


namespace {

constexpr size_t kScratchBytes = SHOT_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) float g_noalloc_scratch[kScratchBytes / sizeof(float)];

constexpr int kMaxDevices = 64;
float* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

int scratch_for_current_device(float** out) {
  int dev = 0;
  SHOT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("shot_heat_apply_noalloc: device ordinal out of range");
    return SHOT_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(noalloc scratch)");
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SHOT_OK;
}

}  // namespace
}  // namespace shot

extern "C" int shot_heat_apply_noalloc(shot_grid gh, double t, const float* in, float* out, int nfields,
                                       void* stream) {
  using namespace shot;
  Grid* g = reinterpret_cast<Grid*>(gh);
  if (!g || !in || !out || nfields < 1 || !(t >= 0.0) || in == out) {
    set_error("shot_heat_apply_noalloc: bad argument");
    return SHOT_ERR_INVALID_ARG;
  }
  if (g->precision != SHOT_FP32) {
    set_error("shot_heat_apply_noalloc: only SHOT_FP32 grids are supported");
    return SHOT_ERR_UNSUPPORTED;
  }
  const int ldc = (2 * nfields + 3) / 4 * 4;
  const size_t nx = ((size_t)g->nblk * g->nh * ldc + 63) / 64 * 64;  // spectra X (and Y), 256-B padded
  const size_t nc = (size_t)g->rows_total * ldc;                      // coefficients C
  const size_t need = (nx + nc) * sizeof(float);
  if (need > kScratchBytes) {
    set_error("shot_heat_apply_noalloc: grid and nfields need " + std::to_string(need) +
              " bytes of scratch, more than the fixed " + std::to_string(kScratchBytes));
    return SHOT_ERR_INVALID_ARG;
  }
  float* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  float* X = scratch;
  float* C = scratch + nx;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if ((rc = launch_heat_mult(*g, t, st))) return rc;
  if ((rc = launch_dft_fwd(*g, in, nfields, nullptr, 0, X, ldc, st))) return rc;
  if ((rc = launch_legendre(*g, nfields, X, C, X, ldc, st))) return rc;
  EpiParams ep{};
  ep.mode = EPI_PLAIN;
  ep.out = out;
  return launch_idft(*g, X, ldc, nfields, ep, st);
}
