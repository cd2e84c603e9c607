// Autotuner for the launch shapes of one grid and field count.
//
// On the first solve with a given number of fields the tuner times, with CUDA events on
// the workspace, every candidate of one tunable at a time (the others at their current
// choice): fields per ring-DFT CTA, fields per inverse-DFT CTA, the FP32 Legendre tile
// width, and the BF16x3 analysis pipeline depth.  None of these choices changes any
// summation order, so the tuned launches give bit-identical results; only their speed
// differs.  The winners are cached in the grid per field count.
#include <float.h>

#include <functional>

#include "shot_internal.cuh"

namespace shot {


namespace {

int time_ms(float* out, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, const std::function<int()>& fn) {
  int rc = fn();  // warm-up (also sets any function attributes)
  if (rc) return rc;
  SHOT_CUDA(cudaEventRecord(e0, st));
  for (int r = 0; r < 3; ++r)
    if ((rc = fn())) return rc;
  SHOT_CUDA(cudaEventRecord(e1, st));
  SHOT_CUDA(cudaEventSynchronize(e1));
  SHOT_CUDA(cudaEventElapsedTime(out, e0, e1));
  return SHOT_OK;
}

}  // namespace

// upd: when given (the solver), the inverse DFT is timed in the solver's form (Sinkhorn
// update + forward transform of the new scaling) rather than as a plain transform.
int autotune(Grid& g, int nf, cudaStream_t st, const EpiParams* upd) {
  for (const Tuning& t : g.tuning)
    if (t.nf == nf) {
      g.active = t;
      return SHOT_OK;
    }
  if (profiling_on()) {   // keep profiled runs free of tuning launches
    g.active = Tuning{};
    return SHOT_OK;
  }
  Workspace& w = g.ws;
  Tuning t;
  t.nf = nf;
  g.active = t;
  cudaEvent_t e0, e1;
  SHOT_CUDA(cudaEventCreate(&e0));
  SHOT_CUDA(cudaEventCreate(&e1));
  const size_t n = g.npix;
  // the solver buffers hold no state yet: use the caller-independent workspace only
  float* fld = nullptr;
  cudaError_t ce = cudaMalloc(&fld, (size_t)nf * n * sizeof(float));
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cuda_status(ce, "autotune buffer");
  }
  int rc = SHOT_OK;
  SHOT_CUDA(cudaMemsetAsync(fld, 0, (size_t)nf * n * sizeof(float), st));
  auto pick = [&](int* slot, std::initializer_list<int> cands, const std::function<int()>& fn) -> int {
    float best = FLT_MAX;
    int arg = 0;
    for (int c : cands) {
      *slot = c;
      g.active = t;
      float ms = 0.f;
      int r = time_ms(&ms, st, e0, e1, fn);
      if (r) return r;
      if (ms < best) {
        best = ms;
        arg = c;
      }
    }
    *slot = arg;
    g.active = t;
    return SHOT_OK;
  };
  EpiParams ep{};
  ep.mode = EPI_PLAIN;
  ep.out = fld;
  std::vector<int> fgs;
  for (int fg : {1, 2, 4, 8})
    if (fg <= nf && fg * g.nlon <= 6400) fgs.push_back(fg);
  if (fgs.empty()) fgs.push_back(1);
  auto run_fwd = [&]() { return launch_dft_fwd(g, fld, nf, nullptr, 0, w.XY, w.ldc, st); };
  EpiParams ep_upd{};
  if (upd) {
    ep_upd = *upd;
    ep_upd.out = fld;
  }
  // the field group only matters for the non-persistent inverse DFT (plain transforms, the final
  // objective, and the update where the persistent kernel does not apply): tune on that
  const bool inv_upd = upd && !idft_is_persistent(g, nf, ep_upd);
  auto run_inv = [&]() { return launch_idft(g, w.XY, w.ldc, nf, inv_upd ? ep_upd : ep, st); };
  auto run_leg = [&]() { return launch_legendre(g, nf, w.XY, w.C, w.XY, w.ldc, st); };
  auto pick_vec = [&](int* slot, const std::vector<int>& c, const std::function<int()>& fn) -> int {
    float best = FLT_MAX;
    int arg = c[0];
    for (int v : c) {
      *slot = v;
      g.active = t;
      float ms = 0.f;
      int r = time_ms(&ms, st, e0, e1, fn);
      if (r) return r;
      if (ms < best) {
        best = ms;
        arg = v;
      }
    }
    *slot = arg;
    g.active = t;
    return SHOT_OK;
  };
  if (!rc) rc = pick_vec(&t.dft_fg, fgs, run_fwd);
  if (!rc) rc = pick_vec(&t.idft_fg, fgs, run_inv);
  if (!rc && g.mode == SHOT_TABLE && g.precision == SHOT_FP32) rc = pick(&t.simt_bn, {32, 48, 64}, run_leg);
  if (!rc && g.mode == SHOT_TABLE && g.precision == SHOT_BF16X3) rc = pick(&t.tc_stages, {2, 3, 4}, run_leg);
  cudaStreamSynchronize(st);
  cudaFree(fld);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    g.active = Tuning{};
    return rc;
  }
  g.tuning.push_back(t);
  g.active = t;
  return SHOT_OK;
}

}  // namespace shot

extern "C" int shot_grid_autotune(shot_grid gh, int nfields, int* choice, void* stream) {
  using namespace shot;
  Grid* g = reinterpret_cast<Grid*>(gh);
  if (!g || nfields < 1) {
    set_error("shot_grid_autotune: bad argument");
    return SHOT_ERR_INVALID_ARG;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = ensure_workspace(*g, nfields, st);
  if (rc) return rc;
  if ((rc = launch_heat_mult(*g, 0.0, st))) return rc;
  if ((rc = autotune(*g, nfields, st))) return rc;
  if (choice) {
    choice[0] = g->active.dft_fg;
    choice[1] = g->active.idft_fg;
    choice[2] = g->active.simt_bn;
    choice[3] = g->active.tc_stages;
  }
  return SHOT_OK;
}
