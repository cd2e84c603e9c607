// C ABI of the SHOT library (declared in include/shot.h) and the Sinkhorn driver.
//
// The driver runs Algorithm 1 (App. C) for a batch of independent problems.  One
// iteration is:  u-step (K v, then u = p/Kv or (p/Kv)^{tau/(tau+eps)}),  v-step (K u,
// then v likewise),  then the gauge (balanced: s = sum u, u/s, s v) or the
// translation-invariant step (c = tau/2 (log sum a p u^{-eps/tau} - log sum a q v^{-eps/tau}),
// u e^{c/eps}, v e^{-c/eps}).  The rescalings are never applied to the stored buffers
// during the loop: each problem keeps u_true = alpha u_buf and v_true = beta v_buf, and
// the forward ring DFT multiplies v_buf by beta on load.  Every C iterations the relative
// marginal error of App. C.3 is evaluated on the device and problems below tol stop.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "shot_internal.cuh"

namespace shot {

static thread_local std::string t_err;

void set_error(const std::string& msg) { t_err = msg; }

int cuda_status(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? SHOT_ERR_OOM : SHOT_ERR_CUDA;
}

int launch_legendre_simt(const Grid& g, int nf, const float* X, float* C, float* Y, int ldc, cudaStream_t st);
int launch_analysis_simt(const Grid& g, int nf, const float* X, float* C, int ldc, bool apply_h, cudaStream_t st);
int launch_synthesis_simt(const Grid& g, int nf, const float* C, float* Y, int ldc, cudaStream_t st);

int launch_legendre(const Grid& g, int nf, const float* X, float* C, float* Y, int ldc, cudaStream_t st) {
  if (g.precision == SHOT_FP32) return launch_legendre_simt(g, nf, X, C, Y, ldc, st);
  return launch_legendre_tc(g, nf, X, nullptr, Y, ldc, true, true, true, st);
}
int launch_analysis_only(const Grid& g, int nf, const float* X, float* C, int ldc, bool apply_h,
                         cudaStream_t st) {
  if (g.precision == SHOT_FP32) return launch_analysis_simt(g, nf, X, C, ldc, apply_h, st);
  return launch_legendre_tc(g, nf, X, C, nullptr, ldc, true, false, apply_h, st);
}
int launch_synthesis_only(const Grid& g, int nf, const float* C, float* Y, int ldc, cudaStream_t st) {
  if (g.precision == SHOT_FP32) return launch_synthesis_simt(g, nf, C, Y, ldc, st);
  int rc = launch_c_to_ct(g, nf, C, ldc, st);
  if (rc) return rc;
  return launch_legendre_tc(g, nf, nullptr, nullptr, Y, ldc, false, true, false, st);
}

namespace {

enum RedMode { RED_U = 0, RED_V = 1, RED_CHECK = 2, RED_FINAL = 3 };

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order reduction of the per-ring-pair partial sums and the per-problem scalar
// steps of Alg. 1 (gauge / TI constant / convergence test / objective).
__global__ void k_reduce(int mode, int nprob, int nh, const double* __restrict__ part, ProbState* ps,
                         int* dev_int, int balanced, double eps, double tau, double tol, int norm_l1) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int kdone = dev_int[0];
  for (int f = wid; f < nprob; f += nw) {
    ProbState* P = ps + f;
    const bool skip = (mode == RED_FINAL) ? (P->status < 0) : (P->active == 0);
    if (skip) continue;
    double s[NPART] = {0.0, 0.0, 0.0, 0.0};
    for (int j = lane; j < nh; j += 32) {
      const double* pt = part + ((size_t)f * nh + j) * NPART;
#pragma unroll
      for (int i = 0; i < NPART; ++i) s[i] += pt[i];
    }
#pragma unroll
    for (int i = 0; i < NPART; ++i) s[i] = wsum(s[i]);
    if (lane != 0) continue;
    if (mode == RED_U || mode == RED_V) {
      if (s[2] > 0.0) {
        P->status = SHOT_ERR_NONPOSITIVE;
        P->active = 0;
        P->iters = kdone + 1;
      } else if (s[3] > 0.0) {
        P->status = SHOT_ERR_NONFINITE;
        P->active = 0;
        P->iters = kdone + 1;
      } else if (mode == RED_U) {
        P->su = s[0];
      } else {
        double al, be;
        if (balanced) {
          al = 1.0 / P->su;
          be = P->su;
        } else {
          const double c = 0.5 * tau * (log(P->su) - log(s[0]));
          al = exp(c / eps);
          be = exp(-c / eps);
        }
        if (!(isfinite(al) && isfinite(be) && al > 0.0 && be > 0.0)) {
          P->status = SHOT_ERR_NONFINITE;
          P->active = 0;
          P->iters = kdone + 1;
        } else {
          P->alpha = al;
          P->beta = be;
        }
      }
    } else if (mode == RED_CHECK) {
      const double e = norm_l1 ? s[0] / s[1] : sqrt(s[0] / s[1]);
      P->err = e;
      if (e < tol) {
        P->active = 0;
        P->iters = kdone;
      }
    } else {
      P->err = norm_l1 ? s[0] / s[1] : sqrt(s[0] / s[1]);
      P->mass = s[2];
      P->ot = s[3];
      P->ot_dual = s[3] - eps * s[2];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (mode == RED_V) dev_int[0] = kdone + 1;
    int na = 0;
    for (int f = 0; f < nprob; ++f) na += ps[f].active;
    dev_int[1] = na;
  }
}

__global__ void k_init_probs(int nprob, ProbState* ps, int* dev_int) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < nprob) {
    ProbState P;
    P.alpha = 1.0;
    P.beta = 1.0;
    P.su = 0.0;
    P.err = nan("");
    P.ot = P.ot_dual = P.mass = nan("");
    P.active = 1;
    P.status = SHOT_OK;
    P.iters = 0;
    P.pad = 0;
    ps[f] = P;
  }
  if (f == 0) {
    dev_int[0] = 0;
    dev_int[1] = nprob;
  }
}

__global__ void k_fill(float* __restrict__ a, size_t n, float v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a[i] = v;
}

// mass m(p) = sum_i a_i p_i of every listed field (FP64), one block per field
__global__ void k_field_mass(const float* const* __restrict__ fl, int nlat, int nlon,
                             const float* __restrict__ a_ring, double* __restrict__ out) {
  __shared__ double red[32];
  const float* f = fl[blockIdx.x];
  double s = 0.0;
  for (size_t i = threadIdx.x; i < (size_t)nlat * nlon; i += blockDim.x)
    s += (double)a_ring[i / nlon] * (double)f[i];
  s = wsum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[blockIdx.x] = t;
  }
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

Grid* as_grid(shot_grid g) { return reinterpret_cast<Grid*>(g); }

int heat_pipeline(Grid& g, const float* in, int nf, int scale_which, cudaStream_t st) {
  Workspace& w = g.ws;
  int rc = launch_dft_fwd(g, in, nf, reinterpret_cast<ProbState*>(w.probs), scale_which, w.XY, w.ldc, st);
  if (rc) return rc;
  return launch_legendre(g, nf, w.XY, w.C, w.XY, w.ldc, st);
}

int reduce(Grid& g, int mode, int nprob, const EpiParams& ep, double tol, cudaStream_t st) {
  ProfScope prof(PK_OTHER, st);
  count_launch();
  k_reduce<<<1, 256, 0, st>>>(mode, nprob, g.nh, g.ws.part, reinterpret_cast<ProbState*>(g.ws.probs),
                              g.ws.dev_int, ep.balanced, ep.eps, ep.tau, tol, ep.norm_l1);
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

struct SolveOut {
  std::vector<ProbState> ps;
  int kdone = 0;
};

// Algorithm 1 on nprob problems with marginal lists P (first) and Q (second).
int run_sinkhorn(Grid& g, const std::vector<const float*>& P, const std::vector<const float*>& Q, double eps,
                 double tau, int T, double tol, int C, int flags, float* u, float* v, cudaStream_t st,
                 SolveOut& out) {
  const int nprob = (int)P.size();
  int rc = ensure_workspace(g, nprob, st);
  if (rc) return rc;
  Workspace& w = g.ws;
  const size_t n = (size_t)g.nlat * g.nlon;
  std::vector<const float*> lists(4 * (size_t)nprob);
  for (int i = 0; i < nprob; ++i) {
    lists[i] = P[i];
    lists[nprob + i] = Q[i];
  }
  SHOT_CUDA(cudaMemcpyAsync(w.marg, lists.data(), 2 * nprob * sizeof(float*), cudaMemcpyHostToDevice, st));
  ProbState* ps = reinterpret_cast<ProbState*>(w.probs);
  count_launch();
  k_init_probs<<<(nprob + 127) / 128, 128, 0, st>>>(nprob, ps, w.dev_int);
  if (!(flags & SHOT_FLAG_WARM_START)) {
    count_launch(2);
    k_fill<<<1024, 256, 0, st>>>(u, n * nprob, 1.f);
    k_fill<<<1024, 256, 0, st>>>(v, n * nprob, 1.f);
  }
  SHOT_CUDA(cudaGetLastError());
  rc = launch_heat_mult(g, eps / 4.0, st);
  if (rc) return rc;

  EpiParams ep{};
  ep.ps = ps;
  ep.part = w.part;
  ep.balanced = isinf(tau) ? 1 : 0;
  ep.gamma = ep.balanced ? 1.f : (float)(tau / (tau + eps));
  ep.eps_over_taueps = ep.balanced ? 0.f : (float)(eps / (tau + eps));
  ep.eps = eps;
  ep.tau = tau;
  ep.norm_l1 = (flags & SHOT_FLAG_NORM_L1) ? 1 : 0;
  const float* const* margP = w.marg;
  const float* const* margQ = w.marg + nprob;

  int k = 0;
  for (k = 1; k <= T; ++k) {
    // u-step: u = p / K(beta v)
    if ((rc = heat_pipeline(g, v, nprob, 1, st))) return rc;
    ep.mode = EPI_UPDATE;
    ep.out = u;
    ep.marg = margP;
    ep.which = 0;
    if ((rc = launch_idft(g, w.XY, w.ldc, nprob, ep, st))) return rc;
    if ((rc = reduce(g, RED_U, nprob, ep, tol, st))) return rc;
    // v-step: v = q / K u
    if ((rc = heat_pipeline(g, u, nprob, 0, st))) return rc;
    ep.out = v;
    ep.marg = margQ;
    ep.which = 1;
    if ((rc = launch_idft(g, w.XY, w.ldc, nprob, ep, st))) return rc;
    if ((rc = reduce(g, RED_V, nprob, ep, tol, st))) return rc;
    if (C > 0 && k % C == 0) {
      if ((rc = heat_pipeline(g, v, nprob, 1, st))) return rc;
      ep.mode = EPI_CHECK;
      ep.other = u;
      ep.marg = margP;
      if ((rc = launch_idft(g, w.XY, w.ldc, nprob, ep, st))) return rc;
      if ((rc = reduce(g, RED_CHECK, nprob, ep, tol, st))) return rc;
      SHOT_CUDA(cudaMemcpyAsync(w.host_int, w.dev_int, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
      SHOT_CUDA(cudaStreamSynchronize(st));
      if (w.host_int[1] == 0) break;
    }
  }
  out.kdone = k > T ? T : k;
  // final K v_true for the objective, mass and marginal error; writes u_true, v_true
  if ((rc = heat_pipeline(g, v, nprob, 1, st))) return rc;
  ep.mode = EPI_FINAL;
  ep.out = v;
  ep.other = u;
  ep.marg = margP;
  ep.marg2 = margQ;
  if ((rc = launch_idft(g, w.XY, w.ldc, nprob, ep, st))) return rc;
  if ((rc = reduce(g, RED_FINAL, nprob, ep, tol, st))) return rc;
  out.ps.resize(nprob);
  SHOT_CUDA(cudaMemcpyAsync(w.host_probs, ps, nprob * sizeof(ProbState), cudaMemcpyDeviceToHost, st));
  SHOT_CUDA(cudaMemcpyAsync(w.host_int, w.dev_int, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
  SHOT_CUDA(cudaStreamSynchronize(st));
  memcpy(out.ps.data(), w.host_probs, nprob * sizeof(ProbState));
  if (w.host_int[4] != 0) {
    SHOT_CUDA(cudaMemsetAsync(w.dev_int + 4, 0, sizeof(int), st));
    set_error("a bounded device-side wait expired in a tensor-core kernel");
    return SHOT_ERR_TIMEOUT;
  }
  for (auto& p : out.ps) {
    if (p.status == SHOT_OK && p.active) {
      p.iters = w.host_int[0];
      if (tol > 0) p.status = SHOT_WARN_NOT_CONVERGED;
    }
    if (p.status < 0) p.ot = p.ot_dual = p.mass = p.err = nan("");
  }
  return SHOT_OK;
}

int worst_status(const std::vector<ProbState>& ps) {
  int w = SHOT_OK;
  for (auto& p : ps) {
    if (p.status < 0 && (w >= 0 || p.status < w)) w = p.status;
    else if (w >= 0 && p.status > w) w = p.status;
  }
  return w;
}

bool finite_pos(double x) { return x > 0.0 && isfinite(x); }

}  // namespace
}  // namespace shot

using namespace shot;

extern "C" {

int shot_last_error(char* buf, int len) {
  const int n = (int)t_err.size();
  if (buf && len > 0) {
    const int c = n < len - 1 ? n : len - 1;
    memcpy(buf, t_err.data(), c);
    buf[c] = 0;
  }
  return n;
}

int shot_grid_init(shot_grid* out, int nlat, int nlon, int lmax, int precision, int legendre_mode,
                   void* stream) {
  if (!out) { set_error("out is NULL"); return SHOT_ERR_INVALID_ARG; }
  *out = nullptr;
  if (lmax == -1) lmax = nlat - 1;
  if (nlat < 2 || lmax < 0 || lmax > nlat - 1 || nlon < 2 * lmax + 1) {
    set_error("need nlat >= 2, 0 <= lmax <= nlat-1, nlon >= 2*lmax+1");
    return SHOT_ERR_INVALID_ARG;
  }
  if (precision != SHOT_FP32 && precision != SHOT_BF16X3) { set_error("unknown precision"); return SHOT_ERR_INVALID_ARG; }
  if (legendre_mode != SHOT_TABLE) { set_error("unknown legendre_mode"); return SHOT_ERR_INVALID_ARG; }
  FftPlan plan;
  if (!make_fft_plan(nlon, &plan)) { set_error("nlon must factor into 2, 3 and 5"); return SHOT_ERR_UNSUPPORTED; }
  Grid* g = new Grid;
  g->nlat = nlat;
  g->nlon = nlon;
  g->lmax = lmax;
  g->nh = (nlat + 1) / 2;
  g->precision = precision;
  g->mode = legendre_mode;
  g->plan = plan;
  cudaGetDevice(&g->dev);
  int rc = build_grid_tables(*g, as_stream(stream));
  if (rc) {
    shot_grid_free(reinterpret_cast<shot_grid>(g));
    return rc;
  }
  *out = reinterpret_cast<shot_grid>(g);
  return SHOT_OK;
}

int shot_grid_free(shot_grid gh) {
  Grid* g = as_grid(gh);
  if (!g) return SHOT_OK;
  void* dptr[] = {g->x_d, g->w_d, g->a_d, g->tw_d, g->h_d, g->tab, g->tab_hi, g->tab_lo, g->tabT_hi, g->tabT_lo,
                  g->ws.ct_hi, g->ws.ct_lo, g->M_d,
                  g->row_off_d, g->tiles_ana, g->tiles_syn, g->ws.XY, g->ws.C, g->ws.part, g->ws.probs,
                  g->ws.marg, g->ws.ubuf, g->ws.vbuf, g->ws.dev_int};
  for (void* p : dptr)
    if (p) cudaFree(p);
  if (g->ws.host_int) cudaFreeHost(g->ws.host_int);
  if (g->ws.host_probs) cudaFreeHost(g->ws.host_probs);
  delete g;
  return SHOT_OK;
}

int shot_grid_info(shot_grid gh, int* nlat, int* nlon, int* lmax, int* precision, int* legendre_mode) {
  Grid* g = as_grid(gh);
  if (!g) { set_error("grid is NULL"); return SHOT_ERR_INVALID_ARG; }
  if (nlat) *nlat = g->nlat;
  if (nlon) *nlon = g->nlon;
  if (lmax) *lmax = g->lmax;
  if (precision) *precision = g->precision;
  if (legendre_mode) *legendre_mode = g->mode;
  return SHOT_OK;
}

int shot_grid_nodes(shot_grid gh, double* x, double* w, double* a_ring) {
  Grid* g = as_grid(gh);
  if (!g) { set_error("grid is NULL"); return SHOT_ERR_INVALID_ARG; }
  for (int j = 0; j < g->nlat; ++j) {
    if (x) x[j] = g->x[j];
    if (w) w[j] = g->w[j];
    if (a_ring) a_ring[j] = g->a_ring[j];
  }
  return SHOT_OK;
}

int shot_grid_reserve(shot_grid gh, int nfields) {
  Grid* g = as_grid(gh);
  if (!g || nfields < 1) { set_error("bad grid or nfields"); return SHOT_ERR_INVALID_ARG; }
  return ensure_workspace(*g, nfields, 0);
}

int shot_heat_apply(shot_grid gh, double t, const float* in, float* out, int nfields, void* stream) {
  Grid* g = as_grid(gh);
  if (!g || !in || !out || nfields < 1 || !(t >= 0.0) || in == out) {
    set_error("shot_heat_apply: bad argument");
    return SHOT_ERR_INVALID_ARG;
  }
  cudaStream_t st = as_stream(stream);
  int rc = ensure_workspace(*g, nfields, st);
  if (rc) return rc;
  if ((rc = launch_heat_mult(*g, t, st))) return rc;
  if ((rc = heat_pipeline(*g, in, nfields, 0, st))) return rc;
  EpiParams ep{};
  ep.mode = EPI_PLAIN;
  ep.out = out;
  return launch_idft(*g, g->ws.XY, g->ws.ldc, nfields, ep, st);
}

int shot_sht_analysis(shot_grid gh, const float* in, float* coeffs, int nfields, void* stream) {
  Grid* g = as_grid(gh);
  if (!g || !in || !coeffs || nfields < 1) { set_error("shot_sht_analysis: bad argument"); return SHOT_ERR_INVALID_ARG; }
  cudaStream_t st = as_stream(stream);
  int rc = ensure_workspace(*g, nfields, st);
  if (rc) return rc;
  Workspace& w = g->ws;
  if ((rc = launch_dft_fwd(*g, in, nfields, nullptr, 0, w.XY, w.ldc, st))) return rc;
  if ((rc = launch_analysis_only(*g, nfields, w.XY, w.C, w.ldc, false, st))) return rc;
  return launch_coeff_gather(*g, w.C, w.ldc, nfields, coeffs, st);
}

int shot_sht_synthesis(shot_grid gh, const float* coeffs, float* out, int nfields, void* stream) {
  Grid* g = as_grid(gh);
  if (!g || !coeffs || !out || nfields < 1) { set_error("shot_sht_synthesis: bad argument"); return SHOT_ERR_INVALID_ARG; }
  cudaStream_t st = as_stream(stream);
  int rc = ensure_workspace(*g, nfields, st);
  if (rc) return rc;
  Workspace& w = g->ws;
  if ((rc = launch_coeff_scatter(*g, coeffs, nfields, w.C, w.ldc, st))) return rc;
  if ((rc = launch_synthesis_only(*g, nfields, w.C, w.XY, w.ldc, st))) return rc;
  EpiParams ep{};
  ep.mode = EPI_PLAIN;
  ep.out = out;
  return launch_idft(*g, w.XY, w.ldc, nfields, ep, st);
}

static int check_solver_args(Grid* g, const float* p, const float* q, int batch, double eps, double tau,
                             int max_iter, int check_every) {
  if (!g || !p || !q || batch < 1 || !finite_pos(eps) || !(tau > 0.0) || isnan(tau) || max_iter < 0 ||
      check_every < 0) {
    set_error("solver: bad argument (need grid, p, q, batch >= 1, eps > 0, tau > 0, max_iter >= 0)");
    return SHOT_ERR_INVALID_ARG;
  }
  return SHOT_OK;
}

int shot_sinkhorn(shot_grid gh, const float* p, const float* q, int batch, double eps, double tau,
                  int max_iter, double tol, int check_every, int flags, float* u, float* v, double* ot,
                  double* ot_dual, double* mass_pi, int* iters, float* err, int* status, void* stream) {
  Grid* g = as_grid(gh);
  int rc = check_solver_args(g, p, q, batch, eps, tau, max_iter, check_every);
  if (rc) return rc;
  if (!u || !v) { set_error("u, v are required"); return SHOT_ERR_INVALID_ARG; }
  const size_t n = (size_t)g->nlat * g->nlon;
  std::vector<const float*> P(batch), Q(batch);
  for (int b = 0; b < batch; ++b) {
    P[b] = p + b * n;
    Q[b] = q + b * n;
  }
  SolveOut so;
  rc = run_sinkhorn(*g, P, Q, eps, tau, max_iter, tol, check_every, flags, u, v, as_stream(stream), so);
  if (rc) return rc;
  for (int b = 0; b < batch; ++b) {
    const ProbState& s = so.ps[b];
    if (ot) ot[b] = s.ot;
    if (ot_dual) ot_dual[b] = s.ot_dual;
    if (mass_pi) mass_pi[b] = s.mass;
    if (iters) iters[b] = s.iters;
    if (err) err[b] = (float)s.err;
    if (status) status[b] = s.status;
  }
  return worst_status(so.ps);
}

int shot_divergence(shot_grid gh, const float* p, const float* q, int batch, double eps, double tau,
                    int max_iter, double tol, int check_every, int flags, double* S, double* S_dual,
                    int* status, float* u3, float* v3, double* ot3, int* iters3, void* stream) {
  Grid* g = as_grid(gh);
  int rc = check_solver_args(g, p, q, batch, eps, tau, max_iter, check_every);
  if (rc) return rc;
  if (!S || !status) { set_error("S and status are required"); return SHOT_ERR_INVALID_ARG; }
  cudaStream_t st = as_stream(stream);
  const size_t n = (size_t)g->nlat * g->nlon;
  const int np = 3 * batch;
  if ((rc = ensure_workspace(*g, np, st))) return rc;
  Workspace& w = g->ws;
  if (!u3 || !v3) {
    if (w.uv_cap < (size_t)np * n) {
      SHOT_CUDA(cudaStreamSynchronize(st));
      cudaFree(w.ubuf);
      cudaFree(w.vbuf);
      w.ubuf = w.vbuf = nullptr;
      w.uv_cap = 0;
      SHOT_CUDA(cudaMalloc(&w.ubuf, (size_t)np * n * sizeof(float)));
      SHOT_CUDA(cudaMalloc(&w.vbuf, (size_t)np * n * sizeof(float)));
      w.uv_cap = (size_t)np * n;
    }
    u3 = w.ubuf;
    v3 = w.vbuf;
  }
  std::vector<const float*> P(np), Q(np);
  for (int b = 0; b < batch; ++b) {
    P[b] = p + b * n;          Q[b] = q + b * n;
    P[batch + b] = p + b * n;  Q[batch + b] = p + b * n;
    P[2 * batch + b] = q + b * n;  Q[2 * batch + b] = q + b * n;
  }
  // masses m(p_b), m(q_b)
  std::vector<const float*> fl(2 * batch);
  for (int b = 0; b < batch; ++b) { fl[b] = p + b * n; fl[batch + b] = q + b * n; }
  const float** fl_d = w.marg + 2 * np;   // spare room in the pointer area
  double* mass_d = w.part;                  // part is free before the solve
  SHOT_CUDA(cudaMemcpyAsync(fl_d, fl.data(), 2 * batch * sizeof(float*), cudaMemcpyHostToDevice, st));
  count_launch();
  k_field_mass<<<2 * batch, 256, 0, st>>>(fl_d, g->nlat, g->nlon, g->a_d, mass_d);
  SHOT_CUDA(cudaGetLastError());
  std::vector<double> masses(2 * batch);
  SHOT_CUDA(cudaMemcpyAsync(masses.data(), mass_d, 2 * batch * sizeof(double), cudaMemcpyDeviceToHost, st));
  SHOT_CUDA(cudaStreamSynchronize(st));

  SolveOut so;
  rc = run_sinkhorn(*g, P, Q, eps, tau, max_iter, tol, check_every, flags, u3, v3, st, so);
  if (rc) return rc;
  for (int b = 0; b < batch; ++b) {
    const ProbState &a = so.ps[b], &pp = so.ps[batch + b], &qq = so.ps[2 * batch + b];
    const double dm = masses[b] - masses[batch + b];
    S[b] = a.ot - 0.5 * (pp.ot + qq.ot) + 0.5 * eps * dm * dm;
    if (S_dual) S_dual[b] = a.ot_dual - 0.5 * (pp.ot_dual + qq.ot_dual);
    int s3[3] = {a.status, pp.status, qq.status};
    int ws = SHOT_OK;
    for (int i = 0; i < 3; ++i) {
      if (s3[i] < 0 && (ws >= 0 || s3[i] < ws)) ws = s3[i];
      else if (ws >= 0 && s3[i] > ws) ws = s3[i];
    }
    status[b] = ws;
  }
  for (int i = 0; i < np; ++i) {
    if (ot3) ot3[i] = so.ps[i].ot;
    if (iters3) iters3[i] = so.ps[i].iters;
  }
  return worst_status(so.ps);
}

}  // extern "C"
