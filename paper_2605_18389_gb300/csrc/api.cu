// C ABI of the SHOT library (declared in include/shot.h) and the host side of the Sinkhorn solver.
//
// The host-side solver runs Algorithm 1 (App. C) for a batch of independent problems.  One
// iteration is:  u-step (K v, then u = p/Kv or (p/Kv)^{tau/(tau+eps)}),  v-step (K u,
// then v likewise),  then the gauge (balanced: s = sum u, u/s, s v) or the
// translation-invariant step (c = tau/2 (log sum a p u^{-eps/tau} - log sum a q v^{-eps/tau}),
// u e^{c/eps}, v e^{-c/eps}).  The rescalings are never applied to the stored buffers
// during the loop: each problem keeps u_true = e^{la} u_buf and v_true = e^{lb} v_buf with
// la, lb in FP64, and every half-step transforms the unscaled buffer of the other side, so
// that no FP32 quantity carries a factor e^{phi/eps}.  The update multiplies its ratio by
// an FP32 factor (ru, rv) that holds the buffer's mean level near 1; its exact effect goes
// into la or lb.  Every C iterations the relative marginal error of App. C.3 is evaluated
// on the device and problems below tol stop.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include <cstdlib>

#include "shot_internal.cuh"

extern "C" int shot_launch_count(long long* n);

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
  // TF32X3 grids run the tensor-core kernels in both Legendre modes (table or checkpoints), and
  // BF16X3 grids in recurrence mode run the same recurrence kernels
  if (tf32_kernels(g)) return launch_legendre_tf32(g, nf, X, nullptr, Y, ldc, true, true, true, st);
  if (g.mode == SHOT_RECURRENCE) return launch_legendre_rec(g, nf, X, C, Y, ldc, true, true, true, st);
  if (g.precision == SHOT_FP32) return launch_legendre_simt(g, nf, X, C, Y, ldc, st);
  return launch_legendre_tc(g, nf, X, nullptr, Y, ldc, true, true, true, st);
}
int launch_analysis_only(const Grid& g, int nf, const float* X, float* C, int ldc, bool apply_h,
                         cudaStream_t st) {
  if (tf32_kernels(g)) return launch_legendre_tf32(g, nf, X, C, nullptr, ldc, true, false, apply_h, st);
  if (g.mode == SHOT_RECURRENCE) return launch_legendre_rec(g, nf, X, C, nullptr, ldc, true, false, apply_h, st);
  if (g.precision == SHOT_FP32) return launch_analysis_simt(g, nf, X, C, ldc, apply_h, st);
  return launch_legendre_tc(g, nf, X, C, nullptr, ldc, true, false, apply_h, st);
}
int launch_synthesis_only(const Grid& g, int nf, const float* C, float* Y, int ldc, cudaStream_t st) {
  if (tf32_kernels(g)) {
    const int rc = launch_c_to_ct32(g, nf, C, ldc, st);
    if (rc) return rc;
    return launch_legendre_tf32(g, nf, nullptr, nullptr, Y, ldc, false, true, false, st);
  }
  if (g.mode == SHOT_RECURRENCE) return launch_legendre_rec(g, nf, nullptr, const_cast<float*>(C), Y, ldc, false, true,
                                                            false, st);
  if (g.precision == SHOT_FP32) return launch_synthesis_simt(g, nf, C, Y, ldc, st);
  int rc = launch_c_to_ct(g, nf, C, ldc, st);
  if (rc) return rc;
  return launch_legendre_tc(g, nf, nullptr, nullptr, Y, ldc, false, true, false, st);
}

namespace {

enum RedMode { RED_U = 0, RED_V = 1, RED_CHECK = 2, RED_FINAL = 3, RED_S = 4 };

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order reduction of the per-ring-pair partial sums and the per-problem scalar
// steps of Alg. 1 (gauge / TI constant / convergence test / objective).  One block per
// problem; the last block to finish (ticket in dev_int[12], reset by that block) counts
// the problems still active and advances the iteration counter.
constexpr int kRedThreads = 128;
constexpr double kLn2 = 0.69314718055994530942;

__global__ void __launch_bounds__(kRedThreads) k_reduce(int mode, int nprob, int nh, const double* __restrict__ part,
                                                        ProbState* ps, int* dev_int, double eps, double tol,
                                                        int norm_l1, double lnpix) {
  __shared__ double red[kRedThreads / 32][NPART];
  __shared__ int last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int f = blockIdx.x;
  const int kdone = dev_int[0];
  ProbState* P = ps + f;
  const bool skip = (mode == RED_FINAL) ? (P->status < 0) : (P->active == 0);
  if (!skip) {
    double s[NPART] = {0.0, 0.0, 0.0, 0.0};
    const double4* pf = reinterpret_cast<const double4*>(part + (size_t)f * nh * NPART);
    for (int j = threadIdx.x; j < nh; j += kRedThreads) {
      const double4 a = pf[j];
      s[0] += a.x;
      s[1] += a.y;
      s[2] += a.z;
      s[3] += a.w;
    }
#pragma unroll
    for (int i = 0; i < NPART; ++i) s[i] = wsum(s[i]);
    if (lane == 0)
#pragma unroll
      for (int i = 0; i < NPART; ++i) red[wid][i] = s[i];
    __syncthreads();
    if (wid == 0) {
      // every lane of warp 0 forms the totals; the scalar step runs on its lanes so that the
      // FP64 logarithms (and exponentials) of one step run side by side, one per lane
#pragma unroll
      for (int i = 0; i < NPART; ++i) {
        double t = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) t += red[w][i];
        s[i] = t;
      }
      if (mode == RED_S) {   // symmetric self-term step: breakdown flags only (no gauge)
        if (lane == 0 && (s[2] > 0.0 || s[3] > 0.0)) {
          P->status = s[2] > 0.0 ? SHOT_ERR_NONPOSITIVE : SHOT_ERR_NONFINITE;
          P->active = 0;
          P->iters = kdone + 1;
        }
      } else if (mode == RED_U || mode == RED_V) {
        const int bal = P->balanced;
        int st = SHOT_OK;
        if (s[2] > 0.0) st = SHOT_ERR_NONPOSITIVE;
        else if (s[3] > 0.0) st = SHOT_ERR_NONFINITE;
        // the new buffer w_buf = (r m / K x_buf)^gamma of this half-step relates to the true
        // scaling (m / K x_true)^gamma, x_true = e^{lx} x_buf, by w_true = e^{lw} w_buf;
        // r = 2^e, so log r is exact
        const double lx = log(lane == 0 ? s[0] : (lane == 1 ? (bal ? s[0] : s[1]) : 1.0));
        const double lsum = __shfl_sync(0xffffffffu, lx, 0), ltot = __shfl_sync(0xffffffffu, lx, 1);
        const double gam = (double)P->gamma;
        const int e = (mode == RED_U) ? P->eu : P->ev;
        const double lw = -gam * ((mode == RED_U ? P->lb : P->la) + e * kLn2);
        // v-step: the plan mass m(pi) = sum a u (K v) = sum a v (K u) (K is self-adjoint in the
        // area inner product), from the new v buffer and the K u it divided by:
        // sum a v_true (K u_true) = e^{lw + la} sum a v_buf (K u_buf), kept by the gauge and the
        // translation-invariant step (they keep the product u v).  Unbalanced, the
        // translation-invariant sum is s[0] = sum a v_buf (K u_buf) / r.  Balanced,
        // v_true (K u_true) = q node by node and the final pass sums a q (mass_v = 0 marks it).
        const double mv = (mode == RED_V && !bal) ? exp(lw + P->la) * ldexp(s[0], e) : 0.0;
        // log of the step's sum over true values: sum w_true (balanced gauge) or
        // sum a m w_true^{-eps/tau} (translation-invariant step)
        const double ls = bal ? lw + lsum : -(eps / P->tau) * lw + lsum;
        // buffer level L = log mean w_buf.  The factors r only keep the FP32 buffers near
        // level 0 (exactness comes from lw): a half-step's level is about
        // gamma (log r + A - L_other) with A a slowly varying term of the marginal's and the
        // kernel's shapes, so each half-step estimates A from what it just produced and the
        // other side's factor is set as soon as the level it will divide by is known.
        const double L = ltot - lnpix;
        const double A = L / gam - e * kLn2 + (mode == RED_U ? P->lvv : P->lvu);
        const double zr = ((mode == RED_U ? P->qv : P->qu) + L) / kLn2;
        const int en = (int)fmin(fmax(rint(zr), -100.0), 100.0);
        if (st == SHOT_OK && !(isfinite(lw) && isfinite(ls) && isfinite(L))) st = SHOT_ERR_NONFINITE;
        double la = P->la, lb = lw;
        if (mode == RED_V) {
          if (bal) {   // u / sum u, v sum u
            la -= P->lsu;
            lb += P->lsu;
          } else {     // c = tau/2 (log su - log sv): u e^{c/eps}, v e^{-c/eps}
            const double c = 0.5 * P->tau * (P->lsu - ls);
            la += c / eps;
            lb -= c / eps;
          }
        }
        // e^{la+lb}, e^{la}, e^{lb} side by side on lanes 0..2
        const double ey = (mode == RED_V) ? exp(lane == 0 ? la + lb : (lane == 1 ? la : (lane == 2 ? lb : 0.0)))
                                          : 0.0;
        const double euv = __shfl_sync(0xffffffffu, ey, 0), eu = __shfl_sync(0xffffffffu, ey, 1),
                     ev = __shfl_sync(0xffffffffu, ey, 2);
        const float cuv = (float)euv;
        if (mode == RED_V && st == SHOT_OK && !(isfinite(la) && isfinite(lb) && cuv > 0.f && cuv < INFINITY))
          st = SHOT_ERR_NONFINITE;
        if (lane == 0) {
          if (st != SHOT_OK) {
            P->status = st;
            P->active = 0;
            P->iters = kdone + 1;
          } else if (mode == RED_U) {
            P->la = lw;
            P->lsu = ls;
            P->qu = -A;      // next u-step: log ru = -A + (level of the v buffer it divides by)
            P->lvu = L;
            P->ev = en;      // this iteration's v-step divides by this u buffer
            P->rv = ldexpf(1.f, en);
          } else {
            P->la = la;
            P->lb = lb;
            P->qv = -A;
            P->lvv = L;
            P->eu = en;
            P->ru = ldexpf(1.f, en);
            P->cuv = cuv;
            P->cu = (float)eu;
            P->cv = (float)ev;
            P->mass_v = mv;
          }
        }
      } else if (lane == 0) {
        if (mode == RED_CHECK) {
          const double e = norm_l1 ? s[0] / s[1] : sqrt(s[0] / s[1]);
          P->err = e;
          if (e < tol) {
            P->active = 0;
            P->iters = kdone;
          }
        } else {
          P->err = norm_l1 ? s[0] / s[1] : sqrt(s[0] / s[1]);
          // m(pi) from the last v-update when there was one (the same quantity as
          // sum a u (K v) of this pass, without the FP32 error of the final K v); balanced, the
          // pass summed a q (see the epilogue)
          const double m = (P->balanced || isnan(P->mass_v)) ? s[2] : P->mass_v;
          P->mass = m;
          P->ot = s[3];
          P->ot_dual = s[3] - eps * m;
        }
      }
    }
  }
  // last block: count the active problems (all blocks' updates are visible after the fence)
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(&dev_int[12], 1) == nprob - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  int na = 0;
  for (int g = threadIdx.x; g < nprob; g += kRedThreads) na += *(volatile int*)&ps[g].active;
  na = __reduce_add_sync(0xffffffffu, na);
  __shared__ int wna[kRedThreads / 32];
  if (lane == 0) wna[wid] = na;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kRedThreads / 32; ++w) t += wna[w];
    if (mode == RED_V || mode == RED_S) dev_int[0] = kdone + 1;
    dev_int[1] = t;
    dev_int[12] = 0;
  }
}

// per-problem state: tau (INFINITY = balanced) from taus[f], gamma = tau/(tau+eps)
__global__ void k_init_probs(int nprob, ProbState* ps, int* dev_int, const double* __restrict__ taus, double eps) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < nprob) {
    ProbState P;
    P.la = P.lb = P.lsu = 0.0;
    P.qu = P.qv = P.lvu = P.lvv = 0.0;
    P.eu = P.ev = 0;
    P.beta = 1.0;
    P.ru = P.rv = P.cuv = P.cu = P.cv = 1.f;
    P.err = nan("");
    P.ot = P.ot_dual = P.mass = P.mass_v = nan("");
    const double tau = taus[f];
    P.tau = tau;
    P.balanced = isinf(tau) ? 1 : 0;
    P.gamma = P.balanced ? 1.f : (float)(tau / (tau + eps));
    P.et = P.balanced ? 0.f : (float)(eps / (tau + eps));
    P.active = 1;
    P.status = SHOT_OK;
    P.iters = 0;
    ps[f] = P;
  }
  if (f == 0) {
    dev_int[0] = 0;
    dev_int[1] = nprob;
    dev_int[12] = 0;   // k_reduce's ticket
  }
}

__global__ void k_fill(float* __restrict__ a, size_t n, float v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a[i] = v;
}

// mass m(p) = sum_i a_i p_i of every listed field (FP64): per-ring partial sums by a
// (ring, field) grid, then a fixed-order sum per field
__global__ void k_field_mass_part(const float* const* __restrict__ fl, int nlat, const int* __restrict__ rlen,
                                  const long long* __restrict__ roff, const float* __restrict__ a_ring,
                                  double* __restrict__ part) {
  __shared__ float red[32];
  const int j = blockIdx.x, f = blockIdx.y;
  const float* row = fl[f] + roff[j];
  const int n = rlen[j];
  float s = 0.f;
  for (int k = threadIdx.x; k < n; k += blockDim.x) s += row[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[(size_t)f * nlat + j] = (double)a_ring[j] * (double)t;
  }
}

__global__ void k_field_mass_sum(int nfl, int nlat, const double* __restrict__ part, double* __restrict__ out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nfl) return;
  double s = 0.0;
  for (int j = 0; j < nlat; ++j) s += part[(size_t)f * nlat + j];
  out[f] = s;
}

// masses of nfl listed fields into out (device); part needs nfl*nlat doubles
int field_masses(const Grid& g, const float* const* fl_d, int nfl, double* part, double* out, cudaStream_t st) {
  count_launch(2);
  k_field_mass_part<<<dim3(g.nlat, nfl), 256, 0, st>>>(fl_d, g.nlat, g.ring_len_d, g.ring_off_d, g.a_d, part);
  k_field_mass_sum<<<(nfl + 127) / 128, 128, 0, st>>>(nfl, g.nlat, part, out);
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

Grid* as_grid(shot_grid g) { return reinterpret_cast<Grid*>(g); }

int heat_pipeline(Grid& g, const float* in, int nf, int scale_which, cudaStream_t st) {
  Workspace& w = g.ws;
  int rc = launch_dft_fwd(g, in, nf, reinterpret_cast<ProbState*>(w.probs), scale_which, w.XY, w.ldc, st);
  if (rc) return rc;
  return launch_legendre(g, nf, w.XY, w.C, w.XY, w.ldc, st);
}

int reduce(Grid& g, int mode, int nprob, double eps, double tol, int norm_l1, cudaStream_t st) {
  ProfScope prof(PK_OTHER, st);
  count_launch();
  k_reduce<<<nprob, kRedThreads, 0, st>>>(mode, nprob, g.nh, g.ws.part, reinterpret_cast<ProbState*>(g.ws.probs),
                              g.ws.dev_int, eps, tol, norm_l1, log((double)g.npix));
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

struct SolveOut {
  std::vector<ProbState> ps;
  int kdone = 0;
};

// One Alg. 1 solve on one grid: nprob problems with marginals P (first), Q (second) and
// per-problem tau; state lives in the grid's workspace, work runs on the grid's stream.
struct Solve {
  Grid* g = nullptr;
  int nprob = 0;
  double eps = 0, tol = 0;
  int C = 0, norm_l1 = 0, potentials = 0;
  int symmetric = 0;   // self terms by the symmetric update (u and v are one buffer)
  float *u = nullptr, *v = nullptr;
  cudaStream_t st = nullptr;
};

int ensure_stream(Grid& g) {
  Workspace& w = g.ws;
  if (!w.stream) {
    SHOT_CUDA(cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking));
    SHOT_CUDA(cudaEventCreateWithFlags(&w.ev0, cudaEventDisableTiming));
    SHOT_CUDA(cudaEventCreateWithFlags(&w.ev1, cudaEventDisableTiming));
    SHOT_CUDA(cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking));
    SHOT_CUDA(cudaEventCreateWithFlags(&w.evf, cudaEventDisableTiming));
    SHOT_CUDA(cudaEventCreateWithFlags(&w.evj, cudaEventDisableTiming));
  }
  return SHOT_OK;
}

EpiParams base_ep(Solve& s);

int solve_prepare(Grid& g, const std::vector<const float*>& P, const std::vector<const float*>& Q,
                  const std::vector<double>& taus, double eps, double tol, int C, int flags, float* u, float* v,
                  cudaStream_t user, Solve& s) {
  const int nprob = (int)P.size();
  int rc = ensure_workspace(g, nprob, user);
  if (rc) return rc;
  if ((rc = ensure_stream(g))) return rc;
  Workspace& w = g.ws;
  s.g = &g;
  s.nprob = nprob;
  s.eps = eps;
  s.tol = tol;
  s.C = C;
  s.norm_l1 = (flags & SHOT_FLAG_NORM_L1) ? 1 : 0;
  s.potentials = (flags & SHOT_FLAG_POTENTIALS) ? 1 : 0;
  s.symmetric = (flags & kFlagSymmetricSolve) ? 1 : 0;
  s.u = u;
  s.v = v;
  s.st = w.stream;
  // the solver stream starts after everything already queued on the caller's stream
  SHOT_CUDA(cudaEventRecord(w.ev0, user));
  SHOT_CUDA(cudaStreamWaitEvent(s.st, w.ev0, 0));
  const size_t n = g.npix;
  std::vector<const float*> lists(2 * (size_t)nprob);
  for (int i = 0; i < nprob; ++i) {
    lists[i] = P[i];
    lists[nprob + i] = Q[i];
  }
  SHOT_CUDA(cudaMemcpyAsync(w.marg, lists.data(), 2 * nprob * sizeof(float*), cudaMemcpyHostToDevice, s.st));
  SHOT_CUDA(cudaMemcpyAsync(w.taus, taus.data(), nprob * sizeof(double), cudaMemcpyHostToDevice, s.st));
  ProbState* ps = reinterpret_cast<ProbState*>(w.probs);
  count_launch();
  k_init_probs<<<(nprob + 127) / 128, 128, 0, s.st>>>(nprob, ps, w.dev_int, w.taus, eps);
  if (!(flags & SHOT_FLAG_WARM_START)) {
    count_launch(2);
    k_fill<<<1024, 256, 0, s.st>>>(u, n * nprob, 1.f);
    k_fill<<<1024, 256, 0, s.st>>>(v, n * nprob, 1.f);
  }
  SHOT_CUDA(cudaGetLastError());
  {  // tune the launch shapes on the solver's own form of the inverse DFT
    EpiParams up = base_ep(s);
    up.mode = EPI_UPDATE;
    up.marg = w.marg;
    up.xout = w.XY;
    if ((rc = autotune(g, nprob, s.st, &up))) return rc;
  }
  if ((rc = launch_heat_mult(g, eps / 4.0, s.st))) return rc;
  // spectra of the starting v
  return launch_dft_fwd(g, v, nprob, nullptr, 0, w.XY, w.ldc, s.st);
}

EpiParams base_ep(Solve& s) {
  Workspace& w = s.g->ws;
  EpiParams ep{};
  ep.ps = reinterpret_cast<ProbState*>(w.probs);
  ep.part = w.part;
  ep.eps = s.eps;
  ep.norm_l1 = s.norm_l1;
  return ep;
}

// nit iterations of Alg. 1, then (optionally) the marginal check; no host synchronisation.
// X always holds the ring spectra of the buffer the next heat convolution needs: each
// half-step's inverse DFT also transforms the scaling it has just produced (fused); the
// buffers' factors e^{la}, e^{lb} enter only the FP64 scalars of k_reduce.
int solve_enqueue(Solve& s, int nit, bool check, cudaStream_t st) {
  Grid& g = *s.g;
  Workspace& w = g.ws;
  const float* const* margP = w.marg;
  const float* const* margQ = w.marg + s.nprob;
  EpiParams ep = base_ep(s);
  int rc;
  // Each half-step's reduction runs on the side stream beside the next heat convolution's
  // Legendre stages (which read no per-problem state); the next update waits for it.  Profiled
  // runs (a CUDA event pair around every launch) keep it on the solver's stream, so that each
  // launch's time is its own.
  bool pending = false;
  const bool side = !profiling_on();
  auto fork_reduce = [&](int mode) -> int {
    if (!side) return reduce(g, mode, s.nprob, s.eps, s.tol, s.norm_l1, st);
    SHOT_CUDA(cudaEventRecord(w.evf, st));
    SHOT_CUDA(cudaStreamWaitEvent(w.side, w.evf, 0));
    const int r = reduce(g, mode, s.nprob, s.eps, s.tol, s.norm_l1, w.side);
    if (r) return r;
    SHOT_CUDA(cudaEventRecord(w.evj, w.side));
    pending = true;
    return SHOT_OK;
  };
  auto join = [&]() -> int {
    if (pending) SHOT_CUDA(cudaStreamWaitEvent(st, w.evj, 0));
    pending = false;
    return SHOT_OK;
  };
  for (int i = 0; s.symmetric && i < nit; ++i) {
    // self term: u = sqrt(u (p / K u)^gamma) in place, and X := F(u)
    if ((rc = launch_legendre(g, s.nprob, w.XY, w.C, w.Yb, w.ldc, st))) return rc;
    ep.mode = EPI_SYM;
    ep.out = s.u;
    ep.marg = margP;
    ep.which = 0;
    ep.xout = w.XY;
    if ((rc = join()) || (rc = launch_idft(g, w.Yb, w.ldc, s.nprob, ep, st))) return rc;
    if ((rc = fork_reduce(RED_S))) return rc;
  }
  for (int i = 0; !s.symmetric && i < nit; ++i) {
    // u-step: u = (ru p / K v)^gamma, and X := F(u)
    if ((rc = launch_legendre(g, s.nprob, w.XY, w.C, w.Yb, w.ldc, st))) return rc;
    ep.mode = EPI_UPDATE;
    ep.out = s.u;
    ep.marg = margP;
    ep.which = 0;
    ep.xout = w.XY;
    // only the block's last iteration leaves u and v in their buffers (the check and the final
    // objective read them); the others feed the fused forward transforms alone
    ep.skip_store = (i + 1 < nit) ? 1 : 0;
    if ((rc = join()) || (rc = launch_idft(g, w.Yb, w.ldc, s.nprob, ep, st))) return rc;
    if ((rc = fork_reduce(RED_U))) return rc;
    // v-step: v = (rv q / K u)^gamma, X := F(v); then the gauge / translation-invariant scalars
    if ((rc = launch_legendre(g, s.nprob, w.XY, w.C, w.Yb, w.ldc, st))) return rc;
    ep.out = s.v;
    ep.marg = margQ;
    ep.which = 1;
    if ((rc = join()) || (rc = launch_idft(g, w.Yb, w.ldc, s.nprob, ep, st))) return rc;
    if ((rc = fork_reduce(RED_V))) return rc;
  }
  if (check) {   // K v from the spectra X, which stay for the next u-step
    if ((rc = launch_legendre(g, s.nprob, w.XY, w.C, w.Yb, w.ldc, st))) return rc;
    ep.mode = EPI_CHECK;
    ep.other = s.u;
    ep.marg = margP;
    ep.xout = nullptr;
    if ((rc = join()) || (rc = launch_idft(g, w.Yb, w.ldc, s.nprob, ep, st))) return rc;
    if ((rc = fork_reduce(RED_CHECK))) return rc;
  }
  return join();
}

int solve_final_enqueue(Solve& s) {
  Grid& g = *s.g;
  Workspace& w = g.ws;
  EpiParams ep = base_ep(s);
  ProbState* ps = reinterpret_cast<ProbState*>(w.probs);
  int rc;
  // final K v for the objective, mass and marginal error; writes u_true, v_true
  if ((rc = launch_legendre(g, s.nprob, w.XY, w.C, w.Yb, w.ldc, s.st))) return rc;
  ep.mode = EPI_FINAL;
  ep.potentials = s.potentials;
  ep.out = s.v;
  ep.other = s.u;
  ep.marg = w.marg;
  ep.marg2 = w.marg + s.nprob;
  if ((rc = launch_idft(g, w.Yb, w.ldc, s.nprob, ep, s.st))) return rc;
  if ((rc = reduce(g, RED_FINAL, s.nprob, s.eps, s.tol, s.norm_l1, s.st))) return rc;
  SHOT_CUDA(cudaMemcpyAsync(w.host_probs, ps, s.nprob * sizeof(ProbState), cudaMemcpyDeviceToHost, s.st));
  SHOT_CUDA(cudaMemcpyAsync(w.host_int, w.dev_int, 8 * sizeof(int), cudaMemcpyDeviceToHost, s.st));
  return SHOT_OK;
}

int solve_collect(Solve& s, cudaStream_t user, SolveOut& out) {
  Workspace& w = s.g->ws;
  SHOT_CUDA(cudaStreamSynchronize(s.st));
  // the caller's stream continues after the solve
  SHOT_CUDA(cudaEventRecord(w.ev1, s.st));
  SHOT_CUDA(cudaStreamWaitEvent(user, w.ev1, 0));
  out.ps.resize(s.nprob);
  memcpy(out.ps.data(), w.host_probs, s.nprob * sizeof(ProbState));
  out.kdone = w.host_int[0];
  if (w.host_int[4] != 0) {
    SHOT_CUDA(cudaMemsetAsync(w.dev_int + 4, 0, sizeof(int), s.st));
    SHOT_CUDA(cudaStreamSynchronize(s.st));
    set_error("a bounded device-side wait expired in a tensor-core kernel");
    return SHOT_ERR_TIMEOUT;
  }
  for (auto& p : out.ps) {
    if (p.status == SHOT_OK && p.active) {
      p.iters = w.host_int[0];
      if (s.tol > 0) p.status = SHOT_WARN_NOT_CONVERGED;
    }
    if (p.status < 0) p.ot = p.ot_dual = p.mass = p.err = nan("");
  }
  return SHOT_OK;
}

// Blocks of B iterations (B = C when checking, else 10), each captured once into a CUDA
// graph and replayed; the host polls the number of active problems after every checked
// block.  Graphs are not used while per-launch profiling is on.
struct Runner {
  std::vector<Solve*> sets;
  cudaStream_t main = nullptr;
  cudaGraphExec_t exec = nullptr;
  int block = 10;
  ~Runner() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

int enqueue_all(Runner& r, int nit, bool check) {
  int rc;
  if (r.sets.size() == 1) return solve_enqueue(*r.sets[0], nit, check, r.main);
  // fork: every set on its own grid stream, joined back into the main stream
  for (Solve* s : r.sets) {
    Workspace& w = s->g->ws;
    if (s->st == r.main) {
      if ((rc = solve_enqueue(*s, nit, check, r.main))) return rc;
      continue;
    }
    SHOT_CUDA(cudaEventRecord(w.ev0, r.main));
    SHOT_CUDA(cudaStreamWaitEvent(w.stream, w.ev0, 0));
    if ((rc = solve_enqueue(*s, nit, check, w.stream))) return rc;
    SHOT_CUDA(cudaEventRecord(w.ev1, w.stream));
    SHOT_CUDA(cudaStreamWaitEvent(r.main, w.ev1, 0));
  }
  return SHOT_OK;
}

int run_blocks(Runner& r, int T) {
  const int C = r.sets[0]->C;
  const int B = C > 0 ? C : 10;
  const bool use_graph = !profiling_on() && T >= 2 * B;
  int k = 0, rc;
  long long per_block = 0;
  // the main stream waits for every set's preparation
  for (Solve* s : r.sets)
    if (s->st != r.main) {
      SHOT_CUDA(cudaEventRecord(s->g->ws.ev0, s->st));
      SHOT_CUDA(cudaStreamWaitEvent(r.main, s->g->ws.ev0, 0));
    }
  while (k < T) {
    const int nit = (T - k < B) ? T - k : B;
    const bool check = C > 0 && nit == B;
    if (use_graph && nit == B) {
      if (!r.exec) {
        cudaGraph_t graph = nullptr;
        long long n0 = 0, n1 = 0;
        shot_launch_count(&n0);
        SHOT_CUDA(cudaStreamBeginCapture(r.main, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_all(r, nit, check);
        cudaError_t e = cudaStreamEndCapture(r.main, &graph);
        shot_launch_count(&n1);
        per_block = n1 - n0;
        count_launch((int)-per_block);   // captured, not launched
        if (rc) {
          if (graph) cudaGraphDestroy(graph);
          return rc;
        }
        if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&r.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate");
      }
      count_launch((int)per_block);
      SHOT_CUDA(cudaGraphLaunch(r.exec, r.main));
    } else {
      if ((rc = enqueue_all(r, nit, check))) return rc;
    }
    k += nit;
    if (check) {
      int active = 0;
      for (Solve* s : r.sets) {
        Workspace& w = s->g->ws;
        SHOT_CUDA(cudaMemcpyAsync(w.host_int + 8, w.dev_int + 1, sizeof(int), cudaMemcpyDeviceToHost, r.main));
      }
      SHOT_CUDA(cudaStreamSynchronize(r.main));
      for (Solve* s : r.sets) active += s->g->ws.host_int[8];
      if (active == 0) break;
    }
  }
  // every set's stream continues after the blocks
  for (Solve* s : r.sets)
    if (s->st != r.main) {
      SHOT_CUDA(cudaEventRecord(s->g->ws.ev1, r.main));
      SHOT_CUDA(cudaStreamWaitEvent(s->st, s->g->ws.ev1, 0));
    }
  return SHOT_OK;
}

// Alg. 1 on nprob problems of one grid with marginal lists P (first) and Q (second).
int run_sinkhorn(Grid& g, const std::vector<const float*>& P, const std::vector<const float*>& Q, double eps,
                 double tau, int T, double tol, int C, int flags, float* u, float* v, cudaStream_t st,
                 SolveOut& out) {
  std::vector<double> taus(P.size(), tau);
  Solve s;
  int rc = solve_prepare(g, P, Q, taus, eps, tol, C, flags, u, v, st, s);
  if (rc) return rc;
  Runner r;
  r.sets.push_back(&s);
  r.main = s.st;
  if ((rc = run_blocks(r, T))) return rc;
  if ((rc = solve_final_enqueue(s))) return rc;
  return solve_collect(s, st, out);
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

int run_sinkhorn_public(Grid& g, const std::vector<const float*>& P, const std::vector<const float*>& Q, double eps,
                        double tau, int T, double tol, int C, int flags, float* u, float* v, cudaStream_t st,
                        std::vector<ProbState>& out, int* kdone) {
  SolveOut so;
  int rc = run_sinkhorn(g, P, Q, eps, tau, T, tol, C, flags, u, v, st, so);
  if (rc) return rc;
  out = so.ps;
  if (kdone) *kdone = so.kdone;
  return SHOT_OK;
}

int divergence_grad(Grid& g, const float* p, const float* q, int batch, double eps, double tau, int T, int ck,
                    int mode, double* S, float* grad, int* status, cudaStream_t st);

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
  return shot_grid_init_quad(out, SHOT_QUAD_GAUSS_LEGENDRE, nlat, nlon, lmax, precision, legendre_mode, stream);
}

int shot_grid_init_quad(shot_grid* out, int quadrature, int nlat, int nlon, int lmax, int precision,
                        int legendre_mode, void* stream) {
  if (!out) { set_error("out is NULL"); return SHOT_ERR_INVALID_ARG; }
  *out = nullptr;
  if (quadrature != SHOT_QUAD_GAUSS_LEGENDRE && quadrature != SHOT_QUAD_CLENSHAW_CURTIS) {
    set_error("unknown quadrature");
    return SHOT_ERR_INVALID_ARG;
  }
  if (quadrature == SHOT_QUAD_CLENSHAW_CURTIS && nlat < 3) {
    set_error("a Clenshaw-Curtis grid needs nlat >= 3");
    return SHOT_ERR_INVALID_ARG;
  }
  if (lmax == -1) lmax = nlat - 1;
  if (nlat < 2 || lmax < 0 || lmax > nlat - 1 || nlon < 2 * lmax + 1) {
    set_error("need nlat >= 2, 0 <= lmax <= nlat-1, nlon >= 2*lmax+1");
    return SHOT_ERR_INVALID_ARG;
  }
  if (precision != SHOT_FP32 && precision != SHOT_BF16X3 && precision != SHOT_TF32X3) {
    set_error("unknown precision");
    return SHOT_ERR_INVALID_ARG;
  }
  if (legendre_mode != SHOT_TABLE && legendre_mode != SHOT_RECURRENCE) {
    set_error("unknown legendre_mode");
    return SHOT_ERR_INVALID_ARG;
  }
  FftPlan plan;
  if (nlon > kFftCap || !make_fft_plan(nlon, &plan)) {
    set_error("nlon above the shared-memory ring FFT's 6400 longitudes");
    return SHOT_ERR_UNSUPPORTED;
  }
  Grid* g = new Grid;
  g->nlat = nlat;
  g->nlon = nlon;
  g->lmax = lmax;
  g->nh = (nlat + 1) / 2;
  g->precision = precision;
  g->mode = legendre_mode;
  g->quad = quadrature;
  {
    const char* e = getenv("SHOT_IDFT_PERSISTENT");   // 0: one item per CTA for the update half-steps too
    g->idft_nonpersistent = (e && e[0] == '0') ? 1 : 0;
    e = getenv("SHOT_TC_STAGES");   // 1..4 fixes the analysis pipeline depth instead of the autotuner
    g->tc_stages_override = (e && e[0] >= '1' && e[0] <= '4') ? e[0] - '0' : 0;
    e = getenv("SHOT_T32_2CTA");   // 0: one CTA of 16 split warps per SM in the TF32 table kernels
    g->t32_two_cta_off = (e && e[0] == '0') ? 1 : 0;
    e = getenv("SHOT_T32_INRING");   // 1..8 caps the input ring of the TF32 recurrence kernels
    g->t32_in_override = (e && e[0] >= '1' && e[0] <= '8') ? e[0] - '0' : 0;
  }
  g->plan = plan;
  cudaGetDevice(&g->dev);
  cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->dev);
  int rc = build_grid_tables(*g, as_stream(stream));
  if (rc) {
    shot_grid_free(reinterpret_cast<shot_grid>(g));
    return rc;
  }
  *out = reinterpret_cast<shot_grid>(g);
  return SHOT_OK;
}

int shot_grid_init_healpix(shot_grid* out, int nside, int lmax, int precision, int legendre_mode, void* stream) {
  if (!out) { set_error("out is NULL"); return SHOT_ERR_INVALID_ARG; }
  *out = nullptr;
  if (nside < 1 || nside > 4096) { set_error("need 1 <= nside <= 4096"); return SHOT_ERR_INVALID_ARG; }
  const int nr = 4 * nside - 1;
  if (lmax == -1) lmax = 3 * nside - 1;
  if (lmax < 0 || lmax > nr - 1) { set_error("need 0 <= lmax <= 4 nside - 2"); return SHOT_ERR_INVALID_ARG; }
  if (precision != SHOT_FP32 && precision != SHOT_BF16X3 && precision != SHOT_TF32X3) {
    set_error("unknown precision");
    return SHOT_ERR_INVALID_ARG;
  }
  if (legendre_mode != SHOT_TABLE && legendre_mode != SHOT_RECURRENCE) {
    set_error("unknown legendre_mode");
    return SHOT_ERR_INVALID_ARG;
  }
  Grid* g = new Grid;
  g->nlat = nr;
  g->nlon = 4 * nside;   // the longest ring
  g->lmax = lmax;
  g->nh = (nr + 1) / 2;
  g->nside = nside;
  g->precision = precision;
  g->mode = legendre_mode;
  g->quad = SHOT_QUAD_HEALPIX;
  g->plan.N = 0;
  g->plan.nst = 0;
  cudaGetDevice(&g->dev);
  cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->dev);
  int rc = build_grid_tables(*g, as_stream(stream));
  if (rc) {
    shot_grid_free(reinterpret_cast<shot_grid>(g));
    return rc;
  }
  *out = reinterpret_cast<shot_grid>(g);
  return SHOT_OK;
}

int shot_grid_npix(shot_grid gh, long long* npix) {
  Grid* g = as_grid(gh);
  if (!g || !npix) { set_error("shot_grid_npix: bad argument"); return SHOT_ERR_INVALID_ARG; }
  *npix = (long long)g->npix;
  return SHOT_OK;
}

int shot_grid_rings(shot_grid gh, int* len, long long* off, double* phi0) {
  Grid* g = as_grid(gh);
  if (!g) { set_error("shot_grid_rings: bad handle"); return SHOT_ERR_INVALID_ARG; }
  for (int i = 0; i < g->nlat; ++i) {
    if (len) len[i] = g->ring_len[i];
    if (off) off[i] = g->ring_off[i];
    if (phi0)
      phi0[i] = g->quad == SHOT_QUAD_HEALPIX ? M_PI * g->ring_phase[i].first / g->ring_phase[i].second : 0.0;
  }
  return SHOT_OK;
}

int shot_grid_free(shot_grid gh) {
  Grid* g = as_grid(gh);
  if (!g) return SHOT_OK;
  void* dptr[] = {g->ring_len_d, g->ring_off_d, g->ring_phase_d, g->hp_plan_d, g->ring_plan_d, g->hp_tw_d, g->hp_tw_base_d, g->xyz_d, g->ws.Yb, g->x_d, g->w_d, g->a_d, g->tw_d, g->h_d, g->tab, g->tabT, g->tab_hi, g->tab_lo,
                  g->ws.ct_hi, g->ws.ct_lo, g->ws.ct32, g->rec_seeds, g->rec_coef, g->rec_coef_off, g->rec_x, g->ck, g->ck_off_d, g->M_d,
                  g->row_off_d, g->tiles_ana, g->tiles_syn, g->ws.XY, g->ws.C, g->ws.part, g->ws.probs,
                  g->ws.marg, g->ws.ubuf, g->ws.vbuf, g->ws.dev_int};
  for (void* p : dptr)
    if (p) cudaFree(p);
  if (g->ws.taus) cudaFree(g->ws.taus);
  if (g->ws.stream) cudaStreamDestroy(g->ws.stream);
  if (g->ws.ev0) cudaEventDestroy(g->ws.ev0);
  if (g->ws.ev1) cudaEventDestroy(g->ws.ev1);
  if (g->ws.side) cudaStreamDestroy(g->ws.side);
  if (g->ws.evf) cudaEventDestroy(g->ws.evf);
  if (g->ws.evj) cudaEventDestroy(g->ws.evj);
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

int shot_grid_check(shot_grid gh, void* stream) {
  Grid* g = as_grid(gh);
  if (!g) { set_error("shot_grid_check: bad grid"); return SHOT_ERR_INVALID_ARG; }
  cudaStream_t st = as_stream(stream);
  SHOT_CUDA(cudaStreamSynchronize(st));
  if (!g->ws.dev_int) return SHOT_OK;   // nothing has run on this grid yet
  int flag = 0;
  SHOT_CUDA(cudaMemcpy(&flag, g->ws.dev_int + 4, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    SHOT_CUDA(cudaMemset(g->ws.dev_int + 4, 0, sizeof(int)));
    set_error("a bounded device-side wait expired in a tensor-core kernel");
    return SHOT_ERR_TIMEOUT;
  }
  return SHOT_OK;
}

int shot_grid_set_wait_limit(shot_grid gh, long long cycles) {
  Grid* g = as_grid(gh);
  if (!g) { set_error("shot_grid_set_wait_limit: bad grid"); return SHOT_ERR_INVALID_ARG; }
  g->wait_cycles = cycles > 0 ? cycles : kDefaultWaitCycles;
  return SHOT_OK;
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
  const size_t n = g->npix;
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
  const size_t n = g->npix;
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
  if ((rc = field_masses(*g, fl_d, 2 * batch, w.part + 2 * batch, mass_d, st))) return rc;
  std::vector<double> masses(2 * batch);
  SHOT_CUDA(cudaMemcpyAsync(masses.data(), mass_d, 2 * batch * sizeof(double), cudaMemcpyDeviceToHost, st));
  SHOT_CUDA(cudaStreamSynchronize(st));

  SolveOut so;
  if (flags & SHOT_FLAG_SYMMETRIC_SELF) {
    // (p_b, q_b) by Alg. 1, then the 2B self terms by the symmetric update in one solve
    const int f1 = flags & ~SHOT_FLAG_SYMMETRIC_SELF;
    std::vector<const float*> P1(P.begin(), P.begin() + batch), Q1(Q.begin(), Q.begin() + batch);
    std::vector<const float*> P2(P.begin() + batch, P.end());
    SolveOut s1, s2;
    if ((rc = run_sinkhorn(*g, P1, Q1, eps, tau, max_iter, tol, check_every, f1, u3, v3, st, s1))) return rc;
    float* us = u3 + (size_t)batch * n;
    if ((rc = run_sinkhorn(*g, P2, P2, eps, tau, max_iter, tol, check_every, f1 | kFlagSymmetricSolve, us, us, st,
                           s2)))
      return rc;
    // v = u for the self terms
    SHOT_CUDA(cudaMemcpyAsync(v3 + (size_t)batch * n, us, (size_t)2 * batch * n * sizeof(float),
                              cudaMemcpyDeviceToDevice, st));
    so.ps = s1.ps;
    so.ps.insert(so.ps.end(), s2.ps.begin(), s2.ps.end());
  } else {
    rc = run_sinkhorn(*g, P, Q, eps, tau, max_iter, tol, check_every, flags, u3, v3, st, so);
    if (rc) return rc;
  }
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

int shot_divergence_multi(const shot_pair_set* sets, int nsets, int max_iter, double tol, int check_every,
                          int flags, void* stream) {
  if (!sets || nsets < 1 || max_iter < 0 || check_every < 0) {
    set_error("shot_divergence_multi: bad argument");
    return SHOT_ERR_INVALID_ARG;
  }
  cudaStream_t user = as_stream(stream);
  // group the sets by grid: one solve per grid with per-problem tau
  std::vector<Grid*> grids;
  std::vector<std::vector<int>> members;
  for (int i = 0; i < nsets; ++i) {
    const shot_pair_set& S = sets[i];
    Grid* g = as_grid(S.grid);
    int rc = check_solver_args(g, S.p, S.q, S.batch, S.eps, S.tau, max_iter, check_every);
    if (rc) return rc;
    if (!S.S || !S.status) { set_error("shot_divergence_multi: S and status are required"); return SHOT_ERR_INVALID_ARG; }
    size_t k = 0;
    while (k < grids.size() && grids[k] != g) ++k;
    if (k == grids.size()) {
      grids.push_back(g);
      members.emplace_back();
    }
    if (!members[k].empty() && sets[members[k][0]].eps != S.eps) {
      set_error("shot_divergence_multi: sets sharing a grid must share eps");
      return SHOT_ERR_INVALID_ARG;
    }
    members[k].push_back(i);
  }
  const size_t G = grids.size();
  std::vector<Solve> solves(G);
  std::vector<std::vector<double>> masses(G);
  int rc;
  for (size_t k = 0; k < G; ++k) {
    Grid& g = *grids[k];
    const size_t n = g.npix;
    std::vector<const float*> P, Q, fl;
    std::vector<double> taus;
    for (int i : members[k]) {
      const shot_pair_set& S = sets[i];
      for (int part = 0; part < 3; ++part)
        for (int b = 0; b < S.batch; ++b) {
          const float* pb = S.p + b * n;
          const float* qb = S.q + b * n;
          P.push_back(part == 2 ? qb : pb);
          Q.push_back(part == 0 ? qb : (part == 1 ? pb : qb));
          taus.push_back(S.tau);
        }
      for (int b = 0; b < S.batch; ++b) fl.push_back(S.p + b * n);
      for (int b = 0; b < S.batch; ++b) fl.push_back(S.q + b * n);
    }
    const int np = (int)P.size();
    if ((rc = ensure_workspace(g, np, user))) return rc;
    Workspace& w = g.ws;
    if (w.uv_cap < (size_t)np * n) {
      SHOT_CUDA(cudaStreamSynchronize(user));
      cudaFree(w.ubuf);
      cudaFree(w.vbuf);
      w.ubuf = w.vbuf = nullptr;
      w.uv_cap = 0;
      SHOT_CUDA(cudaMalloc(&w.ubuf, (size_t)np * n * sizeof(float)));
      SHOT_CUDA(cudaMalloc(&w.vbuf, (size_t)np * n * sizeof(float)));
      w.uv_cap = (size_t)np * n;
    }
    // masses of every field of the grid (FP64), before the solve uses the partial buffer
    const int nfl = (int)fl.size();
    const float** fl_d = w.marg + 2 * np;
    if (nfl > 2 * np) { set_error("internal: mass list too long"); return SHOT_ERR_INVALID_ARG; }
    SHOT_CUDA(cudaMemcpyAsync(fl_d, fl.data(), nfl * sizeof(float*), cudaMemcpyHostToDevice, user));
    if ((rc = field_masses(g, fl_d, nfl, w.part + nfl, w.part, user))) return rc;
    masses[k].resize(nfl);
    SHOT_CUDA(cudaMemcpyAsync(masses[k].data(), w.part, nfl * sizeof(double), cudaMemcpyDeviceToHost, user));
    SHOT_CUDA(cudaStreamSynchronize(user));
    if ((rc = solve_prepare(g, P, Q, taus, sets[members[k][0]].eps, tol, check_every, flags, w.ubuf, w.vbuf, user,
                            solves[k])))
      return rc;
  }
  Runner r;
  for (auto& s : solves) r.sets.push_back(&s);
  r.main = solves[0].st;
  if ((rc = run_blocks(r, max_iter))) return rc;
  int worst = SHOT_OK;
  for (size_t k = 0; k < G; ++k)
    if ((rc = solve_final_enqueue(solves[k]))) return rc;
  for (size_t k = 0; k < G; ++k) {
    SolveOut so;
    if ((rc = solve_collect(solves[k], user, so))) return rc;
    size_t off = 0, moff = 0;
    for (int i : members[k]) {
      const shot_pair_set& S = sets[i];
      const int B = S.batch;
      for (int b = 0; b < B; ++b) {
        const ProbState &a = so.ps[off + b], &pp = so.ps[off + B + b], &qq = so.ps[off + 2 * B + b];
        const double dm = masses[k][moff + b] - masses[k][moff + B + b];
        S.S[b] = a.ot - 0.5 * (pp.ot + qq.ot) + 0.5 * S.eps * dm * dm;
        if (S.S_dual) S.S_dual[b] = a.ot_dual - 0.5 * (pp.ot_dual + qq.ot_dual);
        int ws = SHOT_OK;
        for (int st3 : {a.status, pp.status, qq.status}) {
          if (st3 < 0 && (ws >= 0 || st3 < ws)) ws = st3;
          else if (ws >= 0 && st3 > ws) ws = st3;
        }
        S.status[b] = ws;
        if (ws < 0 && (worst >= 0 || ws < worst)) worst = ws;
        else if (worst >= 0 && ws > worst) worst = ws;
      }
      off += 3 * (size_t)B;
      moff += 2 * (size_t)B;
    }
  }
  return worst;
}

int shot_divergence_grad(shot_grid gh, const float* p, const float* q, int batch, double eps, double tau,
                         int max_iter, int checkpoint_every, int mode, double* S, float* grad_p, int* status,
                         void* stream) {
  Grid* g = as_grid(gh);
  int rc = check_solver_args(g, p, q, batch, eps, tau, max_iter, 0);
  if (rc) return rc;
  if (!S || !grad_p || !status || (mode != SHOT_GRAD_UNROLLED && mode != SHOT_GRAD_ENVELOPE)) {
    set_error("shot_divergence_grad: S, grad_p, status required; mode UNROLLED or ENVELOPE");
    return SHOT_ERR_INVALID_ARG;
  }
  return divergence_grad(*g, p, q, batch, eps, tau, max_iter, checkpoint_every, mode, S, grad_p, status,
                         as_stream(stream));
}

}  // extern "C"
