// Gradient of the Sinkhorn divergence with respect to p (shot_divergence_grad).
//
// The paper differentiates the divergence for its regional attribution (Sec. 4.2,
// "Gradient-based regional attribution": g = grad_mu S from the dual potentials).  Two
// modes:
//   UNROLLED  reverse-mode derivative of S computed by exactly max_iter iterations of
//             Alg. 1 (no early stop), through the gauge / translation-invariant steps;
//   ENVELOPE  the potential form at convergence (balanced: a (phi_pq - (phi_pp+psi_pp)/2)
//             + eps (m_p - m_q) a; unbalanced: the derivative of the dual form S_dual).
//
// Adjoints are carried divided by the area weights ("tilde" form, x_bar = a (.) x~).
// Because K = H diag(a) with H symmetric, K^T (a (.) x) = a (.) K x, so every transpose
// heat convolution of the reverse sweep is a forward heat convolution of a tilde field
// and reuses the forward SHT kernels.  One iteration k of Alg. 1 is
//   u' = (p / K v_{k-1})^g,  v' = (q / K u')^g,  then  u_k = al u', v_k = be v'
// with (al, be) = (1/s, s), s = sum_i u'_i (balanced, g = 1) or (E, 1/E),
// E = exp(c/eps), c = tau/2 (log A - log B), A = sum a p u'^{-eps/tau},
// B = sum a q v'^{-eps/tau} (unbalanced, g = tau/(tau+eps)).  Its reverse, given the
// adjoints u~_k, v~_k of (u_k, v_k):
//   balanced    sbar = -sum a u~ u' / s^2 + sum a v~ v';  u~' = u~/s + sbar/a;  v~' = s v~
//   unbalanced  cbar = (sum a u~ u_k - sum a v~ v_k)/eps;  Abar = cbar tau/(2A);
//               Bbar = -cbar tau/(2B);  u~' = E u~ - Abar (eps/tau) p u'^{-eps/tau-1};
//               v~' = v~/E - Bbar (eps/tau) q v'^{-eps/tau-1};  p~ += Abar u'^{-eps/tau};
//               q~ += Bbar v'^{-eps/tau}
//   both        (Ku)~ = -g v~' v'^{1+1/g} / q;  q~ += g v~' v' / q;  u~' += K (Ku)~;
//               (Kv)~ = -g u~' u'^{1+1/g} / p;  p~ += g u~' u' / p;  v~_{k-1} = K (Kv)~,
// with u~_{k-1} = 0.  The sweep starts from the derivative of Alg. 1's return:
// balanced u~_T = eps p / u_T, p~ = eps log u_T; unbalanced u~_T = eps p u_T^{-eps/tau-1},
// p~ = tau (1 - u_T^{-eps/tau}) (and likewise for v, q).  The forward states u', v' and
// the scalars are recomputed segment by segment from checkpoints of v every
// checkpoint_every iterations.  For the pair b the problems are (p_b, q_b) and
// (p_b, p_b); dS/dp = a (.) [p~_(p,q) - (p~_(p,p) + q~_(p,p))/2] + eps (m_p - m_q) a.
#include <math.h>

#include <vector>

#include "shot_internal.cuh"

namespace shot {

int run_sinkhorn_public(Grid& g, const std::vector<const float*>& P, const std::vector<const float*>& Q, double eps,
                        double tau, int T, double tol, int C, int flags, float* u, float* v, cudaStream_t st,
                        std::vector<ProbState>& out, int* kdone);

namespace {

constexpr int kEw = 256;

// ring layout of a field: ring j holds len[j] nodes starting at off[j]; a field has npix nodes
struct Rings {
  const int* len;
  const long long* off;
  long long npix;
  int nring;
};

__device__ __forceinline__ float block_sum_f(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

struct GScal {      // per problem and iteration of a segment
  double al, be;    // u_k = al u', v_k = be v'
  double A, B;      // unbalanced TI sums (A also holds s for the balanced branch)
};

// forward half-step: out = (m / Kf)^g; partial sums per ring of
//   balanced: sum out;  unbalanced: sum a m out^{-eps/tau}
__global__ void k_g_update(Rings R, const float* __restrict__ a_ring, const float* const* __restrict__ marg,
                           const float* __restrict__ Kf, float* __restrict__ out, int balanced, float gam, float et,
                           double* __restrict__ part) {
  __shared__ float red[32];
  const int j = blockIdx.x, b = blockIdx.y;
  const size_t base = (size_t)b * R.npix + R.off[j];
  const int nk = R.len[j];
  const float* m = marg[b] + R.off[j];
  const float aj = a_ring[j];
  float acc = 0.f;
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    const float mm = m[k];
    const float r = mm / Kf[base + k];
    const float u = balanced ? r : powf(r, gam);
    out[base + k] = u;
    acc += balanced ? u : (mm > 0.f ? aj * mm * powf(u, -et) : 0.f);
  }
  const float t = block_sum_f(acc, red);
  if (threadIdx.x == 0) part[(size_t)b * R.nring + j] = (double)t;
}

// scalars of iteration k after both half-steps: (al, be) and the ProbState beta used by
// the next K v (the ring DFT scales v' by beta on load)
__global__ void k_g_scalars(int nprob, int nlat, const double* __restrict__ partU, const double* __restrict__ partV,
                            int balanced, double eps, double tau, GScal* __restrict__ sc, ProbState* __restrict__ ps) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nprob) return;
  double su = 0.0, sv = 0.0;
  for (int j = 0; j < nlat; ++j) {
    su += partU[(size_t)b * nlat + j];
    sv += partV[(size_t)b * nlat + j];
  }
  GScal s;
  if (balanced) {
    s.al = 1.0 / su;
    s.be = su;
    s.A = su;
    s.B = 0.0;
  } else {
    const double c = 0.5 * tau * (log(su) - log(sv));
    s.al = exp(c / eps);
    s.be = exp(-c / eps);
    s.A = su;
    s.B = sv;
  }
  sc[b] = s;
  ps[b].beta = s.be;
}

__global__ void k_g_init_state(int nprob, ProbState* ps) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nprob) {
    ps[b].beta = 1.0;
  }
}

__global__ void k_g_set_beta(int nprob, const GScal* __restrict__ sc, ProbState* ps) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nprob) ps[b].beta = sc[b].be;
}

// initial adjoints from Alg. 1's return (T = last iteration): u~, v~, p~, q~
__global__ void k_g_seed(Rings R, const float* const* __restrict__ P, const float* const* __restrict__ Q,
                         const float* __restrict__ U, const float* __restrict__ V, const GScal* __restrict__ sc,
                         int balanced, float eps, float tau, float* __restrict__ ut, float* __restrict__ vt,
                         float* __restrict__ pt, float* __restrict__ qt) {
  const int j = blockIdx.x, b = blockIdx.y;
  const size_t base = (size_t)b * R.npix + R.off[j];
  const int nk = R.len[j];
  const float al = (float)sc[b].al, be = (float)sc[b].be;
  const float et = eps / tau;
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    const float p = P[b][R.off[j] + k], q = Q[b][R.off[j] + k];
    const float u = al * U[base + k], v = be * V[base + k];
    if (balanced) {
      ut[base + k] = p > 0.f ? eps * p / u : 0.f;
      vt[base + k] = q > 0.f ? eps * q / v : 0.f;
      pt[base + k] = p > 0.f ? eps * logf(u) : 0.f;
      qt[base + k] = q > 0.f ? eps * logf(v) : 0.f;
    } else {
      const float lu = logf(u), lv = logf(v);
      ut[base + k] = p > 0.f ? eps * p * expf((-et - 1.f) * lu) : 0.f;
      vt[base + k] = q > 0.f ? eps * q * expf((-et - 1.f) * lv) : 0.f;
      pt[base + k] = -tau * expm1f(-et * lu);
      qt[base + k] = -tau * expm1f(-et * lv);
    }
  }
}

// partial sums per ring of  sum a u~ u'  and  sum a v~ v'
__global__ void k_g_rsum(Rings R, const float* __restrict__ a_ring, const float* __restrict__ ut,
                         const float* __restrict__ vt, const float* __restrict__ U, const float* __restrict__ V,
                         double* __restrict__ p1, double* __restrict__ p2) {
  __shared__ float red[32];
  const int j = blockIdx.x, b = blockIdx.y;
  const size_t base = (size_t)b * R.npix + R.off[j];
  const int nk = R.len[j];
  float s1 = 0.f, s2 = 0.f;
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    s1 += ut[base + k] * U[base + k];
    s2 += vt[base + k] * V[base + k];
  }
  const float aj = a_ring[j];
  const float t1 = block_sum_f(s1, red);
  const float t2 = block_sum_f(s2, red);
  if (threadIdx.x == 0) {
    p1[(size_t)b * R.nring + j] = (double)(aj * t1);
    p2[(size_t)b * R.nring + j] = (double)(aj * t2);
  }
}

struct RevScal {
  double sbar;          // balanced
  double Abar, Bbar;    // unbalanced
};

__global__ void k_g_rscal(int nprob, int nlat, const double* __restrict__ p1, const double* __restrict__ p2,
                          const GScal* __restrict__ sc, int balanced, double eps, double tau,
                          RevScal* __restrict__ rs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nprob) return;
  double r1 = 0.0, r2 = 0.0;
  for (int j = 0; j < nlat; ++j) {
    r1 += p1[(size_t)b * nlat + j];
    r2 += p2[(size_t)b * nlat + j];
  }
  const GScal s = sc[b];
  RevScal o{0.0, 0.0, 0.0};
  if (balanced) {
    // r1 = sum a u~ u', r2 = sum a v~ v';  s = A
    o.sbar = -r1 / (s.A * s.A) + r2;
  } else {
    // cbar = (sum a u~ u_k - sum a v~ v_k)/eps with u_k = E u', v_k = v'/E
    const double cbar = (s.al * r1 - s.be * r2) / eps;
    o.Abar = cbar * tau / (2.0 * s.A);
    o.Bbar = -cbar * tau / (2.0 * s.B);
  }
  rs[b] = o;
}

// first pointwise reverse stage: u~' (before + K (Ku)~), (Ku)~, q~ updates
__global__ void k_g_rev1(Rings R, const float* __restrict__ a_ring, const float* const* __restrict__ P,
                         const float* const* __restrict__ Q, const float* __restrict__ U, const float* __restrict__ V,
                         const GScal* __restrict__ sc, const RevScal* __restrict__ rs, int balanced, float gam, float et,
                         float* __restrict__ ut, const float* __restrict__ vt, float* __restrict__ qt,
                         float* __restrict__ kut, float* __restrict__ pt) {
  const int j = blockIdx.x, b = blockIdx.y;
  const size_t base = (size_t)b * R.npix + R.off[j];
  const int nk = R.len[j];
  const float aj = a_ring[j];
  const GScal s = sc[b];
  const RevScal r = rs[b];
  const float al = (float)s.al, be = (float)s.be;
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    const float p = P[b][R.off[j] + k], q = Q[b][R.off[j] + k];
    const float u1 = U[base + k], v1 = V[base + k];
    float uu, vv;
    if (balanced) {
      uu = al * ut[base + k] + (float)(r.sbar / aj);
      vv = be * vt[base + k];
    } else {
      uu = al * ut[base + k] - (p > 0.f ? (float)r.Abar * et * p * powf(u1, -et - 1.f) : 0.f);
      vv = be * vt[base + k] - (q > 0.f ? (float)r.Bbar * et * q * powf(v1, -et - 1.f) : 0.f);
      pt[base + k] += (float)r.Abar * powf(u1, -et);
      qt[base + k] += (float)r.Bbar * powf(v1, -et);
    }
    ut[base + k] = uu;
    if (q > 0.f) {
      const float vg = balanced ? v1 * v1 : v1 * powf(v1, 1.f / gam);
      kut[base + k] = -gam * vv * vg / q;
      qt[base + k] += gam * vv * v1 / q;
    } else {
      kut[base + k] = 0.f;
    }
  }
}

// second pointwise reverse stage: u~' += K (Ku)~ ; (Kv)~ ; p~ update
__global__ void k_g_rev2(Rings R, const float* const* __restrict__ P, const float* __restrict__ U,
                         const float* __restrict__ kku, int balanced, float gam, float* __restrict__ ut,
                         float* __restrict__ kvt, float* __restrict__ pt) {
  const int j = blockIdx.x, b = blockIdx.y;
  const size_t base = (size_t)b * R.npix + R.off[j];
  const int nk = R.len[j];
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    const float p = P[b][R.off[j] + k];
    const float u1 = U[base + k];
    const float uu = ut[base + k] + kku[base + k];
    if (p > 0.f) {
      const float ug = balanced ? u1 * u1 : u1 * powf(u1, 1.f / gam);
      kvt[base + k] = -gam * uu * ug / p;
      pt[base + k] += gam * uu * u1 / p;
    } else {
      kvt[base + k] = 0.f;
    }
    ut[base + k] = 0.f;   // u~_{k-1} = 0: u_{k-1} does not enter iteration k
  }
}

// dS/dp for pair b from the (p,q) problem b and the (p,p) problem B + b
__global__ void k_g_assemble(Rings R, int batch, const float* __restrict__ a_ring,
                             const float* __restrict__ pt, const float* __restrict__ qt, const double* __restrict__ dm,
                             double eps, float* __restrict__ grad) {
  const int j = blockIdx.x, b = blockIdx.y;
  const size_t n = (size_t)R.npix;
  const size_t o = (size_t)b * n + R.off[j];
  const size_t oA = o;
  const size_t oB = (size_t)(batch + b) * n + R.off[j];
  const int nk = R.len[j];
  const float aj = a_ring[j];
  const float mt = (float)(eps * dm[b]);
  for (int k = threadIdx.x; k < nk; k += blockDim.x)
    grad[o + k] = aj * (pt[oA + k] - 0.5f * (pt[oB + k] + qt[oB + k]) + mt);
}

// envelope form from the converged scalings of all 3B problems (u3, v3 hold u_T, v_T)
__global__ void k_g_envelope(Rings R, int batch, const float* __restrict__ a_ring,
                             const float* __restrict__ u3, const float* __restrict__ v3, const double* __restrict__ dm,
                             int balanced, float eps, float tau, float* __restrict__ grad) {
  const int j = blockIdx.x, b = blockIdx.y;
  const size_t n = (size_t)R.npix;
  const size_t o = (size_t)b * n + R.off[j];
  const size_t oB = (size_t)(batch + b) * n + R.off[j];
  const int nk = R.len[j];
  const float aj = a_ring[j];
  const float et = eps / tau;
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    const float la = logf(u3[o + k]), lpp = logf(u3[oB + k]), lqp = logf(v3[oB + k]);
    float g;
    if (balanced) {
      g = eps * (la - 0.5f * (lpp + lqp)) + (float)(eps * dm[b]);
    } else {
      g = -tau * expm1f(-et * la) + 0.5f * tau * (expm1f(-et * lpp) + expm1f(-et * lqp));
    }
    grad[o + k] = aj * g;
  }
}

__global__ void k_g_fill_ones(float* __restrict__ a, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a[i] = 1.f;
}

// m(p_b) - m(q_b) = sum_i a_i (p_b - q_b)_i in FP64, one block per pair
__global__ void k_g_mass_diff(Rings R, const float* __restrict__ p, const float* __restrict__ q,
                              const float* __restrict__ a_ring, double* __restrict__ dm) {
  __shared__ double red[32];
  const size_t n = (size_t)R.npix;
  const float* pb = p + (size_t)blockIdx.x * n;
  const float* qb = q + (size_t)blockIdx.x * n;
  double s = 0.0;
  for (int j = 0; j < R.nring; ++j) {
    float t = 0.f;
    const float* pr = pb + R.off[j];
    const float* qr = qb + R.off[j];
    for (int k = threadIdx.x; k < R.len[j]; k += blockDim.x) t += pr[k] - qr[k];
    s += (double)a_ring[j] * (double)t;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    dm[blockIdx.x] = t;
  }
}

}  // namespace

// out = K (beta (.) in) (beta per problem from ps when ps != nullptr)
static int heat_fields(Grid& g, const float* in, float* out, int nf, const ProbState* ps, cudaStream_t st) {
  Workspace& w = g.ws;
  int rc = launch_dft_fwd(g, in, nf, ps, ps ? 1 : 0, w.XY, w.ldc, st);
  if (rc) return rc;
  if ((rc = launch_legendre(g, nf, w.XY, w.C, w.XY, w.ldc, st))) return rc;
  EpiParams ep{};
  ep.mode = EPI_PLAIN;
  ep.out = out;
  return launch_idft(g, w.XY, w.ldc, nf, ep, st);
}

int divergence_grad(Grid& g, const float* p, const float* q, int batch, double eps, double tau, int T, int ck,
                    int mode, double* S, float* grad, int* status, cudaStream_t st) {
  const size_t n = (size_t)g.npix;
  const Rings rings{g.ring_len_d, g.ring_off_d, (long long)g.npix, g.nlat};
  const int np3 = 3 * batch, np = 2 * batch;
  const bool balanced = isinf(tau);
  int rc;
  // --- forward for S (all three problems of every pair), also the envelope's potentials
  std::vector<const float*> P3(np3), Q3(np3);
  for (int b = 0; b < batch; ++b) {
    P3[b] = p + b * n;          Q3[b] = q + b * n;
    P3[batch + b] = p + b * n;  Q3[batch + b] = p + b * n;
    P3[2 * batch + b] = q + b * n;  Q3[2 * batch + b] = q + b * n;
  }
  float *u3 = nullptr, *v3 = nullptr, *bufs = nullptr;
  double* dbufs = nullptr;
  const float** plist = nullptr;
  auto cleanup = [&]() {
    cudaFree(u3);
    cudaFree(v3);
    cudaFree(bufs);
    cudaFree(dbufs);
    cudaFree(plist);
  };
  SHOT_CUDA(cudaMalloc(&u3, (size_t)np3 * n * sizeof(float)));
  SHOT_CUDA(cudaMalloc(&v3, (size_t)np3 * n * sizeof(float)));
  std::vector<ProbState> pso;
  int kdone = 0;
  rc = run_sinkhorn_public(g, P3, Q3, eps, tau, T, 0.0, 0, 0, u3, v3, st, pso, &kdone);
  if (rc) { cleanup(); return rc; }
  // m(p_b) - m(q_b) (device, FP64)
  SHOT_CUDA(cudaMalloc(&dbufs, (size_t)batch * sizeof(double)));
  count_launch();
  k_g_mass_diff<<<batch, 256, 0, st>>>(rings, p, q, g.a_d, dbufs);
  SHOT_CUDA(cudaGetLastError());
  std::vector<double> dm(batch);
  SHOT_CUDA(cudaMemcpyAsync(dm.data(), dbufs, batch * sizeof(double), cudaMemcpyDeviceToHost, st));
  SHOT_CUDA(cudaStreamSynchronize(st));
  int worst = SHOT_OK;
  for (int b = 0; b < batch; ++b) {
    const ProbState &A = pso[b], &B = pso[batch + b], &Cq = pso[2 * batch + b];
    S[b] = A.ot - 0.5 * (B.ot + Cq.ot) + 0.5 * eps * dm[b] * dm[b];
    int s = SHOT_OK;
    for (int st3 : {A.status, B.status, Cq.status})
      if (st3 < 0 && (s >= 0 || st3 < s)) s = st3;
    status[b] = s;
    if (s < 0 && (worst >= 0 || s < worst)) worst = s;
  }
  dim3 ew(g.nlat, batch);
  if (mode == SHOT_GRAD_ENVELOPE) {
    count_launch();
    k_g_envelope<<<ew, kEw, 0, st>>>(rings, batch, g.a_d, u3, v3, dbufs, balanced ? 1 : 0, (float)eps,
                                     (float)tau, grad);
    SHOT_CUDA(cudaGetLastError());
    SHOT_CUDA(cudaStreamSynchronize(st));
    cleanup();
    return worst;
  }
  if (worst < 0) {   // no derivative through a broken-down iteration
    cleanup();
    return worst;
  }

  // --- unrolled reverse sweep over the problems (p_b, q_b) and (p_b, p_b)
  if (ck < 1) ck = 1;
  if (ck > T) ck = T > 0 ? T : 1;
  const int nseg = T > 0 ? (T + ck - 1) / ck : 0;
  // device buffers: checkpoints of v' (nseg), segment u', v' (ck each), adjoints
  const size_t fld = (size_t)np * n;
  const size_t nflt = fld * ((size_t)nseg + 2 * (size_t)ck + 7);
  SHOT_CUDA(cudaMalloc(&bufs, nflt * sizeof(float)));
  float* ckpt = bufs;                       // [nseg][np][n]
  float* useg = ckpt + (size_t)nseg * fld;  // [ck][np][n]
  float* vseg = useg + (size_t)ck * fld;
  float* ut = vseg + (size_t)ck * fld;
  float* vt = ut + fld;
  float* pt = vt + fld;
  float* qt = pt + fld;
  float* kf = qt + fld;   // K applied to a field
  float* t1 = kf + fld;   // (Ku)~ / (Kv)~
  float* t2 = t1 + fld;
  int rc2 = ensure_workspace(g, np, st);
  if (rc2) { cleanup(); return rc2; }
  Workspace& w = g.ws;
  // per-problem state: the ring DFT scales by ProbState::beta; scalars per segment iteration
  ProbState* ps = reinterpret_cast<ProbState*>(w.probs);
  GScal* sc = nullptr;
  RevScal* rs = nullptr;
  double* parts = nullptr;
  SHOT_CUDA(cudaMalloc(&sc, (size_t)(ck + 1) * np * sizeof(GScal) + (size_t)(nseg + 1) * np * sizeof(GScal)));
  GScal* sck = sc + (size_t)(ck + 1) * np;   // checkpoint scalars (beta of v' at k0)
  SHOT_CUDA(cudaMalloc(&rs, (size_t)np * sizeof(RevScal)));
  SHOT_CUDA(cudaMalloc(&parts, (size_t)4 * np * g.nlat * sizeof(double)));
  SHOT_CUDA(cudaMalloc(&plist, (size_t)2 * np * sizeof(float*)));
  auto cleanup2 = [&]() {
    cudaFree(sc);
    cudaFree(rs);
    cudaFree(parts);
    cleanup();
  };
  {
    std::vector<const float*> pl(2 * np);
    for (int b = 0; b < batch; ++b) {
      pl[b] = p + b * n;          pl[np + b] = q + b * n;
      pl[batch + b] = p + b * n;  pl[np + batch + b] = p + b * n;
    }
    SHOT_CUDA(cudaMemcpyAsync(plist, pl.data(), 2 * np * sizeof(float*), cudaMemcpyHostToDevice, st));
  }
  const float* const* Pl = plist;
  const float* const* Ql = plist + np;
  double* partU = parts;
  double* partV = parts + (size_t)np * g.nlat;
  const float gam = balanced ? 1.f : (float)(tau / (tau + eps));
  const float et = balanced ? 0.f : (float)(eps / tau);
  const int bal = balanced ? 1 : 0;
  dim3 ewp(g.nlat, np);
  const int nb = (np + 127) / 128;
  if ((rc = launch_heat_mult(g, eps / 4.0, st))) { cleanup2(); return rc; }

  // one forward iteration from (vprev, beta in ps) storing u', v' and the scalars at slot
  auto fwd_iter = [&](const float* vprev, float* uo, float* vo, GScal* slot) -> int {
    int r;
    if ((r = heat_fields(g, vprev, kf, np, ps, st))) return r;
    count_launch();
    k_g_update<<<ewp, kEw, 0, st>>>(rings, g.a_d, Pl, kf, uo, bal, gam, et, partU);
    if ((r = heat_fields(g, uo, kf, np, nullptr, st))) return r;
    count_launch(2);
    k_g_update<<<ewp, kEw, 0, st>>>(rings, g.a_d, Ql, kf, vo, bal, gam, et, partV);
    k_g_scalars<<<nb, 128, 0, st>>>(np, g.nlat, partU, partV, bal, eps, tau, slot, ps);
    SHOT_CUDA(cudaGetLastError());
    return SHOT_OK;
  };

  // pass 1: checkpoints of (v', beta) at k0 = 0, ck, 2ck, ...; v_0 = 1
  count_launch(2);
  k_g_init_state<<<nb, 128, 0, st>>>(np, ps);
  {
    // checkpoint 0: v' = 1, beta = 1
    count_launch();
    k_g_fill_ones<<<1024, 256, 0, st>>>(ckpt, fld);
    std::vector<GScal> one(np, GScal{1.0, 1.0, 0.0, 0.0});
    SHOT_CUDA(cudaMemcpyAsync(sck, one.data(), np * sizeof(GScal), cudaMemcpyHostToDevice, st));
  }
  SHOT_CUDA(cudaGetLastError());
  for (int sgi = 0; sgi + 1 < nseg; ++sgi) {
    const int k0 = sgi * ck;
    const float* vprev = ckpt + (size_t)sgi * fld;
    count_launch();
    k_g_set_beta<<<nb, 128, 0, st>>>(np, sck + (size_t)sgi * np, ps);
    for (int k = k0 + 1; k <= k0 + ck; ++k) {
      float* vo = (k == k0 + ck) ? ckpt + (size_t)(sgi + 1) * fld : vseg;
      if ((rc = fwd_iter(vprev, useg, vo, sc))) { cleanup2(); return rc; }
      vprev = vo;
    }
    SHOT_CUDA(cudaMemcpyAsync(sck + (size_t)(sgi + 1) * np, sc, np * sizeof(GScal), cudaMemcpyDeviceToDevice, st));
  }
  // pass 2: segments from the last, recompute forward, then reverse
  bool seeded = false;
  for (int sgi = nseg - 1; sgi >= 0; --sgi) {
    const int k0 = sgi * ck, k1 = (k0 + ck < T) ? k0 + ck : T;
    const int len = k1 - k0;
    count_launch();
    k_g_set_beta<<<nb, 128, 0, st>>>(np, sck + (size_t)sgi * np, ps);
    const float* vprev = ckpt + (size_t)sgi * fld;
    for (int i = 0; i < len; ++i) {
      if ((rc = fwd_iter(vprev, useg + (size_t)i * fld, vseg + (size_t)i * fld, sc + (size_t)i * np))) {
        cleanup2();
        return rc;
      }
      vprev = vseg + (size_t)i * fld;
    }
    for (int i = len - 1; i >= 0; --i) {
      const float* U = useg + (size_t)i * fld;
      const float* V = vseg + (size_t)i * fld;
      const GScal* s_i = sc + (size_t)i * np;
      if (!seeded) {
        count_launch();
        k_g_seed<<<ewp, kEw, 0, st>>>(rings, Pl, Ql, U, V, s_i, bal, (float)eps, (float)tau, ut, vt, pt, qt);
        seeded = true;
      }
      count_launch(3);
      k_g_rsum<<<ewp, kEw, 0, st>>>(rings, g.a_d, ut, vt, U, V, partU, partV);
      k_g_rscal<<<nb, 128, 0, st>>>(np, g.nlat, partU, partV, s_i, bal, eps, tau, rs);
      k_g_rev1<<<ewp, kEw, 0, st>>>(rings, g.a_d, Pl, Ql, U, V, s_i, rs, bal, gam, et, ut, vt, qt, t1, pt);
      SHOT_CUDA(cudaGetLastError());
      if ((rc = heat_fields(g, t1, t2, np, nullptr, st))) { cleanup2(); return rc; }
      count_launch();
      k_g_rev2<<<ewp, kEw, 0, st>>>(rings, Pl, U, t2, bal, gam, ut, t1, pt);
      SHOT_CUDA(cudaGetLastError());
      if ((rc = heat_fields(g, t1, vt, np, nullptr, st))) { cleanup2(); return rc; }
    }
  }
  if (!seeded) {   // T == 0: only the direct terms
    SHOT_CUDA(cudaMemsetAsync(pt, 0, fld * sizeof(float), st));
    SHOT_CUDA(cudaMemsetAsync(qt, 0, fld * sizeof(float), st));
  }
  count_launch();
  k_g_assemble<<<ew, kEw, 0, st>>>(rings, batch, g.a_d, pt, qt, dbufs, eps, grad);
  SHOT_CUDA(cudaGetLastError());
  SHOT_CUDA(cudaStreamSynchronize(st));
  cleanup2();
  return worst;
}

}  // namespace shot
