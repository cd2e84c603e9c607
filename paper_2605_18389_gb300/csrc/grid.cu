// Grid set-up: Gauss-Legendre nodes and weights, area weights, ring-DFT twiddles, the
// parity-folded orthonormal associated Legendre table, tile lists and workspaces.
//
// FP64 is used on the device only here (nodes, weights, table seeds/recurrence), the
// values being rounded to FP32 (or split into bf16 hi + lo) for the hot path.
#include <math.h>
#include <algorithm>
#include <cmath>
#include <functional>
#include <vector>

#include "shot_internal.cuh"

namespace shot {

namespace {

// GL nodes by Newton's method on P_n from cos(pi (k - 1/4)/(n + 1/2)) (App. C.1,
// "Gauss-Legendre": the latitudes are the roots of P_nlat); w = 2/((1-x^2) P_n'(x)^2).
// One thread per north-hemisphere node; the south half is its exact mirror.
__global__ void k_gl_nodes(int n, double* __restrict__ x, double* __restrict__ w) {
  const int nh = (n + 1) / 2;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nh) return;
  double xj = cos(M_PI * (j + 0.75) / (n + 0.5));
  double dp = 1.0;
  for (int it = 0; it < 60; ++it) {
    double p0 = 1.0, p1 = xj;
    for (int l = 2; l <= n; ++l) {
      const double p2 = ((2 * l - 1) * xj * p1 - (l - 1) * p0) / l;
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) { p0 = 1.0; p1 = xj; }
    dp = n * (p0 - xj * p1) / (1.0 - xj * xj);
    const double dx = p1 / dp;
    xj -= dx;
    if (fabs(dx) < 1e-16) break;
  }
  {  // derivative at the converged node
    double p0 = 1.0, p1 = xj;
    for (int l = 2; l <= n; ++l) {
      const double p2 = ((2 * l - 1) * xj * p1 - (l - 1) * p0) / l;
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) { p0 = 1.0; p1 = xj; }
    dp = n * (p0 - xj * p1) / (1.0 - xj * xj);
  }
  if ((n & 1) && j == nh - 1) xj = 0.0;   // the equator node of an odd grid
  const double wj = 2.0 / ((1.0 - xj * xj) * dp * dp);
  x[j] = xj;
  w[j] = wj;
  x[n - 1 - j] = -xj;
  w[n - 1 - j] = wj;
}

// Equiangular Clenshaw-Curtis nodes x_j = cos(pi j/N), N = n-1, both poles included
// (App. C.1, "Equiangular ... Clenshaw-Curtis"), and the closed-form weights of the
// degree-N interpolatory rule on them:
//   w_j = (c_j/N) (1 - sum_{k=1}^{floor(N/2)} b_k cos(2 pi k j / N) / (4k^2 - 1)),
// c_j = 1 for j in {0, N} else 2, b_k = 1 for k = N/2 else 2.  The cosine argument is
// reduced exactly (k j mod N) before sincospi.  One thread per north-half node; the
// south half is its exact mirror.
__global__ void k_cc_nodes(int n, double* __restrict__ x, double* __restrict__ w) {
  const int nh = (n + 1) / 2;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nh) return;
  const int N = n - 1;
  double xj = cospi((double)j / N);
  if (2 * j == N) xj = 0.0;   // the equator ring of an odd grid
  double s = 0.0;
  for (int k = 1; 2 * k <= N; ++k) {
    const long long r = ((long long)k * j) % N;
    const double bk = (2 * k == N) ? 1.0 : 2.0;
    s += bk * cospi(2.0 * (double)r / N) / (4.0 * k * k - 1.0);
  }
  const double cj = (j == 0) ? 1.0 : 2.0;
  const double wj = cj / N * (1.0 - s);
  x[j] = xj;
  w[j] = wj;
  x[n - 1 - j] = -xj;
  w[n - 1 - j] = wj;
}

__global__ void k_area(int nlat, int nlon, const double* __restrict__ w, float* __restrict__ a) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nlat) a[j] = (float)(w[j] * (2.0 * M_PI / nlon));
}

// Orthonormal Pbar_lm(x_jh) (App. B) by the standard recurrences:
//   Pbar_00 = 1/sqrt(4 pi); Pbar_mm = -sqrt((2m+1)/(2m)) sin(theta) Pbar_{m-1,m-1};
//   Pbar_{m+1,m} = sqrt(2m+3) x Pbar_mm;
//   Pbar_lm = a_lm (x Pbar_{l-1,m} - b_lm Pbar_{l-2,m}),
//   a_lm = sqrt((4l^2-1)/(l^2-m^2)), b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)).
// One thread per (m, jh); row l goes to block (m, (l-m) mod 2), row (l-m)/2.
// tabT (optional): the same values at [blk][jh][ldi] (degrees contiguous).
__global__ void k_pbar(int lmax, int nh, const double* __restrict__ x, const long long* __restrict__ row_off,
                       int ldt, float* __restrict__ tab, __nv_bfloat16* __restrict__ hi,
                       __nv_bfloat16* __restrict__ lo, float* __restrict__ tabT, int ldi) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (j >= nh) return;
  const double xj = x[j];
  const double st = sqrt((1.0 - xj) * (1.0 + xj));
  double pmm = 0.28209479177387814;   // 1/sqrt(4 pi)
  for (int k = 1; k <= m; ++k) pmm *= -sqrt((2.0 * k + 1.0) / (2.0 * k)) * st;
  auto store = [&](int l, double val) {
    const int d = l - m;
    const int blk = 2 * m + (d & 1);
    const size_t off = (size_t)(row_off[blk] + (d >> 1)) * ldt + j;
    if (tab) tab[off] = (float)val;
    if (tabT) tabT[((size_t)blk * nh + j) * ldi + (d >> 1)] = (float)val;
    if (hi) {
      const __nv_bfloat16 h = __double2bfloat16(val);
      const __nv_bfloat16 l = __double2bfloat16(val - (double)__bfloat162float(h));
      hi[off] = h;
      lo[off] = l;
    }
  };
  store(m, pmm);
  if (m == lmax) return;
  double p2 = pmm;
  double p1 = sqrt(2.0 * m + 3.0) * xj * pmm;
  store(m + 1, p1);
  for (int l = m + 2; l <= lmax; ++l) {
    const double ll = (double)l * l, mm = (double)m * m, l1 = (double)(l - 1) * (l - 1);
    const double a = sqrt((4.0 * ll - 1.0) / (ll - mm));
    const double b = sqrt((l1 - mm) / (4.0 * l1 - 1.0));
    const double pl = a * (xj * p1 - b * p2);
    store(l, pl);
    p2 = p1;
    p1 = pl;
  }
}

__global__ void k_heat(int lmax, double t, float* __restrict__ h) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l <= lmax) h[l] = (float)exp(-t * (double)l * (double)(l + 1));
}

// C[row_off[blk] + i][2f + {0,1}]  <->  coeffs[f][l][m][{re,im}],  l = m + p + 2i
__global__ void k_coeff_gather(int lmax, int nf, const long long* __restrict__ row_off,
                               const float* __restrict__ C, int ldc, float* __restrict__ coeffs) {
  const int L = lmax + 1;
  const size_t total = (size_t)nf * L * L;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(idx % L);
    const int l = (int)((idx / L) % L);
    const int f = (int)(idx / ((size_t)L * L));
    float2 v = make_float2(0.f, 0.f);
    if (m <= l) {
      const int d = l - m;
      const long long row = row_off[2 * m + (d & 1)] + (d >> 1);
      v = *reinterpret_cast<const float2*>(C + (size_t)row * ldc + 2 * f);
    }
    reinterpret_cast<float2*>(coeffs)[idx] = v;
  }
}

__global__ void k_coeff_scatter(int lmax, int nf, const long long* __restrict__ row_off,
                                const float* __restrict__ coeffs, float* __restrict__ C, int ldc) {
  const int L = lmax + 1;
  const size_t total = (size_t)nf * L * L;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(idx % L);
    const int l = (int)((idx / L) % L);
    const int f = (int)(idx / ((size_t)L * L));
    if (m > l) continue;
    float2 v = reinterpret_cast<const float2*>(coeffs)[idx];
    if (m == 0) v.y = 0.f;
    const int d = l - m;
    const long long row = row_off[2 * m + (d & 1)] + (d >> 1);
    *reinterpret_cast<float2*>(C + (size_t)row * ldc + 2 * f) = v;
  }
}

}  // namespace

// Factorisation of the ring length into the radices the shared-memory FFT has
// butterflies for.  Fewest stages first; then the bank conflicts of the first stage's
// stores (lanes at a stride of R complex values: conflict-free for odd R, gcd(2R, 32)/2-way
// otherwise), which puts an odd radix first when there is one and otherwise the smallest;
// then the smallest largest radix (registers).
bool make_fft_plan(int N, FftPlan* pl) {
  if (N < 1 || N >= (1 << 16)) return false;
  // prime factors above 5 become generic stages, placed first (their stage twiddles are 1)
  std::vector<int> gen;
  {
    int m = N;
    for (int p : {2, 3, 5})
      while (m % p == 0) m /= p;
    for (int p = 7; (long long)p * p <= m; p += 2)
      while (m % p == 0) {
        gen.push_back(p);
        m /= p;
      }
    if (m > 1) gen.push_back(m);
    std::sort(gen.rbegin(), gen.rend());
    for (int p : gen) N /= p;   // the 2,3,5-smooth part goes to the radix search below
  }
  const int Nfull = [&] { int t = N; for (int p : gen) t *= p; return t; }();
  static const int kRad[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
  const int nrad = (int)(sizeof(kRad) / sizeof(kRad[0]));
  auto order = [](std::vector<int> f) {
    std::vector<int> odd, even;
    for (int r : f) (r & 1 ? odd : even).push_back(r);
    std::sort(odd.rbegin(), odd.rend());
    std::sort(even.begin(), even.end());
    odd.insert(odd.end(), even.begin(), even.end());
    return odd;
  };
  auto cost = [](const std::vector<int>& f) {
    if (f.empty()) return 0.0;
    int g = 2 * f[0], b = 32;
    while (b) { const int t = g % b; g = b; b = t; }
    const int deg = (f[0] & 1) ? 1 : g / 2;
    const int mx = *std::max_element(f.begin(), f.end());
    return (double)f.size() + 0.15 * (deg - 1) + 0.01 * mx;
  };
  std::vector<int> best, cur;
  double best_cost = 1e30;
  bool found = false;
  // multisets in non-increasing radix-table order
  std::function<void(int, int)> dfs = [&](int n, int from) {
    if (n == 1) {
      const std::vector<int> f = order(cur);
      const double c = cost(f);
      if (!found || c < best_cost) { best = f; best_cost = c; found = true; }
      return;
    }
    if ((int)cur.size() >= 16) return;
    for (int i = from; i < nrad; ++i)
      if (n % kRad[i] == 0) {
        cur.push_back(kRad[i]);
        dfs(n / kRad[i], i);
        cur.pop_back();
      }
  };
  dfs(N, 0);
  if (!found) return false;
  best.insert(best.begin(), gen.begin(), gen.end());
  if (best.size() > 16) return false;
  N = Nfull;
  pl->N = N;
  pl->nst = (int)best.size();
  // exact division by multiply-high for operands below 2^16
  auto mul = [](uint32_t d) -> uint32_t { return d <= 1 ? 0u : (uint32_t)((((uint64_t)1 << 32) + d - 1) / d); };
  int Ns = 1, off = 0, roff = N;
  for (int s = 0; s < pl->nst; ++s) {
    pl->R[s] = best[s];
    pl->tw_off[s] = off;
    pl->root_off[s] = 0;
    if (!fft_radix_compiled(best[s])) {
      pl->root_off[s] = roff;
      roff += best[s];
    }
    pl->ns_mul[s] = mul((uint32_t)Ns);
    pl->nr_mul[s] = mul((uint32_t)(N / pl->R[s]));
    if (s > 0) off += (pl->R[s] - 1) * Ns;
    Ns *= pl->R[s];
  }
  return true;
}

void fft_plan_twiddles(const FftPlan& pl, std::vector<float2>& tw) {
  const int N = pl.N;
  size_t total = N;
  for (int s = 0; s < pl.nst; ++s)
    if (!fft_radix_compiled(pl.R[s])) total = std::max(total, (size_t)pl.root_off[s] + pl.R[s]);
  tw.assign(total, make_float2(1.f, 0.f));
  for (int s = 0; s < pl.nst; ++s)   // roots W_R^e of the generic stages
    if (!fft_radix_compiled(pl.R[s]))
      for (int e = 0; e < pl.R[s]; ++e) {
        const double a = 2.0 * M_PI * (double)e / pl.R[s];
        tw[pl.root_off[s] + e] = make_float2((float)std::cos(a), (float)-std::sin(a));
      }
  int Ns = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.R[s];
    if (s > 0) {
      const long long tstep = N / (Ns * R);
      for (int r = 1; r < R; ++r)
        for (int k = 0; k < Ns; ++k) {
          const long long e = ((long long)k * r * tstep) % N;   // exact index reduction
          const double a = 2.0 * M_PI * (double)e / N;
          tw[pl.tw_off[s] + (r - 1) * Ns + k] = make_float2((float)std::cos(a), (float)-std::sin(a));
        }
    }
    Ns *= R;
  }
}

int build_grid_tables(Grid& g, cudaStream_t st) {
  const int nlat = g.nlat, nh = g.nh, L = g.lmax + 1;
  SHOT_CUDA(cudaMalloc(&g.x_d, nlat * sizeof(double)));
  SHOT_CUDA(cudaMalloc(&g.w_d, nlat * sizeof(double)));
  SHOT_CUDA(cudaMalloc(&g.a_d, nlat * sizeof(float)));
  SHOT_CUDA(cudaMalloc(&g.tw_d, (size_t)std::max(fft_tw_len(g.plan), g.nlon) * sizeof(float2)));
  SHOT_CUDA(cudaMalloc(&g.h_d, L * sizeof(float)));
  if (g.quad == SHOT_QUAD_HEALPIX) {
    // closed-form ring geometry on the host (FP64), then to the device
    healpix_geometry(g, g.nside);
    std::vector<float> af(g.a_ring.begin(), g.a_ring.end());
    SHOT_CUDA(cudaMemcpyAsync(g.x_d, g.x.data(), nlat * sizeof(double), cudaMemcpyHostToDevice, st));
    SHOT_CUDA(cudaMemcpyAsync(g.w_d, g.w.data(), nlat * sizeof(double), cudaMemcpyHostToDevice, st));
    SHOT_CUDA(cudaMemcpyAsync(g.a_d, af.data(), nlat * sizeof(float), cudaMemcpyHostToDevice, st));
    std::vector<int2> ph(nlat);
    for (int i = 0; i < nlat; ++i) ph[i] = make_int2(g.ring_phase[i].first, g.ring_phase[i].second);
    SHOT_CUDA(cudaMalloc(&g.ring_phase_d, nlat * sizeof(int2)));
    SHOT_CUDA(cudaMemcpyAsync(g.ring_phase_d, ph.data(), nlat * sizeof(int2), cudaMemcpyHostToDevice, st));
    // ring FFT plans: one per distinct length with factors 2, 3, 5 only
    std::vector<FftPlan> plans;
    std::vector<int> ring_plan(nlat, -1), tw_base;
    std::vector<float2> tw_all;
    for (int i = 0; i < nlat; ++i) {
      const int n = g.ring_len[i];
      int pi = -1;
      for (size_t k = 0; k < plans.size(); ++k)
        if (plans[k].N == n) pi = (int)k;
      if (pi < 0) {
        FftPlan pl;
        if (make_fft_plan(n, &pl)) {
          std::vector<float2> tw;
          fft_plan_twiddles(pl, tw);
          pi = (int)plans.size();
          plans.push_back(pl);
          tw_base.push_back((int)tw_all.size());
          tw_all.insert(tw_all.end(), tw.begin(), tw.end());
        }
      }
      ring_plan[i] = pi;
    }
    SHOT_CUDA(cudaMalloc(&g.ring_plan_d, nlat * sizeof(int)));
    SHOT_CUDA(cudaMemcpyAsync(g.ring_plan_d, ring_plan.data(), nlat * sizeof(int), cudaMemcpyHostToDevice, st));
    if (!plans.empty()) {
      SHOT_CUDA(cudaMalloc(&g.hp_plan_d, plans.size() * sizeof(FftPlan)));
      SHOT_CUDA(cudaMalloc(&g.hp_tw_d, tw_all.size() * sizeof(float2)));
      SHOT_CUDA(cudaMalloc(&g.hp_tw_base_d, tw_base.size() * sizeof(int)));
      SHOT_CUDA(cudaMemcpyAsync(g.hp_plan_d, plans.data(), plans.size() * sizeof(FftPlan), cudaMemcpyHostToDevice, st));
      SHOT_CUDA(cudaMemcpyAsync(g.hp_tw_d, tw_all.data(), tw_all.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
      SHOT_CUDA(cudaMemcpyAsync(g.hp_tw_base_d, tw_base.data(), tw_base.size() * sizeof(int), cudaMemcpyHostToDevice,
                                st));
    }
    SHOT_CUDA(cudaStreamSynchronize(st));   // af, ph, the plans and tables are locals
    count_launch();
    k_heat<<<(L + 255) / 256, 256, 0, st>>>(g.lmax, 0.0, g.h_d);
    SHOT_CUDA(cudaGetLastError());
  } else {
    count_launch(3);
    if (g.quad == SHOT_QUAD_CLENSHAW_CURTIS)
      k_cc_nodes<<<(nh + 127) / 128, 128, 0, st>>>(nlat, g.x_d, g.w_d);
    else
      k_gl_nodes<<<(nh + 127) / 128, 128, 0, st>>>(nlat, g.x_d, g.w_d);
    k_area<<<(nlat + 255) / 256, 256, 0, st>>>(nlat, g.nlon, g.w_d, g.a_d);
    k_heat<<<(L + 255) / 256, 256, 0, st>>>(g.lmax, 0.0, g.h_d);
    SHOT_CUDA(cudaGetLastError());
    std::vector<float2> tw;
    fft_plan_twiddles(g.plan, tw);
    SHOT_CUDA(cudaMemcpyAsync(g.tw_d, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    SHOT_CUDA(cudaStreamSynchronize(st));   // tw is a local
    g.ring_len.assign(nlat, g.nlon);
    g.ring_off.assign(nlat + 1, 0);
    for (int i = 0; i < nlat; ++i) g.ring_off[i + 1] = g.ring_off[i] + g.nlon;
    g.npix = (size_t)nlat * g.nlon;
  }
  SHOT_CUDA(cudaMalloc(&g.ring_len_d, nlat * sizeof(int)));
  SHOT_CUDA(cudaMalloc(&g.ring_off_d, (nlat + 1) * sizeof(long long)));
  SHOT_CUDA(cudaMemcpyAsync(g.ring_len_d, g.ring_len.data(), nlat * sizeof(int), cudaMemcpyHostToDevice, st));
  SHOT_CUDA(cudaMemcpyAsync(g.ring_off_d, g.ring_off.data(), (nlat + 1) * sizeof(long long), cudaMemcpyHostToDevice,
                            st));

  // blocks (m, p): rows M = (lmax - m - p)/2 + 1 when lmax - m - p >= 0
  g.nblk = 2 * L;
  g.M.assign(g.nblk, 0);
  g.row_off.assign(g.nblk + 1, 0);
  for (int m = 0; m < L; ++m)
    for (int p = 0; p < 2; ++p) {
      const int d = g.lmax - m - p;
      g.M[2 * m + p] = d >= 0 ? d / 2 + 1 : 0;
    }
  for (int b = 0; b < g.nblk; ++b) g.row_off[b + 1] = g.row_off[b] + g.M[b];
  g.rows_total = g.row_off[g.nblk];
  g.ldt = (nh + 15) / 16 * 16;
  SHOT_CUDA(cudaMalloc(&g.M_d, g.nblk * sizeof(int)));
  SHOT_CUDA(cudaMalloc(&g.row_off_d, (g.nblk + 1) * sizeof(long long)));
  SHOT_CUDA(cudaMemcpyAsync(g.M_d, g.M.data(), g.nblk * sizeof(int), cudaMemcpyHostToDevice, st));
  SHOT_CUDA(cudaMemcpyAsync(g.row_off_d, g.row_off.data(), (g.nblk + 1) * sizeof(long long),
                            cudaMemcpyHostToDevice, st));

  const size_t tab_elems = (size_t)g.rows_total * g.ldt;
  float* tab = nullptr;
  __nv_bfloat16 *hi = nullptr, *lo = nullptr;
  g.ldi = (g.M[0] + 7) / 8 * 8;
  if (g.mode == SHOT_RECURRENCE) {
    int rc = tf32_kernels(g) ? build_tf32_recurrence(g, st) : build_recurrence(g, st);
    if (rc) return rc;
  } else {
  float* tabT = nullptr;
  if (g.precision == SHOT_FP32 || g.precision == SHOT_TF32X3) {
    SHOT_CUDA(cudaMalloc(&g.tab, tab_elems * sizeof(float)));
    SHOT_CUDA(cudaMemsetAsync(g.tab, 0, tab_elems * sizeof(float), st));
    tab = g.tab;
    if (g.precision == SHOT_TF32X3) {
      const size_t tt = (size_t)g.nblk * nh * g.ldi;
      SHOT_CUDA(cudaMalloc(&g.tabT, tt * sizeof(float)));
      SHOT_CUDA(cudaMemsetAsync(g.tabT, 0, tt * sizeof(float), st));
      tabT = g.tabT;
    }
  } else {
    SHOT_CUDA(cudaMalloc(&g.tab_hi, tab_elems * sizeof(__nv_bfloat16)));
    SHOT_CUDA(cudaMalloc(&g.tab_lo, tab_elems * sizeof(__nv_bfloat16)));
    SHOT_CUDA(cudaMemsetAsync(g.tab_hi, 0, tab_elems * sizeof(__nv_bfloat16), st));
    SHOT_CUDA(cudaMemsetAsync(g.tab_lo, 0, tab_elems * sizeof(__nv_bfloat16), st));
    hi = g.tab_hi;
    lo = g.tab_lo;
  }
  dim3 gp((nh + 127) / 128, L);
  count_launch();
  k_pbar<<<gp, 128, 0, st>>>(g.lmax, nh, g.x_d, g.row_off_d, g.ldt, tab, hi, lo, tabT, g.ldi);
  SHOT_CUDA(cudaGetLastError());
  }

  // tile lists: analysis tiles cover the rows i of each block, synthesis tiles the nodes
  std::vector<Tile> ta, ts;
  for (int b = 0; b < g.nblk; ++b) {
    for (int r = 0; r < g.M[b]; r += g.bm_ana) ta.push_back({b, r});
    if (g.M[b] > 0)
      for (int r = 0; r < nh; r += g.bm_syn) ts.push_back({b, r});
  }
  // largest contraction first (synthesis work is proportional to M)
  std::stable_sort(ts.begin(), ts.end(), [&](const Tile& a, const Tile& b) { return g.M[a.blk] > g.M[b.blk]; });
  g.ntiles_ana = (int)ta.size();
  g.ntiles_syn = (int)ts.size();
  SHOT_CUDA(cudaMalloc(&g.tiles_ana, ta.size() * sizeof(Tile)));
  SHOT_CUDA(cudaMalloc(&g.tiles_syn, ts.size() * sizeof(Tile)));
  SHOT_CUDA(cudaMemcpyAsync(g.tiles_ana, ta.data(), ta.size() * sizeof(Tile), cudaMemcpyHostToDevice, st));
  SHOT_CUDA(cudaMemcpyAsync(g.tiles_syn, ts.data(), ts.size() * sizeof(Tile), cudaMemcpyHostToDevice, st));

  if (g.quad != SHOT_QUAD_HEALPIX) {   // nodes and weights were made on the device
    g.x.resize(nlat);
    g.w.resize(nlat);
    g.a_ring.resize(nlat);
    SHOT_CUDA(cudaMemcpyAsync(g.x.data(), g.x_d, nlat * sizeof(double), cudaMemcpyDeviceToHost, st));
    SHOT_CUDA(cudaMemcpyAsync(g.w.data(), g.w_d, nlat * sizeof(double), cudaMemcpyDeviceToHost, st));
    SHOT_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < nlat; ++j) g.a_ring[j] = g.w[j] * (2.0 * M_PI / g.nlon);
  }
  SHOT_CUDA(cudaStreamSynchronize(st));
  return SHOT_OK;
}

int launch_heat_mult(const Grid& g, double t, cudaStream_t st) {
  const int L = g.lmax + 1;
  count_launch();
  k_heat<<<(L + 255) / 256, 256, 0, st>>>(g.lmax, t, g.h_d);
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

int launch_coeff_gather(const Grid& g, const float* C, int ldc, int nf, float* coeffs, cudaStream_t st) {
  count_launch();
  k_coeff_gather<<<1024, 256, 0, st>>>(g.lmax, nf, g.row_off_d, C, ldc, coeffs);
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

int launch_coeff_scatter(const Grid& g, const float* coeffs, int nf, float* C, int ldc, cudaStream_t st) {
  count_launch();
  k_coeff_scatter<<<1024, 256, 0, st>>>(g.lmax, nf, g.row_off_d, coeffs, C, ldc);
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

int ensure_workspace(Grid& g, int nf, cudaStream_t st) {
  Workspace& w = g.ws;
  if (w.dev_int == nullptr) {
    SHOT_CUDA(cudaMalloc(&w.dev_int, 16 * sizeof(int)));
    SHOT_CUDA(cudaMemsetAsync(w.dev_int, 0, 16 * sizeof(int), st));
    SHOT_CUDA(cudaMallocHost(&w.host_int, 16 * sizeof(int)));
  }
  if (nf <= w.nf_cap) return SHOT_OK;
  SHOT_CUDA(cudaStreamSynchronize(st));
  cudaFree(w.XY);
  cudaFree(w.Yb);
  w.Yb = nullptr;
  cudaFree(w.C);
  cudaFree(w.part);
  cudaFree(w.probs);
  cudaFree(w.marg);
  cudaFree(w.ct_hi);
  cudaFree(w.ct_lo);
  cudaFree(w.ct32);
  w.ct32 = nullptr;
  cudaFree(w.taus);
  w.taus = nullptr;
  w.ct_hi = w.ct_lo = nullptr;
  w.nmma_cap = 0;
  if (w.host_probs) cudaFreeHost(w.host_probs);
  w.XY = w.C = nullptr;
  w.part = nullptr;
  w.probs = nullptr;
  w.marg = nullptr;
  w.host_probs = nullptr;
  w.nf_cap = 0;
  const int ldc = (2 * nf + 3) / 4 * 4;
  const size_t xy = (size_t)g.nblk * g.nh * ldc;
  const size_t cc = (size_t)g.rows_total * ldc;
  SHOT_CUDA(cudaMalloc(&w.XY, xy * sizeof(float)));
  SHOT_CUDA(cudaMalloc(&w.Yb, xy * sizeof(float)));
  SHOT_CUDA(cudaMemsetAsync(w.Yb, 0, xy * sizeof(float), st));
  SHOT_CUDA(cudaMalloc(&w.C, cc * sizeof(float)));
  SHOT_CUDA(cudaMalloc(&w.part, (size_t)nf * g.nh * NPART * sizeof(double)));
  SHOT_CUDA(cudaMalloc(&w.probs, (size_t)nf * sizeof(ProbState)));
  SHOT_CUDA(cudaMalloc(&w.marg, (size_t)4 * nf * sizeof(float*)));
  SHOT_CUDA(cudaMalloc(&w.taus, (size_t)nf * sizeof(double)));
  SHOT_CUDA(cudaMallocHost(&w.host_probs, (size_t)nf * sizeof(ProbState)));
  // X and C are never read before written except padding columns; keep them finite
  SHOT_CUDA(cudaMemsetAsync(w.XY, 0, xy * sizeof(float), st));
  SHOT_CUDA(cudaMemsetAsync(w.C, 0, cc * sizeof(float), st));
  if (g.precision == SHOT_BF16X3 && !tf32_kernels(g)) {
    w.nmma_cap = tc_nmma(nf);
    const size_t ct = (size_t)g.nblk * w.nmma_cap * g.ldi;
    SHOT_CUDA(cudaMalloc(&w.ct_hi, ct * sizeof(__nv_bfloat16)));
    SHOT_CUDA(cudaMalloc(&w.ct_lo, ct * sizeof(__nv_bfloat16)));
    SHOT_CUDA(cudaMemsetAsync(w.ct_hi, 0, ct * sizeof(__nv_bfloat16), st));
    SHOT_CUDA(cudaMemsetAsync(w.ct_lo, 0, ct * sizeof(__nv_bfloat16), st));
  }
  if (tf32_kernels(g)) {
    w.nmma_cap = tc_nmma(nf);
    const size_t ct = (size_t)g.nblk * w.nmma_cap * g.ldi;
    SHOT_CUDA(cudaMalloc(&w.ct32, ct * sizeof(float)));
    SHOT_CUDA(cudaMemsetAsync(w.ct32, 0, ct * sizeof(float), st));
  }
  w.ldc = ldc;
  w.nf_cap = nf;
  return SHOT_OK;
}

}  // namespace shot
