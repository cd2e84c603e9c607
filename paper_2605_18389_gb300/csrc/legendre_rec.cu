// Legendre contractions with the associated Legendre values regenerated on the fly
// (SHOT_RECURRENCE): O(n) memory instead of the O(n^{3/2}) table (Sec. 3.2, "O(n)
// memory ... no kernel matrix is ever formed").
//
// Per order m and node x_jh (north hemisphere) the grid keeps a seed: the first degree
// l_s >= m with |Pbar_{l_s m}(x_jh)| >= 2^-100 and the FP64-computed values
// Pbar_{l_s m}, Pbar_{l_s+1, m} (rounded to FP32); below l_s the functions are < 2^-100
// (they underflow in FP32 near the poles at high m) and are taken as 0.  From the seed the
// normalised three-term recurrence of App. B runs in double-float arithmetic (every value
// and coefficient an unevaluated FP32 pair hi + lo, ~44 significant bits; a plain FP32
// recurrence drifts by ~1e-7 per degree, 5e-5 at degree 719):
//   Pbar_lm = a_lm (x Pbar_{l-1,m} - b_lm Pbar_{l-2,m}),
// with a_lm, b_lm from a (lmax+1)(lmax+2)/2 coefficient table (FP64 rounded to pairs).
//   analysis:  a CTA owns (m, parity, 48-column tile); it marches l in chunks, its threads
//              generating 32 rows of the parity into shared memory per chunk, and contracts
//              them against the X tile (also in shared memory), times h_l.
//   synthesis: a thread owns one node and a column tile, marches l in registers and
//              accumulates Y[jh][c] += Pbar_lm(x_jh) C[l][c], reading coefficient rows from
//              shared memory.
#include "shot_internal.cuh"

namespace shot {
namespace {

constexpr int kRecThreads = 128;
constexpr int kRB = 32;     // rows per analysis chunk
constexpr int kRN = 48;     // columns per CTA

struct Seed {
  int ls;
  float p0h, p0l, p1h, p1l;
};

// double-float helpers (Dekker/Knuth error-free transformations with FMA); the _rn
// intrinsics are never contracted, which the transformations rely on
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const float s = __fadd_rn(p, e);
  return DF{s, __fsub_rn(e, __fsub_rn(s, p))};
}
__device__ __forceinline__ DF df_sub(DF a, DF b) {
  const float s = __fsub_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  float e = __fsub_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fadd_rn(b.h, bb));
  e = __fadd_rn(e, __fsub_rn(a.l, b.l));
  const float t = __fadd_rn(s, e);
  return DF{t, __fsub_rn(e, __fsub_rn(t, s))};
}

// next value of the recurrence from (Pbar_{l-1}, Pbar_{l-2}) with ab = (a_h, a_l, b_h, b_l)
__device__ __forceinline__ DF rec_step(DF x, DF pm1, DF pm2, float4 ab) {
  return df_mul(DF{ab.x, ab.y}, df_sub(df_mul(x, pm1), df_mul(DF{ab.z, ab.w}, pm2)));
}

// Analysis, one CTA per (m, parity, column tile): C[i][c] = h_l sum_jh Pbar_lm(x_jh) X[jh][c].
// NPT nodes per thread for the recurrence (nh <= NPT * kAnaThreads).
constexpr int kAnaThreads = 256;

template <int NPT>
__global__ void __launch_bounds__(kAnaThreads) k_ana_rec(int lmax, int nh, const float2* __restrict__ xf,
                                                         const Seed* __restrict__ seeds,
                                                         const float4* __restrict__ coef,
                                                         const long long* __restrict__ coef_off,
                                                         const int* __restrict__ Mrows,
                                                         const long long* __restrict__ row_off,
                                                         const float* __restrict__ X, int ldc, int ncols,
                                                         const float* __restrict__ h, float* __restrict__ C) {
  extern __shared__ float sm[];
  const int blk = blockIdx.x;
  const int m = blk >> 1, p = blk & 1;
  const int M = Mrows[blk];
  if (M == 0) return;
  const int n0 = blockIdx.y * kRN;
  float* Xs = sm;                       // [nh][kRN]
  float* Ps = sm + (size_t)nh * kRN;    // [nh][kRB] (node-major, then row)
  const float* Xb = X + (size_t)blk * nh * ldc;
  for (int idx = threadIdx.x; idx < nh * kRN; idx += blockDim.x) {
    const int k = idx / kRN, c = idx - k * kRN;
    Xs[idx] = (n0 + c < ncols) ? Xb[(size_t)k * ldc + n0 + c] : 0.f;
  }
  DF st1[NPT], st2[NPT], xs[NPT], s0[NPT], s1[NPT];
  int ls[NPT];
#pragma unroll
  for (int r = 0; r < NPT; ++r) {
    const int jh = threadIdx.x + r * kAnaThreads;
    st1[r] = st2[r] = xs[r] = s0[r] = s1[r] = DF{0.f, 0.f};
    ls[r] = 1 << 30;
    if (jh < nh) {
      const Seed sd = seeds[(size_t)m * nh + jh];
      const float2 xx = xf[jh];
      xs[r] = DF{xx.x, xx.y};
      ls[r] = sd.ls;
      s0[r] = DF{sd.p0h, sd.p0l};
      s1[r] = DF{sd.p1h, sd.p1l};
    }
  }
  const float4* cf = coef + coef_off[m];   // (a_h, a_l, b_h, b_l) for l = m .. lmax at index l - m
  // contraction tile: row tr (32 rows), 6 columns from tc*6 (8 groups over 48)
  const int tr = threadIdx.x >> 3, tc = threadIdx.x & 7;
  int l = m;                                 // next degree to generate
  for (int i0 = 0; i0 < M; i0 += kRB) {
    const int rows = min(kRB, M - i0);
    __syncthreads();   // Ps free (and Xs ready on the first chunk)
    // rows i0 .. i0+rows-1 of parity p are the degrees m + p + 2 i; the recurrence
    // marches every degree (both parities) up to the last of them
    const int lend = m + p + 2 * (i0 + rows - 1);
    for (; l <= lend; ++l) {
      const float4 ab = cf[l - m];
      const bool keep = ((l - m) & 1) == p;
      const int row = ((l - m - p) >> 1) - i0;
#pragma unroll
      for (int r = 0; r < NPT; ++r) {
        DF v;
        if (l < ls[r]) v = DF{0.f, 0.f};
        else if (l == ls[r]) v = s0[r];
        else if (l == ls[r] + 1) v = s1[r];
        else v = rec_step(xs[r], st1[r], st2[r], ab);
        st2[r] = st1[r];
        st1[r] = v;
        const int jh = threadIdx.x + r * kAnaThreads;
        if (keep && jh < nh) Ps[(size_t)jh * kRB + row] = v.h;
      }
    }
    __syncthreads();
    if (tr < rows) {
      float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      for (int k = 0; k < nh; ++k) {
        const float a = Ps[(size_t)k * kRB + tr];
        const float2* xb = reinterpret_cast<const float2*>(Xs + (size_t)k * kRN + tc * 6);
        const float2 b0 = xb[0], b1 = xb[1], b2 = xb[2];
        acc[0] = fmaf(a, b0.x, acc[0]);
        acc[1] = fmaf(a, b0.y, acc[1]);
        acc[2] = fmaf(a, b1.x, acc[2]);
        acc[3] = fmaf(a, b1.y, acc[3]);
        acc[4] = fmaf(a, b2.x, acc[4]);
        acc[5] = fmaf(a, b2.y, acc[5]);
      }
      const int i = i0 + tr;
      const float sc = h ? h[m + p + 2 * i] : 1.f;
      float* o = C + (size_t)(row_off[blk] + i) * ldc;
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const int col = n0 + tc * 6 + c;
        if (col < ncols) o[col] = acc[c] * sc;
      }
    }
  }
}

// Synthesis: Y[jh][c] = sum_i Pbar_lm(x_jh) C[i][c] for block (m, p); a thread owns a node
__global__ void __launch_bounds__(kRecThreads) k_syn_rec(int lmax, int nh, const float2* __restrict__ xf,
                                                         const Seed* __restrict__ seeds,
                                                         const float4* __restrict__ coef,
                                                         const long long* __restrict__ coef_off,
                                                         const int* __restrict__ Mrows,
                                                         const long long* __restrict__ row_off,
                                                         const float* __restrict__ C, int ldc, int ncols,
                                                         float* __restrict__ Y) {
  extern __shared__ float sm[];
  const int blk = blockIdx.x;
  const int m = blk >> 1, p = blk & 1;
  const int M = Mrows[blk];
  if (M == 0) return;
  const int n0 = blockIdx.z * kRN;
  const int jh = blockIdx.y * kRecThreads + threadIdx.x;
  float* Cs = sm;   // [M][kRN]
  const float* Cb = C + (size_t)row_off[blk] * ldc;
  for (int idx = threadIdx.x; idx < M * kRN; idx += blockDim.x) {
    const int i = idx / kRN, c = idx - i * kRN;
    Cs[idx] = (n0 + c < ncols) ? Cb[(size_t)i * ldc + n0 + c] : 0.f;
  }
  __syncthreads();
  if (jh >= nh) return;
  const Seed sd = seeds[(size_t)m * nh + jh];
  const float2 xx = xf[jh];
  const DF x{xx.x, xx.y};
  const float4* cf = coef + coef_off[m];
  float acc[kRN];
#pragma unroll
  for (int c = 0; c < kRN; ++c) acc[c] = 0.f;
  DF st1{0.f, 0.f}, st2{0.f, 0.f};
  const int lend = m + p + 2 * (M - 1);
  for (int l = (sd.ls > m ? sd.ls : m); l <= lend; ++l) {
    DF vv;
    if (l == sd.ls) vv = DF{sd.p0h, sd.p0l};
    else if (l == sd.ls + 1) vv = DF{sd.p1h, sd.p1l};
    else vv = rec_step(x, st1, st2, cf[l - m]);
    st2 = st1;
    st1 = vv;
    const float v = vv.h;
    if (((l - m) & 1) == p) {
      const float4* cr = reinterpret_cast<const float4*>(Cs + (size_t)((l - m - p) >> 1) * kRN);
#pragma unroll
      for (int c4 = 0; c4 < kRN / 4; ++c4) {
        const float4 cc = cr[c4];
        acc[4 * c4] = fmaf(v, cc.x, acc[4 * c4]);
        acc[4 * c4 + 1] = fmaf(v, cc.y, acc[4 * c4 + 1]);
        acc[4 * c4 + 2] = fmaf(v, cc.z, acc[4 * c4 + 2]);
        acc[4 * c4 + 3] = fmaf(v, cc.w, acc[4 * c4 + 3]);
      }
    }
  }
  float* o = Y + ((size_t)blk * nh + jh) * ldc;
#pragma unroll
  for (int c = 0; c < kRN; ++c)
    if (n0 + c < ncols) o[n0 + c] = acc[c];
}

// seeds (FP64 recurrence from l = m until |Pbar| >= 2^-100) and the coefficient table
__device__ __forceinline__ float2 split_df(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

__global__ void k_rec_seeds(int lmax, int nh, const double* __restrict__ x, Seed* __restrict__ seeds,
                            float2* __restrict__ xf) {
  const int jh = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (jh >= nh) return;
  if (m == 0) xf[jh] = split_df(x[jh]);
  const double xj = x[jh];
  const double st = sqrt((1.0 - xj) * (1.0 + xj));
  const double thr = 7.888609052210118e-31;   // 2^-100
  double pmm = 0.28209479177387814;           // 1/sqrt(4 pi)
  for (int k = 1; k <= m; ++k) pmm *= -sqrt((2.0 * k + 1.0) / (2.0 * k)) * st;
  double p2 = pmm, p1 = (m < lmax) ? sqrt(2.0 * m + 3.0) * xj * pmm : 0.0;
  int l = m;
  // advance until |Pbar_l| crosses the threshold (or the degrees run out)
  while (fabs(p2) < thr && l < lmax) {
    const int ln = l + 2;
    double pn = 0.0;
    if (ln <= lmax) {
      const double ll = (double)ln * ln, mm = (double)m * m, l1 = (double)(ln - 1) * (ln - 1);
      pn = sqrt((4.0 * ll - 1.0) / (ll - mm)) * (xj * p1 - sqrt((l1 - mm) / (4.0 * l1 - 1.0)) * p2);
    }
    p2 = p1;
    p1 = pn;
    ++l;
  }
  Seed s;
  s.ls = (fabs(p2) < thr) ? (1 << 30) : l;
  const float2 a0 = split_df(p2), a1 = split_df(p1);
  s.p0h = a0.x;
  s.p0l = a0.y;
  s.p1h = a1.x;
  s.p1l = a1.y;
  seeds[(size_t)m * nh + jh] = s;
}

__global__ void k_rec_coef(int lmax, const long long* __restrict__ coef_off, float4* __restrict__ coef) {
  const int m = blockIdx.x;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    float4 ab = make_float4(0.f, 0.f, 0.f, 0.f);
    if (l >= m + 2) {
      const double ll = (double)l * l, mm = (double)m * m, l1 = (double)(l - 1) * (l - 1);
      const float2 a = split_df(sqrt((4.0 * ll - 1.0) / (ll - mm)));
      const float2 b = split_df(sqrt((l1 - mm) / (4.0 * l1 - 1.0)));
      ab = make_float4(a.x, a.y, b.x, b.y);
    }
    coef[coef_off[m] + (l - m)] = ab;
  }
}

}  // namespace

int build_recurrence(Grid& g, cudaStream_t st) {
  const int L = g.lmax + 1;
  std::vector<long long> off(L + 1, 0);
  for (int m = 0; m < L; ++m) off[m + 1] = off[m] + (L - m);
  SHOT_CUDA(cudaMalloc(&g.rec_coef_off, (L + 1) * sizeof(long long)));
  SHOT_CUDA(cudaMemcpyAsync(g.rec_coef_off, off.data(), (L + 1) * sizeof(long long), cudaMemcpyHostToDevice, st));
  SHOT_CUDA(cudaMalloc(&g.rec_coef, off[L] * sizeof(float4)));
  SHOT_CUDA(cudaMalloc(&g.rec_seeds, (size_t)L * g.nh * sizeof(Seed)));
  SHOT_CUDA(cudaMalloc(&g.rec_x, (size_t)g.nh * sizeof(float2)));
  count_launch(2);
  k_rec_coef<<<L, 256, 0, st>>>(g.lmax, g.rec_coef_off, reinterpret_cast<float4*>(g.rec_coef));
  dim3 gs((g.nh + 127) / 128, L);
  k_rec_seeds<<<gs, 128, 0, st>>>(g.lmax, g.nh, g.x_d, reinterpret_cast<Seed*>(g.rec_seeds),
                                  reinterpret_cast<float2*>(g.rec_x));
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

int launch_legendre_rec(const Grid& g, int nf, const float* X, float* C, float* Y, int ldc, bool ana, bool syn,
                        bool apply_h, cudaStream_t st) {
  const int ncols = 2 * nf;
  const int ncol_tiles = (ncols + kRN - 1) / kRN;
  if (g.nh > 6 * kAnaThreads) {
    set_error("recurrence mode supports nlat <= 3072");
    return SHOT_ERR_UNSUPPORTED;
  }
  if (ana) {
    const size_t smem = ((size_t)g.nh * kRN + (size_t)g.nh * kRB) * sizeof(float);
    if (smem > 227 * 1024) {
      set_error("recurrence analysis: grid too large for one CTA's shared memory");
      return SHOT_ERR_UNSUPPORTED;
    }
    const int npt = (g.nh + kAnaThreads - 1) / kAnaThreads;
    auto kern = npt <= 1 ? k_ana_rec<1> : npt <= 2 ? k_ana_rec<2> : npt <= 3 ? k_ana_rec<3> : k_ana_rec<6>;
    SHOT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope prof(PK_ANALYSIS, st);
    count_launch();
    kern<<<dim3(g.nblk, ncol_tiles), kAnaThreads, smem, st>>>(
        g.lmax, g.nh, reinterpret_cast<const float2*>(g.rec_x), reinterpret_cast<const Seed*>(g.rec_seeds),
        reinterpret_cast<const float4*>(g.rec_coef), g.rec_coef_off, g.M_d, g.row_off_d, X, ldc, ncols,
        apply_h ? g.h_d : nullptr, C);
    SHOT_CUDA(cudaGetLastError());
  }
  if (syn) {
    const size_t smem = (size_t)g.M[0] * kRN * sizeof(float);
    SHOT_CUDA(cudaFuncSetAttribute(k_syn_rec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope prof(PK_SYNTHESIS, st);
    count_launch();
    k_syn_rec<<<dim3(g.nblk, (g.nh + kRecThreads - 1) / kRecThreads, ncol_tiles), kRecThreads, smem, st>>>(
        g.lmax, g.nh, reinterpret_cast<const float2*>(g.rec_x), reinterpret_cast<const Seed*>(g.rec_seeds),
        reinterpret_cast<const float4*>(g.rec_coef), g.rec_coef_off, g.M_d, g.row_off_d, C, ldc, ncols, Y);
    SHOT_CUDA(cudaGetLastError());
  }
  return SHOT_OK;
}

}  // namespace shot
