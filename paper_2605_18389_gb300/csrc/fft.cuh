// Shared-memory mixed-radix Stockham FFT for the longitude rings.
//
// The semi-naive SHT (App. C.1, last paragraph) starts with a DFT along every
// iso-latitude ring.  A ring of nlon = N points is transformed in shared memory by the
// Stockham autosort formulation: at the stage with radix R and span Ns, butterfly j
// (0 <= j < N/R) reads in[j + r N/R] (r < R), multiplies input r by W_N^{(j mod Ns) r N/(Ns R)},
// applies an R-point DFT and writes output r to out[(j div Ns) Ns R + (j mod Ns) + r Ns].
//
// Radices go up to 16 so that the rings of the usual grids take three stages
// (1440 = 9 * 10 * 16); a prime factor above 5 becomes a stage of its own with a generic
// butterfly (O(R) work per output, roots of unity from the plan's table), so any ring
// length has a plan.  The composite radices (6, 9, 10, 12, 15, 16) run as two
// register-resident levels of 2-, 3-, 4- and 5-point DFTs (Cooley-Tukey inside the
// butterfly) whose internal twiddles are compile-time constants.  The stage twiddles come
// from a per-stage table, r-major, so that consecutive lanes read consecutive entries.
// Sequences sit at a stride of N + 1 complex values, which staggers the banks of the
// sequences of one CTA.
#pragma once
#include <utility>

#include "shot_internal.cuh"

namespace shot {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---- compile-time roots of unity ----------------------------------------------------
// cos and sin of 2 pi j / R from their Taylor series; the angle is first reduced to
// [-pi, pi], where 40 terms are far below double rounding.  Only evaluated by the
// compiler (constexpr initialisers of the butterflies' internal twiddles).
__host__ __device__ constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 40; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 40; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double root_angle(int j, int R) {
  // 2 pi j / R with j reduced to (-R/2, R/2]
  int r = ((j % R) + R) % R;
  if (2 * r > R) r -= R;
  return 2.0 * 3.14159265358979323846 * r / R;
}

// a * W_R^J with W_R = exp(-2 pi i / R) (forward) or its conjugate (inverse)
template <int R, int J, bool INV>
__device__ __forceinline__ float2 mul_root(float2 a) {
  constexpr int j = ((J % R) + R) % R;
  if constexpr (j == 0) {
    return a;
  } else if constexpr (2 * j == R) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (4 * j == R) {
    return mul_mi<INV>(a);
  } else if constexpr (4 * j == 3 * R) {
    return mul_mi<!INV>(a);
  } else {
    constexpr float c = (float)taylor_cos(root_angle(j, R));
    constexpr float s = (float)taylor_sin(root_angle(j, R));
    constexpr float sy = INV ? s : -s;   // W^j = (c, -s) forward
    return make_float2(fmaf(a.x, c, -a.y * sy), fmaf(a.x, sy, a.y * c));
  }
}

// ---- prime-size butterflies (in place on v[0..R-1]) ---------------------------------
template <bool INV>
__device__ __forceinline__ void bfly2(float2* v) {
  const float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <bool INV>
__device__ __forceinline__ void bfly4(float2* v) {
  const float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]), c = cadd(v[1], v[3]);
  const float2 d = mul_mi<INV>(csub(v[1], v[3]));
  v[0] = cadd(a, c);
  v[2] = csub(a, c);
  v[1] = cadd(b, d);
  v[3] = csub(b, d);
}

template <bool INV>
__device__ __forceinline__ void bfly8(float2* v) {
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  bfly4<INV>(e);
  bfly4<INV>(o);
  o[1] = mul_root<8, 1, INV>(o[1]);
  o[2] = mul_root<8, 2, INV>(o[2]);
  o[3] = mul_root<8, 3, INV>(o[3]);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[i] = cadd(e[i], o[i]);
    v[i + 4] = csub(e[i], o[i]);
  }
}

template <bool INV>
__device__ __forceinline__ void bfly3(float2* v) {
  const float s = 0.86602540378443865f;   // sin(2 pi / 3)
  const float2 t = cadd(v[1], v[2]);
  const float2 d = csub(v[1], v[2]);
  const float2 a = make_float2(fmaf(-0.5f, t.x, v[0].x), fmaf(-0.5f, t.y, v[0].y));
  const float2 b = mul_mi<INV>(make_float2(s * d.x, s * d.y));
  v[0] = cadd(v[0], t);
  v[1] = cadd(a, b);
  v[2] = csub(a, b);
}

template <bool INV>
__device__ __forceinline__ void bfly5(float2* v) {
  const float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;   // cos(2pi/5), cos(4pi/5)
  const float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;    // sin(2pi/5), sin(4pi/5)
  const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  const float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
  const float2 x0 = v[0];
  const float2 a1 = make_float2(fmaf(c2, t2.x, fmaf(c1, t1.x, x0.x)), fmaf(c2, t2.y, fmaf(c1, t1.y, x0.y)));
  const float2 a2 = make_float2(fmaf(c1, t2.x, fmaf(c2, t1.x, x0.x)), fmaf(c1, t2.y, fmaf(c2, t1.y, x0.y)));
  const float2 b1 = mul_mi<INV>(make_float2(fmaf(s1, d1.x, s2 * d2.x), fmaf(s1, d1.y, s2 * d2.y)));
  const float2 b2 = mul_mi<INV>(make_float2(fmaf(s2, d1.x, -s1 * d2.x), fmaf(s2, d1.y, -s1 * d2.y)));
  v[0] = cadd(x0, cadd(t1, t2));
  v[1] = cadd(a1, b1);
  v[4] = csub(a1, b1);
  v[2] = cadd(a2, b2);
  v[3] = csub(a2, b2);
}

template <int R, bool INV>
__device__ __forceinline__ void bfly_prime(float2* v) {
  if constexpr (R == 2) bfly2<INV>(v);
  else if constexpr (R == 3) bfly3<INV>(v);
  else if constexpr (R == 4) bfly4<INV>(v);
  else if constexpr (R == 5) bfly5<INV>(v);
  else bfly8<INV>(v);
}

// R-point DFT of the registers v[O + S i], i < R
template <int R, int O, int S, bool INV>
__device__ __forceinline__ void dft_at(float2* v) {
  float2 t[R];
#pragma unroll
  for (int i = 0; i < R; ++i) t[i] = v[O + S * i];
  bfly_prime<R, INV>(t);
#pragma unroll
  for (int i = 0; i < R; ++i) v[O + S * i] = t[i];
}

// Composite R = R1 R2 with n = R2 n1 + n2, k = k1 + R1 k2:
//   X[k] = sum_{n2} W_R2^{n2 k2} W_R^{n2 k1} sum_{n1} W_R1^{n1 k1} x[R2 n1 + n2].
// After the call X[k1 + R1 k2] is in v[R2 k1 + k2].
template <int R1, int R2, bool INV, int... I>
__device__ __forceinline__ void composite_level1(float2* v, std::integer_sequence<int, I...>) {
  (dft_at<R1, I, R2, INV>(v), ...);
}
template <int R1, int R2, bool INV, int... I>
__device__ __forceinline__ void composite_twiddle(float2* v, std::integer_sequence<int, I...>) {
  // element I = R2 k1 + n2 takes W_R^{n2 k1}
  ((v[I] = mul_root<R1 * R2, (I % R2) * (I / R2), INV>(v[I])), ...);
}
template <int R1, int R2, bool INV, int... I>
__device__ __forceinline__ void composite_level2(float2* v, std::integer_sequence<int, I...>) {
  (dft_at<R2, R2 * I, 1, INV>(v), ...);
}

template <int R1, int R2, bool INV>
__device__ __forceinline__ void bfly_composite(float2* v) {
  composite_level1<R1, R2, INV>(v, std::make_integer_sequence<int, R2>{});
  composite_twiddle<R1, R2, INV>(v, std::make_integer_sequence<int, R1 * R2>{});
  composite_level2<R1, R2, INV>(v, std::make_integer_sequence<int, R1>{});
}

// Radix R butterfly and the register holding its output k.
template <int R>
struct Radix {
  static constexpr int R1 = 1, R2 = R;   // prime-size: output k in v[k]
};
template <> struct Radix<6> { static constexpr int R1 = 2, R2 = 3; };
template <> struct Radix<9> { static constexpr int R1 = 3, R2 = 3; };
template <> struct Radix<10> { static constexpr int R1 = 2, R2 = 5; };
template <> struct Radix<12> { static constexpr int R1 = 4, R2 = 3; };
template <> struct Radix<15> { static constexpr int R1 = 3, R2 = 5; };
template <> struct Radix<16> { static constexpr int R1 = 4, R2 = 4; };

template <int R, bool INV>
__device__ __forceinline__ void butterfly(float2* v) {
  if constexpr (Radix<R>::R1 == 1) bfly_prime<R, INV>(v);
  else bfly_composite<Radix<R>::R1, Radix<R>::R2, INV>(v);
}
template <int R>
__host__ __device__ constexpr int out_reg(int k) {
  return Radix<R>::R1 == 1 ? k : Radix<R>::R2 * (k % Radix<R>::R1) + k / Radix<R>::R1;
}

// Threads of an FFT CTA (launched with at least three CTAs per SM in mind: <= 80
// registers, enough for the radix-16 butterfly without spills); kFftCap (the most elements,
// sequences x length, one CTA transforms) is declared with the grid types.
constexpr int kFftThreads = 256;

// stride of consecutive sequences in the CTA's buffers
__host__ __device__ constexpr int seq_ld(int N) { return N + 1; }

// a / d for 0 <= a < 2^16 and 2 <= d < 2^16 with mul = ceil(2^32 / d) (exact: the
// error a (mul - 2^32/d) / 2^32 < 2^-16 never crosses an integer); mul == 0 means d == 1.
__device__ __forceinline__ int fast_div(int a, uint32_t mul) {
  return mul ? (int)__umulhi((uint32_t)a, mul) : a;
}

template <int R, bool INV>
__device__ __forceinline__ void stockham_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                               const float2* __restrict__ tws, int N, int Ns, int nseq,
                                               uint32_t ns_mul, uint32_t nr_mul) {
  const int NR = N / R;
  const int ld = seq_ld(N);
  const int total = nseq * NR;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int q = fast_div(idx, nr_mul);
    const int j = idx - q * NR;
    const int jd = fast_div(j, ns_mul);
    const int k = j - jd * Ns;
    const float2* s = src + q * ld + j;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[r * NR];
    if (Ns > 1) {   // the first stage's twiddles are all 1
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = tws[(r - 1) * Ns + k];
        v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
      }
    }
    butterfly<R, INV>(v);
    float2* d = dst + q * ld + jd * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) d[r * Ns] = v[out_reg<R>(r)];
  }
}

// Stage with a radix that has no compiled butterfly (a prime above 5): each task computes one
// output r of butterfly j, sum_t v_t W_R^{r t}, with v_t the stage-twiddled input t and the
// roots W_R^e from the plan's table; O(R) work per output.  Tasks run r-major over the
// butterflies, so consecutive threads read consecutive inputs.
template <bool INV>
__device__ __noinline__ void stockham_stage_generic(const float2* __restrict__ src, float2* __restrict__ dst,
                                                    const float2* __restrict__ tws, const float2* __restrict__ roots,
                                                    int N, int R, int Ns, int nseq, uint32_t ns_mul,
                                                    uint32_t nr_mul) {
  const int NR = N / R;
  const int ld = seq_ld(N);
  const int total = nseq * N;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int qr = fast_div(idx, nr_mul);   // q R + r
    const int j = idx - qr * NR;
    const int q = qr / R, r = qr - q * R;
    const int jd = fast_div(j, ns_mul);
    const int k = j - jd * Ns;
    const float2* s = src + q * ld + j;
    float re = 0.f, im = 0.f;
    int e = 0;   // r t mod R
    for (int t = 0; t < R; ++t) {
      float2 v = s[t * NR];
      if (Ns > 1 && t > 0) {
        const float2 w = tws[(t - 1) * Ns + k];
        v = INV ? cmulc(v, w) : cmul(v, w);
      }
      const float2 w = roots[e];
      v = INV ? cmulc(v, w) : cmul(v, w);
      re += v.x;
      im += v.y;
      e += r;
      if (e >= R) e -= R;
    }
    dst[q * ld + jd * Ns * R + k + r * Ns] = make_float2(re, im);
  }
}

// Transforms nseq sequences of length plan.N stored at a[q * seq_ld(N) + k]; b is
// scratch of the same shape; tw holds the plan's stage twiddles (forward sign).  Returns
// the buffer holding the result.  All threads of the block must call it; it
// synchronises after every stage.
template <bool INV>
__device__ float2* fft_smem(float2* a, float2* b, const float2* tw, const FftPlan& pl, int nseq) {
  int Ns = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.R[s];
    const float2* tws = tw + pl.tw_off[s];
    const uint32_t nsm = pl.ns_mul[s], nrm = pl.nr_mul[s];
    switch (R) {
      case 2: stockham_stage<2, INV>(a, b, tws, pl.N, Ns, nseq, nsm, nrm); break;
      case 3: stockham_stage<3, INV>(a, b, tws, pl.N, Ns, nseq, nsm, nrm); break;
      case 4: stockham_stage<4, INV>(a, b, tws, pl.N, Ns, nseq, nsm, nrm); break;
      case 5: stockham_stage<5, INV>(a, b, tws, pl.N, Ns, nseq, nsm, nrm); break;
      case 6: stockham_stage<6, INV>(a, b, tws, pl.N, Ns, nseq, nsm, nrm); break;
      case 8: stockham_stage<8, INV>(a, b, tws, pl.N, Ns, nseq, nsm, nrm); break;
      case 9: stockham_stage<9, INV>(a, b, tws, pl.N, Ns, nseq, nsm, nrm); break;
      case 10: stockham_stage<10, INV>(a, b, tws, pl.N, Ns, nseq, nsm, nrm); break;
      case 12: stockham_stage<12, INV>(a, b, tws, pl.N, Ns, nseq, nsm, nrm); break;
      case 15: stockham_stage<15, INV>(a, b, tws, pl.N, Ns, nseq, nsm, nrm); break;
      case 16: stockham_stage<16, INV>(a, b, tws, pl.N, Ns, nseq, nsm, nrm); break;
      default:
        stockham_stage_generic<INV>(a, b, tws, tw + pl.root_off[s], pl.N, R, Ns, nseq, nsm, nrm);
        break;
    }
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// ---- plans fixed at compile time ---------------------------------------------------
// The same Stockham stages with N, the radices and the spans as template constants: the
// divisions by N/R and Ns become multiply-shifts and every load, twiddle and store offset an
// immediate.  CtPlan<0> is the runtime plan.
template <int N_, int R0_ = 1, int R1_ = 1, int R2_ = 1>
struct CtPlan {
  static constexpr int N = N_, R0 = R0_, R1 = R1_, R2 = R2_;
};
using RuntimePlan = CtPlan<0>;

template <int R, bool INV, int N, int NS, int TWOFF>
__device__ __forceinline__ void stockham_stage_ct(const float2* __restrict__ src, float2* __restrict__ dst,
                                                  const float2* __restrict__ tw, int nseq) {
  constexpr int NR = N / R, LD = N + 1;
  const int total = nseq * NR;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int q = idx / NR;
    const int j = idx - q * NR;
    const int jd = j / NS;
    const int k = j - jd * NS;
    const float2* s = src + q * LD + j;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[r * NR];
    if constexpr (NS > 1) {
      const float2* tws = tw + TWOFF + k;
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = INV ? cmulc(v[r], tws[(r - 1) * NS]) : cmul(v[r], tws[(r - 1) * NS]);
    }
    butterfly<R, INV>(v);
    float2* d = dst + q * LD + jd * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) d[r * NS] = v[out_reg<R>(r)];
  }
}

// three-stage compile-time plan; the twiddle table layout is the runtime plan's (stage s at
// sum over earlier stages s' >= 1 of (R_s' - 1) Ns_s')
template <bool INV, class PL>
__device__ float2* fft_smem_ct(float2* a, float2* b, const float2* tw, int nseq) {
  constexpr int N = PL::N, R0 = PL::R0, R1 = PL::R1, R2 = PL::R2;
  static_assert(R0 * R1 * R2 == N, "plan radices must multiply to N");
  stockham_stage_ct<R0, INV, N, 1, 0>(a, b, tw, nseq);
  __syncthreads();
  stockham_stage_ct<R1, INV, N, R0, 0>(b, a, tw, nseq);
  __syncthreads();
  stockham_stage_ct<R2, INV, N, R0 * R1, (R1 - 1) * R0>(a, b, tw, nseq);
  __syncthreads();
  return b;
}

template <bool INV, class PL>
__device__ __forceinline__ float2* fft_smem_plan(float2* a, float2* b, const float2* tw, const FftPlan& pl,
                                                 int nseq) {
  if constexpr (PL::N == 0) return fft_smem<INV>(a, b, tw, pl, nseq);
  else return fft_smem_ct<INV, PL>(a, b, tw, nseq);
}

}  // namespace shot
