// Shared-memory mixed-radix (2,3,4,5,8) Stockham FFT for the longitude rings.
//
// The semi-naive SHT (App. C.1, last paragraph) starts with a DFT along every
// iso-latitude ring.  A ring of nlon points is transformed in shared memory by the
// Stockham autosort formulation: at the stage with radix R and span Ns, butterfly j
// (0 <= j < N/R) reads in[j + r N/R] (r < R), multiplies by W_N^{(j mod Ns) r N/(Ns R)},
// applies an R-point DFT and writes out[(j div Ns) Ns R + (j mod Ns) + q Ns].
#pragma once
#include "shot_internal.cuh"

namespace shot {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void bfly2(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <bool INV>
__device__ __forceinline__ void bfly4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = mul_mi<INV>(csub(x1, x3));
  x0 = cadd(a, c);
  x2 = csub(a, c);
  x1 = cadd(b, d);
  x3 = csub(b, d);
}

template <bool INV>
__device__ __forceinline__ void bfly8(float2* v) {
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  bfly4<INV>(e0, e1, e2, e3);
  bfly4<INV>(o0, o1, o2, o3);
  const float h = 0.70710678118654752f;
  // w^1 = (1 -+ i)/sqrt2, w^2 = -+i, w^3 = (-1 -+ i)/sqrt2
  float2 w1o1 = INV ? make_float2(h * (o1.x - o1.y), h * (o1.x + o1.y))
                    : make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x));
  float2 w2o2 = mul_mi<INV>(o2);
  float2 w3o3 = INV ? make_float2(h * (-o3.x - o3.y), h * (o3.x - o3.y))
                    : make_float2(h * (o3.y - o3.x), h * (-o3.x - o3.y));
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, w1o1);
  v[5] = csub(e1, w1o1);
  v[2] = cadd(e2, w2o2);
  v[6] = csub(e2, w2o2);
  v[3] = cadd(e3, w3o3);
  v[7] = csub(e3, w3o3);
}

template <bool INV>
__device__ __forceinline__ void bfly3(float2* v) {
  const float s = 0.86602540378443865f;   // sin(2 pi / 3)
  float2 t = cadd(v[1], v[2]);
  float2 d = csub(v[1], v[2]);
  float2 a = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
  float2 b = mul_mi<INV>(make_float2(s * d.x, s * d.y));
  v[0] = cadd(v[0], t);
  v[1] = cadd(a, b);
  v[2] = csub(a, b);
}

template <bool INV>
__device__ __forceinline__ void bfly5(float2* v) {
  const float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;   // cos(2pi/5), cos(4pi/5)
  const float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;    // sin(2pi/5), sin(4pi/5)
  float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
  float2 x0 = v[0];
  float2 a1 = make_float2(x0.x + c1 * t1.x + c2 * t2.x, x0.y + c1 * t1.y + c2 * t2.y);
  float2 a2 = make_float2(x0.x + c2 * t1.x + c1 * t2.x, x0.y + c2 * t1.y + c1 * t2.y);
  float2 b1 = mul_mi<INV>(make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
  float2 b2 = mul_mi<INV>(make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
  v[0] = cadd(x0, cadd(t1, t2));
  v[1] = cadd(a1, b1);
  v[4] = csub(a1, b1);
  v[2] = cadd(a2, b2);
  v[3] = csub(a2, b2);
}

// Threads of an FFT CTA and the most elements (sequences x length) one CTA transforms:
// two ping-pong buffers of kFftCap complex values plus the twiddles stay under ~110 KB, so
// two CTAs fit on one SM.
constexpr int kFftThreads = 512;
constexpr int kFftCap = 6400;

template <int R, bool INV>
__device__ __forceinline__ void butterfly(float2* v) {
  if (R == 2) bfly2<INV>(v);
  if (R == 3) bfly3<INV>(v);
  if (R == 4) bfly4<INV>(v[0], v[1], v[2], v[3]);
  if (R == 5) bfly5<INV>(v);
  if (R == 8) bfly8<INV>(v);
}

// Shared-memory index of complex element i of the sequence buffers: one float2 of padding
// after every 16, which turns the stride-R stores of the early Stockham stages into
// conflict-free 8-byte accesses.
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 4) + 1; }

// a / d for 0 <= a < 2^16 and 2 <= d < 2^16 with mul = ceil(2^32 / d) (exact: the
// error a (mul - 2^32/d) / 2^32 < 2^-16 never crosses an integer); mul == 0 means d == 1.
__device__ __forceinline__ int fast_div(int a, uint32_t mul) {
  return mul ? (int)__umulhi((uint32_t)a, mul) : a;
}

template <int R, bool INV>
__device__ __forceinline__ void stockham_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                               const float2* __restrict__ tw, int N, int Ns, int nseq,
                                               int ld, uint32_t ns_mul, uint32_t nr_mul) {
  const int NR = N / R;
  const int tstep = N / (Ns * R);
  const int total = nseq * NR;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int q = fast_div(idx, nr_mul);
    const int j = idx - q * NR;
    const int jd = fast_div(j, ns_mul);
    const int k = j - jd * Ns;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float2 x = src[pidx(q * ld + j + r * NR)];
      if (r > 0) {
        float2 w = tw[k * r * tstep];
        if (INV) w.y = -w.y;
        x = cmul(x, w);
      }
      v[r] = x;
    }
    butterfly<R, INV>(v);
    const int o = jd * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[pidx(q * ld + o + r * Ns)] = v[r];
  }
}

// Transforms nseq sequences of length plan.N stored at a[q*ld + k]; b is scratch of the
// same shape.  Returns the buffer holding the result.  All threads of the block must
// call it; it synchronises after every stage.
template <bool INV>
__device__ float2* fft_smem(float2* a, float2* b, const float2* tw, const FftPlan& pl, int nseq, int ld) {
  int Ns = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.R[s];
    switch (R) {
      case 2: stockham_stage<2, INV>(a, b, tw, pl.N, Ns, nseq, ld, pl.ns_mul[s], pl.nr_mul[s]); break;
      case 3: stockham_stage<3, INV>(a, b, tw, pl.N, Ns, nseq, ld, pl.ns_mul[s], pl.nr_mul[s]); break;
      case 4: stockham_stage<4, INV>(a, b, tw, pl.N, Ns, nseq, ld, pl.ns_mul[s], pl.nr_mul[s]); break;
      case 5: stockham_stage<5, INV>(a, b, tw, pl.N, Ns, nseq, ld, pl.ns_mul[s], pl.nr_mul[s]); break;
      default: stockham_stage<8, INV>(a, b, tw, pl.N, Ns, nseq, ld, pl.ns_mul[s], pl.nr_mul[s]); break;
    }
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

}  // namespace shot
