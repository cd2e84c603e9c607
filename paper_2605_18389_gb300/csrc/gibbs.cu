// Explicit matrix convolution with the geodesic Gibbs kernel and its comparison with the
// heat convolution (App. "Convolution on S^2").
//
// The matrix convolution applies K_eps(x, y) = exp(-d(x, y)^2 / eps) with the area weights
// of App. C.2:   (K f)_i = sum_j a_j exp(-d_ij^2 / eps) f_j,
// an O(n^2) product computed on the fly (nothing of size n^2 is stored).  d is taken as
// atan2(|x_i x x_j|, x_i . x_j), accurate near 0 and pi where arccos of the dot product
// loses half its digits.  The kernel integrates to C(eps) = 2 pi int_0^pi exp(-th^2/eps)
// sin(th) dth, and by Varadhan's formula the heat kernel at t = eps/4 is close to
// K_eps / C(eps); the comparison rescales the heat output by C(eps) and takes the mean
// absolute difference over the grid nodes.
#include <cmath>
#include <vector>

#include "shot_internal.cuh"

namespace shot {
namespace {

constexpr int kGT = 256;   // threads per CTA, one output node each
constexpr int kGF = 4;     // fields per pass

// node unit vectors (FP64 trig, rounded to FP32), [ring][lon]
__global__ void k_node_xyz(int nlat, int nlon, const double* __restrict__ x, float4* __restrict__ xyz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nlat * nlon) return;
  const int j = i / nlon, k = i - j * nlon;
  const double z = x[j];
  const double st = sqrt((1.0 - z) * (1.0 + z));
  double s, c;
  sincospi(2.0 * k / nlon, &s, &c);
  xyz[i] = make_float4((float)(st * c), (float)(st * s), (float)z, 0.f);
}

__global__ void __launch_bounds__(kGT) k_gibbs(int n, int nlon, const float4* __restrict__ xyz,
                                               const float* __restrict__ a_ring, float inv_eps,
                                               const float* __restrict__ in, float* __restrict__ out, int nf,
                                               int f0) {
  __shared__ float4 sx[kGT];
  __shared__ float sv[kGF][kGT];
  const int i = blockIdx.x * kGT + threadIdx.x;
  const float4 xi = (i < n) ? xyz[i] : make_float4(0.f, 0.f, 1.f, 0.f);
  const int nfp = min(kGF, nf - f0);
  float acc[kGF] = {0.f, 0.f, 0.f, 0.f};
  for (int j0 = 0; j0 < n; j0 += kGT) {
    const int j = j0 + threadIdx.x;
    if (j < n) {
      sx[threadIdx.x] = xyz[j];
      const float aj = a_ring[j / nlon];
#pragma unroll
      for (int q = 0; q < kGF; ++q) sv[q][threadIdx.x] = (q < nfp) ? aj * in[(size_t)(f0 + q) * n + j] : 0.f;
    }
    __syncthreads();
    const int nj = min(kGT, n - j0);
    for (int jj = 0; jj < nj; ++jj) {
      const float4 xj = sx[jj];
      const float dot = fmaf(xi.x, xj.x, fmaf(xi.y, xj.y, xi.z * xj.z));
      const float cx = fmaf(xi.y, xj.z, -xi.z * xj.y);
      const float cy = fmaf(xi.z, xj.x, -xi.x * xj.z);
      const float cz = fmaf(xi.x, xj.y, -xi.y * xj.x);
      const float d = atan2f(sqrtf(fmaf(cx, cx, fmaf(cy, cy, cz * cz))), dot);
      const float w = expf(-d * d * inv_eps);
#pragma unroll
      for (int q = 0; q < kGF; ++q) acc[q] = fmaf(w, sv[q][jj], acc[q]);
    }
    __syncthreads();
  }
  if (i < n)
    for (int q = 0; q < nfp; ++q) out[(size_t)(f0 + q) * n + i] = acc[q];
}

// per field: sum_i |C h_i - k_i| (FP64 partial sums per CTA, fixed order)
__global__ void k_conv_absdiff(int n, double C, const float* __restrict__ h, const float* __restrict__ k,
                               double* __restrict__ part) {
  __shared__ double red[32];
  const int f = blockIdx.y;
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    s += fabs(C * (double)h[(size_t)f * n + i] - (double)k[(size_t)f * n + i]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[(size_t)f * gridDim.x + blockIdx.x] = t;
  }
}

// C(eps) by composite Simpson's rule on [0, c] and [c, pi], c = min(pi, 12 sqrt(eps)), where
// the integrand's mass sits (2^14 panels each; the fourth derivative scales as eps^-2, so
// the rule's error stays near double rounding for eps >= 1e-6)
double gibbs_normaliser_host(double eps) {
  auto f = [&](double th) { return std::exp(-th * th / eps) * std::sin(th); };
  auto simpson = [&](double a, double b) {
    const int n = 1 << 14;
    const double h = (b - a) / n;
    double s = f(a) + f(b);
    for (int i = 1; i < n; ++i) s += (i & 1 ? 4.0 : 2.0) * f(a + i * h);
    return s * h / 3.0;
  };
  const double cut = std::fmin(M_PI, 12.0 * std::sqrt(eps));
  double v = simpson(0.0, cut);
  if (cut < M_PI) v += simpson(cut, M_PI);
  return 2.0 * M_PI * v;
}

int ensure_xyz(Grid& g, cudaStream_t st) {
  if (g.xyz_d) return SHOT_OK;
  const int n = (int)g.npix;
  SHOT_CUDA(cudaMalloc(&g.xyz_d, (size_t)n * sizeof(float4)));
  if (g.quad == SHOT_QUAD_HEALPIX) {   // ring lengths and longitude offsets vary: host, FP64
    std::vector<float4> v((size_t)n);
    for (int i = 0; i < g.nlat; ++i) {
      const double z = g.x[i], st_ = std::sqrt((1.0 - z) * (1.0 + z));
      const double phi0 = M_PI * g.ring_phase[i].first / g.ring_phase[i].second;
      for (int k = 0; k < g.ring_len[i]; ++k) {
        const double ph = phi0 + 2.0 * M_PI * k / g.ring_len[i];
        v[(size_t)g.ring_off[i] + k] = make_float4((float)(st_ * std::cos(ph)), (float)(st_ * std::sin(ph)), (float)z, 0.f);
      }
    }
    SHOT_CUDA(cudaMemcpyAsync(g.xyz_d, v.data(), v.size() * sizeof(float4), cudaMemcpyHostToDevice, st));
    SHOT_CUDA(cudaStreamSynchronize(st));   // v is a local
    return SHOT_OK;
  }
  count_launch();
  k_node_xyz<<<(n + 255) / 256, 256, 0, st>>>(g.nlat, g.nlon, g.x_d, reinterpret_cast<float4*>(g.xyz_d));
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

int launch_gibbs(Grid& g, double eps, const float* in, float* out, int nf, cudaStream_t st) {
  int rc = ensure_xyz(g, st);
  if (rc) return rc;
  const int n = (int)g.npix;
  // node j's area weight is a_ring[j / ring width]: HEALPix pixels all have the same area
  const int width = g.quad == SHOT_QUAD_HEALPIX ? n : g.nlon;
  for (int f0 = 0; f0 < nf; f0 += kGF) {
    count_launch();
    k_gibbs<<<(n + kGT - 1) / kGT, kGT, 0, st>>>(n, width, reinterpret_cast<const float4*>(g.xyz_d), g.a_d,
                                                 (float)(1.0 / eps), in, out, nf, f0);
    SHOT_CUDA(cudaGetLastError());
  }
  return SHOT_OK;
}

}  // namespace
}  // namespace shot

using namespace shot;

extern "C" int shot_gibbs_normaliser(double eps, double* C) {
  if (!C || !(eps > 0.0) || !std::isfinite(eps)) {
    set_error("shot_gibbs_normaliser: need eps > 0 and a result pointer");
    return SHOT_ERR_INVALID_ARG;
  }
  *C = gibbs_normaliser_host(eps);
  return SHOT_OK;
}

extern "C" int shot_gibbs_apply(shot_grid gh, double eps, const float* in, float* out, int nfields, void* stream) {
  Grid* g = reinterpret_cast<Grid*>(gh);
  if (!g || !in || !out || in == out || nfields < 1 || !(eps > 0.0) || !std::isfinite(eps)) {
    set_error("shot_gibbs_apply: bad argument");
    return SHOT_ERR_INVALID_ARG;
  }
  return launch_gibbs(*g, eps, in, out, nfields, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int shot_conv_compare(shot_grid gh, double eps, const float* in, int nfields, double* mae,
                                 void* stream) {
  Grid* g = reinterpret_cast<Grid*>(gh);
  if (!g || !in || !mae || nfields < 1 || !(eps > 0.0) || !std::isfinite(eps)) {
    set_error("shot_conv_compare: bad argument");
    return SHOT_ERR_INVALID_ARG;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int n = (int)g->npix;
  const int nblk = 64;
  float *h = nullptr, *k = nullptr;
  double* part = nullptr;
  int rc = SHOT_OK;
  if (cudaMalloc(&h, (size_t)nfields * n * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&k, (size_t)nfields * n * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&part, (size_t)nfields * nblk * sizeof(double)) != cudaSuccess) {
    cudaFree(h);
    cudaFree(k);
    cudaFree(part);
    set_error("shot_conv_compare: out of device memory");
    return SHOT_ERR_OOM;
  }
  std::vector<double> hp((size_t)nfields * nblk);
  const double C = gibbs_normaliser_host(eps);
  if (!rc) rc = shot_heat_apply(gh, eps / 4.0, in, h, nfields, stream);
  if (!rc) rc = launch_gibbs(*g, eps, in, k, nfields, st);
  if (!rc) {
    count_launch();
    k_conv_absdiff<<<dim3(nblk, nfields), 256, 0, st>>>(n, C, h, k, part);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_status(e, "shot_conv_compare");
  }
  if (!rc)
    for (int f = 0; f < nfields; ++f) {
      double s = 0.0;
      for (int b = 0; b < nblk; ++b) s += hp[(size_t)f * nblk + b];
      mae[f] = s / n;
    }
  cudaFree(h);
  cudaFree(k);
  cudaFree(part);
  return rc;
}
