// Gradient-based regional attribution (Sec. 4.2 and App. E, "Gradient-based regional
// attribution"): the gradient of S is turned into a field (dS/dp_i / a_i), centred by its
// area-weighted mean, and its area-weighted RMS is taken over five latitude bands:
// Tropics |lat| < 23.5, ITCZ |lat| < 10, NH mid-latitudes 30..60 N, SH mid-latitudes
// 30..60 S, Arctic lat > 66.5 (degrees).
#include <math.h>

#include <vector>

#include "shot_internal.cuh"

namespace shot {
namespace {


// per (ring, field): sum_k g and sum_k g^2 of the field form g = grad / a_j; ring j holds
// rlen[j] nodes from roff[j] of a field of npix nodes
__global__ void k_ring_moments(int nring, const int* __restrict__ rlen, const long long* __restrict__ roff,
                               long long npix, const float* __restrict__ grad, const float* __restrict__ a_ring,
                               double* __restrict__ mom) {
  __shared__ float r1[32], r2[32];
  const int j = blockIdx.x, b = blockIdx.y;
  const int nlat = nring;
  const float inv_a = 1.f / a_ring[j];
  const float* row = grad + (size_t)b * npix + roff[j];
  const int nk = rlen[j];
  float s1 = 0.f, s2 = 0.f;
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    const float g = row[k] * inv_a;
    s1 += g;
    s2 += g * g;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = s1;
    r2[threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t1 += r1[w];
      t2 += r2[w];
    }
    mom[((size_t)b * nlat + j) * 2] = t1;
    mom[((size_t)b * nlat + j) * 2 + 1] = t2;
  }
}

}  // namespace
}  // namespace shot

extern "C" int shot_regional_rms(shot_grid gh, const float* grad_p, int batch, double* rms, void* stream) {
  using namespace shot;
  Grid* g = reinterpret_cast<Grid*>(gh);
  if (!g || !grad_p || batch < 1 || !rms) {
    set_error("shot_regional_rms: bad argument");
    return SHOT_ERR_INVALID_ARG;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* mom = nullptr;
  SHOT_CUDA(cudaMalloc(&mom, (size_t)batch * g->nlat * 2 * sizeof(double)));
  count_launch();
  k_ring_moments<<<dim3(g->nlat, batch), 256, 0, st>>>(g->nlat, g->ring_len_d, g->ring_off_d, (long long)g->npix,
                                                        grad_p, g->a_d, mom);
  cudaError_t e = cudaGetLastError();
  std::vector<double> h((size_t)batch * g->nlat * 2);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), mom, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(mom);
  if (e != cudaSuccess) return cuda_status(e, "shot_regional_rms");
  // band membership from the ring latitudes (FP64 nodes)
  const double deg = 180.0 / M_PI;
  for (int b = 0; b < batch; ++b) {
    double s1 = 0.0, area = 0.0;
    for (int j = 0; j < g->nlat; ++j) {
      s1 += g->a_ring[j] * h[((size_t)b * g->nlat + j) * 2];
      area += g->a_ring[j] * g->ring_len[j];
    }
    const double mean = s1 / area;   // area-weighted mean of the field form
    double S0[5] = {0}, S1[5] = {0}, S2[5] = {0};
    for (int j = 0; j < g->nlat; ++j) {
      const double lat = 90.0 - acos(g->x[j]) * deg;
      const bool in[5] = {fabs(lat) < 23.5, fabs(lat) < 10.0, lat >= 30.0 && lat <= 60.0, lat <= -30.0 && lat >= -60.0,
                          lat > 66.5};
      const double a = g->a_ring[j];
      const double m1 = h[((size_t)b * g->nlat + j) * 2], m2 = h[((size_t)b * g->nlat + j) * 2 + 1];
      for (int r = 0; r < 5; ++r)
        if (in[r]) {
          S0[r] += a * g->ring_len[j];
          S1[r] += a * m1;
          S2[r] += a * m2;
        }
    }
    for (int r = 0; r < 5; ++r) {
      // sum a (g - mean)^2 = S2 - 2 mean S1 + mean^2 S0
      const double v = S0[r] > 0 ? (S2[r] - 2.0 * mean * S1[r] + mean * mean * S0[r]) / S0[r] : NAN;
      rms[(size_t)b * 5 + r] = v > 0 ? sqrt(v) : 0.0;
    }
  }
  return SHOT_OK;
}
