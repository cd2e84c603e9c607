// HEALPix grids (App. C.1 "HEALPix"): ring geometry and the ring transforms.
//
// Rings i = 0 .. 4 nside - 2 run north to south; ring i has n_i pixels at longitudes
// phi0_i + 2 pi j / n_i (j = 0 .. n_i - 1) and every pixel the area 4 pi / N, N = 12 nside^2.
// Polar cap (k = i + 1 < nside): z = 1 - k^2/(3 nside^2), n = 4k, phi0 = pi/(4k);
// equatorial belt (nside <= k <= 2 nside): z = 4/3 - 2k/(3 nside), n = 4 nside,
// phi0 = pi (2 - s)/(4 nside), s = (k - nside + 1) mod 2; the south half mirrors the north
// (z -> -z, same n and phi0), so rings i and 4 nside - 2 - i form the same parity pairs as on
// the other grids and the Legendre stage is shared with them unchanged.
//
// A ring's length n_i is 4k, not always a product of 2, 3 and 5, and the band limit
// (3 nside - 1 by default) exceeds n_i / 2 on the polar rings.  The ring transforms run the
// shared-memory Stockham FFT of the rectangular grids on the rings whose length factors into
// 2, 3 and 5 (all equatorial-belt rings at the usual nside = 2^k, and many polar rings) and a
// direct DFT in shared memory on the others, with the aliasing made explicit:
//   forward  F_m = e^{-i m phi0} D_{m mod n},   D_k = sum_j f_j e^{-2 pi i k j / n}
//   inverse  f_j = sum_k Z_k e^{2 pi i k j / n},
//            Z_k = sum_{m = -lmax..lmax, m = k mod n} e^{i m phi0} G_m,   G_{-m} = conj G_m.
// Two rings (j north, J south) travel as one complex sequence, as on the other grids.
#include <cmath>
#include <vector>

#include "epilogue.cuh"
#include "fft.cuh"

namespace shot {
namespace {

constexpr int kHpThreads = 256;

__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// e^{i pi r / d} for an integer r reduced modulo 2d (exact argument reduction)
__device__ __forceinline__ float2 half_turns(long long r, int d) {
  long long rr = r % (2LL * d);
  if (rr < 0) rr += 2LL * d;
  float s, c;
  sincospif((float)rr / (float)d, &s, &c);
  return make_float2(c, s);
}

// ring constants: twiddles tw[t] = e^{-2 pi i t / n} (direct DFT rings; tw may be null);
// phases ph[m] = e^{i m phi0}
__device__ __forceinline__ void ring_tables(float2* tw, float2* ph, int n, int2 phase, int lmax) {
  if (tw)
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const float2 e = half_turns(2LL * t, n);
    tw[t] = make_float2(e.x, -e.y);
  }
  if (ph)
    for (int m = threadIdx.x; m <= lmax; m += blockDim.x) ph[m] = half_turns((long long)m * phase.x, phase.y);
}

// D[q][k] = sum_t zin[q][t] tw[k t mod n] (forward, conj = false) or with conj(tw) (inverse);
// sequences at a stride of ld
template <bool INV>
__device__ __forceinline__ void direct_dft(const float2* zin, float2* zout, const float2* tw, int n, int ld,
                                           int nseq) {
  for (int idx = threadIdx.x; idx < nseq * n; idx += blockDim.x) {
    const int q = idx / n, k = idx - q * n;
    const float2* s = zin + q * ld;
    float re = 0.f, im = 0.f;
    int e = 0;
    for (int t = 0; t < n; ++t) {
      const float2 w = tw[e];
      const float2 v = s[t];
      const float wy = INV ? -w.y : w.y;
      re = fmaf(v.x, w.x, fmaf(-v.y, wy, re));
      im = fmaf(v.x, wy, fmaf(v.y, w.x, im));
      e += k;
      if (e >= n) e -= n;
    }
    zout[q * ld + k] = make_float2(re, im);
  }
}

// The ring transform of nseq sequences (stride seq_ld(n)) in a, b as scratch: the FFT when
// the ring has a plan (pi >= 0), else the direct DFT with the twiddles tw.  Returns the buffer
// holding the result.  All threads call it; it synchronises before returning.
template <bool INV>
__device__ __forceinline__ float2* ring_transform(float2* a, float2* b, const float2* tw, int n, int nseq, int pi,
                                                  const FftPlan* __restrict__ plans,
                                                  const float2* __restrict__ tw_all, const int* __restrict__ tw_base) {
  if (pi >= 0) {
    const FftPlan pl = plans[pi];
    return fft_smem<INV>(a, b, tw_all + tw_base[pi], pl, nseq);
  }
  direct_dft<INV>(a, b, tw, n, seq_ld(n), nseq);
  __syncthreads();
  return b;
}

// from the transformed ring pair D: S = a (F_N + F_S), D = a (F_N - F_S) for m <= lmax into X
template <int FG>
__device__ __forceinline__ void hp_unpack_store(const float2* D, const float2* ph, int n, int nfg, int f0, int lmax,
                                                int nh, int jh, float aj, float* __restrict__ X, int ldc) {
  const int ld = seq_ld(n);
  for (int idx = threadIdx.x; idx < (lmax + 1) * FG; idx += blockDim.x) {
    const int m = idx / FG, q = idx - m * FG;
    if (q >= nfg) continue;
    const int k = m % n, kk = (n - k) % n;
    const float2 zm = D[q * ld + k], zn = D[q * ld + kk];
    float2 FN = make_float2(0.5f * (zm.x + zn.x), 0.5f * (zm.y - zn.y));
    float2 FS = make_float2(0.5f * (zm.y + zn.y), -0.5f * (zm.x - zn.x));
    const float2 e = make_float2(ph[m].x, -ph[m].y);   // e^{-i m phi0}
    FN = c_mul(FN, e);
    FS = c_mul(FS, e);
    const int f = f0 + q;
    *reinterpret_cast<float2*>(X + ((size_t)(2 * m) * nh + jh) * ldc + 2 * f) =
        make_float2(aj * (FN.x + FS.x), aj * (FN.y + FS.y));
    *reinterpret_cast<float2*>(X + ((size_t)(2 * m + 1) * nh + jh) * ldc + 2 * f) =
        make_float2(aj * (FN.x - FS.x), aj * (FN.y - FS.y));
  }
}

template <int FG>
__global__ void __launch_bounds__(kHpThreads) k_hp_fwd(const float* __restrict__ in, int nf, size_t npix,
                                                       const int* __restrict__ rlen,
                                                       const long long* __restrict__ roff,
                                                       const int2* __restrict__ rphase, int nrings, int lmax, int nh,
                                                       float area, float* __restrict__ X, int ldc,
                                                       const int* __restrict__ rplan, const FftPlan* __restrict__ plans,
                                                       const float2* __restrict__ tw_all,
                                                       const int* __restrict__ tw_base,
                                                       const ProbState* __restrict__ ps) {
  extern __shared__ __align__(16) float2 sm[];
  const int jh = blockIdx.y, f0 = blockIdx.x * FG;
  const int nfg = min(FG, nf - f0);
  const int j = jh, J = nrings - 1 - jh;
  const int n = rlen[j], ld = seq_ld(n);
  const int pi = rplan[j];
  float2* zb = sm;               // [FG][ld]
  float2* db = zb + FG * ld;     // [FG][ld]
  float2* tw = db + FG * ld;     // [n] (direct DFT rings)
  float2* ph = tw + n;           // [lmax + 1]
  ring_tables(pi >= 0 ? nullptr : tw, ph, n, rphase[j], lmax);
  for (int q = 0; q < nfg; ++q) {
    const float* fj = in + (size_t)(f0 + q) * npix + roff[j];
    const float* fJ = in + (size_t)(f0 + q) * npix + roff[J];
    const float sc = ps ? (float)ps[f0 + q].beta : 1.f;   // per-field factor (gradient sweeps)
    for (int k = threadIdx.x; k < n; k += blockDim.x)
      zb[q * ld + k] = make_float2(sc * fj[k], J != j ? sc * fJ[k] : 0.f);
  }
  __syncthreads();
  const float2* D = ring_transform<false>(zb, db, tw, n, nfg, pi, plans, tw_all, tw_base);
  hp_unpack_store<FG>(D, ph, n, nfg, f0, lmax, nh, jh, area, X, ldc);
}

template <int FG>
__global__ void __launch_bounds__(kHpThreads) k_hp_idft(const float* __restrict__ Y, int ldc, int nf, size_t npix,
                                                        const int* __restrict__ rlen,
                                                        const long long* __restrict__ roff,
                                                        const int2* __restrict__ rphase, int nrings, int lmax,
                                                        int nh, float area, EpiParams ep,
                                                        const int* __restrict__ rplan,
                                                        const FftPlan* __restrict__ plans,
                                                        const float2* __restrict__ tw_all,
                                                        const int* __restrict__ tw_base) {
  extern __shared__ __align__(16) float2 sm[];
  __shared__ float red[kHpThreads / 32][FG * NPART];
  __shared__ EpiField fi[FG];
  const int jh = blockIdx.y, f0 = blockIdx.x * FG;
  const int nfg = min(FG, nf - f0);
  const int j = jh, J = nrings - 1 - jh;
  const int n = rlen[j], ld = seq_ld(n);
  const int pi = rplan[j];
  const int nm = lmax + 1;
  float2* za = sm;               // [FG][ld]  spectra Z
  float2* zb = za + FG * ld;     // [FG][ld]
  float2* tw = zb + FG * ld;     // [n] (direct DFT rings)
  float2* ph = tw + n;           // [lmax + 1]
  float2* gn = ph + nm;          // [lmax + 1][FG]  G_N = E + O
  float2* gs = gn + nm * FG;     // [lmax + 1][FG]  G_S = E - O
  epi_fields_load<FG>(ep, f0, nfg, fi);
  ring_tables(pi >= 0 ? nullptr : tw, ph, n, rphase[j], lmax);
  for (int idx = threadIdx.x; idx < nm * FG; idx += blockDim.x) {
    const int m = idx / FG, q = idx - m * FG;
    float2 E = make_float2(0.f, 0.f), O = make_float2(0.f, 0.f);
    if (q < nfg) {
      E = *reinterpret_cast<const float2*>(Y + ((size_t)(2 * m) * nh + jh) * ldc + 2 * (f0 + q));
      if (m < lmax) O = *reinterpret_cast<const float2*>(Y + ((size_t)(2 * m + 1) * nh + jh) * ldc + 2 * (f0 + q));
    }
    gn[idx] = make_float2(E.x + O.x, E.y + O.y);
    gs[idx] = make_float2(E.x - O.x, E.y - O.y);
  }
  __syncthreads();
  // Z_k: orders m >= 0 with m = k (mod n) and m = -m' (m' >= 1) with m' = n - k (mod n)
  for (int idx = threadIdx.x; idx < nfg * n; idx += blockDim.x) {
    const int q = idx / n, k = idx - q * n;
    float re = 0.f, im = 0.f;
    for (int m = k; m <= lmax; m += n) {   // e^{i m phi0} (G_N + i G_S)
      const float2 a = gn[m * FG + q], b = gs[m * FG + q];
      const float2 t = c_mul(ph[m], make_float2(a.x - b.y, a.y + b.x));
      re += t.x;
      im += t.y;
    }
    for (int mp = (k == 0) ? n : n - k; mp <= lmax; mp += n) {   // e^{-i m' phi0} (conj G_N + i conj G_S)
      const float2 a = gn[mp * FG + q], b = gs[mp * FG + q];
      const float2 t = c_mul(make_float2(ph[mp].x, -ph[mp].y), make_float2(a.x + b.y, b.x - a.y));
      re += t.x;
      im += t.y;
    }
    za[q * ld + k] = make_float2(re, im);
  }
  __syncthreads();
  float2* z = ring_transform<true>(za, zb, tw, n, nfg, pi, plans, tw_all, tw_base);   // K v on the ring pair
  float2* other = (z == za) ? zb : za;   // receives the new scaling
  const bool two = (J != j);
  ring_pair_epilogue<FG, kHpThreads>(z, other, ld, n, nfg, f0, npix, (size_t)roff[j], (size_t)roff[J], two, area,
                                     nh, jh, ep, red, fi);
  if (ep.mode == EPI_PLAIN) return;
  if ((ep.mode == EPI_UPDATE || ep.mode == EPI_SYM) && ep.xout) {   // transform the new scaling
    __syncthreads();
    const float2* D = ring_transform<false>(other, z, tw, n, nfg, pi, plans, tw_all, tw_base);
    hp_unpack_store<FG>(D, ph, n, nfg, f0, lmax, nh, jh, area, ep.xout, ldc);
  }
}

size_t hp_fwd_smem(int fg, int n, int lmax) {
  return (size_t)(2 * fg * seq_ld(n) + n + lmax + 1) * sizeof(float2);
}
size_t hp_idft_smem(int fg, int n, int lmax) {
  return (size_t)(2 * fg * seq_ld(n) + n + (lmax + 1) * (1 + 2 * fg)) * sizeof(float2);
}

int hp_pick_fg(const Grid& g, int nf, bool inverse) {
  const int n = g.nlon;   // the longest ring
  int fg = 4;
  while (fg > 1 && (fg > nf || (inverse ? hp_idft_smem(fg, n, g.lmax) : hp_fwd_smem(fg, n, g.lmax)) > 100 * 1024))
    fg >>= 1;
  return fg;
}

template <int FG>
int hp_fwd_t(const Grid& g, const float* in, int nf, float* X, int ldc, cudaStream_t st, const ProbState* ps) {
  const size_t smem = hp_fwd_smem(FG, g.nlon, g.lmax);
  SHOT_CUDA(cudaFuncSetAttribute(k_hp_fwd<FG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope prof(PK_DFT, st);
  count_launch();
  k_hp_fwd<FG><<<dim3((nf + FG - 1) / FG, g.nh), kHpThreads, smem, st>>>(
      in, nf, g.npix, g.ring_len_d, g.ring_off_d, g.ring_phase_d, g.nlat, g.lmax, g.nh, (float)g.a_ring[0], X, ldc,
      g.ring_plan_d, g.hp_plan_d, g.hp_tw_d, g.hp_tw_base_d, ps);
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

template <int FG>
int hp_idft_t(const Grid& g, const float* Y, int ldc, int nf, const EpiParams& ep, cudaStream_t st) {
  const size_t smem = hp_idft_smem(FG, g.nlon, g.lmax);
  SHOT_CUDA(cudaFuncSetAttribute(k_hp_idft<FG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope prof(ep.mode == EPI_CHECK || ep.mode == EPI_FINAL ? PK_CHECK : PK_IDFT, st);
  count_launch();
  k_hp_idft<FG><<<dim3((nf + FG - 1) / FG, g.nh), kHpThreads, smem, st>>>(
      Y, ldc, nf, g.npix, g.ring_len_d, g.ring_off_d, g.ring_phase_d, g.nlat, g.lmax, g.nh, (float)g.a_ring[0], ep,
      g.ring_plan_d, g.hp_plan_d, g.hp_tw_d, g.hp_tw_base_d);
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

}  // namespace

int launch_hp_dft_fwd(const Grid& g, const float* in, int nf, float* X, int ldc, cudaStream_t st,
                      const ProbState* ps) {
  switch (hp_pick_fg(g, nf, false)) {
    case 4: return hp_fwd_t<4>(g, in, nf, X, ldc, st, ps);
    case 2: return hp_fwd_t<2>(g, in, nf, X, ldc, st, ps);
    default: return hp_fwd_t<1>(g, in, nf, X, ldc, st, ps);
  }
}

int launch_hp_idft(const Grid& g, const float* Y, int ldc, int nf, const EpiParams& ep, cudaStream_t st) {
  switch (hp_pick_fg(g, nf, true)) {
    case 4: return hp_idft_t<4>(g, Y, ldc, nf, ep, st);
    case 2: return hp_idft_t<2>(g, Y, ldc, nf, ep, st);
    default: return hp_idft_t<1>(g, Y, ldc, nf, ep, st);
  }
}

// Ring geometry of a HEALPix grid of resolution nside (host, FP64), into the Grid: node
// z = cos(theta) per ring, ring lengths, offsets, longitude phases, per-pixel area.
void healpix_geometry(Grid& g, int nside) {
  const int nr = 4 * nside - 1;
  g.x.assign(nr, 0.0);
  g.ring_len.assign(nr, 0);
  g.ring_off.assign(nr + 1, 0);
  g.ring_phase.assign(nr, std::make_pair(0, 1));
  for (int i = 1; i <= nr; ++i) {
    const int k = i <= 2 * nside ? i : nr + 1 - i;   // mirrored into the north half
    double z;
    int n, pn, pd;
    if (k < nside) {
      z = 1.0 - (double)k * k / (3.0 * nside * nside);
      n = 4 * k;
      pn = 1;
      pd = 4 * k;   // phi0 = pi / (4k)
    } else {
      const int s = (k - nside + 1) % 2;
      z = 4.0 / 3.0 - 2.0 * k / (3.0 * nside);
      n = 4 * nside;
      pn = 2 - s;
      pd = 4 * nside;   // phi0 = pi (2 - s) / (4 nside)
    }
    g.x[i - 1] = (i <= 2 * nside) ? z : -z;
    g.ring_len[i - 1] = n;
    g.ring_phase[i - 1] = std::make_pair(pn, pd);
  }
  g.x[2 * nside - 1] = 0.0;   // the equator ring
  for (int i = 0; i < nr; ++i) g.ring_off[i + 1] = g.ring_off[i] + g.ring_len[i];
  g.npix = (size_t)g.ring_off[nr];
  const double area = 4.0 * M_PI / (double)g.npix;
  g.a_ring.assign(nr, area);
  g.w.resize(nr);
  for (int i = 0; i < nr; ++i) g.w[i] = area * g.ring_len[i] / (2.0 * M_PI);   // ring weight, sum 2
}

}  // namespace shot
