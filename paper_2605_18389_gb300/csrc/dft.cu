// Ring DFTs of the semi-naive SHT and the fused Sinkhorn epilogues.
//
// Forward (App. C.1, last paragraph; App. B quadrature): for a field f and ring j,
//   F_m(j) = sum_k f_jk e^{-i m phi_k},  m = 0..lmax.
// Rings j (north) and J = nlat-1-j (south) are transformed together as ONE complex
// sequence z = f_j + i f_J; F_N(m) = (Z(m) + conj Z(N-m))/2, F_S(m) = (Z(m) - conj Z(N-m))/(2i).
// Because Pbar_lm(-x) = (-1)^{l+m} Pbar_lm(x) and GL nodes are symmetric, the quadrature
// sum over j splits into an even part (l-m even) over S = a_j (F_N + F_S) and an odd part
// (l-m odd) over D = a_j (F_N - F_S) on the north half only.  The kernel writes S and D
// into the (m, parity) blocks X[2m+p][jh][2f + {re,im}].
//
// Inverse: the synthesis produces E_m(jh) (even degrees) and O_m(jh) (odd degrees); the
// north ring has G_N = E + O, the south ring G_S = E - O, and
//   (K v)(theta_j, phi_k) = Re G_0(j) + 2 Re sum_{m>=1} G_m(j) e^{i m phi_k}
// is evaluated for both rings by one inverse complex FFT of the Hermitian-extended
// spectrum Z(m) = G_N(m) + i G_S(m), Z(N-m) = conj G_N(m) + i conj G_S(m).
// The epilogue then applies Algorithm 1's pointwise step to K v (update, check or
// final objective) and reduces per-field partial sums (FP64) per ring pair.
#include "fft.cuh"
#include "epilogue.cuh"

namespace shot {

namespace {

constexpr int kThreads = kFftThreads;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }


// Loads rings j (real part) and J = nlat-1-j (imaginary part) of nfg fields into buf.
__device__ __forceinline__ void load_ring_pairs(const float* __restrict__ in, float2* buf, int f0, int nfg,
                                                int nlat, int nlon, int j, int J) {
  const int N = nlon, ld = seq_ld(N);
  for (int q = 0; q < nfg; ++q) {
    const float* fj = in + (size_t)(f0 + q) * nlat * nlon + (size_t)j * nlon;
    const float* fJ = in + (size_t)(f0 + q) * nlat * nlon + (size_t)J * nlon;
    for (int k = threadIdx.x; k < N; k += blockDim.x)
      buf[q * ld + k] = make_float2(__ldg(fj + k), (J != j) ? __ldg(fJ + k) : 0.f);
  }
}

// Two-for-one unpack of the transformed ring pair (j north, J south) and the parity fold:
// F_N(m) = (Z(m) + conj Z(N-m))/2, F_S(m) = (Z(m) - conj Z(N-m))/(2i);
// S = a_j (F_N + F_S) -> block (m, even), D = a_j (F_N - F_S) -> block (m, odd).
template <int FG>
__device__ __forceinline__ void unpack_fold_store(const float2* buf, int nfg, int f0, int N, int lmax, int nh, int jh,
                                                  float aj, const ProbState* __restrict__ ps, int scale_which,
                                                  float* __restrict__ X, int ldc) {
  const int nm = lmax + 1, ld = seq_ld(N);
  for (int idx = threadIdx.x; idx < nm * FG; idx += blockDim.x) {
    const int m = idx / FG, q = idx - m * FG;
    if (q >= nfg) continue;
    const int f = f0 + q;
    float sc = aj;
    if (scale_which == 1) sc *= (float)ps[f].beta;
    const float2 zm = buf[q * ld + m];
    const float2 zn = buf[q * ld + (m ? N - m : 0)];
    const float2 FN = make_float2(0.5f * (zm.x + zn.x), 0.5f * (zm.y - zn.y));
    const float2 FS = make_float2(0.5f * (zm.y + zn.y), -0.5f * (zm.x - zn.x));
    const float2 S = make_float2(sc * (FN.x + FS.x), sc * (FN.y + FS.y));
    const float2 D = make_float2(sc * (FN.x - FS.x), sc * (FN.y - FS.y));
    const size_t oS = ((size_t)(2 * m) * nh + jh) * ldc + 2 * f;
    const size_t oD = ((size_t)(2 * m + 1) * nh + jh) * ldc + 2 * f;
    *reinterpret_cast<float2*>(X + oS) = S;
    *reinterpret_cast<float2*>(X + oD) = D;
  }
}

template <int FG>
__global__ void __launch_bounds__(kThreads, 3) k_dft_fwd(
    const float* __restrict__ in, int nf, int nlat, int nlon, int lmax, int nh,
    const float* __restrict__ a_ring, const ProbState* __restrict__ ps, int scale_which,
    float* __restrict__ X, int ldc, FftPlan pl, const float2* __restrict__ tw_g) {
  extern __shared__ __align__(16) float2 sm[];
  const int N = nlon;
  float2* b0 = sm;
  float2* b1 = b0 + FG * seq_ld(N);
  float2* tw = b1 + FG * seq_ld(N);
  const int jh = blockIdx.y;
  const int f0 = blockIdx.x * FG;
  const int nfg = min(FG, nf - f0);
  const int j = jh, J = nlat - 1 - jh;

  for (int k = threadIdx.x; k < fft_tw_len(pl); k += blockDim.x) tw[k] = tw_g[k];
  load_ring_pairs(in, b0, f0, nfg, nlat, nlon, j, J);
  __syncthreads();
  const float2* buf = fft_smem<false>(b0, b1, tw, pl, nfg);

  unpack_fold_store<FG>(buf, nfg, f0, N, lmax, nh, jh, a_ring[j], ps, scale_which, X, ldc);
}

template <int FG, class PL = RuntimePlan>
__global__ void __launch_bounds__(kThreads, 3) k_idft(
    const float* __restrict__ Y, int ldc, int nf, int nlat, int nlon, int lmax, int nh,
    const float* __restrict__ a_ring, FftPlan pl, const float2* __restrict__ tw_g, EpiParams ep) {
  extern __shared__ __align__(16) float2 sm[];
  __shared__ float red[kThreads / 32][FG * NPART];
  __shared__ EpiField fi[FG];
  const int N = nlon;
  const int ld = seq_ld(N);
  float2* buf = sm;
  float2* b1 = buf + FG * ld;
  float2* tw = b1 + FG * ld;
  const int jh = blockIdx.y;
  const int f0 = blockIdx.x * FG;
  const int nfg = min(FG, nf - f0);
  const int j = jh, J = nlat - 1 - jh;

  // Gather this ring pair's spectra of the CTA's fields, E_m and O_m for every order (the
  // (2m+1) block of m = lmax is empty), into b1 with asynchronous copies: all of them are
  // in flight at once.  Row (blk, jh) holds the fields' (re, im) pairs contiguously; a
  // field group of even size starts on a 16-byte boundary (ldc is a multiple of 4), and
  // reading up to the next even field stays inside the row.
  float2* stg = b1;   // stg[blk * FG + q]
  const int nblk_v = 2 * lmax + 1;
  if constexpr (FG % 2 == 0) {
    constexpr int ch = FG / 2;
    for (int e = threadIdx.x; e < nblk_v * ch; e += blockDim.x) {
      const int blk = e / ch, c = e - blk * ch;
      if (2 * c < nfg) cp_async16(stg + blk * FG + 2 * c, Y + ((size_t)blk * nh + jh) * ldc + 2 * f0 + 4 * c);
    }
  } else {
    for (int blk = threadIdx.x; blk < nblk_v; blk += blockDim.x)
      cp_async8(stg + blk * FG, Y + ((size_t)blk * nh + jh) * ldc + 2 * f0);
  }
  epi_fields_load<FG>(ep, f0, nfg, fi);
  for (int k = threadIdx.x; k < fft_tw_len(pl); k += blockDim.x) tw[k] = tw_g[k];
  // zero the band lmax < m < N - lmax
  const int nz = N - 2 * lmax - 1;
  for (int q = 0; q < nfg; ++q)
    for (int k = threadIdx.x; k < nz; k += blockDim.x) buf[q * ld + lmax + 1 + k] = make_float2(0.f, 0.f);
  cp_async_wait_all();
  __syncthreads();
  epi_prefetch_marginals<FG>(ep, fi, nfg, (size_t)j * nlon, (size_t)(nlat - 1 - jh) * nlon, nlat - 1 - jh != jh, N, f0,
                             (size_t)nlat * nlon);
  const int nm = lmax + 1;
  for (int idx = threadIdx.x; idx < nm * FG; idx += blockDim.x) {
    const int m = idx / FG, q = idx - m * FG;
    if (q >= nfg) continue;
    const float2 E = stg[(2 * m) * FG + q];
    const float2 O = (m < lmax) ? stg[(2 * m + 1) * FG + q] : make_float2(0.f, 0.f);
    const float2 GN = make_float2(E.x + O.x, E.y + O.y);
    const float2 GS = make_float2(E.x - O.x, E.y - O.y);
    if (m == 0) {
      buf[q * ld] = make_float2(GN.x, GS.x);
    } else {
      buf[q * ld + m] = make_float2(GN.x - GS.y, GN.y + GS.x);
      buf[q * ld + N - m] = make_float2(GN.x + GS.y, GS.x - GN.y);
    }
  }
  __syncthreads();
  const float2* z = fft_smem_plan<true, PL>(buf, b1, tw, pl, nfg);
  float2* other = (z == buf) ? b1 : buf;   // input of the fused forward transform

  const float aj = a_ring[j];
  const bool two = (J != j);   // false only for the equator ring of an odd grid
  ring_pair_epilogue<FG, kThreads>(z, other, ld, N, nfg, f0, (size_t)nlat * nlon, (size_t)j * nlon,
                                   (size_t)J * nlon, two, aj, nh, jh, ep, red, fi);
  if (ep.mode == EPI_PLAIN) return;
  if ((ep.mode == EPI_UPDATE || ep.mode == EPI_SYM) && ep.xout) {
    // the new scaling of this ring pair is in `other`: transform it for the next half-step
    __syncthreads();
    const float2* zf = fft_smem_plan<false, PL>(other, const_cast<float2*>(z), tw, pl, nfg);
    unpack_fold_store<FG>(zf, nfg, f0, N, lmax, nh, jh, aj, nullptr, 0, ep.xout, ldc);
  }
}

// ---------------------------------------------------------------------------------
// Persistent form of k_idft for the solver's update half-steps (EPI_UPDATE with the fused
// forward transform of the new scaling) and its marginal checks (EPI_CHECK, no forward
// transform).  A CTA walks over items (ring pair jh, field group)
// item = blockIdx.x + i gridDim.x, consecutive items covering the field groups of one ring
// pair.  Right after it has unpacked one item's spectra it starts the cp.async gather of the
// next item's spectra rows into a staging area and asks L2 for the next item's marginal rows,
// so that neither the gather nor the update waits on DRAM.  The stage twiddles are read
// through L1 (every CTA reads the same N values) rather than copied into shared memory, which
// keeps three CTAs per SM (~68 KB each at 1440 longitudes and two fields).
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// shared-memory layout of k_idft_p (bytes): [buf][b1] sequences, then the spectra staging
// area, 16-byte aligned
struct IdftPLayout {
  size_t stg, total;
};
__host__ __device__ inline IdftPLayout idft_p_layout(int FG, int N, int lmax) {
  IdftPLayout L;
  L.stg = ((size_t)2 * FG * seq_ld(N) * sizeof(float2) + 15) / 16 * 16;
  L.total = L.stg + (size_t)(2 * lmax + 1) * FG * sizeof(float2);
  return L;
}

template <int FG, class PL = RuntimePlan>
__global__ void __launch_bounds__(kThreads, 3) k_idft_p(
    const float* __restrict__ Y, int ldc, int nf, int nlat, int nlon, int lmax, int nh,
    const float* __restrict__ a_ring, FftPlan pl, const float2* __restrict__ tw_g, EpiParams ep, int ngroups) {
  extern __shared__ __align__(16) float2 sm[];
  __shared__ float red[kThreads / 32][FG * NPART];
  __shared__ EpiField fi[2][FG];
  const int N = nlon, ld = seq_ld(N);
  float2* buf = sm;
  float2* b1 = buf + FG * ld;
  float2* stg = reinterpret_cast<float2*>(reinterpret_cast<uint8_t*>(sm) + idft_p_layout(FG, N, lmax).stg);
  const int nblk_v = 2 * lmax + 1;   // the (2m+1) block of m = lmax is empty
  const int nitems = ngroups * nh;

  auto item_geom = [&](int item, int& jh, int& f0, int& nfg) {
    jh = item / ngroups;
    f0 = (item - jh * ngroups) * FG;
    nfg = min(FG, nf - f0);
  };
  auto issue_Y = [&](int item) {   // spectra rows E_m, O_m of the item's fields -> stg[blk][FG]
    if (item >= nitems) return;
    int jh, f0, nfg;
    item_geom(item, jh, f0, nfg);
    if constexpr (FG % 2 == 0) {
      constexpr int ch = FG / 2;
      for (int e = threadIdx.x; e < nblk_v * ch; e += blockDim.x) {
        const int blk = e / ch, c = e - blk * ch;
        if (2 * c < nfg) cp_async16(stg + blk * FG + 2 * c, Y + ((size_t)blk * nh + jh) * ldc + 2 * f0 + 4 * c);
      }
    } else {
      for (int blk = threadIdx.x; blk < nblk_v; blk += blockDim.x)
        cp_async8(stg + blk * FG, Y + ((size_t)blk * nh + jh) * ldc + 2 * f0);
    }
    cp_async_commit();
  };

  int item = blockIdx.x, slot = 0;
  if (item < nitems) {
    int jh, f0, nfg;
    item_geom(item, jh, f0, nfg);
    epi_fields_load<FG>(ep, f0, nfg, fi[0]);
  }
  issue_Y(item);
  __syncthreads();
  if (item < nitems) {
    int jh, f0, nfg;
    item_geom(item, jh, f0, nfg);
    epi_prefetch_marginals<FG>(ep, fi[0], nfg, (size_t)jh * nlon, (size_t)(nlat - 1 - jh) * nlon,
                               nlat - 1 - jh != jh, N, f0, (size_t)nlat * nlon);
  }
  while (item < nitems) {
    const int next = item + gridDim.x;
    int jh, f0, nfg;
    item_geom(item, jh, f0, nfg);
    const int j = jh, J = nlat - 1 - jh;
    cp_async_wait_all();   // this item's spectra
    __syncthreads();
    const int nz = N - 2 * lmax - 1;   // the band lmax < m < N - lmax is zero
    for (int q = 0; q < nfg; ++q)
      for (int k = threadIdx.x; k < nz; k += blockDim.x) buf[q * ld + lmax + 1 + k] = make_float2(0.f, 0.f);
    const int nm = lmax + 1;
    for (int idx = threadIdx.x; idx < nm * FG; idx += blockDim.x) {
      const int m = idx / FG, q = idx - m * FG;
      if (q >= nfg) continue;
      const float2 E = stg[(2 * m) * FG + q];
      const float2 O = (m < lmax) ? stg[(2 * m + 1) * FG + q] : make_float2(0.f, 0.f);
      const float2 GN = make_float2(E.x + O.x, E.y + O.y);
      const float2 GS = make_float2(E.x - O.x, E.y - O.y);
      if (m == 0) {
        buf[q * ld] = make_float2(GN.x, GS.x);
      } else {
        buf[q * ld + m] = make_float2(GN.x - GS.y, GN.y + GS.x);
        buf[q * ld + N - m] = make_float2(GN.x + GS.y, GS.x - GN.y);
      }
    }
    __syncthreads();
    if (next < nitems) {   // the staging area is free again: the next item's state and spectra
      int jn, fn, nn;
      item_geom(next, jn, fn, nn);
      epi_fields_load<FG>(ep, fn, nn, fi[slot ^ 1]);
    }
    issue_Y(next);
    const float2* z = fft_smem_plan<true, PL>(buf, b1, tw_g, pl, nfg);
    float2* other = (z == buf) ? b1 : buf;
    if (next < nitems) {   // fi[slot ^ 1] is visible after the transform's barriers
      int jn, fn, nn;
      item_geom(next, jn, fn, nn);
      epi_prefetch_marginals<FG>(ep, fi[slot ^ 1], nn, (size_t)jn * nlon, (size_t)(nlat - 1 - jn) * nlon,
                                 nlat - 1 - jn != jn, N, fn, (size_t)nlat * nlon);
    }
    const float aj = a_ring[j];
    const bool two = (J != j);
    // the persistent kernel runs updates and checks only: no final-objective branch
    ring_pair_epilogue<FG, kThreads, false>(z, other, ld, N, nfg, f0, (size_t)nlat * nlon, (size_t)j * nlon,
                                            (size_t)J * nlon, two, aj, nh, jh, ep, red, fi[slot]);
    if (ep.xout) {   // the update's new scaling: its spectra for the next half-step
      __syncthreads();
      const float2* zf = fft_smem_plan<false, PL>(other, const_cast<float2*>(z), tw_g, pl, nfg);
      unpack_fold_store<FG>(zf, nfg, f0, N, lmax, nh, jh, aj, nullptr, 0, ep.xout, ldc);
    }
    item = next;
    slot ^= 1;
  }
  cp_async_wait_all();
}

int pick_fg(int N, int nf) {
  int fg = 8;
  while (fg > 1 && (fg * N > kFftCap || fg > nf)) fg >>= 1;
  return fg;
}

template <int FG>
int launch_fwd_t(const Grid& g, const float* in, int nf, const ProbState* ps, int scale_which, float* X,
                 int ldc, cudaStream_t st) {
  const size_t smem = (size_t)(fft_tw_len(g.plan) + 2 * FG * seq_ld(g.nlon)) * sizeof(float2);
  SHOT_CUDA(cudaFuncSetAttribute(k_dft_fwd<FG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((nf + FG - 1) / FG, g.nh);   // field groups of one ring pair run together
  ProfScope prof(PK_DFT, st);
  count_launch();
  k_dft_fwd<FG><<<grid, kThreads, smem, st>>>(in, nf, g.nlat, g.nlon, g.lmax, g.nh, g.a_d, ps, scale_which, X,
                                              ldc, g.plan, g.tw_d);
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

template <int FG, class PL = RuntimePlan>
int launch_idft_t(const Grid& g, const float* Y, int ldc, int nf, const EpiParams& ep, cudaStream_t st) {
  // two sequence buffers (the second also stages the gathered spectra) and the twiddles
  const size_t smem = (size_t)(fft_tw_len(g.plan) + 2 * FG * seq_ld(g.nlon)) * sizeof(float2);
  SHOT_CUDA(cudaFuncSetAttribute(k_idft<FG, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((nf + FG - 1) / FG, g.nh);   // field groups of one ring pair run together
  ProfScope prof(ep.mode == EPI_CHECK || ep.mode == EPI_FINAL ? PK_CHECK : PK_IDFT, st);
  count_launch();
  k_idft<FG, PL><<<grid, kThreads, smem, st>>>(Y, ldc, nf, g.nlat, g.nlon, g.lmax, g.nh, g.a_d, g.plan, g.tw_d, ep);
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

template <int FG, class PL = RuntimePlan>
int launch_idft_p_t(const Grid& g, const float* Y, int ldc, int nf, const EpiParams& ep, cudaStream_t st) {
  const size_t smem = idft_p_layout(FG, g.nlon, g.lmax).total;
  SHOT_CUDA(cudaFuncSetAttribute(k_idft_p<FG, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int ngroups = (nf + FG - 1) / FG;
  const int nitems = ngroups * g.nh;
  const int grid = nitems < 3 * g.num_sms ? nitems : 3 * g.num_sms;
  ProfScope prof(ep.mode == EPI_CHECK || ep.mode == EPI_FINAL ? PK_CHECK : PK_IDFT, st);
  count_launch();
  k_idft_p<FG, PL><<<grid, kThreads, smem, st>>>(Y, ldc, nf, g.nlat, g.nlon, g.lmax, g.nh, g.a_d, g.plan, g.tw_d, ep,
                                                 ngroups);
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

// the runtime plan equals the compile-time one (same N and radices in the same order)
template <class PL>
bool plan_is(const FftPlan& p) {
  return p.N == PL::N && p.nst == 3 && p.R[0] == PL::R0 && p.R[1] == PL::R1 && p.R[2] == PL::R2;
}
using Plan1440 = CtPlan<1440, 15, 8, 12>;   // 720 x 1440 grids
using Plan1024 = CtPlan<1024, 4, 16, 16>;   // 512 x 1024 grids

}  // namespace

int launch_dft_fwd(const Grid& g, const float* in, int nf, const ProbState* ps, int scale_which,
                   float* X, int ldc, cudaStream_t st) {
  if (g.quad == SHOT_QUAD_HEALPIX) {
    if (scale_which && scale_which != 1) {
      set_error("HEALPix ring transform: the per-field factor beta only");
      return SHOT_ERR_UNSUPPORTED;
    }
    return launch_hp_dft_fwd(g, in, nf, X, ldc, st, scale_which == 1 ? ps : nullptr);
  }
  if (g.nlon > kFftCap) {
    set_error("nlon too large for the shared-memory ring FFT");
    return SHOT_ERR_UNSUPPORTED;
  }
  int fg = pick_fg(g.nlon, nf);
  if (g.active.nf == nf && g.active.dft_fg > 0 && g.active.dft_fg * g.nlon <= kFftCap) fg = g.active.dft_fg;
  switch (fg) {
    case 8: return launch_fwd_t<8>(g, in, nf, ps, scale_which, X, ldc, st);
    case 4: return launch_fwd_t<4>(g, in, nf, ps, scale_which, X, ldc, st);
    case 2: return launch_fwd_t<2>(g, in, nf, ps, scale_which, X, ldc, st);
    default: return launch_fwd_t<1>(g, in, nf, ps, scale_which, X, ldc, st);
  }
}

// whether launch_idft runs the persistent kernel (fixed field group of 2) for this epilogue
bool idft_is_persistent(const Grid& g, int nf, const EpiParams& ep) {
  return g.quad != SHOT_QUAD_HEALPIX && g.nlon <= kFftCap &&
         (((ep.mode == EPI_UPDATE || ep.mode == EPI_SYM) && ep.xout) || ep.mode == EPI_CHECK) &&
         !g.idft_nonpersistent && nf >= 2 && idft_p_layout(2, g.nlon, g.lmax).total <= 74 * 1024;
}

int launch_idft(const Grid& g, const float* Y, int ldc, int nf, const EpiParams& ep, cudaStream_t st) {
  if (g.quad == SHOT_QUAD_HEALPIX) return launch_hp_idft(g, Y, ldc, nf, ep, st);
  if (g.nlon > kFftCap) {
    set_error("nlon too large for the shared-memory ring FFT");
    return SHOT_ERR_UNSUPPORTED;
  }
  // the solver's update half-steps and marginal checks: persistent kernel with the next item's
  // inputs prefetched
  if (idft_is_persistent(g, nf, ep)) {
    if (plan_is<Plan1440>(g.plan)) return launch_idft_p_t<2, Plan1440>(g, Y, ldc, nf, ep, st);
    if (plan_is<Plan1024>(g.plan)) return launch_idft_p_t<2, Plan1024>(g, Y, ldc, nf, ep, st);
    return launch_idft_p_t<2>(g, Y, ldc, nf, ep, st);
  }
  int fg = pick_fg(g.nlon, nf);
  if (g.active.nf == nf && g.active.idft_fg > 0 && g.active.idft_fg * g.nlon <= kFftCap) fg = g.active.idft_fg;
  if (fg == 2 || fg == 4) {   // plans compiled for the common ring lengths
    if (plan_is<Plan1440>(g.plan))
      return fg == 2 ? launch_idft_t<2, Plan1440>(g, Y, ldc, nf, ep, st) : launch_idft_t<4, Plan1440>(g, Y, ldc, nf, ep, st);
    if (plan_is<Plan1024>(g.plan))
      return fg == 2 ? launch_idft_t<2, Plan1024>(g, Y, ldc, nf, ep, st) : launch_idft_t<4, Plan1024>(g, Y, ldc, nf, ep, st);
  }
  switch (fg) {
    case 8: return launch_idft_t<8>(g, Y, ldc, nf, ep, st);
    case 4: return launch_idft_t<4>(g, Y, ldc, nf, ep, st);
    case 2: return launch_idft_t<2>(g, Y, ldc, nf, ep, st);
    default: return launch_idft_t<1>(g, Y, ldc, nf, ep, st);
  }
}

}  // namespace shot
