// The Sinkhorn epilogue of the inverse ring transform, shared by the rectangular grids'
// FFT kernel and the HEALPix ring kernel.
//
// z holds K v on the ring pair (real part: ring j, imaginary part: ring J; nseq = nfg
// sequences of N longitudes at stride ld); the epilogue applies Algorithm 1's pointwise step
// of the given mode and reduces the per-field partial sums of the pair into
// ep.part[f][jh][NPART]:
//   EPI_PLAIN   out = K v
//   EPI_UPDATE  u = r p / Kv (balanced) or (r p / Kv)^{tau/(tau+eps)} with the problem's FP32
//               buffer factor r (ProbState ru / rv); sums: sum u (gauge) or sum a p u^{-eps/tau}
//               (translation-invariant step) and sum u (unbalanced buffer level),
//               non-positive and non-finite counts; when ep.xout is set the new scaling is
//               also written into `other` (u_j + i u_J) for the forward transform that follows
//   EPI_CHECK   |u_true (K v_true) - p| sums for the marginal error (L2 or L1, App. C.3)
//   EPI_FINAL   u_true, v_true (or the potentials), the marginal error, m(pi) and the dual
//               objective (in FP64); m(pi) = sum a q when a balanced v-update has run (then
//               v (K u) = q node by node), else sum a u (K v)
//   EPI_SYM     self term (q = p): u = sqrt(u_old (p / Ku)^gamma) in place (ep.out holds u_old),
//               breakdown counts; with ep.xout the new u is also written into `other`
// Field f occupies out[f * fstride ...]; rings j and J start at rj and rJ within a field.
#pragma once
#include "shot_internal.cuh"

namespace shot {

// Per-field state the epilogue needs, read into shared memory by epi_fields_load at the start
// of the kernel (while the spectra gather is in flight), so that the epilogue does not wait on
// the chain problem state -> marginal pointer -> marginal values.
struct EpiField {
  const float* marg;   // p (u-step) or q (v-step) of the field
  int live;            // EPI_FINAL: status >= 0; otherwise active
  int balanced;
  float gamma, et;
  float r;             // EPI_UPDATE: the buffer factor inside the ratio (ru or rv)
};

// Threads 0..FG-1 fill fi[q] for the CTA's fields f0 + q (q < nfg).
template <int FG>
__device__ __forceinline__ void epi_fields_load(const EpiParams& ep, int f0, int nfg, EpiField* fi) {
  const int q = threadIdx.x;
  if (q < FG && q < nfg && ep.mode != EPI_PLAIN) {
    const ProbState* P = ep.ps + f0 + q;
    EpiField e;
    e.marg = ep.marg[f0 + q];
    e.live = (ep.mode == EPI_FINAL) ? (P->status >= 0) : (P->active != 0);
    e.balanced = P->balanced;
    e.gamma = P->gamma;
    e.et = P->et;
    e.r = ep.which ? P->rv : P->ru;
    fi[q] = e;
  }
}

// After fi is visible to the block: asks L2 for the marginal rows j and J of the CTA's live
// fields (UPDATE and CHECK modes) and, for the check, the rows of the u buffer it reads (fields
// f0 + q at stride fstride in ep.other), one 128-byte line per thread, so that the epilogue's
// loads hit L2 instead of waiting on DRAM after the inverse transform.
template <int FG>
__device__ __forceinline__ void epi_prefetch_marginals(const EpiParams& ep, const EpiField* fi, int nfg, size_t rj,
                                                       size_t rJ, bool two, int N, int f0 = 0, size_t fstride = 0) {
  if (ep.mode != EPI_UPDATE && ep.mode != EPI_CHECK && ep.mode != EPI_SYM) return;
  const float* second = ep.mode == EPI_CHECK ? ep.other : (ep.mode == EPI_SYM ? ep.out : nullptr);
  const int nsrc = (second && fstride) ? 2 : 1;   // marginal (+ the u buffer the epilogue reads)
  const int lines = (N + 31) / 32 + 1;   // a row of N floats spans at most this many 128-byte lines
  const int per_field = 2 * nsrc * lines;
  for (int t = threadIdx.x; t < nfg * per_field; t += blockDim.x) {
    const int q = t / per_field, r = t - q * per_field;
    if (!fi[q].live) continue;
    const int src = r / (2 * lines), rr = r - src * 2 * lines;
    const int ring = rr / lines, l = rr - ring * lines;
    if (ring == 1 && !two) continue;
    const float* base = src ? second + (size_t)(f0 + q) * fstride : fi[q].marg;
    const float* row = base + (ring ? rJ : rj);
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(row) & ~uintptr_t(127);
    const uintptr_t a = a0 + (uintptr_t)l * 128;
    if (a < reinterpret_cast<uintptr_t>(row + N))
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
  }
}

__device__ __forceinline__ float epi_warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// kFinal = false compiles the EPI_FINAL branch out (kernels never launched with it)
template <int FG, int NT, bool kFinal = true>
__device__ __forceinline__ void ring_pair_epilogue(const float2* z, float2* other, int ld, int N, int nfg, int f0,
                                                   size_t fstride, size_t rj, size_t rJ, bool two, float aj,
                                                   int nh, int jh, const EpiParams& ep,
                                                   float (*red)[FG * NPART], const EpiField* fi) {
  constexpr int kEpiBatch = 6;   // longitudes per thread whose marginal values are loaded together
  if (ep.mode == EPI_PLAIN) {
    for (int q = 0; q < nfg; ++q) {
      float* oj = ep.out + (size_t)(f0 + q) * fstride + rj;
      float* oJ = ep.out + (size_t)(f0 + q) * fstride + rJ;
      for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const float2 zz = z[q * ld + k];
        oj[k] = zz.x;
        if (two) oJ[k] = zz.y;
      }
    }
    return;
  }
  // Per-element arithmetic is FP32; every thread sums its few elements (<= 2N/512 per
  // field) in FP32, warps reduce in FP32 and the cross-warp / grid sums are FP64.  A
  // thread takes longitude k of both rings of the pair.
  float acc[FG][NPART];
#pragma unroll
  for (int q = 0; q < FG; ++q)
#pragma unroll
    for (int i = 0; i < NPART; ++i) acc[q][i] = 0.f;
  // EPI_FINAL: the dual objective and m(pi) reach the block's FP64 sums through per-thread
  // partials: the potentials' offsets eps la and eps lb cancel between the two marginals' terms
  // and, across the three problems, in the divergence, so the balanced objective is formed per
  // thread as la sum p + lb sum q + sum (p log u_buf + q log v_buf), with the sums of p and q
  // (and the masses) compensated (Kahan) in FP32 and the offsets applied in FP64; per element
  // the work stays FP32.  m(pi) enters S_dual times eps.
  __shared__ double redd[NT / 32][FG][2];   // EPI_FINAL: warp sums of m(pi) and the objective

#pragma unroll
  for (int q = 0; q < FG; ++q) {
    if (q >= nfg) break;
    const int f = f0 + q;
    const size_t fbase = (size_t)f * fstride;
    float* outf = ep.out + fbase;
    float* othf = ep.other ? ep.other + fbase : nullptr;
    const EpiField F = fi[q];
    if (ep.mode == EPI_UPDATE) {
      if (!F.live) {
        if (ep.xout) {   // frozen problem: transform the stored scaling
          for (int k = threadIdx.x; k < N; k += blockDim.x)
            other[q * ld + k] = make_float2(outf[rj + k], two ? outf[rJ + k] : 0.f);
        }
        continue;
      }
      const float* mg = F.marg;
      const int bal = F.balanced;
      const float gam = F.gamma, rr = F.r, rinv = 1.f / F.r;
      for (int k0 = threadIdx.x; k0 < N; k0 += kEpiBatch * NT) {
        // the marginal values of all this thread's longitudes first, then the arithmetic
        float pv[kEpiBatch][2];
#pragma unroll
        for (int b = 0; b < kEpiBatch; ++b) {
          const int k = k0 + b * NT;
          pv[b][0] = (k < N) ? __ldg(mg + rj + k) : 0.f;
          pv[b][1] = (k < N && two) ? __ldg(mg + rJ + k) : 0.f;
        }
#pragma unroll
        for (int b = 0; b < kEpiBatch; ++b) {
          const int k = k0 + b * NT;
          if (k >= N) break;
          const float2 zz = z[q * ld + k];
          float u2[2];
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            if (r == 1 && !two) { u2[1] = 0.f; break; }
            const float kv = r ? zz.y : zz.x;
            const float pm = pv[b][r];
            const float ratio = __fdividef(pm, kv) * rr;   // MUFU reciprocal + multiply, <= 2 ulp
            float u;
            if (bal) {
              u = ratio;
              acc[q][0] += u;
            } else {
              // u = (r p/Kv)^gamma (hardware log2/exp2, ~2^-21 absolute in the exponent); the
              // translation-invariant sum's p u^{-eps/tau} = p (r p/Kv)^{-eps/(tau+eps)} equals
              // u (Kv) / r since gamma + eps/(tau+eps) = 1, so one power serves both (ratio = 0
              // gives u = 0 and adds nothing)
              u = exp2f(gam * __log2f(ratio));
              acc[q][0] += aj * u * kv * rinv;
              acc[q][1] += u;
            }
            // one test on the common path: K v positive and finite, u finite (NaN fails each
            // comparison); the rare failures are sorted into non-positive (first in the status
            // precedence) and non-finite
            if (!(kv > 0.f && kv < INFINITY && fabsf(u) < INFINITY)) {
              if (kv <= 0.f) acc[q][2] += 1.f;
              else acc[q][3] += 1.f;   // NaN or infinite K v, or u overflowed
            }
            if (!ep.skip_store) outf[(r ? rJ : rj) + k] = u;
            u2[r] = u;
          }
          if (ep.xout) other[q * ld + k] = make_float2(u2[0], u2[1]);
        }
      }
    } else if (ep.mode == EPI_SYM) {
      if (!F.live) {
        if (ep.xout) {   // frozen problem: transform the stored scaling
          for (int k = threadIdx.x; k < N; k += blockDim.x)
            other[q * ld + k] = make_float2(outf[rj + k], two ? outf[rJ + k] : 0.f);
        }
        continue;
      }
      const float* mg = F.marg;
      const int bal = F.balanced;
      const float gam = F.gamma;
      for (int k0 = threadIdx.x; k0 < N; k0 += kEpiBatch * NT) {
        // the marginal and old-scaling values of this thread's longitudes first, then the arithmetic
        float pv[kEpiBatch][2], uo[kEpiBatch][2];
#pragma unroll
        for (int b = 0; b < kEpiBatch; ++b) {
          const int k = k0 + b * NT;
          pv[b][0] = (k < N) ? __ldg(mg + rj + k) : 0.f;
          pv[b][1] = (k < N && two) ? __ldg(mg + rJ + k) : 0.f;
          uo[b][0] = (k < N) ? outf[rj + k] : 0.f;
          uo[b][1] = (k < N && two) ? outf[rJ + k] : 0.f;
        }
#pragma unroll
        for (int b = 0; b < kEpiBatch; ++b) {
          const int k = k0 + b * NT;
          if (k >= N) break;
          const float2 zz = z[q * ld + k];
          float u2[2];
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            if (r == 1 && !two) { u2[1] = 0.f; break; }
            const float kv = r ? zz.y : zz.x;
            const float ratio = __fdividef(pv[b][r], kv);
            const float t = bal ? ratio : exp2f(gam * __log2f(ratio));
            const float u = sqrtf(uo[b][r] * t);
            if (!(kv > 0.f && kv < INFINITY && fabsf(u) < INFINITY)) {
              if (kv <= 0.f) acc[q][2] += 1.f;
              else acc[q][3] += 1.f;
            }
            outf[(r ? rJ : rj) + k] = u;
            u2[r] = u;
          }
          if (ep.xout) other[q * ld + k] = make_float2(u2[0], u2[1]);
        }
      }
    } else if (ep.mode == EPI_CHECK) {
      if (!F.live) continue;
      const float* mg = F.marg;
      const float cuv = ep.ps[f].cuv;
      for (int k0 = threadIdx.x; k0 < N; k0 += kEpiBatch * NT) {
        // the marginal and u values of all this thread's longitudes first, then the arithmetic
        float pv[kEpiBatch][2], uv[kEpiBatch][2];
#pragma unroll
        for (int b = 0; b < kEpiBatch; ++b) {
          const int k = k0 + b * NT;
          pv[b][0] = (k < N) ? __ldg(mg + rj + k) : 0.f;
          pv[b][1] = (k < N && two) ? __ldg(mg + rJ + k) : 0.f;
          uv[b][0] = (k < N) ? __ldg(othf + rj + k) : 0.f;
          uv[b][1] = (k < N && two) ? __ldg(othf + rJ + k) : 0.f;
        }
#pragma unroll
        for (int b = 0; b < kEpiBatch; ++b) {
          const int k = k0 + b * NT;
          if (k >= N) break;
          const float2 zz = z[q * ld + k];
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            if (r == 1 && !two) break;
            const float kv = r ? zz.y : zz.x;
            const float pm = pv[b][r];
            const float d = fmaf(cuv * uv[b][r], kv, -pm);
            if (ep.norm_l1) {
              acc[q][0] += aj * fabsf(d);
              acc[q][1] += aj * pm;
            } else {
              acc[q][0] += d * d;
              acc[q][1] += pm * pm;
            }
          }
        }
      }
    } else if constexpr (kFinal) {  // EPI_FINAL: z = K v_buf; ep.other = u buffer, ep.out = v buffer
      if (!F.live) continue;
      const ProbState* P = ep.ps + f;
      const float* pp = ep.marg[f];
      const float* qq = ep.marg2[f];
      const float cu = P->cu, cv = P->cv, cuv = P->cuv;
      // log u_true = la + log u_buf with la split into an FP32 head and a small remainder
      const float la_hi = (float)P->la, lb_hi = (float)P->lb;
      const float la_lo = (float)(P->la - (double)la_hi), lb_lo = (float)(P->lb - (double)lb_hi);
      const int bal = P->balanced;
      // balanced, after a v-update: v (K u) = q at every node, so m(pi) = sum a u (K v) =
      // sum a v (K u) = sum a q (K is self-adjoint in the area inner product)
      const bool mass_q = bal && !isnan(P->mass_v);
      const float epsf = (float)ep.eps, tauf = (float)P->tau, et = bal ? 0.f : (float)(ep.eps / P->tau);
      // balanced: A = sum p, B = sum q (compensated), C = sum p log u_buf + q log v_buf, D = sum
      // u (K v) (m(pi) before any v-update); unbalanced: A = sum u (K v), B = the objective's terms
      float A = 0.f, Ac = 0.f, B = 0.f, Bc = 0.f, C = 0.f, D = 0.f;
      auto kahan = [](float& s, float& c, float x) {
        const float y = x - c, t = s + y;
        c = (t - s) - y;
        s = t;
      };
      for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const float2 zz = z[q * ld + k];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          if (r == 1 && !two) break;
          const float kv = r ? zz.y : zz.x;
          const size_t o = (r ? rJ : rj) + k;
          const float pm = __ldg(pp + o), qm = __ldg(qq + o);
          const float ub = othf[o], vb = outf[o];
          const float lu = la_hi + (logf(ub) + la_lo), lv = lb_hi + (logf(vb) + lb_lo);
          if (ep.potentials) {
            othf[o] = epsf * lu;
            outf[o] = epsf * lv;
          } else {
            othf[o] = cu * ub;
            outf[o] = cv * vb;
          }
          const float ukv = cuv * ub * kv;   // u_true (K v_true)
          const float d = ukv - pm;
          if (ep.norm_l1) {
            acc[q][0] += aj * fabsf(d);
            acc[q][1] += aj * pm;
          } else {
            acc[q][0] += d * d;
            acc[q][1] += pm * pm;
          }
          // phi = eps log u, psi = eps log v (App. C.2); terms with a zero marginal vanish.
          // Balanced: p (la + log u_buf) + q (lb + log v_buf), the offsets applied per thread
          // below; eps and a_j multiply the sums.
          if (bal) {
            kahan(A, Ac, pm);
            kahan(B, Bc, qm);
            C += (pm > 0.f ? pm * logf(ub) : 0.f) + (qm > 0.f ? qm * logf(vb) : 0.f);
            D += ukv;
          } else {  // tau (1 - e^{-phi/tau}) = -tau expm1(-(eps/tau) log u), per node in FP32
            kahan(A, Ac, ukv);
            kahan(B, Bc, (pm > 0.f ? -tauf * expm1f(-et * lu) * pm : 0.f) +
                             (qm > 0.f ? -tauf * expm1f(-et * lv) * qm : 0.f));
          }
        }
      }
      // this thread's m(pi) and objective in FP64, then the warp's sums
      double vm, vo;
      if (bal) {
        vm = mass_q ? (double)B - (double)Bc : (double)D;
        vo = P->la * ((double)A - (double)Ac) + P->lb * ((double)B - (double)Bc) + (double)C;
      } else {
        vm = (double)A - (double)Ac;
        vo = (double)B - (double)Bc;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        vm += __shfl_xor_sync(0xffffffffu, vm, o);
        vo += __shfl_xor_sync(0xffffffffu, vo, o);
      }
      if ((threadIdx.x & 31) == 0) {
        redd[threadIdx.x >> 5][q][0] = vm;
        redd[threadIdx.x >> 5][q][1] = vo;
      }
    }
  }
  // one block reduction for all fields of the CTA
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < FG; ++q)
#pragma unroll
    for (int i = 0; i < NPART; ++i) {
      const float v = epi_warp_sum(acc[q][i]);
      if (lane == 0) red[wid][q * NPART + i] = v;
    }
  __syncthreads();
  if constexpr (kFinal) {
    if (ep.mode == EPI_FINAL && threadIdx.x < 2 * FG) {
      const int q = threadIdx.x >> 1, i = threadIdx.x & 1;
      if (q < nfg && fi[q].live) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += redd[w][q][i];
        // m(pi) sums a_j times the node values; the balanced objective's sums are of
        // p (la + log u_buf) + q (lb + log v_buf): times eps a_j
        const double sc = (i == 1 && fi[q].balanced) ? ep.eps * (double)aj : (double)aj;
        ep.part[((size_t)(f0 + q) * nh + jh) * NPART + 2 + i] = sc * t;
      }
    }
  }
  if (threadIdx.x < FG * NPART) {
    const int q = threadIdx.x / NPART, i = threadIdx.x - q * NPART;
    if (q < nfg && !(ep.mode == EPI_FINAL && i >= 2)) {
      const int f = f0 + q;
      if (fi[q].live) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += (double)red[w][threadIdx.x];
        ep.part[((size_t)f * nh + jh) * NPART + i] = t;
      }
    }
  }
}

}  // namespace shot
