// Per-order Legendre contractions on the 5th-generation tensor cores (tcgen05), BF16x3.
//
// Same contractions as the FP32 path (App. C.1 semi-naive SHT; Sec. 3.2 h_l scaling):
//   analysis   C[i][c] = h_l sum_jh Pbar_lm(x_jh) X[jh][c]        (K = nodes jh)
//   synthesis  Y[jh][c] = sum_i Pbar_lm(x_jh) C[i][c]               (K = degrees i)
// Both operands are split into bf16 hi + lo (v = hi + lo, |lo| <= 2^-9 |v|) and the
// product is accumulated in FP32 in tensor memory as A_hi B_hi + A_hi B_lo + A_lo B_hi
// (the lo*lo term, ~2^-18 relative, is dropped).  Operands are K-major, 128-byte
// swizzled in shared memory: the table tiles come by TMA (the synthesis reads a
// transposed copy of the table so that its A operand is K-major as well); the analysis
// B operand (the FP32 ring spectra X) is split and transposed by four producer warps.
// One elected thread issues tcgen05.mma (M = 128, N = 2*nfields rounded to 16, K = 16);
// tcgen05.commit releases the pipeline stages; four warps read the accumulator with
// tcgen05.ld for the epilogue.  Every mbarrier wait is bounded; on expiry the CTA
// records SHOT_ERR_TIMEOUT in a device flag and still releases its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "shot_internal.cuh"

namespace shot {
namespace {

constexpr int kTcThreads = 256;
constexpr int kBM = 128;          // MMA M
constexpr int kBK = 64;           // K elements per pipeline stage (one 128-byte swizzle row)
constexpr int kMaxStages = 4;
constexpr int kStagesAna = 3;   // one CTA per SM (table + X + B tiles)
constexpr int kStagesSyn = 2;   // two CTAs per SM
constexpr uint32_t kSpinLimit = 1u << 24;
constexpr int kATileBytes = kBM * kBK * 2;   // 16 KB

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait that ignores the abort flag: used to let this CTA's own TMA copies land
// before it exits.
__device__ __forceinline__ void mbar_drain(uint64_t* b, uint32_t parity) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_test(b, parity)) return;
    if ((it & 255u) == 255u) __nanosleep(32);
  }
}

// Warp-uniform bounded wait: lane 0 waits, the verdict is broadcast to the warp (the
// epilogue's tcgen05.ld is .sync.aligned and must be reached by all lanes or none).
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* b, uint32_t parity, volatile int* abort);

// Bounded wait for the phase of the given parity.  Returns false (and raises the CTA's
// abort flag) when the limit expires or another role already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_test(b, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*abort) return false;
      __nanosleep(32);
    }
  }
  *abort = 1;
  return false;
}

__device__ __forceinline__ bool mbar_wait_warp(uint64_t* b, uint32_t parity, volatile int* abort) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(b, parity, abort) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  return ok != 0;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 TMEM lanes x 16 consecutive 32-bit columns into 16 registers per thread
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1 KB apart.
__device__ __forceinline__ uint64_t desc_sw128_kmajor(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: BF16 A and B, FP32 accumulator, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t tmem_cols_for(int n) {
  uint32_t c = 32;
  while ((int)c < n) c <<= 1;
  return c;
}

// byte offset of element (row, k) in a K-major 128B-swizzled tile with 64-element rows
__device__ __forceinline__ uint32_t sw128_offset(int row, int k) {
  const uint32_t chunk = (uint32_t)(k >> 3);   // 16-byte chunk within the 128-byte row
  return (uint32_t)(row >> 3) * 1024u + (uint32_t)(row & 7) * 128u + ((chunk ^ (uint32_t)(row & 7)) << 4) +
         (uint32_t)(k & 7) * 2u;
}

struct TcSmem {
  uint64_t fullA[kMaxStages];
  uint64_t fullB[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t done;
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ uint8_t* align1k(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

struct AnaArgs {
  const Tile* tiles;
  const int* M;
  const long long* row_off;
  int nh;
  const float* X;      // [blk][jh][ldc] FP32
  int ldc, ncols, nmma;
  const float* h;      // h_l or nullptr
  __nv_bfloat16* ct_hi;   // [blk][nmma_cap][ldi]
  __nv_bfloat16* ct_lo;
  int nmma_cap, ldi;
  float* cf;           // optional FP32 [row_off + i][ldc]
  int* err;
};

template <int kStages>
__global__ void __launch_bounds__(kTcThreads, 1) k_legendre_ana_tc(const __grid_constant__ CUtensorMap tm_hi,
                                                                   const __grid_constant__ CUtensorMap tm_lo,
                                                                   const __grid_constant__ CUtensorMap tm_x,
                                                                   AnaArgs a) {
  extern __shared__ uint8_t smraw[];
  __shared__ TcSmem ctl;
  uint8_t* base = align1k(smraw);
  const int bbytes = a.nmma * kBK * 2;
  uint8_t* sA_hi = base;
  uint8_t* sA_lo = sA_hi + kStages * kATileBytes;
  uint8_t* sB_hi = sA_lo + kStages * kATileBytes;
  uint8_t* sB_lo = sB_hi + kStages * bbytes;
  const int xbytes = a.nmma * kBK * 4;     // FP32 X tile [64 nodes][nmma columns]
  uint8_t* sX = sB_lo + kStages * bbytes;

  const Tile tl = a.tiles[blockIdx.x];
  const int blk = tl.blk, i0 = tl.r0;
  const int m = blk >> 1, p = blk & 1;
  const int M = a.M[blk];
  const long long ro = a.row_off[blk];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = (a.nh + kBK - 1) / kBK;
  const uint32_t ncols_alloc = tmem_cols_for(a.nmma);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&ctl.fullA[s], 1);
      mbar_init(&ctl.fullB[s], 128);
      mbar_init(&ctl.empty[s], 1);
    }
    mbar_init(&ctl.done, 1);
    ctl.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&ctl.tmem, ncols_alloc);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = ctl.tmem;
  volatile int* abort = &ctl.abort;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer of the table tiles (A operand)
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % kStages, n = kb / kStages;
        if (kb >= kStages && !mbar_wait(&ctl.empty[s], (n - 1) & 1, abort)) break;
        mbar_arrive_expect_tx(&ctl.fullA[s], 2 * kATileBytes + xbytes);
        tma_load_2d(sA_hi + s * kATileBytes, &tm_hi, &ctl.fullA[s], kb * kBK, (int)(ro + i0));
        tma_load_2d(sA_lo + s * kATileBytes, &tm_lo, &ctl.fullA[s], kb * kBK, (int)(ro + i0));
        tma_load_2d(sX + s * xbytes, &tm_x, &ctl.fullA[s], 0, blk * a.nh + kb * kBK);
        issued = kb + 1;
      }
      for (int kb = issued > kStages ? issued - kStages : 0; kb < issued; ++kb)
        mbar_drain(&ctl.fullA[kb % kStages], (kb / kStages) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = idesc_bf16(kBM, a.nmma);
      bool ok = true;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb % kStages, n = kb / kStages;
        ok = mbar_wait(&ctl.fullA[s], n & 1, abort) && mbar_wait(&ctl.fullB[s], n & 1, abort);
        if (!ok) break;
        tc_fence_after();
        const uint32_t ah = smem_u32(sA_hi + s * kATileBytes), al = smem_u32(sA_lo + s * kATileBytes);
        const uint32_t bh = smem_u32(sB_hi + s * bbytes), bl = smem_u32(sB_lo + s * bbytes);
#pragma unroll
        for (int k = 0; k < kBK / 16; ++k) {
          const uint32_t off = k * 32;
          umma_bf16(taddr, desc_sw128_kmajor(ah + off), desc_sw128_kmajor(bh + off), idesc, (kb | k) != 0);
          umma_bf16(taddr, desc_sw128_kmajor(ah + off), desc_sw128_kmajor(bl + off), idesc, 1);
          umma_bf16(taddr, desc_sw128_kmajor(al + off), desc_sw128_kmajor(bh + off), idesc, 1);
        }
        umma_commit(&ctl.empty[s]);
      }
      umma_commit(&ctl.done);
    }
  } else if (warp >= 4) {
    // producers of the B operand: the FP32 tile X[jh][c] (brought by TMA with the table
    // tiles) -> bf16 hi/lo, K-major [c][jh], 128-byte swizzled
    const int pt = threadIdx.x - 128;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % kStages, n = kb / kStages;
      if (!mbar_wait(&ctl.fullA[s], n & 1, abort)) break;
      const float* xs = reinterpret_cast<const float*>(sX + s * xbytes);
      uint8_t* bh = sB_hi + s * bbytes;
      uint8_t* bl = sB_lo + s * bbytes;
      // one task = 8 consecutive nodes of one column -> one 16-byte swizzle chunk of hi
      // and of lo; rows beyond the block's nodes (or columns beyond the fields) are zero
      for (int e = pt; e < 8 * a.nmma; e += 128) {
        const int r8 = e / a.nmma, c = e - r8 * a.nmma;
        const int jh0 = kb * kBK + r8 * 8;
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
          float v0 = xs[(r8 * 8 + t) * a.nmma + c];
          float v1 = xs[(r8 * 8 + t + 1) * a.nmma + c];
          if (c >= a.ncols || jh0 + t >= a.nh) v0 = 0.f;
          if (c >= a.ncols || jh0 + t + 1 >= a.nh) v1 = 0.f;
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
          const float2 hf = __bfloat1622float2(h2);
          const __nv_bfloat162 l2 = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
          hw[t / 2] = *reinterpret_cast<const uint32_t*>(&h2);
          lw[t / 2] = *reinterpret_cast<const uint32_t*>(&l2);
        }
        const uint32_t o = sw128_offset(c, r8 * 8);
        *reinterpret_cast<uint4*>(bh + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(bl + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
      fence_async_smem();
      mbar_arrive(&ctl.fullB[s]);
    }
    // epilogue: accumulator rows -> h_l scaling -> bf16 hi/lo C^T (and optional FP32 C)
    const int q = warp - 4;   // TMEM lane quadrant
    if (mbar_wait_warp(&ctl.done, 0, abort)) {
      tc_fence_after();
      const int row = q * 32 + lane;
      const int i = i0 + row;
      const float hl = (a.h && i < M) ? a.h[m + p + 2 * i] : 1.f;
      for (int c0 = 0; c0 < a.nmma; c0 += 16) {
        float v[16];
        tmem_ld16(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
        if (i < M) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int c = c0 + t;
            if (c < a.ncols) {
              const float val = v[t] * hl;
              const __nv_bfloat16 hi = __float2bfloat16_rn(val);
              const __nv_bfloat16 lo = __float2bfloat16_rn(val - __bfloat162float(hi));
              const size_t o = ((size_t)blk * a.nmma_cap + c) * a.ldi + i;
              a.ct_hi[o] = hi;
              a.ct_lo[o] = lo;
              if (a.cf) a.cf[(size_t)(ro + i) * a.ldc + c] = val;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(taddr, ncols_alloc);
  }
  if (threadIdx.x == 0 && ctl.abort) atomicExch(a.err, SHOT_ERR_TIMEOUT);
}

struct SynArgs {
  const Tile* tiles;
  const int* M;
  int nh;
  int nmma, nmma_cap, ncols, ldc;
  float* Y;   // [blk][jh][ldc]
  int* err;
};

template <int kStages>
__global__ void __launch_bounds__(kTcThreads, 1) k_legendre_syn_tc(const __grid_constant__ CUtensorMap ta_hi,
                                                                   const __grid_constant__ CUtensorMap ta_lo,
                                                                   const __grid_constant__ CUtensorMap tb_hi,
                                                                   const __grid_constant__ CUtensorMap tb_lo,
                                                                   SynArgs a) {
  extern __shared__ uint8_t smraw[];
  __shared__ TcSmem ctl;
  uint8_t* base = align1k(smraw);
  const int bbytes = a.nmma * kBK * 2;
  uint8_t* sA_hi = base;
  uint8_t* sA_lo = sA_hi + kStages * kATileBytes;
  uint8_t* sB_hi = sA_lo + kStages * kATileBytes;
  uint8_t* sB_lo = sB_hi + kStages * bbytes;

  const Tile tl = a.tiles[blockIdx.x];
  const int blk = tl.blk, j0 = tl.r0;
  const int M = a.M[blk];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = (M + kBK - 1) / kBK;
  const uint32_t ncols_alloc = tmem_cols_for(a.nmma);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&ctl.fullA[s], 1);
      mbar_init(&ctl.fullB[s], 1);
      mbar_init(&ctl.empty[s], 1);
    }
    mbar_init(&ctl.done, 1);
    ctl.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&ctl.tmem, ncols_alloc);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = ctl.tmem;
  volatile int* abort = &ctl.abort;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % kStages, n = kb / kStages;
        if (kb >= kStages && !mbar_wait(&ctl.empty[s], (n - 1) & 1, abort)) break;
        mbar_arrive_expect_tx(&ctl.fullA[s], 2 * kATileBytes + 2 * bbytes);
        tma_load_2d(sA_hi + s * kATileBytes, &ta_hi, &ctl.fullA[s], kb * kBK, blk * a.nh + j0);
        tma_load_2d(sA_lo + s * kATileBytes, &ta_lo, &ctl.fullA[s], kb * kBK, blk * a.nh + j0);
        tma_load_2d(sB_hi + s * bbytes, &tb_hi, &ctl.fullA[s], kb * kBK, blk * a.nmma_cap);
        tma_load_2d(sB_lo + s * bbytes, &tb_lo, &ctl.fullA[s], kb * kBK, blk * a.nmma_cap);
        issued = kb + 1;
      }
      for (int kb = issued > kStages ? issued - kStages : 0; kb < issued; ++kb)
        mbar_drain(&ctl.fullA[kb % kStages], (kb / kStages) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kBM, a.nmma);
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % kStages, n = kb / kStages;
        if (!mbar_wait(&ctl.fullA[s], n & 1, abort)) break;
        tc_fence_after();
        const uint32_t ah = smem_u32(sA_hi + s * kATileBytes), al = smem_u32(sA_lo + s * kATileBytes);
        const uint32_t bh = smem_u32(sB_hi + s * bbytes), bl = smem_u32(sB_lo + s * bbytes);
#pragma unroll
        for (int k = 0; k < kBK / 16; ++k) {
          const uint32_t off = k * 32;
          umma_bf16(taddr, desc_sw128_kmajor(ah + off), desc_sw128_kmajor(bh + off), idesc, (kb | k) != 0);
          umma_bf16(taddr, desc_sw128_kmajor(ah + off), desc_sw128_kmajor(bl + off), idesc, 1);
          umma_bf16(taddr, desc_sw128_kmajor(al + off), desc_sw128_kmajor(bh + off), idesc, 1);
        }
        umma_commit(&ctl.empty[s]);
      }
      umma_commit(&ctl.done);
    }
  } else if (warp >= 4) {
    const int q = warp - 4;
    if (mbar_wait_warp(&ctl.done, 0, abort)) {
      tc_fence_after();
      const int jh = j0 + q * 32 + lane;
      float* yrow = a.Y + ((size_t)blk * a.nh + jh) * a.ldc;
      for (int c0 = 0; c0 < a.nmma; c0 += 16) {
        float v[16];
        tmem_ld16(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
        if (jh < a.nh) {
          if (c0 + 16 <= a.ncols) {
#pragma unroll
            for (int t = 0; t < 16; t += 4)
              *reinterpret_cast<float4*>(yrow + c0 + t) = make_float4(v[t], v[t + 1], v[t + 2], v[t + 3]);
          } else {
#pragma unroll
            for (int t = 0; t < 16; ++t)
              if (c0 + t < a.ncols) yrow[c0 + t] = v[t];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(taddr, ncols_alloc);
  }
  if (threadIdx.x == 0 && ctl.abort) atomicExch(a.err, SHOT_ERR_TIMEOUT);
}

// FP32 coefficients C[row_off + i][ldc] -> bf16 hi/lo C^T[blk][nmma_cap][ldi] (synthesis input)
__global__ void k_c_to_ct(int nblk, const int* __restrict__ Mrows, const long long* __restrict__ row_off,
                          const float* __restrict__ C, int ldc, int ncols, __nv_bfloat16* __restrict__ hi,
                          __nv_bfloat16* __restrict__ lo, int nmma_cap, int ldi) {
  const int blk = blockIdx.x;
  const int M = Mrows[blk];
  const long long ro = row_off[blk];
  for (int idx = threadIdx.x; idx < M * ncols; idx += blockDim.x) {
    const int c = idx / M, i = idx - c * M;
    const float v = C[(size_t)(ro + i) * ldc + c];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const size_t o = ((size_t)blk * nmma_cap + c) * ldi + i;
    hi[o] = h;
    lo[o] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D bf16 tensor [rows][inner] with row stride ld (elements), box {64, box_rows}, 128B swizzle
int make_map(CUtensorMap* map, const void* ptr, uint64_t inner, uint64_t rows, uint64_t ld, uint32_t box_rows) {
  auto enc = get_encode();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return SHOT_ERR_CUDA;
  }
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed");
    return SHOT_ERR_CUDA;
  }
  return SHOT_OK;
}

// 2-D FP32 tensor [rows][inner] (row stride ld elements), box {box_inner, box_rows}, no swizzle
int make_map_f32(CUtensorMap* map, const void* ptr, uint64_t inner, uint64_t rows, uint64_t ld, uint32_t box_inner,
                 uint32_t box_rows) {
  auto enc = get_encode();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return SHOT_ERR_CUDA;
  }
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {ld * 4};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (FP32) failed");
    return SHOT_ERR_CUDA;
  }
  return SHOT_OK;
}

size_t tc_smem_bytes(int nmma, bool with_x, int stages) {
  return 1024 + (size_t)stages * (2 * kATileBytes + 2 * nmma * kBK * 2 + (with_x ? nmma * kBK * 4 : 0));
}

}  // namespace

int tc_nmma(int nf) { return (2 * nf + 15) / 16 * 16; }

int tc_supported_fields(int nf) { return tc_nmma(nf) <= 256; }

int launch_legendre_tc(const Grid& g, int nf, const float* X, float* Cf, float* Y, int ldc, bool ana, bool syn,
                       bool apply_h, cudaStream_t st) {
  const Workspace& w = g.ws;
  const int nmma = tc_nmma(nf);
  if (nmma > 256 || nmma > w.nmma_cap) {
    set_error("BF16X3 path supports at most 128 fields per call");
    return SHOT_ERR_UNSUPPORTED;
  }
  int rc;
  if (ana) {
    // deepest pipeline (<= 3 stages) whose tiles fit in one CTA's shared memory
    int stages = kStagesAna;
    while (stages > 1 && tc_smem_bytes(nmma, true, stages) > 227 * 1024) --stages;
    const size_t smem = tc_smem_bytes(nmma, true, stages);
    CUtensorMap mh, ml, mx;
    if ((rc = make_map(&mh, g.tab_hi, g.nh, g.rows_total, g.ldt, kBM))) return rc;
    if ((rc = make_map(&ml, g.tab_lo, g.nh, g.rows_total, g.ldt, kBM))) return rc;
    if ((rc = make_map_f32(&mx, X, ldc, (uint64_t)g.nblk * g.nh, ldc, nmma, kBK))) return rc;
    AnaArgs a{g.tiles_ana, g.M_d, g.row_off_d, g.nh, X, ldc, 2 * nf, nmma, apply_h ? g.h_d : nullptr,
              w.ct_hi, w.ct_lo, w.nmma_cap, g.ldi, Cf, w.dev_int + 4};
    auto kern = stages == 3 ? k_legendre_ana_tc<3> : stages == 2 ? k_legendre_ana_tc<2> : k_legendre_ana_tc<1>;
    SHOT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope prof(PK_ANALYSIS, st);
    count_launch();
    kern<<<g.ntiles_ana, kTcThreads, smem, st>>>(mh, ml, mx, a);
    SHOT_CUDA(cudaGetLastError());
  }
  if (syn) {
    const size_t smem = tc_smem_bytes(nmma, false, kStagesSyn);
    CUtensorMap ah, al, bh, bl;
    if ((rc = make_map(&ah, g.tabT_hi, g.ldi, (uint64_t)g.nblk * g.nh, g.ldi, kBM))) return rc;
    if ((rc = make_map(&al, g.tabT_lo, g.ldi, (uint64_t)g.nblk * g.nh, g.ldi, kBM))) return rc;
    if ((rc = make_map(&bh, w.ct_hi, g.ldi, (uint64_t)g.nblk * w.nmma_cap, g.ldi, nmma))) return rc;
    if ((rc = make_map(&bl, w.ct_lo, g.ldi, (uint64_t)g.nblk * w.nmma_cap, g.ldi, nmma))) return rc;
    SynArgs a{g.tiles_syn, g.M_d, g.nh, nmma, w.nmma_cap, 2 * nf, ldc, Y, w.dev_int + 4};
    SHOT_CUDA(cudaFuncSetAttribute(k_legendre_syn_tc<kStagesSyn>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    ProfScope prof(PK_SYNTHESIS, st);
    count_launch();
    k_legendre_syn_tc<kStagesSyn><<<g.ntiles_syn, kTcThreads, smem, st>>>(ah, al, bh, bl, a);
    SHOT_CUDA(cudaGetLastError());
  }
  return SHOT_OK;
}

int launch_c_to_ct(const Grid& g, int nf, const float* C, int ldc, cudaStream_t st) {
  const Workspace& w = g.ws;
  count_launch();
  k_c_to_ct<<<g.nblk, 256, 0, st>>>(g.nblk, g.M_d, g.row_off_d, C, ldc, 2 * nf, w.ct_hi, w.ct_lo, w.nmma_cap, g.ldi);
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

}  // namespace shot
