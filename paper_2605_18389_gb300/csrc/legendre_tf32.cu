// Per-order Legendre contractions on the tensor cores in split TF32 (TF32x3).
//
// Same contractions as the other paths (App. C.1 semi-naive SHT; Sec. 3.2 h_l scaling):
//   analysis   C[i][c] = h_l sum_jh Pbar_lm(x_jh) X[jh][c]        (K = nodes jh)
//   synthesis  Y[jh][c] = sum_i Pbar_lm(x_jh) C[i][c]               (K = degrees i)
// Every FP32 operand v is split into two TF32 values: hi = v rounded to the nearest TF32
// (10 stored mantissa bits), lo = v - hi (exact in FP32, |lo| <= 2^-11 |v|) rounded to the
// nearest TF32 as well, so that both are exact TF32 values and the tensor core reads them
// as they are.  The product is accumulated in FP32 in tensor memory as
// A_hi B_hi + A_hi B_lo + A_lo B_hi (tcgen05.mma kind::tf32, K = 8 per instruction); the
// rounding of lo (<= 2^-22 |v|) and the dropped lo*lo term (<= 2^-22 |AB|) leave
// <= ~2^-20 relative error per product, of either sign, against ~2^-16 for BF16x3.  The
// HBM traffic is that of the BF16x3 path: the table is read once as FP32 (4 bytes an entry,
// as bf16 hi + lo) and split in shared memory.
//
// Both operands are K-major, 128-byte swizzled, 32 FP32 values (one swizzle row) per
// pipeline stage along K:
//   analysis   A = table tile [128 degree rows][32 nodes]        (TMA, the table [i][jh])
//              B = X^T [columns][32 nodes]                        (transposed from the FP32
//                                                                  spectra tile in smem)
//   synthesis  A = transposed table tile [128 nodes][32 degrees]  (TMA, a second copy of the
//                                                                  table laid out [blk][jh][i])
//              B = C^T [columns][32 degrees]                      (TMA, FP32 C^T written by
//                                                                  the analysis epilogue)
// kind::tf32 is used with K-major operands only, hence the transposed table copy.
// Warp roles: 0 TMA producer, 1 MMA issuer, 2-9 split (eight warps, two per SM sub-partition:
// the table tile alone is 16 KB per stage), 10-13 epilogue over a double-buffered accumulator
// (a warp reads the TMEM lane quadrant warp % 4).  Every mbarrier wait
// is bounded; on expiry the CTA records SHOT_ERR_TIMEOUT and still frees its tensor memory.
#include "tc_ptx.cuh"

namespace shot {
namespace {

constexpr int kSplitWarps = 8;                   // warps 2..9 (two per SM sub-partition)
constexpr int kSplitThreads = 32 * kSplitWarps;
constexpr int kT32Threads = 32 * (2 + kSplitWarps + 4);   // + TMA, MMA and four epilogue warps
constexpr int kTK = 32;                          // K per stage (one 128-byte row of FP32)
constexpr int kTTile = kBM * kTK * 4;            // 16 KB: 128 rows x 32 FP32
constexpr int kT32MaxStages = 4;
constexpr uint32_t kTf32Mask = 0xFFFFE000u;      // sign, exponent and 10 stored mantissa bits
constexpr uint32_t kTf32Half = 0x00001000u;      // half a unit in the last TF32 place

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

// Instruction descriptor, kind::tf32: TF32 A and B (format 2), FP32 accumulator, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// v rounded to the nearest TF32 value (ties away from zero): add half a TF32 unit to the
// magnitude bits, then clear the 13 low mantissa bits (a carry moves into the exponent, as it
// should).  Finite inputs below the FP32 maximum only (the operands here are far below it).
__device__ __forceinline__ float tf32_rn(float v) {
  return __uint_as_float((__float_as_uint(v) + kTf32Half) & kTf32Mask);
}
// hi/lo split of four values: hi = rn(v), lo = rn(v - hi)
__device__ __forceinline__ void tf32_split4(const float (&v)[4], float4& h, float4& l) {
  h = make_float4(tf32_rn(v[0]), tf32_rn(v[1]), tf32_rn(v[2]), tf32_rn(v[3]));
  l = make_float4(tf32_rn(v[0] - h.x), tf32_rn(v[1] - h.y), tf32_rn(v[2] - h.z), tf32_rn(v[3] - h.w));
}

// byte offset of FP32 element (row, k) in a K-major 128B-swizzled tile with 32-element rows
__device__ __forceinline__ uint32_t sw128_offset32(int row, int k) {
  const uint32_t chunk = (uint32_t)(k >> 2);   // 16-byte chunk (4 values) within the row
  return (uint32_t)(row >> 3) * 1024u + (uint32_t)(row & 7) * 128u + ((chunk ^ (uint32_t)(row & 7)) << 4) +
         (uint32_t)(k & 3) * 4u;
}

// Element-wise split of a tile (the swizzle does not matter): raw -> hi (in place), lo.
// Each thread loads kSplitBatch chunks before it stores any, so the loads overlap.
constexpr int kSplitBatch = 4;   // 16 KB / (256 threads x 16 B) = 4 chunks per thread
__device__ __forceinline__ void split_inplace(uint8_t* raw, uint8_t* lo, int nbytes, int pt) {
  for (int base = 0; base < nbytes; base += kSplitBatch * kSplitThreads * 16) {
    float4 v[kSplitBatch];
#pragma unroll
    for (int i = 0; i < kSplitBatch; ++i) {
      const int o = base + (pt + i * kSplitThreads) * 16;
      if (o < nbytes) v[i] = *reinterpret_cast<const float4*>(raw + o);
    }
#pragma unroll
    for (int i = 0; i < kSplitBatch; ++i) {
      const int o = base + (pt + i * kSplitThreads) * 16;
      if (o < nbytes) {
        const float w[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
        float4 h, l;
        tf32_split4(w, h, l);
        *reinterpret_cast<float4*>(raw + o) = h;
        *reinterpret_cast<float4*>(lo + o) = l;
      }
    }
  }
}

// X^T operand: xs[32 nodes][nmma] (row-major FP32, by TMA) -> hi/lo [c][32 nodes], K-major
// SW128.  One task = 4 consecutive nodes of one column (one 16-byte chunk); nodes past the
// block (jh0 + k >= nh) and columns past the fields are zero.
// Two tasks per thread are loaded before either is stored.
__device__ __forceinline__ void split_xt(const float* xs, int nmma, int ncols, int jh0, int nh, uint8_t* bh,
                                         uint8_t* bl, int pt) {
  const int ntask = nmma * (kTK / 4);
  for (int e0 = pt; e0 < ntask; e0 += 2 * kSplitThreads) {
    float v[2][4];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int e = e0 + b * kSplitThreads;
      const int c = e % nmma, k4 = (e / nmma) * 4;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        v[b][q] = (e < ntask && c < ncols && jh0 + k4 + q < nh) ? xs[(k4 + q) * nmma + c] : 0.f;
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int e = e0 + b * kSplitThreads;
      if (e < ntask) {
        const int c = e % nmma, k4 = (e / nmma) * 4;
        float4 h, l;
        tf32_split4(v[b], h, l);
        const uint32_t o = sw128_offset32(c, k4);
        *reinterpret_cast<float4*>(bh + o) = h;
        *reinterpret_cast<float4*>(bl + o) = l;
      }
    }
  }
}

// The X^T split with each thread's tasks fixed for the whole kernel (they are the same at every
// stage): the tile offsets of the four node values, the chunk's offset in the swizzled B tile and
// whether the column is a field column; a stage then only loads, splits and stores.
constexpr int kXtTasks = 4;   // nmma x 8 tasks <= 4 x 256 threads (nmma <= 128)
struct XtPlan {
  int c[kXtTasks];         // column (-1: no task)
  int k4[kXtTasks];        // first of the task's four nodes within the 32-node chunk
  uint32_t o[kXtTasks];    // byte offset of the 16-byte chunk in the hi (and lo) tile
  __device__ __forceinline__ void init(int nmma, int pt) {
    const int ntask = nmma * (kTK / 4);
#pragma unroll
    for (int i = 0; i < kXtTasks; ++i) {
      const int e = pt + i * kSplitThreads;
      c[i] = -1;
      k4[i] = 0;
      o[i] = 0;
      if (e < ntask) {
        c[i] = e % nmma;
        k4[i] = (e / nmma) * 4;
        o[i] = sw128_offset32(c[i], k4[i]);
      }
    }
  }
  __device__ __forceinline__ void run(const float* xs, int nmma, int ncols, int jh0, int nh, uint8_t* bh,
                                      uint8_t* bl) const {
    float v[kXtTasks][4];
#pragma unroll
    for (int i = 0; i < kXtTasks; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        v[i][q] = (c[i] >= 0 && c[i] < ncols && jh0 + k4[i] + q < nh) ? xs[(k4[i] + q) * nmma + c[i]] : 0.f;
#pragma unroll
    for (int i = 0; i < kXtTasks; ++i) {
      if (c[i] < 0) continue;
      float4 h, l;
      tf32_split4(v[i], h, l);
      *reinterpret_cast<float4*>(bh + o[i]) = h;
      *reinterpret_cast<float4*>(bl + o[i]) = l;
    }
  }
};

struct T32Args {
  const Tile* tiles;
  int ntiles;
  const int* M;
  const long long* row_off;
  int nh, ldc, ncols, nmma;
  const float* h;             // analysis: h_l, or nullptr
  float* ct;                  // analysis output: C^T [blk][nmma_cap][ldi] FP32
  float* cf;                  // analysis output (optional): C [row_off + i][ldc] FP32
  int nmma_cap, ldi;
  float* Y;                   // synthesis output [blk][jh][ldc]
  int* err;
};

// Persistent, warp-specialised TF32x3 Legendre GEMM (roles in the file header).  Stage s
// holds [A hi (TMA'd raw, split in place)][A lo][B hi][B lo][X raw (analysis)].
template <int kStages, bool ANA, bool BCAT>
__global__ void __launch_bounds__(kT32Threads, 1) k_legendre_tf32(const __grid_constant__ CUtensorMap ta,
                                                                  const __grid_constant__ CUtensorMap tb,
                                                                  T32Args a) {
  extern __shared__ uint8_t smraw[];
  __shared__ TcSmem ctl;
  uint8_t* base = align1k(smraw);
  const int nmma = a.nmma, nh = a.nh;
  const int bbytes = nmma * kTK * 4;   // one B tile (hi or lo); the analysis X tile has the same size
  const int sbytes = 2 * kTTile + (ANA ? 3 : 2) * bbytes;
  auto sA_hi = [&](int s) { return base + s * sbytes; };
  auto sA_lo = [&](int s) { return base + s * sbytes + kTTile; };
  auto sB_hi = [&](int s) { return base + s * sbytes + 2 * kTTile; };
  auto sB_lo = [&](int s) { return base + s * sbytes + 2 * kTTile + bbytes; };
  auto sX = [&](int s) { return base + s * sbytes + 2 * kTTile + 2 * bbytes; };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // BCAT (2 nmma <= 256): B hi and B lo are adjacent in shared memory and form one operand
  // of N = 2 nmma, so A_hi [B_hi | B_lo] and A_lo B_hi are two MMAs per K step instead of
  // three (one fewer read of the A tile); the accumulator then holds two halves that the
  // epilogue adds.
  constexpr bool bcat = BCAT;
  const int nacc = bcat ? 2 * nmma : nmma;
  const uint32_t ncols_alloc = tmem_cols_for(nacc);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&ctl.fullA[s], 1);
      mbar_init(&ctl.fullB[s], kSplitThreads);
      mbar_init(&ctl.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl.tfull[b], 1);
      mbar_init(&ctl.tempty[b], 128);
    }
    ctl.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&ctl.tmem, 2 * ncols_alloc);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = ctl.tmem;
  volatile int* abort = &ctl.abort;
  auto nkb_of = [&](int blk) { return ANA ? (nh + kTK - 1) / kTK : (a.M[blk] + kTK - 1) / kTK; };

  if (warp == 0) {
    if (lane == 0) {  // TMA producer, runs ahead across tiles
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        const Tile tl = a.tiles[t];
        const int nkb = nkb_of(tl.blk);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % kStages, n = it / kStages;
          if (it >= kStages && !(ok = mbar_wait(&ctl.empty[s], (n - 1) & 1, abort))) break;
          mbar_arrive_expect_tx(&ctl.fullA[s], kTTile + bbytes);
          if (ANA) {   // table rows i of the tile x nodes of this K-chunk; spectra rows = nodes
            tma_load_2d(sA_hi(s), &ta, &ctl.fullA[s], kb * kTK, (int)(a.row_off[tl.blk] + tl.r0));
            tma_load_2d(sX(s), &tb, &ctl.fullA[s], 0, tl.blk * nh + kb * kTK);
          } else {     // transposed table: nodes of the tile x degrees of this K-chunk; C^T rows = columns
            tma_load_2d(sA_hi(s), &ta, &ctl.fullA[s], kb * kTK, tl.blk * nh + tl.r0);
            tma_load_2d(sB_hi(s), &tb, &ctl.fullA[s], kb * kTK, tl.blk * a.nmma_cap);
          }
        }
      }
      // let this CTA's copies land before it can exit
      for (int k = it > kStages ? it - kStages : 0; k < it; ++k)
        mbar_drain(&ctl.fullA[k % kStages], (k / kStages) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer: every operand it reads was written by the split warps
      const uint32_t idesc = idesc_tf32(kBM, nmma), idesc2 = idesc_tf32(kBM, nacc);
      int it = 0, lt = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++lt) {
        const Tile tl = a.tiles[t];
        const int nkb = nkb_of(tl.blk);
        const int acc = lt & 1, u = lt >> 1;
        if (lt >= 2 && !(ok = mbar_wait(&ctl.tempty[acc], (u - 1) & 1, abort))) break;
        tc_fence_after();
        const uint32_t d = taddr + (uint32_t)(acc * ncols_alloc);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % kStages, n = it / kStages;
          if (!(ok = mbar_wait(&ctl.fullB[s], n & 1, abort))) break;
          tc_fence_after();
          const uint32_t ah = smem_u32(sA_hi(s)), al = smem_u32(sA_lo(s));
          const uint32_t bh = smem_u32(sB_hi(s)), bl = smem_u32(sB_lo(s));
#pragma unroll
          for (int k = 0; k < kTK / 8; ++k) {   // 8 TF32 = 32 bytes per instruction
            const uint32_t off = k * 32;
            const uint64_t a_h = desc_sw128_kmajor(ah + off), a_l = desc_sw128_kmajor(al + off);
            const uint64_t b_h = desc_sw128_kmajor(bh + off), b_l = desc_sw128_kmajor(bl + off);
            if constexpr (BCAT) {   // b_h spans B_hi and B_lo (2 nmma rows)
              umma_tf32(d, a_h, b_h, idesc2, (kb | k) != 0);
              umma_tf32(d, a_l, b_h, idesc, 1);
            } else {
              umma_tf32(d, a_h, b_h, idesc, (kb | k) != 0);
              umma_tf32(d, a_h, b_l, idesc, 1);
              umma_tf32(d, a_l, b_h, idesc, 1);
            }
          }
          umma_commit(&ctl.empty[s]);
        }
        if (!ok) break;
        umma_commit(&ctl.tfull[acc]);
      }
    }
  } else if (warp < 2 + kSplitWarps) {
    // split warps: table tile in place -> hi, lo; analysis: X -> X^T hi/lo; synthesis: C^T in place
    const int pt = threadIdx.x - 64;
    const bool pre = ANA && nmma * (kTK / 4) <= kXtTasks * kSplitThreads;
    XtPlan xp;
    xp.init(pre ? nmma : 0, pt);
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
      const Tile tl = a.tiles[t];
      const int nkb = nkb_of(tl.blk);
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = it % kStages, n = it / kStages;
        if (!(ok = mbar_wait(&ctl.fullA[s], n & 1, abort))) break;
        split_inplace(sA_hi(s), sA_lo(s), kTTile, pt);
        if (ANA && pre)
          xp.run(reinterpret_cast<const float*>(sX(s)), nmma, a.ncols, kb * kTK, nh, sB_hi(s), sB_lo(s));
        else if (ANA)
          split_xt(reinterpret_cast<const float*>(sX(s)), nmma, a.ncols, kb * kTK, nh, sB_hi(s), sB_lo(s), pt);
        else
          split_inplace(sB_hi(s), sB_lo(s), bbytes, pt);
        fence_async_smem();
        mbar_arrive(&ctl.fullB[s]);
      }
    }
  } else {
    // epilogue: drain the accumulator of every tile of this CTA (warp 8 + q reads lanes 32q..)
    const int q = warp & 3;   // a warp reaches only TMEM lanes 32 (warp % 4) ..
    int lt = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++lt) {
      const Tile tl = a.tiles[t];
      const int acc = lt & 1, u = lt >> 1;
      if (!mbar_wait_warp(&ctl.tfull[acc], u & 1, abort)) break;
      tc_fence_after();
      const uint32_t d = taddr + (uint32_t)(acc * ncols_alloc) + ((uint32_t)(q * 32) << 16);
      const int row = tl.r0 + q * 32 + lane;
      if (ANA) {
        const int blk = tl.blk, m = blk >> 1, p = blk & 1;
        const int M = a.M[blk];
        const long long ro = a.row_off[blk];
        const float hl = (a.h && row < M) ? a.h[m + p + 2 * row] : 1.f;
        for (int c0 = 0; c0 < nmma; c0 += 16) {
          float v[16];
          tmem_ld16(d + (uint32_t)c0, v);
          if constexpr (BCAT) {   // + A_hi B_lo, accumulated in the second half
            float w[16];
            tmem_ld16(d + (uint32_t)(nmma + c0), w);
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] += w[e];
          }
          if (row < M) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int c = c0 + e;
              if (c < a.ncols) {
                const float val = v[e] * hl;
                a.ct[((size_t)blk * a.nmma_cap + c) * a.ldi + row] = val;
                if (a.cf) a.cf[(size_t)(ro + row) * a.ldc + c] = val;
              }
            }
          }
        }
      } else {
        float* yrow = a.Y + ((size_t)tl.blk * nh + row) * a.ldc;
        for (int c0 = 0; c0 < nmma; c0 += 16) {
          float v[16];
          tmem_ld16(d + (uint32_t)c0, v);
          if constexpr (BCAT) {   // + A_hi B_lo, accumulated in the second half
            float w[16];
            tmem_ld16(d + (uint32_t)(nmma + c0), w);
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] += w[e];
          }
          if (row < nh) {
            if (c0 + 16 <= a.ncols) {
#pragma unroll
              for (int e = 0; e < 16; e += 4)
                *reinterpret_cast<float4*>(yrow + c0 + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
            } else {
#pragma unroll
              for (int e = 0; e < 16; ++e)
                if (c0 + e < a.ncols) yrow[c0 + e] = v[e];
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&ctl.tempty[acc]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(taddr, 2 * ncols_alloc);
  }
  if (threadIdx.x == 0 && ctl.abort) atomicExch(a.err, SHOT_ERR_TIMEOUT);
}

// FP32 coefficients C[row_off + i][ldc] -> C^T[blk][nmma_cap][ldi] (synthesis-only input)
__global__ void k_c_to_ct32(const int* __restrict__ Mrows, const long long* __restrict__ row_off,
                            const float* __restrict__ C, int ldc, int ncols, float* __restrict__ ct, int nmma_cap,
                            int ldi) {
  const int blk = blockIdx.x;
  const int M = Mrows[blk];
  const long long ro = row_off[blk];
  for (int idx = threadIdx.x; idx < M * ncols; idx += blockDim.x) {
    const int c = idx / M, i = idx - c * M;
    ct[((size_t)blk * nmma_cap + c) * ldi + i] = C[(size_t)(ro + i) * ldc + c];
  }
}

size_t tf32_smem_bytes(int nmma, bool ana, int stages) {
  return 1024 + (size_t)stages * (2 * kTTile + (ana ? 3 : 2) * (size_t)nmma * kTK * 4);
}

}  // namespace

int tf32_nmma(int nf) { return (2 * nf + 15) / 16 * 16; }

int launch_legendre_tf32(const Grid& g, int nf, const float* X, float* Cf, float* Y, int ldc, bool ana, bool syn,
                         bool apply_h, cudaStream_t st) {
  const Workspace& w = g.ws;
  const int nmma = tf32_nmma(nf);
  if (nmma > 256 || nmma > w.nmma_cap || !w.ct32 || !g.tab || !g.tabT) {
    set_error("TF32X3 path supports at most 128 fields per call");
    return SHOT_ERR_UNSUPPORTED;
  }
  int rc;
  // deepest pipeline (<= 4 stages) whose tiles fit in one CTA's shared memory, with 2 KB
  // left for the static control block
  auto pick = [&](bool a_) {
    int s = kT32MaxStages;
    while (s > 1 && tf32_smem_bytes(nmma, a_, s) + 2048 > 227 * 1024) --s;
    return s;
  };
  auto launch = [&](bool a_, const CUtensorMap& ma, const CUtensorMap& mb, const T32Args& args, int ntiles) -> int {
    const int stages = pick(a_);
    const size_t smem = tf32_smem_bytes(nmma, a_, stages);
    const bool bc = 2 * nmma <= 256;
    auto kern = bc ? (a_ ? (stages == 4 ? k_legendre_tf32<4, true, true> : stages == 3 ? k_legendre_tf32<3, true, true>
                            : stages == 2 ? k_legendre_tf32<2, true, true> : k_legendre_tf32<1, true, true>)
                         : (stages == 4 ? k_legendre_tf32<4, false, true> : stages == 3 ? k_legendre_tf32<3, false, true>
                            : stages == 2 ? k_legendre_tf32<2, false, true> : k_legendre_tf32<1, false, true>))
                   : (a_ ? (stages == 4 ? k_legendre_tf32<4, true, false> : stages == 3 ? k_legendre_tf32<3, true, false>
                            : stages == 2 ? k_legendre_tf32<2, true, false> : k_legendre_tf32<1, true, false>)
                         : (stages == 4 ? k_legendre_tf32<4, false, false> : stages == 3 ? k_legendre_tf32<3, false, false>
                            : stages == 2 ? k_legendre_tf32<2, false, false> : k_legendre_tf32<1, false, false>));
    SHOT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = ntiles < g.num_sms ? ntiles : g.num_sms;
    ProfScope prof(a_ ? PK_ANALYSIS : PK_SYNTHESIS, st);
    count_launch();
    kern<<<grid, kT32Threads, smem, st>>>(ma, mb, args);
    SHOT_CUDA(cudaGetLastError());
    return SHOT_OK;
  };
  if (ana) {
    CUtensorMap ma, mx;
    if ((rc = make_map_f32(&ma, g.tab, g.nh, g.rows_total, g.ldt, kTK, kBM, true))) return rc;
    if ((rc = make_map_f32(&mx, X, ldc, (uint64_t)g.nblk * g.nh, ldc, nmma, kTK))) return rc;
    const T32Args args{g.tiles_ana, g.ntiles_ana, g.M_d, g.row_off_d, g.nh, ldc, 2 * nf, nmma,
                       apply_h ? g.h_d : nullptr, w.ct32, Cf, w.nmma_cap, g.ldi, nullptr, w.dev_int + 4};
    if ((rc = launch(true, ma, mx, args, g.ntiles_ana))) return rc;
  }
  if (syn) {
    CUtensorMap ma, mb;
    if ((rc = make_map_f32(&ma, g.tabT, g.ldi, (uint64_t)g.nblk * g.nh, g.ldi, kTK, kBM, true))) return rc;
    if ((rc = make_map_f32(&mb, w.ct32, g.ldi, (uint64_t)g.nblk * w.nmma_cap, g.ldi, kTK, nmma, true))) return rc;
    const T32Args args{g.tiles_syn, g.ntiles_syn, g.M_d, g.row_off_d, g.nh, ldc, 2 * nf, nmma,
                       nullptr, nullptr, nullptr, w.nmma_cap, g.ldi, Y, w.dev_int + 4};
    if ((rc = launch(false, ma, mb, args, g.ntiles_syn))) return rc;
  }
  return SHOT_OK;
}

int launch_c_to_ct32(const Grid& g, int nf, const float* C, int ldc, cudaStream_t st) {
  const Workspace& w = g.ws;
  count_launch();
  k_c_to_ct32<<<g.nblk, 256, 0, st>>>(g.M_d, g.row_off_d, C, ldc, 2 * nf, w.ct32, w.nmma_cap, g.ldi);
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

}  // namespace shot
