// Per-order Legendre contractions on the 5th-generation tensor cores (tcgen05), BF16x3.
//
// Same contractions as the FP32 path (App. C.1 semi-naive SHT; Sec. 3.2 h_l scaling):
//   analysis   C[i][c] = h_l sum_jh Pbar_lm(x_jh) X[jh][c]        (K = nodes jh)
//   synthesis  Y[jh][c] = sum_i Pbar_lm(x_jh) C[i][c]               (K = degrees i)
// Both operands are split into bf16 hi + lo (v = hi + lo, |lo| <= 2^-9 |v|) and the
// product is accumulated in FP32 in tensor memory as A_hi B_hi + A_hi B_lo + A_lo B_hi
// (the lo*lo term, ~2^-18 relative, is dropped).  Operands are 128-byte swizzled in
// shared memory.  The table [i][jh] (jh contiguous) comes by TMA and serves both
// contractions: K-major A of the analysis (K = jh), MN-major A of the synthesis (M = jh).
// The analysis B operand (the FP32 ring spectra X, [jh][c]) is split into hi/lo by two
// warps in the MN-major layout it already has; the
// synthesis B operand is C^T (K-major, bf16 hi/lo, written by the analysis epilogue).
// One elected thread issues tcgen05.mma (M = 128, N = 2*nfields rounded to 16, K = 16);
// tcgen05.commit releases the pipeline stages; four warps read the accumulator with
// tcgen05.ld for the epilogue.  Every mbarrier wait is bounded; on expiry the CTA
// records SHOT_ERR_TIMEOUT in a device flag and still releases its tensor memory.
#include "tc_ptx.cuh"

namespace shot {
namespace {

// B operand of the analysis, MN-major (N = columns contiguous): nmma columns in atoms of 64
// (8 KB apart, 128-byte rows, one row per node).
__host__ __device__ constexpr int mn_atoms(int nmma) { return (nmma + 63) / 64; }

// Splits the FP32 spectra tile xs[64 nodes][nmma] (TMA, row-major) into bf16 hi and lo in
// the MN-major layout above.  One task = 8 consecutive columns of one node: one 16-byte
// swizzled chunk of hi and one of lo.  Nodes past the block (jh0 + r >= nh) and columns
// past the fields are zero.  nt threads (pt = 0..nt-1); each loads two tasks before it
// stores either, so the shared-memory loads overlap.
__device__ __forceinline__ void split_x_mn(const float* xs, int nmma, int ncols, int jh0, int nh, uint8_t* bh,
                                           uint8_t* bl, int pt, int nt = 64) {
  const int ch = nmma >> 3;
  const int ntask = 64 * ch;
  for (int e0 = pt; e0 < ntask; e0 += 2 * nt) {
    float4 ld[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int e = e0 + i * nt;
      if (e < ntask) {
        const int r = e / ch, c0 = (e - r * ch) * 8;
        ld[i][0] = *reinterpret_cast<const float4*>(xs + r * nmma + c0);
        ld[i][1] = *reinterpret_cast<const float4*>(xs + r * nmma + c0 + 4);
      }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int e = e0 + i * nt;
      if (e >= ntask) break;
      const int r = e / ch, c0 = (e - r * ch) * 8;
      const float4 a = ld[i][0];
      const float4 b = ld[i][1];
      float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
      const bool row_ok = jh0 + r < nh;
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        const float v0 = (row_ok && c0 + q < ncols) ? v[q] : 0.f;
        const float v1 = (row_ok && c0 + q + 1 < ncols) ? v[q + 1] : 0.f;
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
        const float2 hf = __bfloat1622float2(h2);
        const __nv_bfloat162 l2 = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
        hw[q / 2] = *reinterpret_cast<const uint32_t*>(&h2);
        lw[q / 2] = *reinterpret_cast<const uint32_t*>(&l2);
      }
      const uint32_t o = (uint32_t)((c0 >> 6) * (64 * 64 * 2)) + sw128_offset(r, c0 & 63);
      *reinterpret_cast<uint4*>(bh + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4*>(bl + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
  }
}

// The same split with each thread's tasks fixed for the whole kernel: the offsets into the
// FP32 tile and into the atoms, the task's node and its valid-column mask are computed once
// (the tasks are the same at every stage), so a stage costs only the loads, the conversions
// and the stores.  Up to kXcTasks tasks per thread (64 x nmma/8 <= kXcTasks x threads).
constexpr int kXcTasks = 4;
struct XConv {
  int xoff[kXcTasks];     // float offset of the task's 8 values in the FP32 tile (-1: no task)
  uint32_t so[kXcTasks];  // byte offset of its 16-byte chunk in the hi (and lo) atoms
  int r[kXcTasks];        // node within the 64-node chunk
  uint32_t cm[kXcTasks];  // bit q: column c0 + q < ncols

  __device__ __forceinline__ void init(int nmma, int ncols, int pt, int nt) {
    const int ch = nmma >> 3, ntask = 64 * ch;
#pragma unroll
    for (int i = 0; i < kXcTasks; ++i) {
      const int e = pt + i * nt;
      xoff[i] = -1;
      so[i] = 0;
      r[i] = 0;
      cm[i] = 0;
      if (e < ntask) {
        const int rr = e / ch, c0 = (e - rr * ch) * 8;
        xoff[i] = rr * nmma + c0;
        so[i] = (uint32_t)((c0 >> 6) * (64 * 64 * 2)) + sw128_offset(rr, c0 & 63);
        r[i] = rr;
        uint32_t m = 0;
        for (int q = 0; q < 8; ++q) m |= (c0 + q < ncols) ? (1u << q) : 0u;
        cm[i] = m;
      }
    }
  }

  __device__ __forceinline__ void run(const float* xs, int jh0, int nh, uint8_t* bh, uint8_t* bl) const {
    float4 a[kXcTasks], b[kXcTasks];
#pragma unroll
    for (int i = 0; i < kXcTasks; ++i)
      if (xoff[i] >= 0) {
        a[i] = *reinterpret_cast<const float4*>(xs + xoff[i]);
        b[i] = *reinterpret_cast<const float4*>(xs + xoff[i] + 4);
      }
#pragma unroll
    for (int i = 0; i < kXcTasks; ++i) {
      if (xoff[i] < 0) continue;
      const uint32_t m = (jh0 + r[i] < nh) ? cm[i] : 0u;
      const float v[8] = {a[i].x, a[i].y, a[i].z, a[i].w, b[i].x, b[i].y, b[i].z, b[i].w};
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        const float v0 = (m >> q) & 1u ? v[q] : 0.f;
        const float v1 = (m >> (q + 1)) & 1u ? v[q + 1] : 0.f;
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
        const float2 hf = __bfloat1622float2(h2);
        const __nv_bfloat162 l2 = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
        hw[q / 2] = *reinterpret_cast<const uint32_t*>(&h2);
        lw[q / 2] = *reinterpret_cast<const uint32_t*>(&l2);
      }
      *reinterpret_cast<uint4*>(bh + so[i]) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4*>(bl + so[i]) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
  }
};

struct AnaArgs {
  const Tile* tiles;
  int ntiles;
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
  long long wait;      // limit of every bounded wait (SM clock cycles)
};

struct SynArgs {
  const Tile* tiles;
  int ntiles;
  const int* M;
  const long long* row_off;
  int nh;
  int nmma, nmma_cap, ncols, ldc;
  float* Y;   // [blk][jh][ldc]
  int* err;
  long long wait;
};

// Persistent, warp-specialised Legendre GEMM.  Warp 0: TMA producer (runs ahead across
// tiles); warp 1: MMA issuer; the converter warps (analysis only) split the FP32 X tile into
// the bf16 hi/lo B operand; four epilogue warps.  The accumulator is double-buffered in TMEM
// so the epilogue of one tile overlaps the MMAs of the next.
constexpr int kXsBoxBytes = 64 * 64 * 2;   // one MN-major B atom: 64 columns x 64 nodes, bf16

// The analysis runs eight converter warps (2-9, two on each SM sub-partition) and its
// epilogue on warps 10-13 (448 threads); the synthesis keeps two idle converter slots (2-3)
// and warps 4-7 (256 threads).
template <bool ANA>
__host__ __device__ constexpr int tc_conv_warps() { return ANA ? 8 : 2; }
template <bool ANA>
__host__ __device__ constexpr int tc_threads() { return 32 * (2 + tc_conv_warps<ANA>() + 4); }
static_assert(tc_threads<true>() == 448 && tc_threads<false>() == kTcThreads, "warp roles");

template <int kStages, bool ANA, int kBR = 2, bool BCAT = false>
__global__ void __launch_bounds__(tc_threads<ANA>(), 1) k_legendre_tc(const __grid_constant__ CUtensorMap ta_hi,
                                                               const __grid_constant__ CUtensorMap ta_lo,
                                                               const __grid_constant__ CUtensorMap tb_hi,
                                                               const __grid_constant__ CUtensorMap tb_lo,
                                                               AnaArgs aa, SynArgs sa) {
  extern __shared__ uint8_t smraw[];
  __shared__ TcSmem ctl;
  uint8_t* base = align1k(smraw);
  const int nmma = ANA ? aa.nmma : sa.nmma;
  const int nh = ANA ? aa.nh : sa.nh;
  const int ntiles = ANA ? aa.ntiles : sa.ntiles;
  const Tile* tiles = ANA ? aa.tiles : sa.tiles;
  const int* Mr = ANA ? aa.M : sa.M;
  const int bbytes = ANA ? mn_atoms(nmma) * kXsBoxBytes : nmma * kBK * 2;
  const int xbytes = ANA ? nmma * kBK * 4 : 0;
  // Analysis from FP32 spectra: the split B operand lives in its own ring of kBR
  // buffers (released by the MMAs), so the TMA ring holds only what streams from memory
  // (table tiles and the FP32 spectra tile) and can run one stage deeper in the same shared
  // memory.
  // Each ring buffer holds the hi atoms followed by the lo atoms, so that for up to 128
  // columns (BCAT) [B_hi | B_lo] is one MN-major operand of N = 2 x 64 x atoms: a K step is
  // then A_hi [B_hi | B_lo] + A_lo B_hi, two MMAs instead of three (the A tile is read from
  // shared memory twice instead of three times), and the epilogue adds the accumulator's
  // second half.  Pad columns of the atoms stay zero.
  constexpr bool kBRing = ANA;
  constexpr int nB = kBRing ? kBR : kStages;
  const int bstride = kBRing ? 2 * bbytes : bbytes;   // between the B buffers
  uint8_t* sA_hi = base;
  uint8_t* sA_lo = sA_hi + kStages * kATileBytes;
  uint8_t* sB_hi = sA_lo + kStages * kATileBytes;
  uint8_t* sB_lo = kBRing ? sB_hi + bbytes : sB_hi + nB * bbytes;
  uint8_t* sX = sB_hi + 2 * nB * bbytes;
  const int ncat = 2 * 64 * mn_atoms(nmma);   // N of [B_hi | B_lo] (BCAT)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ncols_alloc = tmem_cols_for(BCAT ? ncat : nmma);
  if (kBRing) {   // the atoms' pad columns are never written by the converter: zero them once
    for (int o = threadIdx.x * 16; o < 2 * nB * bbytes; o += blockDim.x * 16)
      *reinterpret_cast<uint4*>(sB_hi + o) = make_uint4(0, 0, 0, 0);
    fence_async_smem();
  }

  constexpr int kConv = 32 * tc_conv_warps<ANA>();   // converter threads
  constexpr int kEpiWarp0 = 2 + tc_conv_warps<ANA>();
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&ctl.fullA[s], 1);
      mbar_init(&ctl.empty[s], 1);
    }
    for (int s = 0; s < (kStages > nB ? kStages : nB); ++s) mbar_init(&ctl.fullB[s], kConv);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl.tfull[b], 1);
      mbar_init(&ctl.tempty[b], 128);
    }
    for (int b = 0; b < kBR; ++b) mbar_init(&ctl.bempty[b], 1);
    mbar_init(&ctl.drain, 1);
    ctl.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&ctl.tmem, 2 * ncols_alloc);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = ctl.tmem;
  volatile int* abort = &ctl.abort;
  const long long wl = (ANA ? aa.wait : sa.wait);   // wait limit (cycles)
  auto nkb_of = [&](int blk) { return ANA ? (nh + kBK - 1) / kBK : (Mr[blk] + kBK - 1) / kBK; };

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const Tile tl = tiles[t];
        const int nkb = nkb_of(tl.blk);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % kStages, n = it / kStages;
          if (it >= kStages && !(ok = mbar_wait(&ctl.empty[s], (n - 1) & 1, abort, wl))) break;
          if (ANA) {
            mbar_arrive_expect_tx(&ctl.fullA[s], 2 * kATileBytes + xbytes);
            const int y = (int)(aa.row_off[tl.blk] + tl.r0);
            tma_load_2d(sA_hi + s * kATileBytes, &ta_hi, &ctl.fullA[s], kb * kBK, y);
            tma_load_2d(sA_lo + s * kATileBytes, &ta_lo, &ctl.fullA[s], kb * kBK, y);
            tma_load_2d(sX + s * xbytes, &tb_hi, &ctl.fullA[s], 0, tl.blk * nh + kb * kBK);
          } else {
            // A = the table's rows i (K) of this K-chunk, nodes r0 .. r0+127 (M, contiguous):
            // two 64-node boxes 8 KB apart, read as an MN-major operand
            mbar_arrive_expect_tx(&ctl.fullA[s], 2 * kATileBytes + 2 * bbytes);
            const int y = (int)sa.row_off[tl.blk] + kb * kBK;
            tma_load_2d(sA_hi + s * kATileBytes, &ta_hi, &ctl.fullA[s], tl.r0, y);
            tma_load_2d(sA_hi + s * kATileBytes + kATileBytes / 2, &ta_hi, &ctl.fullA[s], tl.r0 + 64, y);
            tma_load_2d(sA_lo + s * kATileBytes, &ta_lo, &ctl.fullA[s], tl.r0, y);
            tma_load_2d(sA_lo + s * kATileBytes + kATileBytes / 2, &ta_lo, &ctl.fullA[s], tl.r0 + 64, y);
            tma_load_2d(sB_hi + s * bbytes, &tb_hi, &ctl.fullA[s], kb * kBK, tl.blk * sa.nmma_cap);
            tma_load_2d(sB_lo + s * bbytes, &tb_lo, &ctl.fullA[s], kb * kBK, tl.blk * sa.nmma_cap);
          }
        }
      }
      // let this CTA's copies land before it can exit
      for (int k = it > kStages ? it - kStages : 0; k < it; ++k)
        mbar_drain(&ctl.fullA[k % kStages], (k / kStages) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      // analysis: A (table) K-major, B (spectra) MN-major; synthesis: A (table) MN-major,
      // B (C^T) K-major
      const uint32_t idesc = ANA ? (idesc_bf16(kBM, nmma) | (1u << 16)) : idesc_bf16_amn(kBM, nmma);
      const uint32_t idesc_cat = idesc_bf16(kBM, BCAT ? ncat : nmma) | (1u << 16);
      int it = 0, lt = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
        const Tile tl = tiles[t];
        const int nkb = nkb_of(tl.blk);
        const int acc = lt & 1, u = lt >> 1;
        if (lt >= 2 && !(ok = mbar_wait(&ctl.tempty[acc], (u - 1) & 1, abort, wl))) break;
        tc_fence_after();
        const uint32_t d = taddr + (uint32_t)(acc * ncols_alloc);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % kStages, n = it / kStages;
          const int sb = kBRing ? (it % kBR) : s;   // B buffer of this iteration
          ok = mbar_wait(&ctl.fullA[s], n & 1, abort, wl);
          if (ok && kBRing) ok = mbar_wait(&ctl.fullB[sb], (it / kBR) & 1, abort, wl);
          if (!ok) break;
          tc_fence_after();
          const uint32_t ah = smem_u32(sA_hi + s * kATileBytes), al = smem_u32(sA_lo + s * kATileBytes);
          const uint32_t bh = smem_u32(sB_hi + sb * bstride), bl = smem_u32(sB_lo + sb * bstride);
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k) {
            const uint32_t off = k * 32;
            uint64_t b_h, b_l;
            if (ANA) {   // 16 K-rows = two 8-row groups of the MN-major atoms
              b_h = desc_sw128_mnmajor(bh + k * 2048, kXsBoxBytes, 1024);
              b_l = desc_sw128_mnmajor(bl + k * 2048, kXsBoxBytes, 1024);
            } else {
              b_h = desc_sw128_kmajor(bh + off);
              b_l = desc_sw128_kmajor(bl + off);
            }
            uint64_t a_h, a_l;
            if (ANA) {
              a_h = desc_sw128_kmajor(ah + off);
              a_l = desc_sw128_kmajor(al + off);
            } else {   // 16 K-rows (two 8-row groups) of two 64-node atoms
              a_h = desc_sw128_mnmajor(ah + k * 2048, kATileBytes / 2, 1024);
              a_l = desc_sw128_mnmajor(al + k * 2048, kATileBytes / 2, 1024);
            }
            if constexpr (BCAT) {   // b_h starts [B_hi | B_lo]
              umma_bf16(d, a_h, b_h, idesc_cat, (kb | k) != 0);
              umma_bf16(d, a_l, b_h, idesc, 1);
            } else {
              umma_bf16(d, a_h, b_h, idesc, (kb | k) != 0);
              umma_bf16(d, a_h, b_l, idesc, 1);
              umma_bf16(d, a_l, b_h, idesc, 1);
            }
          }
          umma_commit(&ctl.empty[s]);
          if (kBRing) umma_commit(&ctl.bempty[sb]);
        }
        umma_commit(&ctl.tfull[acc]);
      }
      // every MMA issued here completes before the CTA frees its tensor memory (after an abort too)
      umma_commit(&ctl.drain);
      mbar_drain(&ctl.drain, 0);
    }
  } else if (warp < kEpiWarp0) {
    if (ANA) {
      // split the FP32 X tile (TMA, with the table tiles) into bf16 hi/lo, MN-major [jh][c]
      const int pt = threadIdx.x - 64;
      const bool pre = 64 * (nmma >> 3) <= kXcTasks * kConv;   // the tasks fit the fixed plan
      XConv xc;
      xc.init(pre ? nmma : 0, aa.ncols, pt, kConv);
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const Tile tl = tiles[t];
        const int nkb = nkb_of(tl.blk);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % kStages, n = it / kStages;
          const int sb = it % kBR, nb = it / kBR;
          if (!(ok = mbar_wait(&ctl.fullA[s], n & 1, abort, wl))) break;
          // the MMAs of iteration it - kBR have finished reading this B buffer
          if (nb > 0 && !(ok = mbar_wait(&ctl.bempty[sb], (nb - 1) & 1, abort, wl))) break;
          if (pre)
            xc.run(reinterpret_cast<const float*>(sX + s * xbytes), kb * kBK, nh, sB_hi + sb * bstride,
                   sB_lo + sb * bstride);
          else
            split_x_mn(reinterpret_cast<const float*>(sX + s * xbytes), nmma, aa.ncols, kb * kBK, nh,
                       sB_hi + sb * bstride, sB_lo + sb * bstride, pt, kConv);
          fence_async_smem();
          mbar_arrive(&ctl.fullB[sb]);
        }
      }
    }
  } else {
    // epilogue: drain the accumulator of every tile of this CTA
    const int q = warp & 3;   // a warp reaches only TMEM lanes 32 (warp % 4) .. 32 (warp % 4) + 31
    int lt = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      const Tile tl = tiles[t];
      const int acc = lt & 1, u = lt >> 1;
      if (!mbar_wait_warp(&ctl.tfull[acc], u & 1, abort, wl)) break;
      tc_fence_after();
      const uint32_t d = taddr + (uint32_t)(acc * ncols_alloc) + ((uint32_t)(q * 32) << 16);
      const int row = tl.r0 + q * 32 + lane;
      if (ANA) {
        const int blk = tl.blk, m = blk >> 1, p = blk & 1;
        const int M = Mr[blk];
        const long long ro = aa.row_off[blk];
        const float hl = (aa.h && row < M) ? aa.h[m + p + 2 * row] : 1.f;
        for (int c0 = 0; c0 < nmma; c0 += 16) {
          float v[16];
          tmem_ld16(d + (uint32_t)c0, v);
          if constexpr (BCAT) {   // + A_hi B_lo from the second half
            float w[16];
            tmem_ld16(d + (uint32_t)(ncat / 2 + c0), w);
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] += w[e];
          }
          if (row < M) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int c = c0 + e;
              if (c < aa.ncols) {
                const float val = v[e] * hl;
                const __nv_bfloat16 hi = __float2bfloat16_rn(val);
                const __nv_bfloat16 lo = __float2bfloat16_rn(val - __bfloat162float(hi));
                const size_t o = ((size_t)blk * aa.nmma_cap + c) * aa.ldi + row;
                aa.ct_hi[o] = hi;
                aa.ct_lo[o] = lo;
                if (aa.cf) aa.cf[(size_t)(ro + row) * aa.ldc + c] = val;
              }
            }
          }
        }
      } else {
        float* yrow = sa.Y + ((size_t)tl.blk * nh + row) * sa.ldc;
        for (int c0 = 0; c0 < nmma; c0 += 16) {
          float v[16];
          tmem_ld16(d + (uint32_t)c0, v);
          if (row < nh) {
            if (c0 + 16 <= sa.ncols) {
#pragma unroll
              for (int e = 0; e < 16; e += 4)
                *reinterpret_cast<float4*>(yrow + c0 + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
            } else {
#pragma unroll
              for (int e = 0; e < 16; ++e)
                if (c0 + e < sa.ncols) yrow[c0 + e] = v[e];
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
  if (threadIdx.x == 0 && ctl.abort) atomicExch(ANA ? aa.err : sa.err, SHOT_ERR_TIMEOUT);
}


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

// with_x: analysis (MN-major B of mn_atoms(nmma) 8 KB atoms, plus the FP32 spectra tile);
// otherwise synthesis (K-major B of nmma rows)
size_t tc_smem_bytes(int nmma, bool with_x, int stages, int br = 2) {
  if (with_x)   // analysis: table tiles and the FP32 spectra tile per stage, B in a ring of br buffers
    return 1024 + (size_t)stages * (2 * kATileBytes + (size_t)nmma * kBK * 4) +
           (size_t)br * 2 * (size_t)mn_atoms(nmma) * kXsBoxBytes;
  return 1024 + (size_t)stages * (2 * kATileBytes + 2 * (size_t)nmma * kBK * 2);
}

}  // namespace

int tc_nmma(int nf) { return (2 * nf + 15) / 16 * 16; }

static int host_tmem_cols(int n) {
  int c = 32;
  while (c < n) c <<= 1;
  return c;
}

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
  AnaArgs aa{};
  SynArgs sa{};
  if (ana) {
    // deepest pipeline (<= 3 stages) whose tiles fit in one CTA's shared memory
    int stages = kStagesAna;
    if (g.active.nf == nf && g.active.tc_stages > 0) stages = g.active.tc_stages;
    if (g.tc_stages_override > 0) stages = g.tc_stages_override;
    // split spectra ring: three buffers when they fit beside at least two TMA stages
    const int br = (tc_smem_bytes(nmma, true, 2, 3) + 1024 <= 227 * 1024) ? 3 : 2;
    while (stages > 1 && tc_smem_bytes(nmma, true, stages, br) + 1024 > 227 * 1024) --stages;
    const size_t smem = tc_smem_bytes(nmma, true, stages, br);
    CUtensorMap mh, ml, mx;
    if ((rc = make_map(&mh, g.tab_hi, g.nh, g.rows_total, g.ldt, kBM))) return rc;
    if ((rc = make_map(&ml, g.tab_lo, g.nh, g.rows_total, g.ldt, kBM))) return rc;
    if ((rc = make_map_f32(&mx, X, ldc, (uint64_t)g.nblk * g.nh, ldc, nmma, kBK))) return rc;
    aa = AnaArgs{g.tiles_ana, g.ntiles_ana, g.M_d, g.row_off_d, g.nh, X, ldc, 2 * nf, nmma,
                 apply_h ? g.h_d : nullptr, w.ct_hi, w.ct_lo, w.nmma_cap, g.ldi, Cf, w.dev_int + 4,
                 g.wait_cycles};
    // [B_hi | B_lo] as one operand up to 128 columns (N = 2 x 64 x atoms <= 256)
    const bool bcat = 2 * 64 * mn_atoms(nmma) <= 256;
    auto kern = bcat ? (br == 3 ? (stages == 4   ? k_legendre_tc<4, true, 3, true>
                                   : stages == 3 ? k_legendre_tc<3, true, 3, true>
                                   : stages == 2 ? k_legendre_tc<2, true, 3, true>
                                                 : k_legendre_tc<1, true, 3, true>)
                                : (stages == 4   ? k_legendre_tc<4, true, 2, true>
                                   : stages == 3 ? k_legendre_tc<3, true, 2, true>
                                   : stages == 2 ? k_legendre_tc<2, true, 2, true>
                                                 : k_legendre_tc<1, true, 2, true>))
                     : (br == 3 ? (stages == 4   ? k_legendre_tc<4, true, 3>
                                   : stages == 3 ? k_legendre_tc<3, true, 3>
                                   : stages == 2 ? k_legendre_tc<2, true, 3>
                                                 : k_legendre_tc<1, true, 3>)
                                : (stages == 4   ? k_legendre_tc<4, true, 2>
                                   : stages == 3 ? k_legendre_tc<3, true, 2>
                                   : stages == 2 ? k_legendre_tc<2, true, 2>
                                                 : k_legendre_tc<1, true, 2>));
    SHOT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // CTAs per SM: both shared memory and the 512 TMEM columns (two accumulators each) must fit
    const int acc_cols = host_tmem_cols(bcat ? 2 * 64 * mn_atoms(nmma) : nmma);
    const int per_sm = (smem <= 113 * 1024 && 2 * 2 * acc_cols <= 512) ? 2 : 1;
    const int grid = g.ntiles_ana < per_sm * g.num_sms ? g.ntiles_ana : per_sm * g.num_sms;
    ProfScope prof(PK_ANALYSIS, st);
    count_launch();
    kern<<<grid, tc_threads<true>(), smem, st>>>(mh, ml, mx, mx, aa, sa);
    SHOT_CUDA(cudaGetLastError());
  }
  if (syn) {
    const size_t smem = tc_smem_bytes(nmma, false, kStagesSyn);
    CUtensorMap ah, al, bh, bl;
    if ((rc = make_map(&ah, g.tab_hi, g.nh, g.rows_total, g.ldt, 64))) return rc;
    if ((rc = make_map(&al, g.tab_lo, g.nh, g.rows_total, g.ldt, 64))) return rc;
    if ((rc = make_map(&bh, w.ct_hi, g.ldi, (uint64_t)g.nblk * w.nmma_cap, g.ldi, nmma))) return rc;
    if ((rc = make_map(&bl, w.ct_lo, g.ldi, (uint64_t)g.nblk * w.nmma_cap, g.ldi, nmma))) return rc;
    sa = SynArgs{g.tiles_syn, g.ntiles_syn, g.M_d, g.row_off_d, g.nh, nmma, w.nmma_cap, 2 * nf, ldc, Y, w.dev_int + 4,
                 g.wait_cycles};
    auto kern = k_legendre_tc<kStagesSyn, false>;
    SHOT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // CTAs per SM: both shared memory and the 512 TMEM columns (two accumulators each) must fit
    const int per_sm = (smem <= 113 * 1024 && 2 * 2 * host_tmem_cols(nmma) <= 512) ? 2 : 1;
    const int grid = g.ntiles_syn < per_sm * g.num_sms ? g.ntiles_syn : per_sm * g.num_sms;
    ProfScope prof(PK_SYNTHESIS, st);
    count_launch();
    kern<<<grid, kTcThreads, smem, st>>>(ah, al, bh, bl, aa, sa);
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
