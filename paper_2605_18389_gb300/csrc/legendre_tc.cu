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
// warps in the MN-major layout it already has (or arrives split, bf16 hi/lo, by TMA); the
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
};

// Persistent, warp-specialised Legendre GEMM.  Warp 0: TMA producer (runs ahead across
// tiles); warp 1: MMA issuer; warps 2-3 (analysis only): split the FP32 X tile into the
// bf16 hi/lo B operand; warps 4-7: epilogue.  The accumulator is double-buffered in TMEM
// so the epilogue of one tile overlaps the MMAs of the next.
// XS (analysis only): the spectra come as bf16 hi/lo arrays [blk nh + jh][ldc] and are
// loaded by TMA as an MN-major B operand (64 columns x 64 nodes per box); the split warps
// are idle.
constexpr int kXsBoxBytes = 64 * 64 * 2;

// Analysis from FP32 spectra runs eight converter warps (2-9, two on each SM sub-partition)
// and its epilogue on warps 10-13 (448 threads); the other forms keep two converter slots
// (2-3) and warps 4-7 (256 threads).
template <bool ANA, bool XS>
__host__ __device__ constexpr int tc_conv_warps() { return (ANA && !XS) ? 8 : 2; }
template <bool ANA, bool XS>
__host__ __device__ constexpr int tc_threads() { return 32 * (2 + tc_conv_warps<ANA, XS>() + 4); }
static_assert(tc_threads<true, false>() == 448 && tc_threads<false, false>() == kTcThreads, "warp roles");

template <int kStages, bool ANA, bool XS = false, int kBR = 2, bool BCAT = false>
__global__ void __launch_bounds__(tc_threads<ANA, XS>(), 1) k_legendre_tc(const __grid_constant__ CUtensorMap ta_hi,
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
  const int xbytes = (ANA && !XS) ? nmma * kBK * 4 : 0;
  // Analysis from FP32 spectra: the split B operand lives in its own ring of kBR
  // buffers (released by the MMAs), so the TMA ring holds only what streams from memory
  // (table tiles and the FP32 spectra tile) and can run one stage deeper in the same shared
  // memory.
  // Each ring buffer holds the hi atoms followed by the lo atoms, so that for up to 128
  // columns (BCAT) [B_hi | B_lo] is one MN-major operand of N = 2 x 64 x atoms: a K step is
  // then A_hi [B_hi | B_lo] + A_lo B_hi, two MMAs instead of three (the A tile is read from
  // shared memory twice instead of three times), and the epilogue adds the accumulator's
  // second half.  Pad columns of the atoms stay zero.
  constexpr bool kBRing = ANA && !XS;
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

  constexpr int kConv = 32 * tc_conv_warps<ANA, XS>();   // converter threads
  constexpr int kEpiWarp0 = 2 + tc_conv_warps<ANA, XS>();
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
    ctl.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&ctl.tmem, 2 * ncols_alloc);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = ctl.tmem;
  volatile int* abort = &ctl.abort;
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
          if (it >= kStages && !(ok = mbar_wait(&ctl.empty[s], (n - 1) & 1, abort))) break;
          if (ANA && XS) {
            mbar_arrive_expect_tx(&ctl.fullA[s], 2 * kATileBytes + 2 * kXsBoxBytes);
            const int y = (int)(aa.row_off[tl.blk] + tl.r0);
            tma_load_2d(sA_hi + s * kATileBytes, &ta_hi, &ctl.fullA[s], kb * kBK, y);
            tma_load_2d(sA_lo + s * kATileBytes, &ta_lo, &ctl.fullA[s], kb * kBK, y);
            tma_load_2d(sB_hi + s * bbytes, &tb_hi, &ctl.fullA[s], 0, tl.blk * nh + kb * kBK);
            tma_load_2d(sB_lo + s * bbytes, &tb_lo, &ctl.fullA[s], 0, tl.blk * nh + kb * kBK);
          } else if (ANA) {
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
        if (lt >= 2 && !(ok = mbar_wait(&ctl.tempty[acc], (u - 1) & 1, abort))) break;
        tc_fence_after();
        const uint32_t d = taddr + (uint32_t)(acc * ncols_alloc);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % kStages, n = it / kStages;
          const int sb = kBRing ? (it % kBR) : s;   // B buffer of this iteration
          ok = mbar_wait(&ctl.fullA[s], n & 1, abort);
          if (ok && kBRing) ok = mbar_wait(&ctl.fullB[sb], (it / kBR) & 1, abort);
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
    }
  } else if (warp < kEpiWarp0) {
    if (ANA && !XS) {
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
          if (!(ok = mbar_wait(&ctl.fullA[s], n & 1, abort))) break;
          // the MMAs of iteration it - kBR have finished reading this B buffer
          if (nb > 0 && !(ok = mbar_wait(&ctl.bempty[sb], (nb - 1) & 1, abort))) break;
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
      if (!mbar_wait_warp(&ctl.tfull[acc], u & 1, abort)) break;
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


// ---------------------------------------------------------------------------------
// Transposed analysis: C^T[c][i] = h_l sum_jh X[jh][c] Pbar[i][jh], i.e. D = A B with
//   A = X^T  (M = 128 lanes: the spectra columns c, only 2 nf of them filled; K = jh),
//             MN-major in shared memory, split into hi/lo by two warps (same layout as the
//             analysis B operand of k_legendre_tc);
//   B = Pbar (N = the tile's degree rows, up to 256 in 32-row TMA boxes; K = jh), K-major.
// A tile is a run of at most 256 degree rows of one block, so a block wastes < 32 rows to
// padding (an M = 128 row tiling wastes ~64), and the epilogue holds 16 consecutive degrees
// of one column per tcgen05.ld: C^T rows are written as 32-byte vectors, directly in the
// K-major layout the synthesis reads.  Only used by the heat application (no FP32 C).
constexpr int kRowBox = 32;           // degree rows per TMA box
constexpr int kRowBoxBytes = kRowBox * kBK * 2;   // 4 KB

struct AnaTArgs {
  const TileR* tiles;
  int ntiles;
  const long long* row_off;
  const int* M;
  int nh;
  const float* X;
  int ldc, ncols, nmma;
  const float* h;
  __nv_bfloat16* ct_hi;
  __nv_bfloat16* ct_lo;
  int nmma_cap, ldi;
  int* err;
};

template <int kStages>
__global__ void __launch_bounds__(kTcThreads, 1) k_ana_tc_t(const __grid_constant__ CUtensorMap t_hi,
                                                            const __grid_constant__ CUtensorMap t_lo,
                                                            const __grid_constant__ CUtensorMap t_x, AnaTArgs aa) {
  extern __shared__ uint8_t smraw[];
  __shared__ TcSmem ctl;
  uint8_t* base = align1k(smraw);
  const int nmma = aa.nmma, nh = aa.nh;
  constexpr int kBTile = 256 * kBK * 2;          // table tile (hi or lo), 256 rows
  constexpr int kATile = 2 * kXsBoxBytes;        // X^T (hi or lo): two 64-column atoms
  const int xbytes = nmma * kBK * 4;
  const int sbytes = 2 * kBTile + 2 * kATile + xbytes;
  auto sB_hi = [&](int s) { return base + s * sbytes; };
  auto sB_lo = [&](int s) { return base + s * sbytes + kBTile; };
  auto sA_hi = [&](int s) { return base + s * sbytes + 2 * kBTile; };
  auto sA_lo = [&](int s) { return base + s * sbytes + 2 * kBTile + kATile; };
  auto sX = [&](int s) { return base + s * sbytes + 2 * kBTile + 2 * kATile; };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr uint32_t kAccCols = 256;
  const int nkb = (nh + kBK - 1) / kBK;

  // the A atoms of columns 64..127 hold only zeros (2 nf <= 64): clear them once
  for (int s = 0; s < kStages; ++s)
    for (int o = threadIdx.x * 16; o < kXsBoxBytes; o += blockDim.x * 16) {
      *reinterpret_cast<uint4*>(sA_hi(s) + kXsBoxBytes + o) = make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4*>(sA_lo(s) + kXsBoxBytes + o) = make_uint4(0, 0, 0, 0);
    }
  fence_async_smem();
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&ctl.fullA[s], 1);
      mbar_init(&ctl.fullB[s], 64);
      mbar_init(&ctl.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl.tfull[b], 1);
      mbar_init(&ctl.tempty[b], 128);
    }
    ctl.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&ctl.tmem, 2 * kAccCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = ctl.tmem;
  volatile int* abort = &ctl.abort;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < aa.ntiles && ok; t += gridDim.x) {
        const TileR tl = aa.tiles[t];
        const int nbox = (tl.rows + kRowBox - 1) / kRowBox;
        const int y0 = (int)aa.row_off[tl.blk] + tl.r0;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % kStages, n = it / kStages;
          if (it >= kStages && !(ok = mbar_wait(&ctl.empty[s], (n - 1) & 1, abort))) break;
          mbar_arrive_expect_tx(&ctl.fullA[s], 2 * nbox * kRowBoxBytes + xbytes);
          for (int b = 0; b < nbox; ++b) {
            tma_load_2d(sB_hi(s) + b * kRowBoxBytes, &t_hi, &ctl.fullA[s], kb * kBK, y0 + b * kRowBox);
            tma_load_2d(sB_lo(s) + b * kRowBoxBytes, &t_lo, &ctl.fullA[s], kb * kBK, y0 + b * kRowBox);
          }
          tma_load_2d(sX(s), &t_x, &ctl.fullA[s], 0, tl.blk * nh + kb * kBK);
        }
      }
      for (int k = it > kStages ? it - kStages : 0; k < it; ++k)
        mbar_drain(&ctl.fullA[k % kStages], (k / kStages) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      int it = 0, lt = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < aa.ntiles && ok; t += gridDim.x, ++lt) {
        const TileR tl = aa.tiles[t];
        const int nrow = (tl.rows + kRowBox - 1) / kRowBox * kRowBox;   // N, a multiple of 32
        const uint32_t idesc = idesc_bf16_amn(kBM, nrow);
        const int acc = lt & 1, u = lt >> 1;
        if (lt >= 2 && !(ok = mbar_wait(&ctl.tempty[acc], (u - 1) & 1, abort))) break;
        tc_fence_after();
        const uint32_t d = taddr + (uint32_t)(acc * kAccCols);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % kStages, n = it / kStages;
          ok = mbar_wait(&ctl.fullA[s], n & 1, abort);
          if (ok) ok = mbar_wait(&ctl.fullB[s], n & 1, abort);
          if (!ok) break;
          tc_fence_after();
          const uint32_t ah = smem_u32(sA_hi(s)), al = smem_u32(sA_lo(s));
          const uint32_t bh = smem_u32(sB_hi(s)), bl = smem_u32(sB_lo(s));
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k) {
            // A: 16 K-rows (jh) of the two 64-column atoms; B: the table rows, K-major
            const uint64_t a_h = desc_sw128_mnmajor(ah + k * 2048, kXsBoxBytes, 1024);
            const uint64_t a_l = desc_sw128_mnmajor(al + k * 2048, kXsBoxBytes, 1024);
            const uint64_t b_h = desc_sw128_kmajor(bh + k * 32), b_l = desc_sw128_kmajor(bl + k * 32);
            umma_bf16(d, a_h, b_h, idesc, (kb | k) != 0);
            umma_bf16(d, a_h, b_l, idesc, 1);
            umma_bf16(d, a_l, b_h, idesc, 1);
          }
          umma_commit(&ctl.empty[s]);
        }
        if (!ok) break;
        umma_commit(&ctl.tfull[acc]);
      }
    }
  } else if (warp < 4) {
    // split the FP32 spectra tile (TMA) into the A operand X^T, hi/lo, MN-major
    const int pt = threadIdx.x - 64;
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < aa.ntiles && ok; t += gridDim.x) {
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = it % kStages, n = it / kStages;
        if (!(ok = mbar_wait(&ctl.fullA[s], n & 1, abort))) break;
        split_x_mn(reinterpret_cast<const float*>(sX(s)), nmma, aa.ncols, kb * kBK, nh, sA_hi(s), sA_lo(s), pt);
        fence_async_smem();
        mbar_arrive(&ctl.fullB[s]);
      }
    }
  } else {
    // epilogue: lane c of quadrant q holds column 32 q + lane; 16 degree rows per load
    const int q = warp - 4;
    const int c = q * 32 + lane;
    const bool qlive = q * 32 < aa.ncols;   // warp-uniform
    int lt = 0;
    for (int t = blockIdx.x; t < aa.ntiles; t += gridDim.x, ++lt) {
      const TileR tl = aa.tiles[t];
      const int acc = lt & 1, u = lt >> 1;
      if (!mbar_wait_warp(&ctl.tfull[acc], u & 1, abort)) break;
      tc_fence_after();
      if (qlive) {
        const int blk = tl.blk, m = blk >> 1, p = blk & 1;
        const uint32_t d = taddr + (uint32_t)(acc * kAccCols) + ((uint32_t)(q * 32) << 16);
        const size_t row0 = ((size_t)blk * aa.nmma_cap + c) * aa.ldi + tl.r0;
        for (int i0 = 0; i0 < tl.rows; i0 += 16) {
          float v[16];
          tmem_ld16(d + (uint32_t)i0, v);
          if (c < aa.ncols) {
            uint32_t hw[8], lw[8];
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
              const int i = tl.r0 + i0 + e;   // rows past the tile (i0 + e >= rows) are not stored
              const float h0 = (aa.h && i0 + e < tl.rows) ? aa.h[m + p + 2 * i] : 1.f;
              const float h1 = (aa.h && i0 + e + 1 < tl.rows) ? aa.h[m + p + 2 * (i + 1)] : 1.f;
              const float v0 = v[e] * h0, v1 = v[e + 1] * h1;
              const __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
              const float2 hf = __bfloat1622float2(h2);
              const __nv_bfloat162 l2 = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
              hw[e / 2] = *reinterpret_cast<const uint32_t*>(&h2);
              lw[e / 2] = *reinterpret_cast<const uint32_t*>(&l2);
            }
            __nv_bfloat16* dh = aa.ct_hi + row0 + i0;
            __nv_bfloat16* dl = aa.ct_lo + row0 + i0;
            if (i0 + 16 <= tl.rows) {   // 16-byte aligned: ldi, r0 and i0 are multiples of 8
              reinterpret_cast<uint4*>(dh)[0] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              reinterpret_cast<uint4*>(dh)[1] = make_uint4(hw[4], hw[5], hw[6], hw[7]);
              reinterpret_cast<uint4*>(dl)[0] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
              reinterpret_cast<uint4*>(dl)[1] = make_uint4(lw[4], lw[5], lw[6], lw[7]);
            } else {   // the block's last rows: rows past M stay zero for the synthesis
              for (int e = 0; e < tl.rows - i0; ++e) {
                const uint32_t wh = hw[e / 2], wl = lw[e / 2];
                dh[e] = __ushort_as_bfloat16((unsigned short)((e & 1) ? (wh >> 16) : (wh & 0xFFFFu)));
                dl[e] = __ushort_as_bfloat16((unsigned short)((e & 1) ? (wl >> 16) : (wl & 0xFFFFu)));
              }
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
    tmem_dealloc(taddr, 2 * kAccCols);
  }
  if (threadIdx.x == 0 && ctl.abort) atomicExch(aa.err, SHOT_ERR_TIMEOUT);
}

// ---------------------------------------------------------------------------------
// Fused heat application per (m, parity) block: the analysis of the block (all its
// 128-row tiles), h_l and the per-field gauge factor in the epilogue, the coefficients
// kept in shared memory as the bf16 hi/lo B operand, then the synthesis of the block
// (all its 128-node tiles) with the SAME table tiles read as an MN-major A operand:
//   analysis   C[i][c] = h_l sum_jh Pbar[i][jh] X[jh][c]      A = Pbar (K = jh contiguous)
//   synthesis  Y[jh][c] = sum_i Pbar[i][jh] C[i][c]            A = Pbar^T (M = jh contiguous)
// The second read of each table tile comes shortly after the first, from L2, so the table
// streams from HBM once per heat application, and no coefficients go through global memory.
// Roles as in k_legendre_tc; a persistent CTA takes whole blocks, largest first, in
// snake order over the grid.
constexpr int kMaxSlots = 8;   // TMEM accumulators per CTA (analysis tiles + synthesis tiles)

struct HeatTcSmem {
  uint64_t full[kMaxStages];
  uint64_t fullB[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t afull[kMaxSlots], aempty[kMaxSlots];
  uint64_t sfull[kMaxSlots], sempty[kMaxSlots];
  uint64_t cready;
  uint32_t tmem;
  int abort;
};

struct HeatArgs {
  const int* order;   // blocks with rows, largest first
  int nwork;
  const int* M;
  const long long* row_off;
  int nh, ldc, ncols, nmma;
  int nmt_max;        // 128-row tiles of the largest block
  int kc_max;         // 64-row chunks of the largest block
  const float* h;     // h_l or nullptr
  float* Y;           // [blk][jh][ldc]
  int* err;
};

__device__ __forceinline__ int heat_work(int r, int c, int G) { return r * G + ((r & 1) ? G - 1 - c : c); }

template <int kStages, bool XS>
__global__ void __launch_bounds__(kTcThreads, 1) k_heat_tc(const __grid_constant__ CUtensorMap t_hi,
                                                           const __grid_constant__ CUtensorMap t_lo,
                                                           const __grid_constant__ CUtensorMap t_x,
                                                           const __grid_constant__ CUtensorMap t_x2, HeatArgs ha) {
  extern __shared__ uint8_t smraw[];
  __shared__ HeatTcSmem ctl;
  uint8_t* base = align1k(smraw);
  const int nmma = ha.nmma, nh = ha.nh;
  const int bbytes = mn_atoms(nmma) * kXsBoxBytes;   // analysis B, MN-major
  const int xbytes = XS ? 0 : nmma * kBK * 4;
  const int sbytes = 2 * kATileBytes + xbytes + 2 * bbytes;   // one pipeline stage
  const int cbytes = nmma * 128;                              // one 64-row chunk of C (hi or lo)
  uint8_t* cbuf_hi = base + kStages * sbytes;
  uint8_t* cbuf_lo = cbuf_hi + ha.kc_max * cbytes;
  auto sA_hi = [&](int s) { return base + s * sbytes; };
  auto sA_lo = [&](int s) { return base + s * sbytes + kATileBytes; };
  auto sX = [&](int s) { return base + s * sbytes + 2 * kATileBytes; };
  auto sB_hi = [&](int s) { return base + s * sbytes + 2 * kATileBytes + xbytes; };
  auto sB_lo = [&](int s) { return base + s * sbytes + 2 * kATileBytes + xbytes + bbytes; };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ncols_alloc = tmem_cols_for(nmma);
  const int nnt = (nh + kBM - 1) / kBM;
  const int nkbA = (nh + kBK - 1) / kBK;
  const int G = gridDim.x;
  const int rounds = (ha.nwork + G - 1) / G;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&ctl.full[s], 1);
      mbar_init(&ctl.fullB[s], 64);
      mbar_init(&ctl.empty[s], 1);
    }
    for (int b = 0; b < kMaxSlots; ++b) {
      mbar_init(&ctl.afull[b], 1);
      mbar_init(&ctl.aempty[b], 128);
      mbar_init(&ctl.sfull[b], 1);
      mbar_init(&ctl.sempty[b], 128);
    }
    mbar_init(&ctl.cready, 128);
    ctl.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&ctl.tmem, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = ctl.tmem;
  volatile int* abort = &ctl.abort;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int it = 0;
      bool ok = true;
      for (int r = 0; r < rounds && ok; ++r) {
        const int w = heat_work(r, blockIdx.x, G);
        if (w >= ha.nwork) continue;
        const int blk = ha.order[w];
        const int M = ha.M[blk];
        const int ro = (int)ha.row_off[blk];
        const int nmt = (M + kBM - 1) / kBM, nkbS = (M + kBK - 1) / kBK;
        for (int mt = 0; mt < nmt && ok; ++mt)
          for (int kb = 0; kb < nkbA; ++kb, ++it) {
            const int s = it % kStages, n = it / kStages;
            if (it >= kStages && !(ok = mbar_wait(&ctl.empty[s], (n - 1) & 1, abort))) break;
            mbar_arrive_expect_tx(&ctl.full[s], 2 * kATileBytes + (XS ? 2 * kXsBoxBytes : xbytes));
            const int y = ro + mt * kBM, x = kb * kBK;
            tma_load_2d(sA_hi(s), &t_hi, &ctl.full[s], x, y);
            tma_load_2d(sA_hi(s) + kATileBytes / 2, &t_hi, &ctl.full[s], x, y + 64);
            tma_load_2d(sA_lo(s), &t_lo, &ctl.full[s], x, y);
            tma_load_2d(sA_lo(s) + kATileBytes / 2, &t_lo, &ctl.full[s], x, y + 64);
            if (XS) {
              tma_load_2d(sB_hi(s), &t_x, &ctl.full[s], 0, blk * nh + kb * kBK);
              tma_load_2d(sB_lo(s), &t_x2, &ctl.full[s], 0, blk * nh + kb * kBK);
            } else {
              tma_load_2d(sX(s), &t_x, &ctl.full[s], 0, blk * nh + kb * kBK);
            }
          }
        for (int nt = 0; nt < nnt && ok; ++nt)
          for (int kb = 0; kb < nkbS; ++kb, ++it) {
            const int s = it % kStages, n = it / kStages;
            if (it >= kStages && !(ok = mbar_wait(&ctl.empty[s], (n - 1) & 1, abort))) break;
            mbar_arrive_expect_tx(&ctl.full[s], 2 * kATileBytes);
            const int y = ro + kb * kBK, x = nt * kBM;
            tma_load_2d(sA_hi(s), &t_hi, &ctl.full[s], x, y);
            tma_load_2d(sA_hi(s) + kATileBytes / 2, &t_hi, &ctl.full[s], x + 64, y);
            tma_load_2d(sA_lo(s), &t_lo, &ctl.full[s], x, y);
            tma_load_2d(sA_lo(s) + kATileBytes / 2, &t_lo, &ctl.full[s], x + 64, y);
          }
      }
      for (int k = it > kStages ? it - kStages : 0; k < it; ++k)
        mbar_drain(&ctl.full[k % kStages], (k / kStages) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      // analysis: A K-major; B K-major (split in shared memory) or MN-major (XS, from TMA)
      const uint32_t id_a = idesc_bf16(kBM, nmma) | (1u << 16);
      const uint32_t id_s = idesc_bf16_amn(kBM, nmma);   // synthesis: A (table) MN-major
      int it = 0, nb = 0;
      int ause[kMaxSlots] = {0}, suse[kMaxSlots] = {0};
      bool ok = true;
      for (int r = 0; r < rounds && ok; ++r) {
        const int w = heat_work(r, blockIdx.x, G);
        if (w >= ha.nwork) continue;
        const int blk = ha.order[w];
        const int M = ha.M[blk];
        const int nmt = (M + kBM - 1) / kBM, nkbS = (M + kBK - 1) / kBK;
        for (int mt = 0; mt < nmt && ok; ++mt) {
          if (ause[mt] > 0 && !(ok = mbar_wait(&ctl.aempty[mt], (ause[mt] - 1) & 1, abort))) break;
          tc_fence_after();
          const uint32_t d = taddr + (uint32_t)(mt * ncols_alloc);
          for (int kb = 0; kb < nkbA; ++kb, ++it) {
            const int s = it % kStages, n = it / kStages;
            ok = mbar_wait(&ctl.full[s], n & 1, abort);
            if (ok && !XS) ok = mbar_wait(&ctl.fullB[s], n & 1, abort);
            if (!ok) break;
            tc_fence_after();
            const uint32_t ah = smem_u32(sA_hi(s)), al = smem_u32(sA_lo(s));
            const uint32_t bh = smem_u32(sB_hi(s)), bl = smem_u32(sB_lo(s));
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k) {
              const uint32_t off = k * 32;
              const uint64_t b_h = desc_sw128_mnmajor(bh + k * 2048, kXsBoxBytes, 1024);
              const uint64_t b_l = desc_sw128_mnmajor(bl + k * 2048, kXsBoxBytes, 1024);
              umma_bf16(d, desc_sw128_kmajor(ah + off), b_h, id_a, (kb | k) != 0);
              umma_bf16(d, desc_sw128_kmajor(ah + off), b_l, id_a, 1);
              umma_bf16(d, desc_sw128_kmajor(al + off), b_h, id_a, 1);
            }
            umma_commit(&ctl.empty[s]);
          }
          if (!ok) break;
          umma_commit(&ctl.afull[mt]);
          ++ause[mt];
        }
        if (!ok) break;
        // the coefficients of this block must be in shared memory
        if (!(ok = mbar_wait(&ctl.cready, nb & 1, abort))) break;
        tc_fence_after();
        const uint32_t ch = smem_u32(cbuf_hi), cl = smem_u32(cbuf_lo);
        for (int nt = 0; nt < nnt && ok; ++nt) {
          const int slot = ha.nmt_max + nt;
          if (suse[nt] > 0 && !(ok = mbar_wait(&ctl.sempty[nt], (suse[nt] - 1) & 1, abort))) break;
          tc_fence_after();
          const uint32_t d = taddr + (uint32_t)(slot * ncols_alloc);
          for (int kb = 0; kb < nkbS; ++kb, ++it) {
            const int s = it % kStages, n = it / kStages;
            ok = mbar_wait(&ctl.full[s], n & 1, abort);
            if (ok && !XS) ok = mbar_wait(&ctl.fullB[s], n & 1, abort);   // keeps the stage phases aligned
            if (!ok) break;
            tc_fence_after();
            const uint32_t ah = smem_u32(sA_hi(s)), al = smem_u32(sA_lo(s));
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k) {
              // A: 16 K-rows (two 8-row groups, 1 KB apart) of two 64-node atoms (8 KB apart)
              const uint64_t a_h = desc_sw128_mnmajor(ah + k * 2048, kATileBytes / 2, 1024);
              const uint64_t a_l = desc_sw128_mnmajor(al + k * 2048, kATileBytes / 2, 1024);
              const uint32_t boff = (uint32_t)(kb * cbytes + k * 32);
              const uint64_t b_h = desc_sw128_kmajor(ch + boff), b_l = desc_sw128_kmajor(cl + boff);
              umma_bf16(d, a_h, b_h, id_s, (kb | k) != 0);
              umma_bf16(d, a_h, b_l, id_s, 1);
              umma_bf16(d, a_l, b_h, id_s, 1);
            }
            umma_commit(&ctl.empty[s]);
          }
          if (!ok) break;
          umma_commit(&ctl.sfull[nt]);
          ++suse[nt];
        }
        ++nb;
      }
    }
  } else if (warp < 4) {
    // split the FP32 X tile of every analysis stage into bf16 hi/lo, K-major [c][jh]; every
    // stage (analysis or synthesis) is released to the MMA issuer through fullB (not used
    // with XS: the spectra arrive split)
    const int pt = threadIdx.x - 64;
    int it = 0;
    bool ok = !XS;
    for (int r = 0; r < rounds && ok; ++r) {
      const int w = heat_work(r, blockIdx.x, G);
      if (w >= ha.nwork) continue;
      const int blk = ha.order[w];
      const int M = ha.M[blk];
      const int nmt = (M + kBM - 1) / kBM, nkbS = (M + kBK - 1) / kBK;
      for (int mt = 0; mt < nmt && ok; ++mt)
        for (int kb = 0; kb < nkbA; ++kb, ++it) {
          const int s = it % kStages, n = it / kStages;
          if (!(ok = mbar_wait(&ctl.full[s], n & 1, abort))) break;
          split_x_mn(reinterpret_cast<const float*>(sX(s)), nmma, ha.ncols, kb * kBK, nh, sB_hi(s), sB_lo(s), pt);
          fence_async_smem();
          mbar_arrive(&ctl.fullB[s]);
        }
      // synthesis stages carry no X, but every stage completes one fullB phase, so that the
      // phase count of each stage's barriers stays the same for every role
      for (int k = 0; k < nnt * nkbS && ok; ++k, ++it) {
        const int s = it % kStages, n = it / kStages;
        if (!(ok = mbar_wait(&ctl.full[s], n & 1, abort))) break;
        mbar_arrive(&ctl.fullB[s]);
      }
    }
  } else {
    // epilogue: coefficients into shared memory, then the synthesis output to Y
    const int q = warp - 4;   // TMEM lane quadrant
    int ause[kMaxSlots] = {0}, suse[kMaxSlots] = {0};
    bool ok = true;
    for (int r = 0; r < rounds && ok; ++r) {
      const int w = heat_work(r, blockIdx.x, G);
      if (w >= ha.nwork) continue;
      const int blk = ha.order[w];
      const int M = ha.M[blk];
      const int m = blk >> 1, p = blk & 1;
      const int nmt = (M + kBM - 1) / kBM, kext = ((M + kBK - 1) / kBK) * kBK;
      for (int mt = 0; mt < nmt; ++mt) {
        if (!(ok = mbar_wait_warp(&ctl.afull[mt], ause[mt] & 1, abort))) break;
        tc_fence_after();
        const uint32_t d = taddr + (uint32_t)(mt * ncols_alloc) + ((uint32_t)(q * 32) << 16);
        const int i = mt * kBM + q * 32 + lane;   // degree row within the block
        const float hl = (i < M) ? (ha.h ? ha.h[m + p + 2 * i] : 1.f) : 0.f;
        const uint32_t cb = (uint32_t)((i >> 6) * cbytes);
        for (int c0 = 0; c0 < nmma; c0 += 16) {
          float v[16];
          tmem_ld16(d + (uint32_t)c0, v);
          if (i < kext) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int c = c0 + e;
              float val = 0.f;
              if (c < ha.ncols) val = v[e] * hl;
              const __nv_bfloat16 hi = __float2bfloat16_rn(val);
              const __nv_bfloat16 lo = __float2bfloat16_rn(val - __bfloat162float(hi));
              const uint32_t o = cb + sw128_offset(c, i & 63);
              *reinterpret_cast<__nv_bfloat16*>(cbuf_hi + o) = hi;
              *reinterpret_cast<__nv_bfloat16*>(cbuf_lo + o) = lo;
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&ctl.aempty[mt]);
        ++ause[mt];
      }
      if (!ok) break;
      fence_async_smem();   // the generic-proxy writes of C become visible to the MMAs
      mbar_arrive(&ctl.cready);
      for (int nt = 0; nt < nnt; ++nt) {
        if (!(ok = mbar_wait_warp(&ctl.sfull[nt], suse[nt] & 1, abort))) break;
        tc_fence_after();
        const int slot = ha.nmt_max + nt;
        const uint32_t d = taddr + (uint32_t)(slot * ncols_alloc) + ((uint32_t)(q * 32) << 16);
        const int jh = nt * kBM + q * 32 + lane;
        float* yrow = ha.Y + ((size_t)blk * nh + jh) * ha.ldc;
        for (int c0 = 0; c0 < nmma; c0 += 16) {
          float v[16];
          tmem_ld16(d + (uint32_t)c0, v);
          if (jh < nh) {
            if (c0 + 16 <= ha.ncols) {
#pragma unroll
              for (int e = 0; e < 16; e += 4)
                *reinterpret_cast<float4*>(yrow + c0 + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
            } else {
#pragma unroll
              for (int e = 0; e < 16; ++e)
                if (c0 + e < ha.ncols) yrow[c0 + e] = v[e];
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&ctl.sempty[nt]);
        ++suse[nt];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(taddr, 512);
  }
  if (threadIdx.x == 0 && ctl.abort) atomicExch(ha.err, SHOT_ERR_TIMEOUT);
}

// ---------------------------------------------------------------------------------
// Merged heat kernel: each persistent CTA owns whole (m, p) blocks and runs both contractions
// for them, the coefficients C^T going through global memory (L2) as in the two-kernel path:
//   analysis  C^T = h_l Pbar X   (block b's table rows from DRAM, the split spectra operand
//                                 built by eight converter warps as in k_legendre_tc)
//   synthesis Y = Pbar^T C       (the same table rows again, shortly after: from L2)
// Units run in the order A1, A2, S1, A3, S2, ..., Ak, S(k-1), Sk (A = analysis of a block,
// S = its synthesis), so that the write-back of a block's coefficients (epilogue -> global ->
// TMA) is hidden behind the next block's analysis.  The producer loads a synthesis unit's C^T
// only after the epilogue has stored it: the epilogue threads fence their global stores for the
// async proxy and arrive on cready[i & 1] (two barriers alternate, so a producer wait never
// sees a phase two blocks ahead).  Up to 32 fields ([B_hi | B_lo] as one operand of N = 128).
struct MergedArgs {
  const int* order;   // blocks with rows, largest first
  int nwork;
  const int* M;
  const long long* row_off;
  int nh, ldc, ncols, nmma;
  const float* h;                 // h_l
  __nv_bfloat16* ct_hi;           // C^T [blk][nmma_cap][ldi] (hi, lo)
  __nv_bfloat16* ct_lo;
  int nmma_cap, ldi;
  float* Y;                       // [blk][jh][ldc]
  int* err;
};

struct MergedSmem {
  uint64_t full[kMaxStages], empty[kMaxStages];
  uint64_t fullB[3], bempty[3];   // split spectra ring
  uint64_t tfull[2], tempty[2];
  uint64_t cready[2];
  uint32_t tmem;
  int abort;
};

// unit u of a CTA with k blocks: (block index within the CTA's list, synthesis?)
__device__ __forceinline__ void merged_unit(int u, int k, int& i, bool& syn) {
  if (u == 0) { i = 0; syn = false; }
  else if (u == 2 * k - 1) { i = k - 1; syn = true; }
  else if (u & 1) { i = (u + 1) / 2; syn = false; }
  else { i = u / 2 - 1; syn = true; }
}

constexpr int kMgConvWarps = 8;
constexpr int kMgThreads = 32 * (2 + kMgConvWarps + 4);
constexpr int kMgBR = 3;

template <int kStages>
__global__ void __launch_bounds__(kMgThreads, 1) k_heat_merged(
    const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,   // table, 128-row boxes
    const __grid_constant__ CUtensorMap ts_hi, const __grid_constant__ CUtensorMap ts_lo,   // table, 64-row boxes
    const __grid_constant__ CUtensorMap tx,                                                  // FP32 spectra
    const __grid_constant__ CUtensorMap tc_hi, const __grid_constant__ CUtensorMap tc_lo,   // C^T
    MergedArgs a) {
  extern __shared__ uint8_t smraw[];
  __shared__ MergedSmem ctl;
  uint8_t* base = align1k(smraw);
  const int nmma = a.nmma, nh = a.nh;
  const int bbytes = mn_atoms(nmma) * kXsBoxBytes;   // analysis B atoms (hi or lo)
  const int xbytes = nmma * kBK * 4;                 // FP32 spectra tile = synthesis C^T hi + lo
  const int sbytes = 2 * kATileBytes + xbytes;
  auto sA_hi = [&](int s) { return base + s * sbytes; };
  auto sA_lo = [&](int s) { return base + s * sbytes + kATileBytes; };
  auto sX = [&](int s) { return base + s * sbytes + 2 * kATileBytes; };   // ana: X; syn: C^T hi then lo
  uint8_t* sB = base + kStages * sbytes;                                   // ring: [hi atoms][lo atoms]
  const int ncat = 2 * 64 * mn_atoms(nmma);
  const uint32_t ncols_alloc = tmem_cols_for(ncat);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kConv = 32 * kMgConvWarps;
  constexpr int kEpiWarp0 = 2 + kMgConvWarps;
  const int G = gridDim.x;
  const int rounds = (a.nwork + G - 1) / G;
  int kblk = 0;   // blocks of this CTA
  for (int r = 0; r < rounds; ++r)
    if (heat_work(r, blockIdx.x, G) < a.nwork) ++kblk;
  auto blk_of = [&](int i) { return a.order[heat_work(i, blockIdx.x, G)]; };
  const int nunits = 2 * kblk;
  const int nkbA = (nh + kBK - 1) / kBK;
  const int nnt = (nh + kBM - 1) / kBM;

  for (int o = threadIdx.x * 16; o < kMgBR * 2 * bbytes; o += blockDim.x * 16)   // pad columns stay zero
    *reinterpret_cast<uint4*>(sB + o) = make_uint4(0, 0, 0, 0);
  fence_async_smem();
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&ctl.full[s], 1);
      mbar_init(&ctl.empty[s], 1);
    }
    for (int b = 0; b < kMgBR; ++b) {
      mbar_init(&ctl.fullB[b], kConv);
      mbar_init(&ctl.bempty[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl.tfull[b], 1);
      mbar_init(&ctl.tempty[b], 128);
      mbar_init(&ctl.cready[b], 128);
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

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int it = 0;
      bool ok = true;
      for (int u = 0; u < nunits && ok; ++u) {
        int i;
        bool syn;
        merged_unit(u, kblk, i, syn);
        const int blk = blk_of(i), M = a.M[blk], ro = (int)a.row_off[blk];
        if (!syn) {
          const int nmt = (M + kBM - 1) / kBM;
          for (int mt = 0; mt < nmt && ok; ++mt)
            for (int kb = 0; kb < nkbA; ++kb, ++it) {
              const int s = it % kStages, n = it / kStages;
              if (it >= kStages && !(ok = mbar_wait(&ctl.empty[s], (n - 1) & 1, abort))) break;
              mbar_arrive_expect_tx(&ctl.full[s], 2 * kATileBytes + xbytes);
              tma_load_2d(sA_hi(s), &ta_hi, &ctl.full[s], kb * kBK, ro + mt * kBM);
              tma_load_2d(sA_lo(s), &ta_lo, &ctl.full[s], kb * kBK, ro + mt * kBM);
              tma_load_2d(sX(s), &tx, &ctl.full[s], 0, blk * nh + kb * kBK);
            }
        } else {
          // the block's coefficients are in global memory once its analysis epilogue arrived
          if (!(ok = mbar_wait(&ctl.cready[i & 1], (i >> 1) & 1, abort))) break;
          asm volatile("fence.proxy.async.global;" ::: "memory");
          const int nkbS = (M + kBK - 1) / kBK;
          for (int nt = 0; nt < nnt && ok; ++nt)
            for (int kb = 0; kb < nkbS; ++kb, ++it) {
              const int s = it % kStages, n = it / kStages;
              if (it >= kStages && !(ok = mbar_wait(&ctl.empty[s], (n - 1) & 1, abort))) break;
              mbar_arrive_expect_tx(&ctl.full[s], 2 * kATileBytes + xbytes);
              const int y = ro + kb * kBK, x = nt * kBM;
              tma_load_2d(sA_hi(s), &ts_hi, &ctl.full[s], x, y);
              tma_load_2d(sA_hi(s) + kATileBytes / 2, &ts_hi, &ctl.full[s], x + 64, y);
              tma_load_2d(sA_lo(s), &ts_lo, &ctl.full[s], x, y);
              tma_load_2d(sA_lo(s) + kATileBytes / 2, &ts_lo, &ctl.full[s], x + 64, y);
              tma_load_2d(sX(s), &tc_hi, &ctl.full[s], kb * kBK, blk * a.nmma_cap);
              tma_load_2d(sX(s) + nmma * kBK * 2, &tc_lo, &ctl.full[s], kb * kBK, blk * a.nmma_cap);
            }
        }
      }
      for (int k = it > kStages ? it - kStages : 0; k < it; ++k)
        mbar_drain(&ctl.full[k % kStages], (k / kStages) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t id_ana = idesc_bf16(kBM, nmma) | (1u << 16);   // B MN-major
      const uint32_t id_cat = idesc_bf16(kBM, ncat) | (1u << 16);
      const uint32_t id_syn = idesc_bf16_amn(kBM, nmma);            // A MN-major
      int it = 0, ia = 0, lt = 0;
      bool ok = true;
      for (int u = 0; u < nunits && ok; ++u) {
        int i;
        bool syn;
        merged_unit(u, kblk, i, syn);
        const int blk = blk_of(i), M = a.M[blk];
        const int ntile = syn ? nnt : (M + kBM - 1) / kBM;
        const int nkb = syn ? (M + kBK - 1) / kBK : nkbA;
        for (int tile = 0; tile < ntile && ok; ++tile, ++lt) {
          const int acc = lt & 1, uu = lt >> 1;
          if (lt >= 2 && !(ok = mbar_wait(&ctl.tempty[acc], (uu - 1) & 1, abort))) break;
          tc_fence_after();
          const uint32_t d = taddr + (uint32_t)(acc * ncols_alloc);
          for (int kb = 0; kb < nkb; ++kb, ++it) {
            const int s = it % kStages, n = it / kStages;
            const int sb = ia % kMgBR;
            ok = mbar_wait(&ctl.full[s], n & 1, abort);
            if (ok && !syn) ok = mbar_wait(&ctl.fullB[sb], (ia / kMgBR) & 1, abort);
            if (!ok) break;
            tc_fence_after();
            const uint32_t ah = smem_u32(sA_hi(s)), al = smem_u32(sA_lo(s));
            if (!syn) {
              const uint32_t bh = smem_u32(sB + sb * 2 * bbytes);
#pragma unroll
              for (int k = 0; k < kBK / 16; ++k) {
                const uint64_t b_cat = desc_sw128_mnmajor(bh + k * 2048, kXsBoxBytes, 1024);
                umma_bf16(d, desc_sw128_kmajor(ah + k * 32), b_cat, id_cat, (kb | k) != 0);
                umma_bf16(d, desc_sw128_kmajor(al + k * 32), b_cat, id_ana, 1);
              }
              umma_commit(&ctl.empty[s]);
              umma_commit(&ctl.bempty[sb]);
              ++ia;
            } else {
              const uint32_t bh = smem_u32(sX(s)), bl = bh + (uint32_t)(nmma * kBK * 2);
#pragma unroll
              for (int k = 0; k < kBK / 16; ++k) {
                const uint64_t a_h = desc_sw128_mnmajor(ah + k * 2048, kATileBytes / 2, 1024);
                const uint64_t a_l = desc_sw128_mnmajor(al + k * 2048, kATileBytes / 2, 1024);
                const uint64_t b_h = desc_sw128_kmajor(bh + k * 32), b_l = desc_sw128_kmajor(bl + k * 32);
                umma_bf16(d, a_h, b_h, id_syn, (kb | k) != 0);
                umma_bf16(d, a_h, b_l, id_syn, 1);
                umma_bf16(d, a_l, b_h, id_syn, 1);
              }
              umma_commit(&ctl.empty[s]);
            }
          }
          if (!ok) break;
          umma_commit(&ctl.tfull[acc]);
        }
      }
    }
  } else if (warp < kEpiWarp0) {
    // converters: the analysis stages' FP32 spectra tiles -> [B_hi | B_lo] ring buffers
    const int pt = threadIdx.x - 64;
    XConv xc;
    xc.init(nmma, a.ncols, pt, kConv);
    int it = 0, ia = 0;
    bool ok = true;
    for (int u = 0; u < nunits && ok; ++u) {
      int i;
      bool syn;
      merged_unit(u, kblk, i, syn);
      const int blk = blk_of(i), M = a.M[blk];
      if (syn) {   // the synthesis stages take their operands straight from TMA
        it += nnt * ((M + kBK - 1) / kBK);
        continue;
      }
      const int nmt = (M + kBM - 1) / kBM;
      for (int mt = 0; mt < nmt && ok; ++mt)
        for (int kb = 0; kb < nkbA; ++kb, ++it, ++ia) {
          const int s = it % kStages, n = it / kStages;
          const int sb = ia % kMgBR, nb = ia / kMgBR;
          if (!(ok = mbar_wait(&ctl.full[s], n & 1, abort))) break;
          if (nb > 0 && !(ok = mbar_wait(&ctl.bempty[sb], (nb - 1) & 1, abort))) break;
          uint8_t* bh = sB + sb * 2 * bbytes;
          xc.run(reinterpret_cast<const float*>(sX(s)), kb * kBK, nh, bh, bh + bbytes);
          fence_async_smem();
          mbar_arrive(&ctl.fullB[sb]);
        }
    }
  } else {
    // epilogue: analysis tiles -> C^T (bf16 hi/lo, global), synthesis tiles -> Y
    const int q = warp & 3;   // a warp reaches only TMEM lanes 32 (warp % 4) ..
    int lt = 0;
    bool ok = true;
    for (int u = 0; u < nunits && ok; ++u) {
      int i;
      bool syn;
      merged_unit(u, kblk, i, syn);
      const int blk = blk_of(i), M = a.M[blk];
      const int m = blk >> 1, p = blk & 1;
      const int ntile = syn ? nnt : (M + kBM - 1) / kBM;
      for (int tile = 0; tile < ntile; ++tile, ++lt) {
        const int acc = lt & 1, uu = lt >> 1;
        if (!(ok = mbar_wait_warp(&ctl.tfull[acc], uu & 1, abort))) break;
        tc_fence_after();
        const uint32_t d = taddr + (uint32_t)(acc * ncols_alloc) + ((uint32_t)(q * 32) << 16);
        const int row = tile * kBM + q * 32 + lane;
        if (!syn) {
          const float hl = (a.h && row < M) ? a.h[m + p + 2 * row] : 1.f;
          for (int c0 = 0; c0 < nmma; c0 += 16) {
            float v[16], w[16];
            tmem_ld16(d + (uint32_t)c0, v);
            tmem_ld16(d + (uint32_t)(ncat / 2 + c0), w);   // + A_hi B_lo
            if (row < M) {
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const int c = c0 + e;
                if (c < a.ncols) {
                  const float val = (v[e] + w[e]) * hl;
                  const __nv_bfloat16 hi = __float2bfloat16_rn(val);
                  const __nv_bfloat16 lo = __float2bfloat16_rn(val - __bfloat162float(hi));
                  const size_t o = ((size_t)blk * a.nmma_cap + c) * a.ldi + row;
                  a.ct_hi[o] = hi;
                  a.ct_lo[o] = lo;
                }
              }
            }
          }
        } else {
          float* yrow = a.Y + ((size_t)blk * nh + row) * a.ldc;
          for (int c0 = 0; c0 < nmma; c0 += 16) {
            float v[16];
            tmem_ld16(d + (uint32_t)c0, v);
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
      if (ok && !syn) {   // this block's C^T is stored: hand it to the producer's TMA loads
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
        mbar_arrive(&ctl.cready[i & 1]);
      }
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
                       bool apply_h, cudaStream_t st, int xsplit) {
  const Workspace& w = g.ws;
  const int nmma = tc_nmma(nf);
  if (nmma > 256 || nmma > w.nmma_cap) {
    set_error("BF16X3 path supports at most 128 fields per call");
    return SHOT_ERR_UNSUPPORTED;
  }
  int rc;
  AnaArgs aa{};
  SynArgs sa{};
  if (ana && !Cf && !xsplit && nmma <= 64 && g.ntiles_ana_t > 0 && g.ana_transposed) {
    // transposed analysis (fields on M, degree rows on N), C^T written by the epilogue
    constexpr int stages = 2;
    const size_t smem = 1024 + (size_t)stages * (2 * 256 * kBK * 2 + 2 * 2 * kXsBoxBytes + (size_t)nmma * kBK * 4);
    CUtensorMap mh, ml, mx;
    if ((rc = make_map(&mh, g.tab_hi, g.nh, g.rows_total, g.ldt, kRowBox))) return rc;
    if ((rc = make_map(&ml, g.tab_lo, g.nh, g.rows_total, g.ldt, kRowBox))) return rc;
    if ((rc = make_map_f32(&mx, X, ldc, (uint64_t)g.nblk * g.nh, ldc, nmma, kBK))) return rc;
    AnaTArgs ta{g.tiles_ana_t, g.ntiles_ana_t, g.row_off_d, g.M_d, g.nh, X, ldc, 2 * nf, nmma,
                apply_h ? g.h_d : nullptr, w.ct_hi, w.ct_lo, w.nmma_cap, g.ldi, w.dev_int + 4};
    SHOT_CUDA(cudaFuncSetAttribute(k_ana_tc_t<stages>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = g.ntiles_ana_t < g.num_sms ? g.ntiles_ana_t : g.num_sms;
    ProfScope prof(PK_ANALYSIS, st);
    count_launch();
    k_ana_tc_t<stages><<<grid, kTcThreads, smem, st>>>(mh, ml, mx, ta);
    SHOT_CUDA(cudaGetLastError());
  } else if (ana && xsplit) {
    // spectra already split (bf16 hi/lo [blk nh + jh][ldc]): B by TMA, four stages
    if (nmma > 64 || ldc % 8 != 0) {
      set_error("split spectra need at most 32 fields and ldc a multiple of 8");
      return SHOT_ERR_UNSUPPORTED;
    }
    const __nv_bfloat16* Xh = reinterpret_cast<const __nv_bfloat16*>(X);
    const __nv_bfloat16* Xl = Xh + (size_t)g.nblk * g.nh * ldc;
    constexpr int stages = 4;
    const size_t smem = 1024 + (size_t)stages * (2 * kATileBytes + 2 * kXsBoxBytes);
    CUtensorMap mh, ml, xh, xl;
    if ((rc = make_map(&mh, g.tab_hi, g.nh, g.rows_total, g.ldt, kBM))) return rc;
    if ((rc = make_map(&ml, g.tab_lo, g.nh, g.rows_total, g.ldt, kBM))) return rc;
    if ((rc = make_map(&xh, Xh, ldc, (uint64_t)g.nblk * g.nh, ldc, kBK))) return rc;
    if ((rc = make_map(&xl, Xl, ldc, (uint64_t)g.nblk * g.nh, ldc, kBK))) return rc;
    aa = AnaArgs{g.tiles_ana, g.ntiles_ana, g.M_d, g.row_off_d, g.nh, nullptr, ldc, 2 * nf, nmma,
                 apply_h ? g.h_d : nullptr, w.ct_hi, w.ct_lo, w.nmma_cap, g.ldi, Cf, w.dev_int + 4};
    auto kern = k_legendre_tc<stages, true, true>;
    SHOT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int per_sm = (smem <= 113 * 1024 && 2 * 2 * host_tmem_cols(nmma) <= 512) ? 2 : 1;
    const int grid = g.ntiles_ana < per_sm * g.num_sms ? g.ntiles_ana : per_sm * g.num_sms;
    ProfScope prof(PK_ANALYSIS, st);
    count_launch();
    kern<<<grid, kTcThreads, smem, st>>>(mh, ml, xh, xl, aa, sa);
    SHOT_CUDA(cudaGetLastError());
  } else if (ana) {
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
                 apply_h ? g.h_d : nullptr, w.ct_hi, w.ct_lo, w.nmma_cap, g.ldi, Cf, w.dev_int + 4};
    // [B_hi | B_lo] as one operand up to 128 columns (N = 2 x 64 x atoms <= 256)
    const bool bcat = 2 * 64 * mn_atoms(nmma) <= 256;
    auto kern = bcat ? (br == 3 ? (stages == 4   ? k_legendre_tc<4, true, false, 3, true>
                                   : stages == 3 ? k_legendre_tc<3, true, false, 3, true>
                                   : stages == 2 ? k_legendre_tc<2, true, false, 3, true>
                                                 : k_legendre_tc<1, true, false, 3, true>)
                                : (stages == 4   ? k_legendre_tc<4, true, false, 2, true>
                                   : stages == 3 ? k_legendre_tc<3, true, false, 2, true>
                                   : stages == 2 ? k_legendre_tc<2, true, false, 2, true>
                                                 : k_legendre_tc<1, true, false, 2, true>))
                     : (br == 3 ? (stages == 4   ? k_legendre_tc<4, true, false, 3>
                                   : stages == 3 ? k_legendre_tc<3, true, false, 3>
                                   : stages == 2 ? k_legendre_tc<2, true, false, 3>
                                                 : k_legendre_tc<1, true, false, 3>)
                                : (stages == 4   ? k_legendre_tc<4, true, false, 2>
                                   : stages == 3 ? k_legendre_tc<3, true, false, 2>
                                   : stages == 2 ? k_legendre_tc<2, true, false, 2>
                                                 : k_legendre_tc<1, true, false, 2>));
    SHOT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // CTAs per SM: both shared memory and the 512 TMEM columns (two accumulators each) must fit
    const int acc_cols = host_tmem_cols(bcat ? 2 * 64 * mn_atoms(nmma) : nmma);
    const int per_sm = (smem <= 113 * 1024 && 2 * 2 * acc_cols <= 512) ? 2 : 1;
    const int grid = g.ntiles_ana < per_sm * g.num_sms ? g.ntiles_ana : per_sm * g.num_sms;
    ProfScope prof(PK_ANALYSIS, st);
    count_launch();
    kern<<<grid, tc_threads<true, false>(), smem, st>>>(mh, ml, mx, mx, aa, sa);
    SHOT_CUDA(cudaGetLastError());
  }
  if (syn) {
    const size_t smem = tc_smem_bytes(nmma, false, kStagesSyn);
    CUtensorMap ah, al, bh, bl;
    if ((rc = make_map(&ah, g.tab_hi, g.nh, g.rows_total, g.ldt, 64))) return rc;
    if ((rc = make_map(&al, g.tab_lo, g.nh, g.rows_total, g.ldt, 64))) return rc;
    if ((rc = make_map(&bh, w.ct_hi, g.ldi, (uint64_t)g.nblk * w.nmma_cap, g.ldi, nmma))) return rc;
    if ((rc = make_map(&bl, w.ct_lo, g.ldi, (uint64_t)g.nblk * w.nmma_cap, g.ldi, nmma))) return rc;
    sa = SynArgs{g.tiles_syn, g.ntiles_syn, g.M_d, g.row_off_d, g.nh, nmma, w.nmma_cap, 2 * nf, ldc, Y, w.dev_int + 4};
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

// Fused analysis + synthesis (k_heat_tc) for the solver's heat applications.  Returns
// SHOT_ERR_UNSUPPORTED (without launching) when the configuration does not fit: more than
// 32 fields, TMEM slots, or shared memory; the caller then runs the two-kernel path.
int launch_heat_tc(const Grid& g, int nf, const float* X, float* Y, int ldc, cudaStream_t st, int xsplit) {
  const Workspace& w = g.ws;
  const int nmma = tc_nmma(nf);
  if (nmma > 64 || g.nwork == 0) return SHOT_ERR_UNSUPPORTED;
  const int ncols_alloc = host_tmem_cols(nmma);
  const int nnt = (g.nh + kBM - 1) / kBM;
  if (g.nmt_max + nnt > 512 / ncols_alloc || g.nmt_max + nnt > kMaxSlots) return SHOT_ERR_UNSUPPORTED;
  if (xsplit && ldc % 8 != 0) return SHOT_ERR_UNSUPPORTED;
  const size_t sbytes = 2 * kATileBytes + 2 * (size_t)mn_atoms(nmma) * kXsBoxBytes +
                        (xsplit ? 0 : (size_t)nmma * kBK * 4);
  const size_t cbytes = (size_t)nmma * 128;
  int stages = 3;
  while (stages > 2 && 1024 + stages * sbytes + 2 * g.kc_max * cbytes > 227 * 1024) --stages;
  size_t smem = 1024 + stages * sbytes + 2 * g.kc_max * cbytes;
  if (smem > 227 * 1024) return SHOT_ERR_UNSUPPORTED;
  if (smem < 120 * 1024) smem = 120 * 1024;   // one CTA per SM: it allocates all 512 TMEM columns
  int rc;
  CUtensorMap mh, ml, mx, mx2;
  if ((rc = make_map(&mh, g.tab_hi, g.nh, g.rows_total, g.ldt, 64))) return rc;
  if ((rc = make_map(&ml, g.tab_lo, g.nh, g.rows_total, g.ldt, 64))) return rc;
  if (xsplit) {
    const __nv_bfloat16* Xh = reinterpret_cast<const __nv_bfloat16*>(X);
    const __nv_bfloat16* Xl = Xh + (size_t)g.nblk * g.nh * ldc;
    if ((rc = make_map(&mx, Xh, ldc, (uint64_t)g.nblk * g.nh, ldc, kBK))) return rc;
    if ((rc = make_map(&mx2, Xl, ldc, (uint64_t)g.nblk * g.nh, ldc, kBK))) return rc;
  } else {
    if ((rc = make_map_f32(&mx, X, ldc, (uint64_t)g.nblk * g.nh, ldc, nmma, kBK))) return rc;
    mx2 = mx;
  }
  HeatArgs ha{g.blk_order_d, g.nwork, g.M_d, g.row_off_d, g.nh, ldc, 2 * nf, nmma, g.nmt_max, g.kc_max,
              g.h_d, Y, w.dev_int + 4};
  auto kern = xsplit ? (stages == 3 ? k_heat_tc<3, true> : k_heat_tc<2, true>)
                     : (stages == 3 ? k_heat_tc<3, false> : k_heat_tc<2, false>);
  SHOT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = g.nwork < g.num_sms ? g.nwork : g.num_sms;
  ProfScope prof(PK_ANALYSIS, st);
  count_launch();
  kern<<<grid, kTcThreads, smem, st>>>(mh, ml, mx, mx2, ha);
  SHOT_CUDA(cudaGetLastError());
  return SHOT_OK;
}

// Merged heat kernel (k_heat_merged) for the BF16X3 heat applications, up to 32 fields with
// FP32 spectra.  Returns SHOT_ERR_UNSUPPORTED (without launching) otherwise.
int launch_heat_merged(const Grid& g, int nf, const float* X, float* Y, int ldc, cudaStream_t st) {
  const Workspace& w = g.ws;
  const int nmma = tc_nmma(nf);
  if (nmma > 64 || g.nwork == 0 || nmma > w.nmma_cap) return SHOT_ERR_UNSUPPORTED;
  const size_t sbytes = 2 * kATileBytes + (size_t)nmma * kBK * 4;
  const size_t ring = (size_t)kMgBR * 2 * mn_atoms(nmma) * kXsBoxBytes;
  int stages = kMaxStages;
  while (stages > 2 && 1024 + stages * sbytes + ring + 2048 > 227 * 1024) --stages;
  const size_t smem = 1024 + stages * sbytes + ring;
  if (smem + 2048 > 227 * 1024) return SHOT_ERR_UNSUPPORTED;
  int rc;
  CUtensorMap ah, al, sh, sl, mx, ch, cl;
  if ((rc = make_map(&ah, g.tab_hi, g.nh, g.rows_total, g.ldt, kBM))) return rc;
  if ((rc = make_map(&al, g.tab_lo, g.nh, g.rows_total, g.ldt, kBM))) return rc;
  if ((rc = make_map(&sh, g.tab_hi, g.nh, g.rows_total, g.ldt, 64))) return rc;
  if ((rc = make_map(&sl, g.tab_lo, g.nh, g.rows_total, g.ldt, 64))) return rc;
  if ((rc = make_map_f32(&mx, X, ldc, (uint64_t)g.nblk * g.nh, ldc, nmma, kBK))) return rc;
  if ((rc = make_map(&ch, w.ct_hi, g.ldi, (uint64_t)g.nblk * w.nmma_cap, g.ldi, nmma))) return rc;
  if ((rc = make_map(&cl, w.ct_lo, g.ldi, (uint64_t)g.nblk * w.nmma_cap, g.ldi, nmma))) return rc;
  MergedArgs ma{g.blk_order_d, g.nwork, g.M_d, g.row_off_d, g.nh, ldc, 2 * nf, nmma, g.h_d,
                w.ct_hi, w.ct_lo, w.nmma_cap, g.ldi, Y, w.dev_int + 4};
  auto kern = stages == 4 ? k_heat_merged<4> : stages == 3 ? k_heat_merged<3> : k_heat_merged<2>;
  SHOT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = g.nwork < g.num_sms ? g.nwork : g.num_sms;
  ProfScope prof(PK_ANALYSIS, st);
  count_launch();
  kern<<<grid, kMgThreads, smem, st>>>(ah, al, sh, sl, mx, ch, cl, ma);
  SHOT_CUDA(cudaGetLastError());
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
