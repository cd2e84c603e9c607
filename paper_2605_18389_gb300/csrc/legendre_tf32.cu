// Per-order Legendre contractions on the tensor cores in split TF32 (TF32x3).
//
// Same contractions as the other paths (App. C.1 semi-naive SHT; Sec. 3.2 h_l scaling):
//   analysis   C[i][c] = h_l sum_jh Pbar_lm(x_jh) X[jh][c]        (K = nodes jh)
//   synthesis  Y[jh][c] = sum_i Pbar_lm(x_jh) C[i][c]               (K = degrees i)
// Every FP32 operand v is split into two TF32 values, hi = v rounded to the nearest TF32 and
// lo = v - hi rounded likewise (|lo| <= 2^-11 |v|, either sign), both written to shared memory
// as exact TF32 values (the tensor core reads a 32-bit kind::tf32 operand by ignoring its 13
// low mantissa bits, checked bit for bit against operands written with the bits cleared, so a
// value that is not exact TF32 would be truncated).  The product is accumulated in FP32 in
// tensor memory as A_hi B_hi + A_hi B_lo + A_lo B_hi (tcgen05.mma kind::tf32, K = 8 per
// instruction); the rounding of lo (<= 2^-22 |v|) and the dropped lo*lo term (<= 2^-22 |AB|)
// leave ~2^-21 relative error per product, of either sign, against ~2^-16 for BF16x3.  The
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
//
// Recurrence mode (SHOT_RECURRENCE): no table.  The grid keeps checkpoints (a quarter of one
// table's entries: O(n^{3/2}) memory with a small constant, not the FP32 path's O(n)), for
// each parity par, Pbar at the degrees (m + 16 s + par, m + 16 s + par + 2) of every order m and
// north-hemisphere node (FP64 recurrence of App. B, rounded to FP32; four values per 16 degrees),
// and the same-parity two-step form of App. B's recurrence,
// P_{l+2} = (A x^2 + B) P_l + C P_{l-2}, as FP32 coefficients (A, B, C) per degree.  A stage's
// checkpoint box (of its parity) comes by TMA and its coefficient slice by a bulk copy with the
// spectra (analysis) or C^T (synthesis) tile into the input ring, and the split warps regenerate
// the A tile of a stage of generated operands
// in FP32, at most 6 two-degree steps from a checkpoint, writing the values' TF32 hi and lo
// straight into the swizzled K-major operand:
//   analysis  A = [128 degree rows of block (m, p)][32 nodes]: eight of the split warps, a thread
//             per (node pair, 16-degree segment), 16 segments per tile, a half-warp's 16 lanes
//             the 32 nodes of one row; the other eight split X^T meanwhile;
//   synthesis A = [128 nodes][32 degree rows]: a thread per (node, segment), 4 segments per
//             stage, each segment's 8 rows of the block's parity stored as two 16-byte chunks.
// The FP32 two-step recurrence over at most 6 steps from FP32-rounded checkpoints carries
// ~1e-7 rms error relative to each order's largest value (6e-6 at worst near the turning
// degrees), the level of the FP32 table it replaces.
// Warp roles: 0 TMA producer, 1 MMA issuer, 2-17 split (sixteen warps, four per SM
// sub-partition, so that the split and recurrence arithmetic, which bounds the kernel, hides
// its latencies), 18-21 epilogue over a double-buffered accumulator
// (a warp reads the TMEM lane quadrant warp % 4).  Every mbarrier wait
// is bounded; on expiry the CTA records SHOT_ERR_TIMEOUT and still frees its tensor memory.
#include "tc_ptx.cuh"

namespace shot {
namespace {

constexpr int kSplitWarps = 16;                  // warps 2..17 (four per SM sub-partition)
constexpr int kSplitThreads = 32 * kSplitWarps;
// (one CTA of 16 split warps: 32 * (2 + 16 + 4) threads, the TMA, MMA and four epilogue warps besides)
constexpr int kTK = 32;                          // K per stage (one 128-byte row of FP32)
constexpr int kTTile = kBM * kTK * 4;            // 16 KB: 128 rows x 32 FP32
constexpr int kT32MaxStages = 4;
constexpr uint32_t kTf32Mask = 0xFFFFE000u;      // sign, exponent and 10 stored mantissa bits

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
constexpr uint32_t kTf32Half = 0x00001000u;
__device__ __forceinline__ float tf32_rn(float v) {
  return __uint_as_float((__float_as_uint(v) + kTf32Half) & kTf32Mask);
}
// hi = rn(v), lo = rn(v - hi)
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

// Element-wise split of a tile (the swizzle does not matter as long as the three tiles share
// their 1024-byte phase): hi = rn(v), lo = rn(v - hi); hi may be the raw tile itself.  Each
// thread loads kSplitBatch chunks before it stores any, so the loads overlap.
constexpr int kSplitBatch = 2;   // 16 KB / (512 threads x 16 B) = 2 chunks per thread
template <int NT = kSplitThreads>   // split threads
__device__ __forceinline__ void split_tile(const uint8_t* raw, uint8_t* hi, uint8_t* lo, int nbytes, int pt) {
  for (int base = 0; base < nbytes; base += kSplitBatch * NT * 16) {
    float4 v[kSplitBatch];
#pragma unroll
    for (int i = 0; i < kSplitBatch; ++i) {
      const int o = base + (pt + i * NT) * 16;
      if (o < nbytes) v[i] = *reinterpret_cast<const float4*>(raw + o);
    }
#pragma unroll
    for (int i = 0; i < kSplitBatch; ++i) {
      const int o = base + (pt + i * NT) * 16;
      if (o < nbytes) {
        const float w[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
        float4 h, l;
        tf32_split4(w, h, l);
        *reinterpret_cast<float4*>(hi + o) = h;
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
                                         uint8_t* bl, int pt, int nthr) {
  const int ntask = nmma * (kTK / 4);
  for (int e0 = pt; e0 < ntask; e0 += 2 * nthr) {
    float v[2][4];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int e = e0 + b * nthr;
      const int c = e % nmma, k4 = (e / nmma) * 4;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        v[b][q] = (e < ntask && c < ncols && jh0 + k4 + q < nh) ? xs[(k4 + q) * nmma + c] : 0.f;
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int e = e0 + b * nthr;
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
constexpr int kXtTasks = 2;   // nmma x 8 tasks <= 2 x threads (wider batches take split_xt's loop)
struct XtPlan {
  int c[kXtTasks];         // column (-1: no task)
  int k4[kXtTasks];        // first of the task's four nodes within the 32-node chunk
  uint32_t o[kXtTasks];    // byte offset of the 16-byte chunk in the hi (and lo) tile
  __device__ __forceinline__ void init(int nmma, int pt, int nthr) {
    const int ntask = nmma * (kTK / 4);
#pragma unroll
    for (int i = 0; i < kXtTasks; ++i) {
      const int e = pt + i * nthr;
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
  long long wait;             // limit of every bounded wait (SM clock cycles)
  // recurrence mode
  const long long* ck_off;    // first checkpoint row of order m (in either parity plane)
  long long ck_rows;          // rows per parity plane
  const float4* coef;         // two-step coefficients (A, B, C, 0) of degree l at m * cstride + (l - m),
                              // zero past l = lmax
  int cstride;
  const float* xnode;         // x_jh^2 in FP32
  int nin;                    // input ring depth (REC)
  int lmax;
};

// Recurrence mode: checkpoint segments of 16 degrees; per stage a checkpoint box and the
// stage's coefficient slice arrive with the spectra / C^T tile.
constexpr int kSeg = 16;
constexpr int kAnaSegs = 2 * kBM / kSeg;             // 16 segments cover a 128-row tile of one parity
constexpr int kSynSegs = 2 * kTK / kSeg;             // 4 segments cover a 32-row K chunk
constexpr int kCkBytes = kAnaSegs * kTK * 8;         // analysis box: 16 segments x 32 nodes x 2 values
static_assert(kCkBytes == kSynSegs * kBM * 8, "both checkpoint boxes are 4 KB");
constexpr int kCfAna = 2 * kBM;                      // coefficients per analysis stage (its tile's degrees)
constexpr int kCfSyn = 2 * kTK;                      // coefficients per synthesis stage (its K chunk's degrees)
constexpr int kCfBytes = kCfAna * 16;                // room for either slice
constexpr int kMaxIn = 8;                            // deepest input ring
static_assert(kMaxIn <= (int)(sizeof(TcSmem::infull) / sizeof(uint64_t)), "input ring barriers");

// One 16-degree segment of the recurrence at one node, all of the parity par: it starts from
// its checkpoint ck = (P_{d0+par}, P_{d0+par+2}) and steps two degrees at a time by the
// same-parity form of App. B's recurrence,
//   P_{l+2} = (A x^2 + B) P_l + C P_{l-2},
//   A = a_{l+2} a_{l+1},  B = -a_{l+2} (a_{l+1} b_{l+1} / a_l + b_{l+2}),  C = -a_{l+2} a_{l+1} b_{l+1} b_l
// (eliminate P_{l+1} and P_{l-1} from three consecutive steps), with (A, B, C) of degree
// d0 + par + 2k at cf[cb + 2k] (cb = d0 + par relative to the stage's coefficient slice).  The
// coefficients are zero past the order's last degree, so the values there come out zero and no
// step needs a bounds test.  emit(k, value) receives P_{d0 + par + 2k}, k = 0 .. 7.
template <class F>
__device__ __forceinline__ void rec_segment(float2 ck, float x2, const float4* cf, int cb, F&& emit) {
  float a0 = ck.x, b0 = ck.y;
  emit(0, a0);
  emit(1, b0);
#pragma unroll
  for (int k = 2; k < kSeg / 2; ++k) {
    const float4 e = cf[cb + 2 * k];
    const float c0 = fmaf(fmaf(e.x, x2, e.y), b0, e.z * a0);
    emit(k, c0);
    a0 = b0;
    b0 = c0;
  }
}

// The same segment at two nodes side by side (independent chains on the same coefficients):
// ck = (P_{d0+par}, P_{d0+par+2}) at node 0, then at node 1; x2 = (x0^2, x1^2); emit(k, v0, v1)
// receives P_{d0 + par + 2k} at both nodes.
template <class F>
__device__ __forceinline__ void rec_node_pair(float4 ck, float2 x2, const float4* cf, int cb, F&& emit) {
  float a0 = ck.x, b0 = ck.y, a1 = ck.z, b1 = ck.w;
  emit(0, a0, a1);
  emit(1, b0, b1);
#pragma unroll
  for (int k = 2; k < kSeg / 2; ++k) {
    const float4 e = cf[cb + 2 * k];
    const float c0 = fmaf(fmaf(e.x, x2.x, e.y), b0, e.z * a0);
    const float c1 = fmaf(fmaf(e.x, x2.y, e.y), b1, e.z * a1);
    emit(k, c0, c1);
    a0 = b0;
    b0 = c0;
    a1 = b1;
    b1 = c1;
  }
}

// Persistent, warp-specialised TF32x3 Legendre GEMM (roles in the file header).  Table mode:
// stage s holds [A hi][A lo][B hi][B lo][X raw (analysis)], A hi the raw table tile by TMA.
// Recurrence mode (REC) runs two rings, so that the TMA latency hides behind a deep ring of
// the small inputs while the large generated operands need only a few stages: kStages output
// stages [A hi][A lo][B hi][B lo] (written by the split warps, read by the MMAs) and a.nin
// input stages [X or C^T raw][checkpoint box][coefficient slice] (written by TMA, read by the
// split warps, released as soon as they are read), then x^2 of the nodes.
// SW split warps: 16 with one CTA per SM; 8 (table mode) with two CTAs per SM, whose independent
// pipelines hide each other's handshake and copy latencies.
template <int kStages, bool ANA, bool BCAT, bool REC = false, int SW = kSplitWarps>
__global__ void __launch_bounds__(32 * (2 + SW + 4), SW == 8 ? 2 : 1)
    k_legendre_tf32(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, T32Args a) {
  static_assert(SW == 16 || (SW == 8 && !REC), "the recurrence generators are laid out for 16 split warps");
  constexpr int kSW = SW, kST = 32 * SW;   // split warps, split threads
  extern __shared__ uint8_t smraw[];
  __shared__ TcSmem ctl;
  uint8_t* base = align1k(smraw);
  const int nmma = a.nmma, nh = a.nh;
  const int bbytes = nmma * kTK * 4;   // one B tile (hi or lo); the analysis X tile has the same size
  const int sbytes = 2 * kTTile + (REC ? 2 : (ANA ? 3 : 2)) * bbytes;   // one (output) stage
  const int ibytes = bbytes + kCkBytes + kCfBytes;                         // one REC input stage
  uint8_t* ibase = base + kStages * sbytes;
  auto sA_hi = [&](int s) { return base + s * sbytes; };
  auto sA_lo = [&](int s) { return base + s * sbytes + kTTile; };
  auto sB_hi = [&](int s) { return base + s * sbytes + 2 * kTTile; };
  auto sB_lo = [&](int s) { return base + s * sbytes + 2 * kTTile + bbytes; };
  // analysis X raw: the table-mode stage's fifth tile, or the REC input stage's first
  auto sIn = [&](int i) { return ibase + i * ibytes; };   // REC: the input stage's X or C^T raw tile
  auto sX = [&](int s) { return REC ? sIn(s) : base + s * sbytes + 2 * kTTile + 2 * bbytes; };
  auto sCk = [&](int i) { return reinterpret_cast<const float2*>(ibase + i * ibytes + bbytes); };
  auto sCf = [&](int i) { return reinterpret_cast<const float4*>(ibase + i * ibytes + bbytes + kCkBytes); };
  const int nin = REC ? a.nin : 1;
  float* sXn = reinterpret_cast<float*>(ibase + (REC ? nin * ibytes : 0));   // REC: x^2 of the nodes [nh]
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
      mbar_init(&ctl.fullB[s], kSW);   // one arrival per split warp
      mbar_init(&ctl.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl.tfull[b], 1);
      mbar_init(&ctl.tempty[b], 4);   // one arrival per epilogue warp
    }
    for (int i = 0; REC && i < nin; ++i) {
      mbar_init(&ctl.infull[i], 1);
      mbar_init(&ctl.inempty[i], kSW);
    }
    mbar_init(&ctl.drain, 1);
    ctl.abort = 0;
    fence_mbar_init();
  }
  if (REC)
    for (int j = threadIdx.x; j < nh; j += blockDim.x) sXn[j] = a.xnode[j];
  if (warp == 1) tmem_alloc(&ctl.tmem, 2 * ncols_alloc);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = ctl.tmem;
  volatile int* abort = &ctl.abort;
  const long long wl = a.wait;   // wait limit (cycles)
  auto nkb_of = [&](int blk) { return ANA ? (nh + kTK - 1) / kTK : (a.M[blk] + kTK - 1) / kTK; };

  if (warp == 0) {
    if (lane == 0) {  // TMA producer, runs ahead across tiles
      const int depth = REC ? nin : kStages;
      int it = 0, s = 0, ph = 0;   // slot of the ring and its phase parity, advanced by counting
      bool ok = true;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        const Tile tl = a.tiles[t];
        const int nkb = nkb_of(tl.blk);
        // checkpoint rows of order m in the plane of the tile's parity (planes of ck_rows rows)
        const long long ck_base = REC ? (tl.blk & 1) * a.ck_rows + a.ck_off[tl.blk >> 1] : 0;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          // REC fills the input ring (freed by the split warps), the table mode the stages (freed
          // by the MMAs)
          uint64_t* full = REC ? &ctl.infull[s] : &ctl.fullA[s];
          if (it >= depth && !(ok = mbar_wait(REC ? &ctl.inempty[s] : &ctl.empty[s], ph ^ 1, abort, wl))) break;
          mbar_arrive_expect_tx(full, (REC ? kCkBytes + (ANA ? kCfAna : kCfSyn) * 16 : kTTile) + bbytes);
          if (REC) {   // checkpoint box of the stage (segments x nodes), FP32 pairs, and coefficients
            const int m = tl.blk >> 1;
            uint8_t* ck = reinterpret_cast<uint8_t*>(const_cast<float2*>(sCk(s)));
            uint8_t* cf = reinterpret_cast<uint8_t*>(const_cast<float4*>(sCf(s)));
            // checkpoint plane of the tile's parity: rows ck_base (see the producer's tile set-up)
            if (ANA) {   // 16 segments of the tile's degrees 2 r0 .. 2 r0 + 255 x the 32 nodes of this chunk
              tma_load_2d(ck, &ta, full, 2 * kb * kTK, (int)(ck_base + tl.r0 / 8));
              bulk_load(cf, a.coef + (size_t)m * a.cstride + 2 * tl.r0, kCfAna * 16, full);
            } else {     // the 4 segments of this K chunk's degrees 64 kb .. 64 kb + 63 x the tile's 128 nodes
              tma_load_2d(ck, &ta, full, 2 * tl.r0, (int)(ck_base + kb * kSynSegs));
              bulk_load(cf, a.coef + (size_t)m * a.cstride + 2 * kb * kTK, kCfSyn * 16, full);
            }
          } else if (ANA) {   // table rows i of the tile x nodes of this K-chunk
            tma_load_2d(sA_hi(s), &ta, full, kb * kTK, (int)(a.row_off[tl.blk] + tl.r0));
          } else {     // transposed table: nodes of the tile x degrees of this K-chunk
            tma_load_2d(sA_hi(s), &ta, full, kb * kTK, tl.blk * nh + tl.r0);
          }
          if (ANA)     // spectra rows = nodes of this K chunk
            tma_load_2d(sX(s), &tb, full, 0, tl.blk * nh + kb * kTK);
          else         // C^T rows = columns, degrees of this K chunk
            tma_load_2d(REC ? sIn(s) : sB_hi(s), &tb, full, kb * kTK, tl.blk * a.nmma_cap);
          if (++s == depth) {
            s = 0;
            ph ^= 1;
          }
        }
      }
      // let this CTA's copies land before it can exit
      for (int k = it > depth ? it - depth : 0; k < it; ++k)
        mbar_drain(REC ? &ctl.infull[k % depth] : &ctl.fullA[k % depth], (k / depth) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer: waits until the split warps have written the stage's lo parts
      const uint32_t idesc = idesc_tf32(kBM, nmma), idesc2 = idesc_tf32(kBM, nacc);
      // operand descriptors: the start-address field is (address >> 4) in the low 14 bits (all
      // of shared memory fits), so every descriptor is the first stage's A hi descriptor plus
      // a constant: stage s at s sbytes, A lo / B hi / B lo at fixed offsets, K step k at 32 k
      // bytes; the issuer spends a few adds per MMA instead of rebuilding descriptors
      const uint64_t dbase = desc_sw128_kmajor(smem_u32(sA_hi(0)));
      const uint64_t d_al = (uint64_t)(kTTile >> 4), d_bh = (uint64_t)((2 * kTTile) >> 4);
      const uint64_t d_bl = d_bh + (uint64_t)(bbytes >> 4), d_stage = (uint64_t)(sbytes >> 4);
      int lt = 0, s = 0, ph = 0;
      uint64_t dstage = dbase;   // descriptor of stage s's A hi
      bool ok = true;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++lt) {
        const Tile tl = a.tiles[t];
        const int nkb = nkb_of(tl.blk);
        const int acc = lt & 1, u = lt >> 1;
        if (lt >= 2 && !(ok = mbar_wait(&ctl.tempty[acc], (u - 1) & 1, abort, wl))) break;
        tc_fence_after();
        const uint32_t d = taddr + (uint32_t)(acc * ncols_alloc);
        for (int kb = 0; kb < nkb; ++kb) {
          if (!(ok = mbar_wait(&ctl.fullB[s], ph, abort, wl))) break;
          tc_fence_after();
#pragma unroll
          for (int k = 0; k < kTK / 8; ++k) {   // 8 TF32 = 32 bytes per instruction
            const uint64_t off = dstage + (uint64_t)(2 * k);
            const uint64_t a_h = off, a_l = off + d_al, b_h = off + d_bh, b_l = off + d_bl;
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
          dstage += d_stage;
          if (++s == kStages) {
            s = 0;
            ph ^= 1;
            dstage = dbase;
          }
        }
        if (!ok) break;
        umma_commit(&ctl.tfull[acc]);
      }
      // every MMA issued here completes before the CTA frees its tensor memory (after an abort too)
      umma_commit(&ctl.drain);
      mbar_drain(&ctl.drain, 0);
    }
  } else if (warp < 2 + kSW) {
    // split warps: table tile -> lo (the raw tile is hi) or (REC) the regenerated A tile hi/lo;
    // analysis: X -> X^T hi/lo; synthesis: C^T -> hi/lo (in place in table mode)
    const int pt = threadIdx.x - 64;
    // REC analysis: split warps 0-7 regenerate A (node pairs), 8-15 split X^T; otherwise every
    // split warp does both parts.  bt / nbt: this thread among the X^T threads.
    constexpr bool kRoles = REC && ANA;
    constexpr int nbt = kRoles ? kST / 2 : kST;
    const bool agen = !kRoles || pt < kST / 2, bsplit = !kRoles || pt >= kST / 2;
    const int bt = kRoles ? pt - kST / 2 : pt;
    const bool pre = ANA && nmma * (kTK / 4) <= kXtTasks * nbt;
    XtPlan xp;
    xp.init(pre && bsplit ? nmma : 0, bt, nbt);
    const int gw = pt >> 5;   // split warp 0..15
    // it counts stages; s / ph: the stage written and its phase parity; i / iph: the REC input
    // slot and its phase (table mode: the stage itself), advanced by counting
    int it = 0, s = 0, ph = 0, i = 0, iph = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
      const Tile tl = a.tiles[t];
      const int nkb = nkb_of(tl.blk);
      const int m = tl.blk >> 1, par = tl.blk & 1;
      const int dmax = a.lmax - m;   // largest relative degree of order m
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        // REC: the inputs are in slot i of the input ring, and stage s must also be free (its
        // previous MMAs done).  Every thread waits (each must observe the copies' phase
        // itself); the outcome is made warp-uniform so that a warp leaves together and its
        // single arrivals below stay valid.
        if (!REC) i = s;
        bool w = REC ? mbar_wait(&ctl.infull[i], iph, abort, wl) : mbar_wait(&ctl.fullA[s], ph, abort, wl);
        if (REC && w && it >= kStages) w = mbar_wait(&ctl.empty[s], ph ^ 1, abort, wl);
        if (!(ok = __all_sync(0xffffffffu, w))) break;
        if (REC && ANA) {
          if (agen) {
            // thread = (node pair np of the K chunk, segment sr of the tile): nodes 2 np, 2 np + 1
            // run as two chains on the same coefficients; the degree of parity par
            // 2 r0 + 16 sr + 2 k + par is tile row 8 sr + k, the pair's columns one 8-byte store
            const int np = pt & 15, sr = pt >> 4;
            const int node = kb * kTK + 2 * np;
            const float2 x2 = make_float2(node < nh ? sXn[node] : 0.f, node + 1 < nh ? sXn[node + 1] : 0.f);
            const int d0 = 2 * tl.r0 + kSeg * sr;
            const float4 ck = d0 <= dmax ? reinterpret_cast<const float4*>(sCk(i))[(sr * kTK) / 2 + np]
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
            uint8_t* ah = sA_hi(s);
            uint8_t* al = sA_lo(s);
            rec_node_pair(ck, x2, sCf(i), kSeg * sr + par, [&](int k, float v0, float v1) {
              const uint32_t o = sw128_offset32(kSeg / 2 * sr + k, 2 * np);
              const float h0 = tf32_rn(v0), h1 = tf32_rn(v1);
              *reinterpret_cast<float2*>(ah + o) = make_float2(h0, h1);
              *reinterpret_cast<float2*>(al + o) = make_float2(tf32_rn(v0 - h0), tf32_rn(v1 - h1));
            });
          }
        } else if (REC) {
          // node tl.r0 + 32 (gw & 3) + lane (tile row); segment gw >> 2 of the K chunk (degrees
          // 64 kb + 16 sr ..): its 8 degrees of parity par are K positions 8 sr .. 8 sr + 7,
          // stored as two 16-byte chunks (zero past the order's last degree)
          const int row = 32 * (gw & 3) + lane;
          const int node = tl.r0 + row;
          const float x2 = node < nh ? sXn[node] : 0.f;
          const int sr = gw >> 2;
          const int d0 = 2 * kb * kTK + kSeg * sr;
          const float2 c = d0 <= dmax ? sCk(i)[sr * kBM + row] : make_float2(0.f, 0.f);
          float v[8];
          rec_segment(c, x2, sCf(i), kSeg * sr + par, [&](int k, float val) { v[k] = val; });
          uint8_t* ah = sA_hi(s);
          uint8_t* al = sA_lo(s);
          const float w0[4] = {v[0], v[1], v[2], v[3]};
          const float w1[4] = {v[4], v[5], v[6], v[7]};
          const uint32_t o0 = sw128_offset32(row, 8 * sr), o1 = sw128_offset32(row, 8 * sr + 4);
          float4 h0, l0, h1, l1;
          tf32_split4(w0, h0, l0);
          tf32_split4(w1, h1, l1);
          *reinterpret_cast<float4*>(ah + o0) = h0;
          *reinterpret_cast<float4*>(ah + o1) = h1;
          *reinterpret_cast<float4*>(al + o0) = l0;
          *reinterpret_cast<float4*>(al + o1) = l1;
        } else {
          split_tile<kST>(sA_hi(s), sA_hi(s), sA_lo(s), kTTile, pt);
        }
        if (ANA && pre && bsplit)
          xp.run(reinterpret_cast<const float*>(sX(i)), nmma, a.ncols, kb * kTK, nh, sB_hi(s), sB_lo(s));
        else if (ANA && bsplit)
          split_xt(reinterpret_cast<const float*>(sX(i)), nmma, a.ncols, kb * kTK, nh, sB_hi(s), sB_lo(s), bt, nbt);
        else if (!ANA)
          split_tile<kST>(REC ? sIn(i) : sB_hi(s), sB_hi(s), sB_lo(s), bbytes, pt);
        // one arrival per warp, after __syncwarp has ordered all its lanes' accesses before it
        if (REC) {   // inputs read: the producer may refill the slot
          __syncwarp();
          if (lane == 0) mbar_arrive(&ctl.inempty[i]);
        }
        fence_async_smem();   // this thread's operand writes, made visible to the tensor core
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl.fullB[s]);
        if (++s == kStages) {
          s = 0;
          ph ^= 1;
        }
        if (REC && ++i == nin) {
          i = 0;
          iph ^= 1;
        }
      }
    }
  } else {
    // epilogue: drain the accumulator of every tile of this CTA (a warp reads the TMEM lanes of its quadrant warp % 4)
    const int q = warp & 3;   // a warp reaches only TMEM lanes 32 (warp % 4) ..
    int lt = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++lt) {
      const Tile tl = a.tiles[t];
      const int acc = lt & 1, u = lt >> 1;
      if (!mbar_wait_warp(&ctl.tfull[acc], u & 1, abort, wl)) break;
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
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl.tempty[acc]);
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

// Recurrence mode, grid set-up: checkpoints of every order m, 16-degree segment s and
// north-hemisphere node, one plane per parity par: (Pbar_{m+16s+par}, Pbar_{m+16s+par+2}) by the
// FP64 recurrences of App. B (k_pbar's), rounded to FP32, at
// ck[(par * ck_rows + ck_off[m] + s) * ckld + 2 jh + {0, 1}]; degrees past lmax and nodes past nh
// stay zero (the buffer is cleared first).  Also x_jh^2 in FP32.
__global__ void k_ck_build(int lmax, int nh, const double* __restrict__ x, const long long* __restrict__ ck_off,
                           long long ck_rows, int ckld, float* __restrict__ ck, float* __restrict__ x2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (j >= nh) return;
  const double xj = x[j];
  if (m == 0) x2[j] = (float)(xj * xj);
  const double st = sqrt((1.0 - xj) * (1.0 + xj));
  double pmm = 0.28209479177387814;   // 1/sqrt(4 pi)
  for (int k = 1; k <= m; ++k) pmm *= -sqrt((2.0 * k + 1.0) / (2.0 * k)) * st;
  double p2 = 0.0, p1 = pmm;   // Pbar_{l-2}, Pbar_{l-1} entering degree l = m + 1
  for (int l = m; l <= lmax; ++l) {
    double pl;
    if (l == m) {
      pl = pmm;
    } else if (l == m + 1) {
      pl = sqrt(2.0 * m + 3.0) * xj * pmm;
    } else {
      const double ll = (double)l * l, mm = (double)m * m, l1 = (double)(l - 1) * (l - 1);
      pl = sqrt((4.0 * ll - 1.0) / (ll - mm)) * (xj * p1 - sqrt((l1 - mm) / (4.0 * l1 - 1.0)) * p2);
    }
    if (l > m) {
      p2 = p1;
      p1 = pl;
    }
    const int d = l - m, r = d % kSeg;
    if (r < 4) {   // offsets 0, 2 -> plane 0; 1, 3 -> plane 1; first or second value by r / 2
      const int par = r & 1;
      ck[((size_t)par * ck_rows + ck_off[m] + d / kSeg) * ckld + 2 * j + (r >> 1)] = (float)pl;
    }
  }
}

// Two-step coefficients (A, B, C, 0) of degree l (from l - 2 and l - 4) for m + 4 <= l <= lmax at
// m * cstride + (l - m), in FP64 from a_lm = sqrt((4l^2-1)/(l^2-m^2)), b_lm =
// sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)), rounded to FP32; the rest of the row stays zero (cleared
// first), so that the recurrence run past lmax gives zeros
__global__ void k_coef32_build(int lmax, int cstride, float4* __restrict__ coef) {
  const int m = blockIdx.x;
  auto al = [&](int l) {
    const double ll = (double)l * l, mm = (double)m * m;
    return sqrt((4.0 * ll - 1.0) / (ll - mm));
  };
  auto be = [&](int l) {
    const double mm = (double)m * m, l1 = (double)(l - 1) * (l - 1);
    return sqrt((l1 - mm) / (4.0 * l1 - 1.0));
  };
  for (int t = m + 4 + threadIdx.x; t <= lmax; t += blockDim.x) {
    const int l = t - 2;   // P_t = (A x^2 + B) P_l + C P_{l-2}
    const double A = al(l + 2) * al(l + 1);
    const double B = -al(l + 2) * (al(l + 1) * be(l + 1) / al(l) + be(l + 2));
    const double C = -al(l + 2) * al(l + 1) * be(l + 1) * be(l);
    coef[(size_t)m * cstride + (t - m)] = make_float4((float)A, (float)B, (float)C, 0.f);
  }
}

// dynamic shared memory of k_legendre_tf32: 1 KB alignment slack, the stages, and in recurrence
// mode the input ring and x^2 of the nodes
size_t tf32_smem_bytes(int nmma, bool ana, int stages, bool rec, int nin, int nh) {
  const size_t bb = (size_t)nmma * kTK * 4;
  if (!rec) return 1024 + (size_t)stages * (2 * kTTile + (ana ? 3 : 2) * bb);
  return 1024 + (size_t)stages * (2 * kTTile + 2 * bb) + (size_t)nin * (bb + kCkBytes + kCfBytes) +
         (size_t)((nh + 3) & ~3) * 4;
}

template <bool REC>
void* tf32_kernel(bool ana, bool bc, int stages, bool two_cta) {
  if constexpr (!REC) {
    if (two_cta) {   // 8 split warps, two CTAs per SM
#define SHOT_T32K8(S, A, B) reinterpret_cast<void*>(k_legendre_tf32<S, A, B, false, 8>)
      if (bc) {
        if (ana) return stages == 2 ? SHOT_T32K8(2, true, true) : SHOT_T32K8(1, true, true);
        return stages == 2 ? SHOT_T32K8(2, false, true) : SHOT_T32K8(1, false, true);
      }
      if (ana) return stages == 2 ? SHOT_T32K8(2, true, false) : SHOT_T32K8(1, true, false);
      return stages == 2 ? SHOT_T32K8(2, false, false) : SHOT_T32K8(1, false, false);
#undef SHOT_T32K8
    }
  }
#define SHOT_T32K(S, A, B) reinterpret_cast<void*>(k_legendre_tf32<S, A, B, REC>)
  if (bc) {
    if (ana) return stages == 4 ? SHOT_T32K(4, true, true) : stages == 3 ? SHOT_T32K(3, true, true)
                  : stages == 2 ? SHOT_T32K(2, true, true) : SHOT_T32K(1, true, true);
    return stages == 4 ? SHOT_T32K(4, false, true) : stages == 3 ? SHOT_T32K(3, false, true)
         : stages == 2 ? SHOT_T32K(2, false, true) : SHOT_T32K(1, false, true);
  }
  if (ana) return stages == 4 ? SHOT_T32K(4, true, false) : stages == 3 ? SHOT_T32K(3, true, false)
                : stages == 2 ? SHOT_T32K(2, true, false) : SHOT_T32K(1, true, false);
  return stages == 4 ? SHOT_T32K(4, false, false) : stages == 3 ? SHOT_T32K(3, false, false)
       : stages == 2 ? SHOT_T32K(2, false, false) : SHOT_T32K(1, false, false);
#undef SHOT_T32K
}

}  // namespace

int tf32_nmma(int nf) { return (2 * nf + 15) / 16 * 16; }

int build_tf32_recurrence(Grid& g, cudaStream_t st) {
  const int L = g.lmax + 1, nh = g.nh;
  std::vector<long long> ckoff(L + 1, 0);
  for (int m = 0; m < L; ++m) ckoff[m + 1] = ckoff[m] + (L - m + kSeg - 1) / kSeg;
  g.ck_ld = 2 * ((nh + 3) / 4 * 4);   // floats per checkpoint row (16-byte multiple)
  g.ck_rows = ckoff[L];
  // coefficient rows: every stage's slice (up to 2 r0 + 256 <= lmax + 256 degrees) stays in its row
  g.cstride = (L + 255) / 256 * 256 + 256;
  SHOT_CUDA(cudaMalloc(&g.ck_off_d, (L + 1) * sizeof(long long)));
  SHOT_CUDA(cudaMemcpyAsync(g.ck_off_d, ckoff.data(), (L + 1) * sizeof(long long), cudaMemcpyHostToDevice, st));
  g.ck_off = ckoff;
  SHOT_CUDA(cudaMalloc(&g.rec_coef, (size_t)L * g.cstride * sizeof(float4)));
  SHOT_CUDA(cudaMemsetAsync(g.rec_coef, 0, (size_t)L * g.cstride * sizeof(float4), st));
  SHOT_CUDA(cudaMalloc(&g.rec_x, (size_t)nh * sizeof(float)));
  SHOT_CUDA(cudaMalloc(&g.ck, (size_t)2 * g.ck_rows * g.ck_ld * sizeof(float)));   // two parity planes
  SHOT_CUDA(cudaMemsetAsync(g.ck, 0, (size_t)2 * g.ck_rows * g.ck_ld * sizeof(float), st));
  count_launch(2);
  k_coef32_build<<<L, 256, 0, st>>>(g.lmax, g.cstride, reinterpret_cast<float4*>(g.rec_coef));
  k_ck_build<<<dim3((nh + 127) / 128, L), 128, 0, st>>>(g.lmax, nh, g.x_d, g.ck_off_d, g.ck_rows, g.ck_ld, g.ck,
                                                        g.rec_x);
  SHOT_CUDA(cudaGetLastError());
  SHOT_CUDA(cudaStreamSynchronize(st));   // ckoff is a local
  return SHOT_OK;
}

int launch_legendre_tf32(const Grid& g, int nf, const float* X, float* Cf, float* Y, int ldc, bool ana, bool syn,
                         bool apply_h, cudaStream_t st) {
  const Workspace& w = g.ws;
  const int nmma = tf32_nmma(nf);
  const bool rec = g.mode == SHOT_RECURRENCE;
  if (nmma > 256 || nmma > w.nmma_cap || !w.ct32 || (rec ? !g.ck : (!g.tab || !g.tabT))) {
    set_error("TF32X3 path supports at most 128 fields per call");
    return SHOT_ERR_UNSUPPORTED;
  }
  int rc;
  // Table mode: the deepest pipeline (<= 4 stages) whose tiles fit in one CTA's shared memory,
  // with 2 KB left for the static control block.  Recurrence mode: 3 stages of generated
  // operands (2, then 1, where the fields leave no room) and the deepest input ring (<= 8)
  // beside them; SHOT_TC_STAGES / SHOT_T32_INRING fix either depth.
  constexpr size_t kSmemCap = 227 * 1024 - 2048;
  auto bytes = [&](bool a_, int s, int in) { return tf32_smem_bytes(nmma, a_, s, rec, in, g.nh); };
  // Table mode: two CTAs per SM (8 split warps each, two stages) where each CTA's tensor memory
  // (two accumulators of at most 128 columns) and two stages in half the SM's shared memory fit;
  // SHOT_T32_2CTA=0 keeps one CTA of 16 split warps.
  const int nacc_h = 2 * nmma <= 256 ? 2 * nmma : nmma;
  int tcols = 32;
  while (tcols < nacc_h) tcols <<= 1;
  constexpr size_t kSmemHalf = 112 * 1024 - 2048;
  bool two_cta = false;
  auto pick = [&](bool a_, int& s, int& in) {
    if (!rec) {
      in = 0;
      two_cta = !g.t32_two_cta_off && tcols <= 128 && bytes(a_, 2, 0) <= kSmemHalf;
      if (two_cta) {
        s = 2;
        return;
      }
      s = g.tc_stages_override > 0 ? g.tc_stages_override : kT32MaxStages;
      while (s > 1 && bytes(a_, s, 0) > kSmemCap) --s;
      return;
    }
    const size_t ib = bytes(a_, 1, 1) - bytes(a_, 1, 0);
    for (s = g.tc_stages_override > 0 ? g.tc_stages_override : 3; s >= 1; --s) {
      const size_t fixed = bytes(a_, s, 0);
      in = fixed < kSmemCap ? (int)std::min<size_t>(kMaxIn, (kSmemCap - fixed) / ib) : 0;
      if (g.t32_in_override > 0 && g.t32_in_override < in) in = g.t32_in_override;
      if (in >= (s > 2 ? 4 : s) || s == 1) return;
    }
  };
  auto launch = [&](bool a_, const CUtensorMap& ma, const CUtensorMap& mb, T32Args args, int ntiles) -> int {
    int stages, nin;
    pick(a_, stages, nin);
    const size_t smem = bytes(a_, stages, nin);
    if (smem > kSmemCap || (rec && nin < 1)) {
      set_error("TF32X3: the grid's recurrence buffers do not fit in shared memory");
      return SHOT_ERR_UNSUPPORTED;
    }
    args.nin = nin;
    const bool bc = 2 * nmma <= 256;
    void* kern = rec ? tf32_kernel<true>(a_, bc, stages, false) : tf32_kernel<false>(a_, bc, stages, two_cta);
    SHOT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int nthreads = 32 * (2 + (two_cta ? 8 : kSplitWarps) + 4);
    const int ctas = (two_cta ? 2 : 1) * g.num_sms;   // persistent: one or two CTAs per SM
    const int grid = ntiles < ctas ? ntiles : ctas;
    ProfScope prof(a_ ? PK_ANALYSIS : PK_SYNTHESIS, st);
    count_launch();
    void* params[] = {const_cast<CUtensorMap*>(&ma), const_cast<CUtensorMap*>(&mb), const_cast<T32Args*>(&args)};
    SHOT_CUDA(cudaLaunchKernel(kern, dim3(grid), dim3(nthreads), params, smem, st));
    return SHOT_OK;
  };
  T32Args rx{};
  CUtensorMap mck_a, mck_s;
  if (rec) {
    rx.ck_off = g.ck_off_d;
    rx.coef = reinterpret_cast<const float4*>(g.rec_coef);
    rx.cstride = g.cstride;
    rx.xnode = g.rec_x;
    rx.ck_rows = g.ck_rows;
    rx.lmax = g.lmax;
    // checkpoint rows (segments) of ck_ld floats: boxes of 16 segments x 32 nodes (analysis)
    // and 4 segments x 128 nodes (synthesis)
    if ((rc = make_map_f32(&mck_a, g.ck, g.ck_ld, (uint64_t)2 * g.ck_rows, g.ck_ld, 2 * kTK, kAnaSegs))) return rc;
    if ((rc = make_map_f32(&mck_s, g.ck, g.ck_ld, (uint64_t)2 * g.ck_rows, g.ck_ld, 2 * kBM, kSynSegs))) return rc;
  }
  if (ana) {
    CUtensorMap ma, mx;
    if (rec) ma = mck_a;
    else if ((rc = make_map_f32(&ma, g.tab, g.nh, g.rows_total, g.ldt, kTK, kBM, true))) return rc;
    if ((rc = make_map_f32(&mx, X, ldc, (uint64_t)g.nblk * g.nh, ldc, nmma, kTK))) return rc;
    T32Args args = rx;
    args.tiles = g.tiles_ana;
    args.ntiles = g.ntiles_ana;
    args.M = g.M_d;
    args.row_off = g.row_off_d;
    args.nh = g.nh;
    args.ldc = ldc;
    args.ncols = 2 * nf;
    args.nmma = nmma;
    args.h = apply_h ? g.h_d : nullptr;
    args.ct = w.ct32;
    args.cf = Cf;
    args.nmma_cap = w.nmma_cap;
    args.ldi = g.ldi;
    args.Y = nullptr;
    args.err = w.dev_int + 4;
    args.wait = g.wait_cycles;
    if ((rc = launch(true, ma, mx, args, g.ntiles_ana))) return rc;
  }
  if (syn) {
    CUtensorMap ma, mb;
    if (rec) ma = mck_s;
    else if ((rc = make_map_f32(&ma, g.tabT, g.ldi, (uint64_t)g.nblk * g.nh, g.ldi, kTK, kBM, true))) return rc;
    if ((rc = make_map_f32(&mb, w.ct32, g.ldi, (uint64_t)g.nblk * w.nmma_cap, g.ldi, kTK, nmma, true))) return rc;
    T32Args args = rx;
    args.tiles = g.tiles_syn;
    args.ntiles = g.ntiles_syn;
    args.M = g.M_d;
    args.row_off = g.row_off_d;
    args.nh = g.nh;
    args.ldc = ldc;
    args.ncols = 2 * nf;
    args.nmma = nmma;
    args.h = nullptr;
    args.ct = nullptr;
    args.cf = nullptr;
    args.nmma_cap = w.nmma_cap;
    args.ldi = g.ldi;
    args.Y = Y;
    args.err = w.dev_int + 4;
    args.wait = g.wait_cycles;
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
