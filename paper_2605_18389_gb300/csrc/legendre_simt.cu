// Per-order Legendre contractions of the semi-naive SHT in FP32 (SIMT FFMA).
//
// Analysis (App. B, quadrature form; the area weights a_j are already folded into X by
// the ring DFT), for every block (m, p) and every column c = (field, re/im):
//   C[i][c] = h_{l} * sum_{jh < nh} Pbar_{l m}(x_jh) X[jh][c],   l = m + p + 2 i
// with h_l = exp(-t l(l+1)) (Sec. 3.2) or 1 for a plain transform.
// Synthesis, the transpose contraction over degrees:
//   Y[jh][c] = sum_i Pbar_{l m}(x_jh) C[i][c]
// Both are GEMMs with N = 2 * nfields columns.  The table is stored [i][jh] (jh
// contiguous): it is the K-contiguous A operand of the analysis and the M-contiguous A
// operand of the synthesis.  One CTA computes a 128 x BN tile; the tile lists are built
// at grid set-up so that large blocks are scheduled first.
#include "shot_internal.cuh"

namespace shot {

namespace {

constexpr int BM = 128, BK = 16, NT = 128, APAD = 4;

template <int BN, bool ANALYSIS>
__global__ void __launch_bounds__(NT) k_legendre_simt(
    const Tile* __restrict__ tiles, const float* __restrict__ tab, int ldt,
    const long long* __restrict__ row_off, const int* __restrict__ Mrows, int nh,
    const float* __restrict__ Bsrc, int ldc, int ncols, float* __restrict__ out,
    const float* __restrict__ h) {
  constexpr int TN = BN / 8;
  constexpr int BF4 = BK * BN / 4;                 // float4 per B chunk
  constexpr int BL = (BF4 + NT - 1) / NT;          // float4 loads per thread
  __shared__ __align__(16) float As[2][BK][BM + APAD];
  __shared__ __align__(16) float Bs[2][BK][BN];

  const Tile tl = tiles[blockIdx.x];
  const int blk = tl.blk, r0 = tl.r0;
  const int m = blk >> 1, p = blk & 1;
  const int M = Mrows[blk];
  const long long ro = row_off[blk];
  const int n0 = blockIdx.y * BN;
  const int K = ANALYSIS ? nh : M;
  const int mvalid = ANALYSIS ? M : nh;   // rows of the output block
  const float* Ab = tab + ro * ldt;
  const float* Bb = ANALYSIS ? (Bsrc + (size_t)blk * nh * ldc) : (Bsrc + ro * ldc);

  const int tid = threadIdx.x;
  const int tn = tid & 7, tm = tid >> 3;

  float4 ra[4];
  float4 rb[BL];

  auto load = [&](int kt) {
    if (ANALYSIS) {
      // A(i, k) = Ab[i*ldt + k], rows r0..r0+127, k in [kt, kt+16): 4 threads per row
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int idx = tid + s * NT;         // 0..511
        const int row = idx >> 2, kq = idx & 3;
        const int i = r0 + row;
        if (i < M) ra[s] = __ldg(reinterpret_cast<const float4*>(Ab + (size_t)i * ldt + kt + kq * 4));
        else ra[s] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    } else {
      // A(jh, i) = Ab[i*ldt + jh], k = i in [kt, kt+16), jh in [r0, r0+128)
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int idx = tid + s * NT;
        const int kr = idx >> 5, c4 = idx & 31;
        const int i = kt + kr, jh = r0 + c4 * 4;
        if (i < M && jh < ldt) ra[s] = __ldg(reinterpret_cast<const float4*>(Ab + (size_t)i * ldt + jh));
        else ra[s] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int s = 0; s < BL; ++s) {
      const int idx = tid + s * NT;
      const int kr = idx / (BN / 4), c4 = idx - kr * (BN / 4);
      const int k = kt + kr, c = n0 + c4 * 4;
      if (idx < BF4 && k < K && c < ncols) rb[s] = __ldg(reinterpret_cast<const float4*>(Bb + (size_t)k * ldc + c));
      else rb[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto store = [&](int buf) {
    if (ANALYSIS) {
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int idx = tid + s * NT;
        const int row = idx >> 2, kq = idx & 3;
        As[buf][kq * 4 + 0][row] = ra[s].x;
        As[buf][kq * 4 + 1][row] = ra[s].y;
        As[buf][kq * 4 + 2][row] = ra[s].z;
        As[buf][kq * 4 + 3][row] = ra[s].w;
      }
    } else {
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int idx = tid + s * NT;
        const int kr = idx >> 5, c4 = idx & 31;
        *reinterpret_cast<float4*>(&As[buf][kr][c4 * 4]) = ra[s];
      }
    }
#pragma unroll
    for (int s = 0; s < BL; ++s) {
      const int idx = tid + s * NT;
      if (idx < BF4) {
        const int kr = idx / (BN / 4), c4 = idx - kr * (BN / 4);
        *reinterpret_cast<float4*>(&Bs[buf][kr][c4 * 4]) = rb[s];
      }
    }
  };

  float acc[8][TN];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) acc[r][c] = 0.f;

  const int nk = (K + BK - 1) / BK;
  if (nk > 0) {
    load(0);
    store(0);
    __syncthreads();
  }
  for (int t = 0; t < nk; ++t) {
    const int cur = t & 1;
    if (t + 1 < nk) load((t + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][tm * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][tm * 8 + 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float b[TN];
      if (TN % 4 == 0) {
#pragma unroll
        for (int c = 0; c < TN; c += 4) {
          const float4 bb = *reinterpret_cast<const float4*>(&Bs[cur][kk][tn * TN + c]);
          b[c] = bb.x; b[c + 1] = bb.y; b[c + 2] = bb.z; b[c + 3] = bb.w;
        }
      } else {
#pragma unroll
        for (int c = 0; c < TN; c += 2) {
          const float2 bb = *reinterpret_cast<const float2*>(&Bs[cur][kk][tn * TN + c]);
          b[c] = bb.x; b[c + 1] = bb.y;
        }
      }
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    if (t + 1 < nk) store(cur ^ 1);
    __syncthreads();
  }

#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int row = r0 + tm * 8 + r;
    if (row >= mvalid) continue;
    float sc = 1.f;
    float* o;
    if (ANALYSIS) {
      if (h) sc = h[m + p + 2 * row];
      o = out + (size_t)(ro + row) * ldc;
    } else {
      o = out + ((size_t)blk * nh + row) * ldc;
    }
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      const int col = n0 + tn * TN + c;
      if (col < ncols) o[col] = acc[r][c] * sc;
    }
  }
}

template <int BN>
int launch_pair(const Grid& g, int nf, const float* X, float* C, float* Y, int ldc, bool ana, bool syn,
                const float* h, cudaStream_t st) {
  const int ncols = 2 * nf;
  const int ny = (ncols + BN - 1) / BN;
  if (ana) {
    dim3 grid(g.ntiles_ana, ny);
    ProfScope prof(PK_ANALYSIS, st);
    count_launch();
    k_legendre_simt<BN, true><<<grid, NT, 0, st>>>(g.tiles_ana, g.tab, g.ldt, g.row_off_d, g.M_d, g.nh, X,
                                                    ldc, ncols, C, h);
    SHOT_CUDA(cudaGetLastError());
  }
  if (syn) {
    dim3 grid(g.ntiles_syn, ny);
    ProfScope prof(PK_SYNTHESIS, st);
    count_launch();
    k_legendre_simt<BN, false><<<grid, NT, 0, st>>>(g.tiles_syn, g.tab, g.ldt, g.row_off_d, g.M_d, g.nh, C,
                                                     ldc, ncols, Y, nullptr);
    SHOT_CUDA(cudaGetLastError());
  }
  return SHOT_OK;
}

int dispatch(const Grid& g, int nf, const float* X, float* C, float* Y, int ldc, bool ana, bool syn,
             const float* h, cudaStream_t st) {
  const int ncols = 2 * nf;
  if (g.active.nf == nf && g.active.simt_bn > 0) {
    if (g.active.simt_bn == 32) return launch_pair<32>(g, nf, X, C, Y, ldc, ana, syn, h, st);
    if (g.active.simt_bn == 48) return launch_pair<48>(g, nf, X, C, Y, ldc, ana, syn, h, st);
    return launch_pair<64>(g, nf, X, C, Y, ldc, ana, syn, h, st);
  }
  if (ncols <= 32) return launch_pair<32>(g, nf, X, C, Y, ldc, ana, syn, h, st);
  if (ncols <= 48) return launch_pair<48>(g, nf, X, C, Y, ldc, ana, syn, h, st);
  return launch_pair<64>(g, nf, X, C, Y, ldc, ana, syn, h, st);
}

}  // namespace

int launch_legendre_simt(const Grid& g, int nf, const float* X, float* C, float* Y, int ldc, cudaStream_t st) {
  return dispatch(g, nf, X, C, Y, ldc, true, true, g.h_d, st);
}

int launch_analysis_simt(const Grid& g, int nf, const float* X, float* C, int ldc, bool apply_h,
                         cudaStream_t st) {
  return dispatch(g, nf, X, C, nullptr, ldc, true, false, apply_h ? g.h_d : nullptr, st);
}

int launch_synthesis_simt(const Grid& g, int nf, const float* C, float* Y, int ldc, cudaStream_t st) {
  return dispatch(g, nf, nullptr, const_cast<float*>(C), Y, ldc, false, true, nullptr, st);
}

}  // namespace shot
