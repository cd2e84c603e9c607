// Internal declarations shared by the CUDA translation units of the SHOT library.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <utility>
#include <vector>

#include "../../include/shot.h"

namespace shot {

// Default limit of the bounded device-side waits of the tensor-core kernels (SM clock cycles).
constexpr long long kDefaultWaitCycles = 1LL << 30;

// ---------------------------------------------------------------------------------
// Error reporting (thread-local message, status codes of shot.h)
void set_error(const std::string& msg);
int cuda_status(cudaError_t e, const char* what);   // SHOT_OK or SHOT_ERR_CUDA/OOM + message
#define SHOT_CUDA(call)                                          \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return ::shot::cuda_status(e_, #call); \
  } while (0)

// ---------------------------------------------------------------------------------
// Launch accounting (prof.cu).  Kinds of shot_profile_read.
// profiled launch kinds: ring DFT, Legendre analysis / synthesis, inverse DFT with the update
// (or a plain inverse transform), other (reductions, set-up), inverse DFT with the marginal
// check or the final objective
enum ProfKind { PK_DFT = 0, PK_ANALYSIS = 1, PK_SYNTHESIS = 2, PK_IDFT = 3, PK_OTHER = 4, PK_CHECK = 5, PK_NKINDS = 6 };
void count_launch(int n = 1);
class ProfScope {
 public:
  ProfScope(int kind, cudaStream_t st);
  ~ProfScope();
 private:
  int kind_;
  cudaStream_t st_;
  cudaEvent_t b_ = nullptr, e_ = nullptr;
};

// ---------------------------------------------------------------------------------
// Ring FFT plan: nlon = prod R[s], radices in {2,3,4,5,8}, Stockham ordering.
// The most elements (sequences x length) one ring-FFT CTA transforms: two ping-pong buffers
// of kFftCap complex values plus the twiddles stay under ~110 KB (at least two CTAs per SM);
// also the longest ring a grid may have.
constexpr int kFftCap = 6400;

struct FftPlan {
  int N;
  int nst;
  int R[16];
  int tw_off[16];        // offset of stage s's twiddles ((R - 1) x Ns, r-major) in the table
  int root_off[16];      // stages with a radix outside {2..6, 8, 9, 10, 12, 15, 16} (primes > 5):
                         // offset of the R roots W_R^e (forward sign) in the table, else 0
  uint32_t ns_mul[16];   // ceil(2^32 / Ns) of stage s (0 when Ns == 1)
  uint32_t nr_mul[16];   // ceil(2^32 / (N / R)) of stage s (0 when N / R == 1)
};
// radices with a compiled butterfly; any other radix runs the generic O(R) per output stage
__host__ __device__ inline bool fft_radix_compiled(int R) {
  return R == 2 || R == 3 || R == 4 || R == 5 || R == 6 || R == 8 || R == 9 || R == 10 || R == 12 || R == 15 ||
         R == 16;
}
// entries of the plan's twiddle table (N, plus the roots of its generic stages)
__host__ __device__ inline int fft_tw_len(const FftPlan& p) {
  int t = p.N;
  for (int s = 0; s < p.nst; ++s)
    if (!fft_radix_compiled(p.R[s]) && p.root_off[s] + p.R[s] > t) t = p.root_off[s] + p.R[s];
  return t;
}
bool make_fft_plan(int N, FftPlan* plan);
// the plan's stage twiddles W_N^{k r N/(Ns R)} (forward sign), then the roots of its generic
// stages: N + (sum of their radices) complex values
void fft_plan_twiddles(const FftPlan& plan, std::vector<float2>& tw);

// ---------------------------------------------------------------------------------
// Spectral layout.  For order m and parity p (p = (l - m) mod 2) the block (m,p)
// holds the degrees l = m + p + 2 i, i = 0 .. M_mp - 1, M_mp = (lmax - m - p)/2 + 1.
//   table   : [block][i][ldt] Pbar_lm(x_jh) at the north-hemisphere nodes jh < nh
//   X / Y   : [block][jh][ldc] ring spectra folded by parity (see dft.cu)
//   C       : [row_off[block] + i][ldc] Legendre coefficients
// ldc >= 2 * nfields (re, im per field), a multiple of 4.
struct Tile {
  int blk;    // 2*m + p
  int r0;     // first row of the tile (i for analysis, jh for synthesis)
};

struct Workspace {
  int nf_cap = 0;       // fields the buffers hold
  int ldc = 0;
  float* XY = nullptr;  // X (analysis input) and Y (synthesis output) share storage
  float* Yb = nullptr;  // the solver keeps X and Y apart: X survives for the next K application
  float* C = nullptr;
  double* part = nullptr;   // per-(field, ring pair) partial sums [nf][nh][NPART]
  size_t part_cap = 0;
  void* probs = nullptr;    // ProbState[nf]
  const float** marg = nullptr;  // device pointer lists [2*nf]
  float* ubuf = nullptr;    // internal u, v storage for the divergence [3*nf*n] each
  float* vbuf = nullptr;
  size_t uv_cap = 0;
  __nv_bfloat16* ct_hi = nullptr;   // BF16X3: scaled coefficients C^T [blk][nmma_cap][ldi]
  __nv_bfloat16* ct_lo = nullptr;
  float* ct32 = nullptr;            // TF32X3: scaled coefficients C^T [blk][nmma_cap][ldi], FP32
  int nmma_cap = 0;
  int* dev_int = nullptr;   // device counters: [0] iterations, [1] active, [4] timeout flag
  int* host_int = nullptr;  // pinned mirror
  void* host_probs = nullptr;  // pinned ProbState mirror
  size_t host_probs_cap = 0;
  double* taus = nullptr;      // per-problem tau (device) [nf]
  cudaStream_t stream = nullptr;   // internal solver stream (capturable)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaStream_t side = nullptr;     // the solver's per-problem reductions (overlap the next analysis)
  cudaEvent_t evf = nullptr, evj = nullptr;
};

// Tunable launch shapes for one field count (0 = the built-in default).
struct Tuning {
  int nf = 0;
  int dft_fg = 0;      // fields per ring-DFT CTA (1, 2, 4, 8)
  int idft_fg = 0;     // fields per inverse-DFT CTA
  int simt_bn = 0;     // FP32 Legendre tile width (32, 48, 64)
  int tc_stages = 0;   // BF16x3 analysis pipeline depth (1..4)
};

struct Grid {
  int nlat = 0, nlon = 0, lmax = 0, nh = 0;
  std::vector<Tuning> tuning;   // per field count, filled by the autotuner
  Tuning active;                // the entry in force for the current launch sequence
  int precision = SHOT_FP32, mode = SHOT_TABLE, quad = SHOT_QUAD_GAUSS_LEGENDRE;
  int dev = 0;
  int num_sms = 148;
  FftPlan plan{};
  // host copies (FP64)
  std::vector<double> x, w, a_ring;
  // blocks
  int nblk = 0;                 // 2*(lmax+1)
  std::vector<int> M;           // rows per block
  std::vector<long long> row_off;  // prefix sum of M
  long long rows_total = 0;
  int ldt = 0;                  // table row stride (elements), multiple of 16
  // device
  double* x_d = nullptr;
  double* w_d = nullptr;
  float* a_d = nullptr;         // per-ring area weight (FP32)
  float2* tw_d = nullptr;       // the ring FFT plan's twiddle table, fft_tw_len(plan) entries
  float* h_d = nullptr;         // heat multipliers for the current call, [lmax+1]
  float* tab = nullptr;         // FP32 folded table [row][ldt] (FP32 and TF32X3 grids)
  float* tabT = nullptr;        // TF32X3: the table transposed per block, [blk][jh][ldi], zero for i >= M
  __nv_bfloat16* tab_hi = nullptr;  // BF16X3 split table [row][ldt]
  __nv_bfloat16* tab_lo = nullptr;
  int ldi = 0;                  // row stride of C^T (>= the largest block, multiple of 8)
  // SHOT_RECURRENCE: seeds per (m, node) and recurrence coefficients (O(n) memory)
  void* rec_seeds = nullptr;
  void* rec_coef = nullptr;
  long long* rec_coef_off = nullptr;
  float* rec_x = nullptr;
  // SHOT_RECURRENCE on TF32X3 grids: FP32 checkpoints, per parity plane par, Pbar at degrees
  // (m + 16 s + par, m + 16 s + par + 2) at [par ck_rows + ck_off[m] + s][ck_ld floats: 2 per node];
  // two-step coefficients (A, B, C, 0) per degree in rec_coef (row stride cstride); x^2 of the
  // nodes in rec_x
  float* ck = nullptr;
  long long* ck_off_d = nullptr;
  std::vector<long long> ck_off;
  long long ck_rows = 0;       // rows per parity plane
  int ck_ld = 0;
  int cstride = 0;              // TF32X3 recurrence: coefficient row stride (entries per order)
  int* M_d = nullptr;
  long long* row_off_d = nullptr;
  Tile* tiles_ana = nullptr;
  Tile* tiles_syn = nullptr;
  int tc_stages_override = 0;   // SHOT_TC_STAGES: pipeline depth of the tensor-core kernels (0 = tuned)
  long long wait_cycles = kDefaultWaitCycles;   // limit of the tensor-core kernels' waits (cycles)
  int t32_in_override = 0;
  int t32_two_cta_off = 0;      // SHOT_T32_2CTA=0: TF32 table kernels with one CTA of 16 split warps per SM      // SHOT_T32_INRING: input ring depth of the TF32 recurrence kernels (0 = deepest)
  int idft_nonpersistent = 0;   // SHOT_IDFT_PERSISTENT=0: update half-steps use the one-item-per-CTA k_idft
  void* xyz_d = nullptr;        // node unit vectors (float4), made on first use
  // ring geometry (every grid): ring i holds ring_len[i] nodes starting at ring_off[i] of a
  // field of npix nodes; HEALPix rings also carry the longitude of their first pixel,
  // phi0 = pi * ring_phase.first / ring_phase.second
  int nside = 0;
  size_t npix = 0;
  std::vector<int> ring_len;
  std::vector<long long> ring_off;
  std::vector<std::pair<int, int>> ring_phase;
  int* ring_len_d = nullptr;
  long long* ring_off_d = nullptr;
  int2* ring_phase_d = nullptr;
  // HEALPix: FFT plans for the ring lengths that factor into 2, 3 and 5 (the other rings use
  // direct DFTs); ring_plan_d[i] = plan index or -1, each plan's stage twiddles at
  // hp_tw_d + hp_tw_base_d[plan]
  FftPlan* hp_plan_d = nullptr;
  int* ring_plan_d = nullptr;
  float2* hp_tw_d = nullptr;
  int* hp_tw_base_d = nullptr;
  int ntiles_ana = 0, ntiles_syn = 0;
  int bm_ana = 128, bm_syn = 128;
  Workspace ws;
};

// ---------------------------------------------------------------------------------
// Per-problem solver state (device), see sinkhorn.cu.
struct ProbState {
  // The solver's buffers hold scalings up to factors kept as FP64 logarithms:
  // u_true = e^{la} u_buf, v_true = e^{lb} v_buf (unbalanced potentials eps log u reach
  // tau |log m(p)/m(q)| / 2, far outside the FP32 exponent range when tau/eps is large).
  double la, lb;
  double lsu;       // pending log of the u-step's sum (sum u_true or sum a p u_true^{-eps/tau})
  double lvu, lvv;  // levels log mean u_buf, log mean v_buf of the latest half-steps
  double qu, qv;    // log ru (resp. rv) minus the level of the buffer that step divides by
  double beta;      // factor the forward ring DFT applies with scale_which 1 (gradient sweeps)
  double err;       // last marginal error
  double ot, ot_dual, mass;
  double mass_v;    // unbalanced: m(pi) = sum a v (K u) from the latest v-update; balanced: 0
                    // once a v-update has run (then m(pi) = sum a q); NaN before the first
  double tau;       // marginal penalty of this problem (INFINITY: balanced)
  float gamma;      // tau/(tau+eps), 1 when balanced
  float et;         // eps/(tau+eps), 0 when balanced
  float ru, rv;     // FP32 factors inside the update ratio: u_buf = (ru p / K v_buf)^gamma
  int eu, ev;       // ru = 2^eu, rv = 2^ev
  float cuv;        // e^{la+lb}: u_true (K v_true) = cuv u_buf (K v_buf)
  float cu, cv;     // e^{la}, e^{lb} in FP32 (saturate for extreme potentials)
  int balanced;
  int active;
  int status;
  int iters;
};

// Epilogue modes of the inverse DFT kernel
enum EpiMode { EPI_PLAIN = 0, EPI_UPDATE = 1, EPI_CHECK = 2, EPI_FINAL = 3, EPI_SYM = 4 };
// solve_prepare flag (internal, above the public SHOT_FLAG_* bits): the problems are self terms
// (q = p) solved by the symmetric averaged update u <- sqrt(u (p / K u)^gamma)
constexpr int kFlagSymmetricSolve = 1 << 30;
constexpr int NPART = 4;   // partial sums per (field, ring pair)

struct EpiParams {
  int mode;
  float* out;                 // EPI_PLAIN: Kv output; EPI_UPDATE: u or v buffer
  const float* const* marg;   // per-field marginal pointers (p or q)
  const float* const* marg2;  // EPI_FINAL: the other marginal
  float* other;               // EPI_CHECK/FINAL: the other scaling buffer (v for the u-side)
  ProbState* ps;              // per-problem state incl. tau-derived constants
  double* part;               // [nf][nh][NPART]
  double eps;
  int norm_l1;
  int which;                  // 0: u-step (marginal p), 1: v-step (marginal q)
  float* xout;                // EPI_UPDATE: when set, the CTA also ring-transforms the new
                              // scaling (unscaled) into the folded spectra xout[.][jh][ldc]
  int potentials;             // EPI_FINAL: write eps log u, eps log v instead of u, v
  int skip_store;             // EPI_UPDATE: the new scaling feeds only the fused forward
                              // transform (no later launch reads this iteration's buffer)
};
bool profiling_on();

// ---------------------------------------------------------------------------------
// Launchers (return SHOT status)
int launch_dft_fwd(const Grid& g, const float* in, int nf, const ProbState* ps, int scale_which,
                   float* X, int ldc, cudaStream_t st);
int launch_idft(const Grid& g, const float* Y, int ldc, int nf, const EpiParams& ep, cudaStream_t st);
bool idft_is_persistent(const Grid& g, int nf, const EpiParams& ep);
// Grids whose Legendre contractions run the TF32x3 tensor-core kernels: TF32X3 grids, and BF16X3
// grids in recurrence mode (the recurrence kernels are bound by generating the A operand, not by
// the MMA's operand width, so a bf16 split of the generated values would gain nothing; TF32x3
// is also the more accurate)
inline bool tf32_kernels(const Grid& g) {
  return g.precision == SHOT_TF32X3 || (g.precision == SHOT_BF16X3 && g.mode == SHOT_RECURRENCE);
}
int launch_legendre(const Grid& g, int nf, const float* X, float* C, float* Y, int ldc, cudaStream_t st);
int launch_heat_mult(const Grid& g, double t, cudaStream_t st);
int launch_coeff_gather(const Grid& g, const float* C, int ldc, int nf, float* coeffs, cudaStream_t st);
int launch_coeff_scatter(const Grid& g, const float* coeffs, int nf, float* C, int ldc, cudaStream_t st);
int launch_synthesis_only(const Grid& g, int nf, const float* C, float* Y, int ldc, cudaStream_t st);
int launch_analysis_only(const Grid& g, int nf, const float* X, float* C, int ldc, bool apply_h,
                         cudaStream_t st);
int build_grid_tables(Grid& g, cudaStream_t st);
// selects g.active for nf (tunes on first use)
int autotune(Grid& g, int nf, cudaStream_t st, const EpiParams* upd = nullptr);
int launch_legendre_tc(const Grid& g, int nf, const float* X, float* Cf, float* Y, int ldc, bool ana, bool syn,
                       bool apply_h, cudaStream_t st);
int launch_c_to_ct(const Grid& g, int nf, const float* C, int ldc, cudaStream_t st);
int launch_legendre_tf32(const Grid& g, int nf, const float* X, float* Cf, float* Y, int ldc, bool ana, bool syn,
                         bool apply_h, cudaStream_t st);
int launch_c_to_ct32(const Grid& g, int nf, const float* C, int ldc, cudaStream_t st);
int build_recurrence(Grid& g, cudaStream_t st);
int build_tf32_recurrence(Grid& g, cudaStream_t st);
int launch_legendre_rec(const Grid& g, int nf, const float* X, float* C, float* Y, int ldc, bool ana, bool syn,
                        bool apply_h, cudaStream_t st);
int tc_nmma(int nf);
int ensure_workspace(Grid& g, int nf, cudaStream_t st);
// HEALPix
void healpix_geometry(Grid& g, int nside);
// ps != nullptr: every field is multiplied by its ProbState::beta on load
int launch_hp_dft_fwd(const Grid& g, const float* in, int nf, float* X, int ldc, cudaStream_t st,
                      const ProbState* ps = nullptr);
int launch_hp_idft(const Grid& g, const float* Y, int ldc, int nf, const EpiParams& ep, cudaStream_t st);

}  // namespace shot
