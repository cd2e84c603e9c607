/*
 * shot.h -- C ABI of the GB300 heat-kernel Sinkhorn library (SHOT: Spherical
 * Harmonic Optimal Transport).
 *
 * The library applies the heat kernel K_t on S^2 to batches of fields sampled on a
 * Gauss-Legendre (GL) grid and runs Algorithm 1 ("Spherical Harmonic Sinkhorn",
 * App. C) and the Sinkhorn divergence of eq. (sinkhorn-divergence) on top of it.
 *
 * Conventions shared by every call
 * --------------------------------
 * - A FIELD is nlat*nlon contiguous float32 values, row-major [nlat][nlon].  Row j
 *   is the GL ring with x_j = cos(theta_j) DESCENDING (north to south); column k is
 *   longitude phi_k = 2*pi*k/nlon.  Batches are [batch][nlat][nlon], contiguous.
 * - The band limit is lmax (degrees 0..lmax, orders 0..lmax, triangular).  The
 *   default lmax = nlat-1 makes the GL quadrature exact for every product of two
 *   band-limited fields (App. C.1, "Gauss-Legendre").
 * - Area weights (App. C.2): every node of ring j has a_j = w_j * 2*pi/nlon with w_j
 *   the GL weight, so that sum_i a_i = 4*pi.
 * - Field pointers are DEVICE pointers owned by the caller.  Per-problem scalar
 *   outputs of the solver calls are HOST pointers (those calls synchronise the
 *   stream before they return).  shot_heat_apply and the transform calls are
 *   asynchronous on the given stream.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 * - A grid handle owns its tables and a workspace that grows on demand; calls that
 *   use the same handle must not run concurrently (serialise them on one stream).
 * - Every call returns an int status: SHOT_OK (0), a positive warning, or a
 *   negative error.  No C++ exception crosses this boundary.  shot_last_error()
 *   gives a message for the calling thread's last error.
 */
#ifndef SHOT_H
#define SHOT_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define SHOT_OK                  0
#define SHOT_WARN_NOT_CONVERGED  1   /* tol > 0 and the marginal check never passed within max_iter */
#define SHOT_ERR_INVALID_ARG    -1   /* bad size, NULL pointer, eps <= 0, tau <= 0, ... */
#define SHOT_ERR_CUDA           -2   /* a CUDA runtime call failed (message in shot_last_error) */
#define SHOT_ERR_OOM            -3   /* device allocation failed */
#define SHOT_ERR_UNSUPPORTED    -4   /* nlon beyond the ring FFT (> 6400 longitudes), or an unbuilt mode */
#define SHOT_ERR_NONPOSITIVE    -5   /* some K v <= 0: the update of Alg. 1 is undefined (App. C.4) */
#define SHOT_ERR_NONFINITE      -6   /* a scaling became inf/NaN (FP32 range exceeded) */
#define SHOT_ERR_TIMEOUT        -7   /* a bounded device-side wait expired */

/* ---- precision of the Legendre contractions ----------------------------- */
#define SHOT_FP32    0   /* FP32 SIMT FFMA */
#define SHOT_BF16X3  1   /* tcgen05 tensor cores, bf16 hi/lo split of both operands, 3 products, FP32 accumulate */
#define SHOT_TF32X3  2   /* tcgen05 tensor cores, tf32 hi/lo split of both operands, 3 products, FP32 accumulate;
                            ~2^-21 relative per product; keeps a second, transposed FP32 table */

/* ---- source of the associated Legendre values ---------------------------- */
#define SHOT_TABLE       0   /* precomputed parity-folded table, O(nlat^3) memory */
#define SHOT_RECURRENCE  1   /* values regenerated on the fly by the normalised three-term
                                recurrence (App. B): SHOT_FP32 grids from per-(m, node) seeds,
                                O(nlat^2) memory; SHOT_TF32X3 grids on the tensor cores from
                                FP32 checkpoints, four values per 16 degrees (a quarter of
                                the table's entries), by the two-step same-parity form;
                                SHOT_BF16X3 grids run the same TF32x3 recurrence kernels (the
                                generation, not the operand width, bounds them) */

/* ---- latitudinal quadrature (App. C.1) ----------------------------------- */
#define SHOT_QUAD_GAUSS_LEGENDRE  0  /* nodes = roots of P_nlat; exact to degree 2 nlat - 1 */
#define SHOT_QUAD_CLENSHAW_CURTIS 1  /* equiangular theta_j = pi j/(nlat-1), both poles included,
                                        Clenshaw-Curtis weights; exact to degree nlat - 1 */
#define SHOT_QUAD_HEALPIX         2  /* HEALPix rings (shot_grid_init_healpix): equal-area pixels,
                                        no exact quadrature */

/* ---- solver flags -------------------------------------------------------- */
#define SHOT_FLAG_NORM_L1     0x1  /* check sum_i a_i|u_i(Kv)_i - p_i| / sum_i a_i p_i instead of the relative L2 */
#define SHOT_FLAG_WARM_START  0x2  /* u and v hold the initial scalings instead of 1 */
#define SHOT_FLAG_POTENTIALS  0x4  /* return the potentials phi = eps log u, psi = eps log v in u, v */
#define SHOT_FLAG_SYMMETRIC_SELF 0x8  /* shot_divergence: self terms OT(p,p), OT(q,q) by the symmetric
                                        averaged update u <- sqrt(u (p/Ku)^gamma) (Feydy et al.,
                                        2019), one heat convolution per iteration, instead of
                                        Alg. 1 with q := p; same fixed point */

typedef struct shot_grid_s* shot_grid;

/* Message of the calling thread's last error ("" if none).  Copies at most
 * len-1 bytes into buf and NUL-terminates; returns the full message length. */
int shot_last_error(char* buf, int len);

/* Build a GL grid: nodes and weights by Newton's method on P_nlat in FP64 on the
 * device (App. C.1), area weights (App. C.2) and the orthonormal associated
 * Legendre table Pbar_lm(x_j) (App. B), folded by parity over the two hemispheres.
 *   out        receives the handle (host pointer)
 *   nlat >= 2; 2*lmax+1 <= nlon <= 6400 (any factorisation: prime factors above 5 run generic
 *              O(p)-per-output FFT stages, so 2,3,5-smooth nlon are fastest); lmax = -1 means nlat-1,
 *              else 0 <= lmax <= nlat-1
 *   precision  SHOT_FP32, SHOT_BF16X3 or SHOT_TF32X3; legendre_mode SHOT_TABLE or SHOT_RECURRENCE
 * Memory: about 2*(lmax+1)(lmax+2)/2 * ceil(nlat/2) * 4 bytes of table (0.37 GB at 720);
 *   SHOT_TF32X3 adds the transposed copy, 2(lmax+1) ceil(nlat/2) ceil(M_max/8)*8 * 4 bytes (0.75 GB at 720).
 *   SHOT_RECURRENCE keeps no table: FP32 grids ~(lmax+1) ceil(nlat/2) * 20 bytes of seeds; TF32X3
 *   grids the checkpoints, ~(lmax+1)(lmax+2)/32 rows of 2 ceil(nlat/2) floats in each of two parity
 *   planes (95 MB at 720, a quarter of the FP32 table; TF32X3's table mode keeps two tables).
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.  Synchronises `stream`. */
int shot_grid_init(shot_grid* out, int nlat, int nlon, int lmax, int precision,
                   int legendre_mode, void* stream);

/* Same as shot_grid_init with a choice of latitudinal quadrature (App. C.1):
 *   quadrature  SHOT_QUAD_GAUSS_LEGENDRE (what shot_grid_init builds) or
 *               SHOT_QUAD_CLENSHAW_CURTIS: the equiangular grid the paper runs its
 *               timings on (Sec. 4.1), ring j at colatitude pi j/(nlat-1) (ring 0 the
 *               north pole, ring nlat-1 the south pole), weights
 *               w_j = (c_j/N)(1 - sum_{k=1}^{N/2} b_k cos(2 pi k j/N)/(4k^2-1)), N = nlat-1,
 *               c_j = 1 at the poles and 2 elsewhere, b_k = 1 for k = N/2 and 2 otherwise,
 *               computed in FP64 on the device.  The heat operator on any node set is
 *               H diag(a) (the addition theorem), so lmax may go up to nlat-1 as on GL;
 *               the analysis is an exact inverse of the synthesis only when
 *               2*lmax <= nlat-1.  Every field-shaped argument of the other calls has the
 *               same [nlat][nlon] layout on either quadrature.
 * Other arguments, memory and errors as shot_grid_init; nlat >= 3 for Clenshaw-Curtis. */
int shot_grid_init_quad(shot_grid* out, int quadrature, int nlat, int nlon, int lmax, int precision,
                        int legendre_mode, void* stream);

/* Build a HEALPix grid (App. C.1 "HEALPix"): N = 12 nside^2 equal-area pixels on 4 nside - 1
 * iso-latitude rings.  Ring i (north to south, k = i + 1 mirrored into the north half) has
 *   polar cap k < nside:  z = 1 - k^2/(3 nside^2), 4k pixels, first pixel at phi0 = pi/(4k);
 *   belt nside <= k <= 2 nside: z = 4/3 - 2k/(3 nside), 4 nside pixels,
 *                         phi0 = pi (2 - s)/(4 nside), s = (k - nside + 1) mod 2;
 * pixel j of a ring at phi0 + 2 pi j / n (the HEALPix pixel centres; the cyclic order in a
 * ring starts at phi0), every pixel with area 4 pi / N.  Fields are flat FP32 arrays of the N
 * pixels in ring order ([batch][N] wherever the other calls say [batch][nlat][nlon]).  There is
 * no exact quadrature: the heat operator is H diag(a) on the pixel centres (addition theorem).
 *   nside in 1..4096; lmax = -1 means 3 nside - 1, else 0 <= lmax <= 4 nside - 2;
 *   precision, legendre_mode as shot_grid_init.  shot_grid_info reports nlat = 4 nside - 1
 *   rings and nlon = 4 nside (the longest ring).
 * Supported on HEALPix grids: shot_heat_apply(_noalloc), shot_sht_analysis/synthesis,
 * shot_sinkhorn, shot_divergence(_multi), shot_divergence_grad, shot_regional_rms,
 * shot_gibbs_apply, shot_conv_compare.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.
 * Synchronises `stream`. */
int shot_grid_init_healpix(shot_grid* out, int nside, int lmax, int precision, int legendre_mode, void* stream);

/* Number of nodes of one field (nlat * nlon, or 12 nside^2 on HEALPix) into *npix. */
int shot_grid_npix(shot_grid g, long long* npix);

/* Ring geometry into host arrays of nlat entries (any may be NULL): nodes per ring, offset of
 * the ring's first node within a field, longitude of that node (0 on GL/CC grids). */
int shot_grid_rings(shot_grid g, int* len, long long* off, double* phi0);

/* Release every device resource of the handle (NULL is a no-op). */
int shot_grid_free(shot_grid g);

/* nlat, nlon, lmax, precision, legendre_mode of the handle (host outputs; any may be NULL). */
int shot_grid_info(shot_grid g, int* nlat, int* nlon, int* lmax, int* precision, int* legendre_mode);

/* Nodes x_j = cos(theta_j) (descending) and quadrature weights w_j (sum 2) into host arrays of nlat
 * doubles, and the per-ring area weights a_j = w_j*2*pi/nlon (App. C.2).  Any
 * pointer may be NULL. */
int shot_grid_nodes(shot_grid g, double* x, double* w, double* a_ring);

/* Pre-size the workspace for calls on up to `nfields` fields (optional; calls grow it). */
int shot_grid_reserve(shot_grid g, int nfields);

/* Device-side status of the asynchronous calls on this grid.  Every wait inside the
 * tensor-core kernels is bounded (about 0.5 s of SM clock); one that expires makes its CTA
 * stop, release its tensor memory and raise a flag in the grid's workspace.  The solver
 * entry points (shot_sinkhorn, shot_divergence, shot_divergence_grad) read the flag
 * themselves; the asynchronous transforms (shot_heat_apply, shot_sht_analysis,
 * shot_sht_synthesis) cannot without synchronising, so their caller checks here:
 * synchronises `stream`, returns SHOT_ERR_TIMEOUT if the flag is set (and clears it), else
 * SHOT_OK.  Not part of the paper's method: a check on the device path.
 * Errors: INVALID_ARG (NULL grid), CUDA, TIMEOUT. */
int shot_grid_check(shot_grid g, void* stream);

/* Limit of the bounded device-side waits in this grid's tensor-core kernels, in SM clock
 * cycles, for the launches that follow (cycles <= 0 restores the default 2^30, about 0.5 s).
 * A limit below 2^20 makes every wait probe without blocking and read the clock after each
 * probe, so that it expires on time: a way to exercise the timeout path (status
 * SHOT_ERR_TIMEOUT from shot_grid_check, tensor memory released, the grid usable again).
 * The waits that only let a CTA's own copies and MMAs finish before it exits keep the
 * default.  Not part of the paper's method.  Errors: INVALID_ARG (NULL grid). */
int shot_grid_set_wait_limit(shot_grid g, long long cycles);

/* Heat convolution, Sec. 3.2: out = HeatConv(in; h), h_l = exp(-t l(l+1)), for
 * nfields fields:  ring real-DFT -> per-order Legendre analysis with area weights ->
 * scaling by h_l -> Legendre synthesis -> inverse ring DFT.
 *   in, out   device [nfields][nlat][nlon] float32 (may not alias)
 *   t >= 0    heat time (Alg. 1 uses t = eps/4)
 * Asynchronous on `stream`.  Errors: INVALID_ARG, OOM, CUDA; a device-side timeout is
 * reported by shot_grid_check. */
int shot_heat_apply(shot_grid g, double t, const float* in, float* out, int nfields, void* stream);

/* Spherical harmonic analysis (App. B: c_lm = <f, Y_lm> by GL quadrature) of nfields
 * real fields.  coeffs: device float32 [nfields][lmax+1][lmax+1][2] (re, im) with
 * entry [l][m] for 0 <= m <= l; entries with m > l are written as 0.  Orthonormal
 * Y_lm with the Condon-Shortley phase.  Asynchronous. */
int shot_sht_analysis(shot_grid g, const float* in, float* coeffs, int nfields, void* stream);

/* Inverse of shot_sht_analysis for real fields: out = sum_{l,|m|<=l} c_lm Y_lm using
 * c_{l,-m} = (-1)^m conj(c_lm).  Entries with m > l and Im c_l0 are ignored.  Asynchronous. */
int shot_sht_synthesis(shot_grid g, const float* coeffs, float* out, int nfields, void* stream);

/* Algorithm 1 (App. C) on `batch` independent problems, each stopping on its own.
 *   p, q        device [batch][nlat][nlon] float32 marginals (p_i, q_i >= 0)
 *   eps > 0     entropic parameter; the heat time is t = eps/4 (Alg. 1, step 1)
 *   tau         marginal penalty; INFINITY = balanced branch, else tau > 0 selects the
 *               unbalanced branch with the translation-invariant step
 *   max_iter    T;  tol = delta;  check_every = C (0 disables the periodic check)
 *   flags       SHOT_FLAG_* ; WARM_START reads u, v as the initial scalings
 *   u, v        device [batch][nlat][nlon] float32 outputs (inputs with WARM_START): the
 *               scalings, or with SHOT_FLAG_POTENTIALS the potentials eps log u, eps log v.
 *               The solver keeps each scaling as an FP32 buffer times an FP64 factor
 *               e^{la}, so the iteration and ot/err/mass stay valid when eps log u lies
 *               outside FP32's exponent range (unbalanced, large tau/eps, unequal masses);
 *               only the returned scalings then saturate to 0 or inf.
 *   ot          host [batch] or NULL: Alg. 1's return (dual form of App. C.2)
 *   ot_dual     host [batch] or NULL: ot - eps * m(pi)
 *   mass_pi     host [batch] or NULL: m(pi) = sum_i a_i u_i (K v)_i
 *   iters       host [batch] or NULL: iterations run (the breakdown iteration on error)
 *   err         host [batch] or NULL: marginal error of the returned u, v
 *   status      host [batch] or NULL: per-problem SHOT_OK / SHOT_WARN_NOT_CONVERGED /
 *               SHOT_ERR_NONPOSITIVE / SHOT_ERR_NONFINITE
 * Returns the most severe per-problem status (or an argument/CUDA error).
 * Outputs of a problem that broke down are NaN.  Synchronises `stream`. */
int shot_sinkhorn(shot_grid g, const float* p, const float* q, int batch,
                  double eps, double tau, int max_iter, double tol, int check_every, int flags,
                  float* u, float* v, double* ot, double* ot_dual, double* mass_pi,
                  int* iters, float* err, int* status, void* stream);

/* Sinkhorn divergence, eq. (sinkhorn-divergence), for `batch` pairs (p_b, q_b):
 *   S      = OT(p,q) - (OT(p,p) + OT(q,q))/2 + eps/2 (m(p) - m(q))^2  with OT = Alg. 1's return
 *   S_dual = the same with OT replaced by OT - eps*m(pi) and no mass-difference term
 * (the two coincide for converged balanced problems).  The 3*batch problems run in
 * one batch ordered [(p_b,q_b)]_b, [(p_b,p_b)]_b, [(q_b,q_b)]_b.
 *   S, S_dual, status  host [batch] (S_dual may be NULL)
 *   u3, v3             device [3*batch][nlat][nlon] or NULL: the scalings of all problems
 *   ot3, iters3        host [3*batch] or NULL
 * Other arguments as in shot_sinkhorn.  Synchronises `stream`. */
int shot_divergence(shot_grid g, const float* p, const float* q, int batch, double eps, double tau,
                    int max_iter, double tol, int check_every, int flags,
                    double* S, double* S_dual, int* status,
                    float* u3, float* v3, double* ot3, int* iters3, void* stream);

/* Many batches of pairs on several grids in one solve (the batched uneven-grid
 * workload): every set's problems (p_b,q_b), (p_b,p_b), (q_b,q_b) join one Alg. 1 solve
 * per grid (sets sharing a grid may differ in tau, not in eps); the grids' solves run on
 * separate streams inside one CUDA graph per block of check_every iterations, replayed
 * until max_iter or until every problem passed the check.
 *   sets[i].grid, p, q (device [batch][nlat][nlon]), batch, eps, tau (INFINITY = balanced),
 *   S, S_dual (may be NULL), status: host [batch] outputs as in shot_divergence.
 * Each grid's internal u, v storage grows to its problem count.  Returns the most severe
 * status.  Synchronises `stream`. */
typedef struct shot_pair_set {
  shot_grid grid;
  const float* p;
  const float* q;
  int batch;
  double eps;
  double tau;
  double* S;
  double* S_dual;
  int* status;
} shot_pair_set;
int shot_divergence_multi(const shot_pair_set* sets, int nsets, int max_iter, double tol, int check_every,
                          int flags, void* stream);

/* Gradient of the Sinkhorn divergence S (the Alg. 1-return form of shot_divergence,
 * including eps/2 (m(p)-m(q))^2) with respect to the node values of p, as used for the
 * gradient-based regional attribution of Sec. 4.2.
 *   mode SHOT_GRAD_UNROLLED: exact reverse-mode derivative of S computed by exactly
 *        max_iter iterations of Alg. 1 (no early stop), through the gauge and the
 *        translation-invariant steps; forward states are checkpointed every
 *        checkpoint_every iterations and recomputed segment by segment.
 *   mode SHOT_GRAD_ENVELOPE: the potential form, valid at convergence: balanced
 *        a (.) [phi_pq - (phi_pp + psi_pp)/2] + eps (m(p)-m(q)) a; unbalanced, the
 *        derivative of S_dual: a (.) [tau(1-e^{-phi_pq/tau}) - (tau(1-e^{-phi_pp/tau}) +
 *        tau(1-e^{-psi_pp/tau}))/2].
 *   grad_p  device [batch][nlat][nlon] float32: dS/dp_i (Euclidean; carries the factor
 *           a_i; balanced S is defined modulo c*a, so compare along directions with
 *           sum_i a_i d_i = 0)
 *   S, status host [batch].  Allocates its checkpoint buffers on the device (about
 *   (max_iter/checkpoint_every + 2 checkpoint_every + 7) * 2 * batch fields).
 * No derivative is produced for a pair whose iteration broke down (status < 0).
 * Synchronises `stream`. */
#define SHOT_GRAD_UNROLLED 0
#define SHOT_GRAD_ENVELOPE 1
int shot_divergence_grad(shot_grid g, const float* p, const float* q, int batch, double eps, double tau,
                         int max_iter, int checkpoint_every, int mode, double* S, float* grad_p, int* status,
                         void* stream);

/* Regional attribution of a divergence gradient (Sec. 4.2, App. E): the field form
 * g_i = grad_p_i / a_i centred by its area-weighted mean, then the area-weighted RMS
 * sqrt(sum_R a (g - mean)^2 / sum_R a) over the bands R = Tropics (|lat| < 23.5 deg),
 * ITCZ (|lat| < 10), NH mid-latitudes (30..60 N), SH mid-latitudes (30..60 S), Arctic (> 66.5 N).
 *   grad_p  device [batch][nlat][nlon] float32 (as written by shot_divergence_grad)
 *   rms     host [batch][5] in that band order (NaN for a band without nodes)
 * Synchronises `stream`. */
int shot_regional_rms(shot_grid g, const float* grad_p, int batch, double* rms, void* stream);

/* ---- heat convolution without device allocation (no counterpart in the paper) ----
 * For callers that cannot call cudaMalloc where they need K_t: code running while
 * another component owns the allocator (a pool that must not grow, a framework step
 * that forbids allocation, a stream another party is capturing into a CUDA graph), or
 * processes held to a device-memory budget fixed at start-up.  shot_heat_apply may
 * grow the grid's workspace; this variant never allocates: its scratch (ring spectra
 * and Legendre coefficients) lives in a fixed file-scope __device__ array of
 * SHOT_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until exit.
 *   Same arguments and result as shot_heat_apply; SHOT_FP32 grids only.
 *   Needs (2(lmax+1)ceil(nlat/2) + (lmax+1)(lmax+2)/2) * ldc * 4 bytes with
 *   ldc = 2*nfields rounded up to a multiple of 4; larger requests return
 *   SHOT_ERR_INVALID_ARG with the sizes in shot_last_error().
 *   The first call on a device resolves the array's device address
 *   (cudaGetSymbolAddress) with that device current; make it before any stream capture.
 *   All calls share the array: calls whose kernels may overlap on the GPU race and must
 *   be serialised by the caller.  A call also writes the grid's heat multipliers h_l for its
 *   t, so it races too with any overlapping call on the same grid (shot_heat_apply, a solve),
 *   which reads them.  Asynchronous on `stream`. */
#define SHOT_NOALLOC_SCRATCH_BYTES (8u << 20)
int shot_heat_apply_noalloc(shot_grid g, double t, const float* in, float* out, int nfields, void* stream);

/* Autotune the launch shapes used for calls on `nfields` fields (fields per ring-DFT and
 * inverse-DFT CTA, FP32 Legendre tile width, BF16x3 analysis pipeline depth) by timing the
 * candidates with CUDA events; the solvers do this automatically on their first call for
 * a field count.  choice: host int[4] or NULL, receives the four selections (0 = the
 * default).  The choices change no summation order (results are bit-identical).
 * Allocates one temporary field batch.  Synchronises `stream`. */
int shot_grid_autotune(shot_grid g, int nfields, int* choice, void* stream);

/* ---- heat convolution vs explicit matrix convolution -----------------------
 * The comparison of App. "Convolution on S^2": the matrix convolution applies the
 * unnormalised geodesic Gibbs kernel K_eps(x, y) = exp(-d(x, y)^2 / eps), which
 * integrates over the sphere to C(eps); by Varadhan's formula the heat kernel at
 * t = eps/4 is close to K_eps / C(eps), so the heat output is rescaled by C(eps) before
 * the two are compared.
 *
 * shot_gibbs_normaliser: C(eps) = 2 pi int_0^pi exp(-theta^2/eps) sin(theta) dtheta
 *   (host computation, composite Simpson's rule).  eps > 0; *C receives the value.
 * shot_gibbs_apply: out[f][i] = sum_j a_j exp(-d(x_i, x_j)^2 / eps) in[f][j] with the
 *   grid's area weights a (App. C.2) and d the great-circle distance, evaluated pair by
 *   pair in FP32 (O(n^2) per field, nothing of size n^2 stored; meant for the small grids
 *   of the comparison).  in, out: device [nfields][nlat][nlon] FP32, distinct.
 *   Asynchronous on `stream`; the first call on a grid also builds its node vectors.
 * shot_conv_compare: for each field, the mean over the grid nodes of
 *   |C(eps) (H_{eps/4} in)_i - (K_eps in)_i| into mae[f] (host array of nfields doubles);
 *   allocates and frees its two temporary field batches; synchronises `stream`.
 * Errors: INVALID_ARG (eps <= 0, NULL pointers, nfields < 1, in == out), OOM, CUDA. */
int shot_gibbs_normaliser(double eps, double* C);
int shot_gibbs_apply(shot_grid g, double eps, const float* in, float* out, int nfields, void* stream);
int shot_conv_compare(shot_grid g, double eps, const float* in, int nfields, double* mae, void* stream);

/* ---- measurement helpers (no counterpart in the paper) -------------------
 * shot_launch_count: total number of CUDA kernels this library has launched in the
 *   process (host counter; *n receives it).
 * shot_profile_enable(1): from now on every launch is bracketed by two CUDA events on
 *   its stream; shot_profile_enable(0) stops recording.
 * shot_profile_read: waits for the recorded events, then writes per kind the summed
 *   device time in ms and the number of launches, and clears the records.  Kinds:
 *   0 ring DFT (forward), 1 Legendre analysis, 2 Legendre synthesis,
 *   3 inverse ring DFT + Sinkhorn update (or a plain inverse transform), 4 reductions and
 *   small kernels, 5 inverse ring DFT + marginal check or final objective.
 *   ms, launches: host arrays of nkinds entries. */
int shot_launch_count(long long* n);
int shot_profile_enable(int on);
int shot_profile_read(double* ms, long long* launches, int nkinds);

#ifdef __cplusplus
}
#endif
#endif /* SHOT_H */
