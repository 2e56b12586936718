/*
 * distil.h -- C interface of the B300 distilled-nucleon library.
 *
 * Computes, on one GPU, the hot path of the nucleon operators with quark
 * distillation profiles (paper: "Improving hadron creation operators for
 * charmonium, glueballs and baryons", Sec. 2.1 "Improved nucleon
 * operators"):
 *
 *   elementals   Phi[p,t]_ijk = sum_x exp(-i p.x) eps_abc v_i^a v_j^b v_k^c
 *                (the nucleon elementals / "triplets" the paper rescales;
 *                the paper names them but prints no formula, this is the
 *                standard baryon elemental without displacement or 1/V3),
 *   correlate    the N_B x N_B matrix C_ab(t) of the profiled elementals
 *                Phi^(a) = g^(a)_i g^(a)_j g^(a)_k Phi_ijk (Sec. 2.1,
 *                displayed equation, no sums) between a sink at t and a
 *                source at t0 = 0 through perambulators tau(t, t0), with the
 *                positive-parity C gamma_5 nucleon spin structure and the
 *                direct minus exchange u-quark Wick terms,
 *   gevp         the generalized eigenvalues of C(t) u = lambda C(t0) u
 *                (Sec. 2.1, "solve a GEVP").
 *
 * Conventions common to every call
 * --------------------------------
 *  - Complex numbers are interleaved (re, im) pairs: "c128" = two doubles,
 *    "c64" = two floats.  Arrays are row-major, last index fastest.
 *  - All array pointers are DEVICE pointers on the context's device, owned
 *    by the caller; the library never frees them.  Exceptions are named
 *    (the momentum list is a host pointer).
 *  - Calls are asynchronous on the given CUDA stream (0 = legacy default
 *    stream) unless stated.  Workspace passed to a call must stay untouched
 *    until the stream has passed the call.
 *  - Alignment: a workspace pointer must be 256-byte aligned (cudaMalloc
 *    and torch allocations are); every array must be aligned to its element
 *    (16 bytes for c128, 8 for c64 and f64).  Misaligned pointers are
 *    rejected with DISTIL_EINVAL.
 *  - Every call returns a distil_status.  On error nothing has been
 *    enqueued (argument errors) or the stream may hold partial results
 *    (DISTIL_ECUDA, DISTIL_ETIMEOUT); distil_last_error() gives a message.
 *    No call traps or aborts the device on bad input.
 *  - Site order s = x + L*(y + L*z).  Momentum p = 2*pi*n/L for integer n.
 *  - Packed triples: i<j<k stored at colex rank C(k,3) + C(j,2) + i,
 *    T3 = nv*(nv-1)*(nv-2)/6 entries.
 *  - Spin-mode index of a perambulator: I = alpha*nv + i (alpha in 0..3),
 *    Dirac-Pauli basis with gamma_4 = diag(1,1,-1,-1).
 */
#ifndef DISTIL_H
#define DISTIL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* distil_stream; /* same type as cudaStream_t */

typedef enum {
  DISTIL_OK = 0,
  DISTIL_EINVAL = 1,   /* bad argument (null pointer, size, mode)          */
  DISTIL_ENOMEM = 2,   /* workspace too small / allocation failed          */
  DISTIL_ECUDA = 3,    /* a CUDA runtime or driver call failed             */
  DISTIL_ETIMEOUT = 4, /* a bounded device-side wait expired               */
  DISTIL_ENOTSUP = 5   /* mode or size not supported by the library       */
} distil_status;

/* Arithmetic of a call.
 * Storage types: FP64 reads and writes c128 everywhere.  FP32 reads and
 * writes c64 (eigenvectors, perambulators, elementals).  The tensor-core
 * modes read c64 eigenvectors and perambulators and keep the elementals in
 * c128 (distil_elementals writes c128, distil_correlate reads c128).  The
 * correlation matrix and the GEVP are always c128.
 * Tensor-core modes split every operand row (power-of-two exponent of its
 * largest entry) into 16-bit pieces and accumulate in TMEM:
 *   FP16X6  fixed-point slices of 9 + 11 + 11 bits (10 + 11 + 11 in the
 *           elementals), 6 products; the leading product is integer-valued
 *           and sums exactly (about 2^-31 of the row maximum per GEMM).  The
 *           accurate mode.
 *   BF16X6  fixed-point slices of 8 + 8 + 8 bits, 6 products (2^-24).
 *   BF16X3  fixed-point slices of 8 + 8 bits, 3 products (2^-16).
 *   FP16X3  floating pieces h + l (22 bits), 3 products; not exact: the
 *           tensor core's FP32 accumulation error grows with K. */
typedef enum {
  DISTIL_FP64 = 0,         /* plain FP64 on CUDA cores                        */
  DISTIL_FP32 = 1,         /* plain FP32 on CUDA cores, FP64 final sums       */
  DISTIL_MIXED_BF16X6 = 2, /* tensor cores, see above                         */
  DISTIL_MIXED_BF16X3 = 3,
  DISTIL_MIXED_FP16X3 = 4,
  DISTIL_MIXED_FP16X6 = 5
} distil_mode;

typedef struct distil_ctx distil_ctx;

/* Create a context on CUDA device `device` (makes it current for the
 * calling thread).  *out receives the handle.  One context per device. */
int distil_create(int device, distil_ctx** out);

/* Release the context and the small device buffers it owns (error word,
 * phase tables).  Waits for nothing: synchronise the streams first. */
void distil_destroy(distil_ctx* ctx);

/* Message of the last failed call made by this thread ("" if none).  The
 * string is owned by the library and valid until the next call. */
const char* distil_last_error(void);

/* ------------------------------------------------------------------ */
/* Elementals                                                          */
/* ------------------------------------------------------------------ */

/* Bytes of device workspace distil_elementals needs for these sizes. */
int distil_elementals_workspace(int L, int nt, int nv, int np, int mode, size_t* bytes);

/* Phi[t][q][r] = sum_s exp(-i p_q.x_s) det[v_i(s), v_j(s), v_k(s)] for the
 * triple of rank r, for t < nt and q < np.
 *   v    [nt][nv][L^3][3]   c128 (FP64) or c64 (other modes), device
 *   mom  [np][3] int32      integer momenta n, HOST pointer, read during the call
 *   phi  [nt][np][T3]       c64 in FP32 mode, c128 in FP64 and in every
 *                           tensor-core mode; device, fully overwritten
 * Sizes: 1 <= L <= 256, nt >= 1, nv >= 1 (nv < 3 gives T3 = 0), np >= 1.
 * The elementals are the paper's Phi[p,t]_ijk before profiles (Sec. 2.1). */
int distil_elementals(distil_ctx* ctx, const void* v, int L, int nt, int nv,
                      const int32_t* mom, int np, int mode, void* phi,
                      void* workspace, size_t ws_bytes, distil_stream stream);

/* ------------------------------------------------------------------ */
/* Correlation matrix                                                  */
/* ------------------------------------------------------------------ */

int distil_correlate_workspace(int nt, int nv, int np, int nb, int mode, size_t* bytes);

/* C[q][a][b][t] = sum_{mu nu} P+_{nu mu} sum Psi^(a)mu_{IJK}(t) tau_II' tau_JJ' tau_KK'
 *                 [Psi^(b)nu_{I'J'K'}(0) - Psi^(b)nu_{K'J'I'}(0)]^*
 * with Psi^(a)mu_{(alpha i)(beta j)(gamma k)} = g^(a)_i g^(a)_j g^(a)_k
 * Phi_ijk (C gamma_5)_{alpha beta} delta_{gamma mu}.
 *   phi_snk [nt][np][T3]      sink elementals at t: c64 in FP32 mode, c128
 *                             in FP64 and in every tensor-core mode
 *   phi_src [np][T3]          source elementals at t0 = 0 (same type)
 *   tau     [nt][4nv][4nv]    tau(t, t0) spin-major: c128 in FP64 mode,
 *                             else c64
 *   prof    [nb][nv] f64, or [nt][nb][nv] when prof_per_t != 0 (sink uses
 *           g[t], source g[0]); device pointer
 *   C       [np][nb][nb][nt]  c128, device, fully overwritten
 * Sizes: nv >= 1, nt >= 1, np >= 1, 1 <= nb <= 16. */
int distil_correlate(distil_ctx* ctx, const void* phi_snk, const void* phi_src,
                     const void* tau, int nt, int nv, int np,
                     const double* prof, int nb, int prof_per_t, int mode,
                     void* C, void* workspace, size_t ws_bytes, distil_stream stream);

/* One sink timeslice of the correlation matrix, for workloads processed
 * one timeslice at a time (the eigenvectors and perambulators of one t at
 * a time on the device).  Computes C[q][a][b][t] for every q, a, b of an
 * array with nt timeslices and leaves the other columns of C untouched;
 * the arithmetic is the one of distil_correlate for that timeslice.
 *   phi_snk_t [np][T3]      sink elementals at timeslice t (types as above)
 *   phi_src   [np][T3]      source elementals at t0 = 0
 *   tau_t     [4nv][4nv]    tau(t, t0)
 *   prof_snk  [nb][nv] f64  sink profiles g^(a)[t] (Sec. 2.1: g_i^(a)[t])
 *   prof_src  [nb][nv] f64  source profiles g^(b)[t0]
 *   C         [np][nb][nb][nt] c128, column t written
 * Workspace: distil_correlate_workspace(1, nv, np, nb, mode).
 * Sizes: 0 <= t < nt, nv, np >= 1, 1 <= nb <= 16. */
int distil_correlate_slice(distil_ctx* ctx, const void* phi_snk_t, const void* phi_src,
                           const void* tau_t, int nv, int np, const double* prof_snk,
                           const double* prof_src, int nb, int mode, void* C, int nt, int t,
                           void* workspace, size_t ws_bytes, distil_stream stream);

/* ------------------------------------------------------------------ */
/* GEVP                                                                */
/* ------------------------------------------------------------------ */

/* lambda[q][t][n] = generalized eigenvalues of C[q][:][:][t] u = lambda
 * C[q][:][:][t0] u, FP64, sorted by |lambda| descending.  General
 * (non-Hermitian) pencils: C(t0)^{-1} C(t) by LU with partial pivoting,
 * then Hessenberg reduction and shifted complex QR.  A singular C(t0) or
 * a QR sweep that fails to converge gives NaN eigenvalues for that (q, t)
 * and the call still returns DISTIL_OK.
 *   C       [np][nb][nb][nt] c128 device;  lambda [np][nt][nb] c128 device.
 * Sizes: 1 <= nb <= 16, 0 <= t0 < nt. */
int distil_gevp(distil_ctx* ctx, const void* C, int np, int nb, int nt, int t0,
                void* lambda, distil_stream stream);

/* The GEVP of distil_gevp for the timeslices t_begin <= t < t_begin +
 * t_count only (lambda entries of other timeslices untouched), and
 * optionally its right eigenvectors (Sec. 2.1: the GEVP whose eigenvectors
 * combine the N_B profiled operators into the optimal one):
 *   vecs [np][nt][nb][nb] c128 device or NULL: vecs[q][t][n][:] solves
 *        C(t) u = lambda_n C(t0) u for the n-th eigenvalue of lambda[q][t],
 *        scaled to unit 2-norm with its largest-modulus component real and
 *        positive (NaN where lambda is NaN).
 * Eigenvectors come from the complex Schur form of C(t0)^{-1} C(t) (the
 * accumulated Householder and Givens transformations) and back substitution.
 * Sizes: as distil_gevp, 0 <= t_begin, t_begin + t_count <= nt. */
int distil_gevp_range(distil_ctx* ctx, const void* C, int np, int nb, int nt, int t0,
                      int t_begin, int t_count, void* lambda, void* vecs, distil_stream stream);

/* Correlators of the optimal operators (Sec. 2.1: the N_B profiled
 * operators combined with the weights of a GEVP eigenvector, the optimal
 * profile combination for each state) and their effective masses:
 *   copt[q][n][t] = u^H C[q][:][:][t] u,  u = vecs[q][td][n][:]
 *   meff[q][n][t] = log(|copt[q][n][t]| / |copt[q][n][t+1]|), NaN at t = nt-1
 *   C    [np][nb][nb][nt] c128 device;  vecs [np][nt][nb][nb] c128 device,
 *        as written by distil_gevp_range (its timeslice td is used)
 *   copt [np][nb][nt] c128 device;  meff [np][nb][nt] f64 device or NULL.
 * The moduli make the effective mass defined for complex correlators.
 * Sizes: 1 <= nb <= 16, 0 <= td < nt. */
int distil_optimal(distil_ctx* ctx, const void* C, int np, int nb, int nt, const void* vecs,
                   int td, void* copt, double* meff, distil_stream stream);

/* Quark distillation profiles as functions of the Laplacian eigenvalues
 * (Sec. 2.1: the profiles "can be a function of the 3D Laplacian
 * eigenvalues" and of t), Gaussian in the eigenvalue:
 *   prof[t][b][i] = exp(-(lam[t][i] / sigma[b])^2)
 *   lam   [nt][nv] f64 device: eigenvalue of distillation vector i at t
 *   sigma [nb] f64 HOST, each > 0, read during the call
 *   prof  [nt][nb][nv] f64 device: the per-timeslice profiles
 *         distil_correlate takes with prof_per_t = 1 (nt = 1: the
 *         t-independent [nb][nv] form)
 * Sizes: nt, nv >= 1, 1 <= nb <= 16. */
int distil_profiles_eigen(distil_ctx* ctx, const double* lam, int nt, int nv, const double* sigma,
                          int nb, double* prof, distil_stream stream);

/* ------------------------------------------------------------------ */
/* Split-precision complex GEMM (the tensor-core engine on its own)    */
/* ------------------------------------------------------------------ */

int distil_cgemm_workspace(int M, int N, int K, int batch, int mode, size_t* bytes);

/* C[b][m][n] = sum_k A[b][m][k] * B[b][n][k]  (complex64, no conjugation),
 * for b < batch, with a tensor-core mode (DISTIL_MIXED_*): both operands are
 * scaled by powers of two, split into 16-bit pieces and multiplied on
 * tcgen05 tensor cores with FP32 accumulation.  This is the contraction
 * engine of distil_correlate; the paper has no separate counterpart (it is
 * the building block of the mode contractions of Sec. 2.1).
 *   A [batch][M][K], B [batch][N][K], C [batch][M][N]  c64, device.
 * Sizes: M, N, K >= 1, 1 <= batch <= 65535.  EINVAL for a CUDA-core mode. */
int distil_cgemm(distil_ctx* ctx, const void* A, const void* B, void* C, int M, int N, int K,
                 int batch, int mode, void* workspace, size_t ws_bytes, distil_stream stream);

/* ------------------------------------------------------------------ */
/* Correlation matrix without device allocation                        */
/* ------------------------------------------------------------------ */

/* Same result as distil_correlate in the FP64 or FP32 mode, for callers that
 * cannot allocate device memory where they need it: a process that works
 * inside a device-memory budget reserved up front, or a latency-critical
 * pipeline that cannot afford the device-wide synchronisation cudaMalloc /
 * cudaFree may imply.  The call allocates nothing; its scratch is a fixed
 * 16 MiB device array inside the library, held by every GPU that loads the
 * library until the process exits.  (The paper has no counterpart; this is
 * an interface convenience.)
 *  - Arguments, layouts and alignment rules as distil_correlate, without
 *    workspace; mode must be DISTIL_FP64 or DISTIL_FP32 (else
 *    DISTIL_EINVAL).  Misaligned arrays return DISTIL_EINVAL before any
 *    launch.
 *  - Sizes needing more scratch than the array (FP64 about 352 N_B N_v^3
 *    bytes: N_v = 16 with N_B <= 11, N_v = 20 with N_B <= 5, N_v = 24 with
 *    N_B <= 3; FP32 about half) return DISTIL_ENOMEM without touching the
 *    device.
 *  - Every call made outside stream capture looks up the array's device
 *    address (cudaGetSymbolAddress) and caches it per device; a call made
 *    while `stream` is being captured uses that cached address.  So make a
 *    first call on each device before any stream capture.
 *  - Every call shares the one array, which keeps the last call's contents.
 *    Calls that overlap on the GPU (different streams, or several host
 *    threads) race on it: serialise them. */
int distil_correlate_noalloc(distil_ctx* ctx, const void* phi_snk, const void* phi_src,
                             const void* tau, int nt, int nv, int np,
                             const double* prof, int nb, int prof_per_t, int mode,
                             void* C, distil_stream stream);

/* ------------------------------------------------------------------ */
/* Batched ensembles: tuning, graph-captured plans                     */
/* ------------------------------------------------------------------ */

/* Tensor-core kernel variant of each mode-contraction site of the mixed
 * correlator, variants[3] = {step i (K = N_v), step j (K = 4 N_v), the T
 * contraction Z = W T^c of the final sum (K = 5 N_v)}:
 *   0  one 128 x NT tile per CTA, NT = 128 (or 80 / 64, whichever pads
 *      less, at the sites that keep three accumulator pairs)
 *   1  persistent CTAs with two accumulator sets, 128 x 64 tiles (128 x 32
 *      with three pairs)
 *   2  step i only: persistent with the whole-K A tile resident in shared
 *      memory (used when N_v <= 128, else variant 1)
 *   3  one 128 x 64 tile per CTA
 *   4  persistent, 128 x 32 tiles
 *   5  persistent with one accumulator set of the variant-0 tile (the MMAs
 *      of a tile wait for the previous tile's epilogue while the operand
 *      copies of the next tile already run)
 * Every variant of a site gives identical results; only the speed differs.
 * The defaults are {5, 5, 5}.  The library has no counterpart of this in
 * the paper: it is a property of this implementation. */
int distil_set_tuning(distil_ctx* ctx, const int* variants);
int distil_get_tuning(const distil_ctx* ctx, int* variants);

/* An ensemble of gauge configurations sharing L, nt, the momenta, nb and
 * the mode, each with its own N_v (Sec. 2.1: the correlators of a
 * configuration follow from its eigenvectors and perambulators; the
 * paper's ensembles are processed configuration by configuration). */
typedef struct {
  int L, nt, np, nb;
  int t0;                /* GEVP reference timeslice, 0 <= t0 < nt */
  int mode;              /* distil_mode */
  const int32_t* mom;    /* [np][3] integers (host), p = 2 pi n / L */
} distil_batch_shape;

typedef struct {
  int nv;                /* eigenvectors of this configuration (>= 1) */
  const void* v;         /* [nt][nv][L^3][3] c128 (FP64 mode) or c64, device */
  const void* tau;       /* [nt][4nv][4nv] c128 (FP64) or c64, device, tau(t, 0) */
  const double* prof;    /* [nb][nv] f64, device */
  void* C;               /* [np][nb][nb][nt] c128 output, device */
  void* lambda;          /* [np][nt][nb] c128 GEVP output, device, or NULL */
} distil_batch_cfg;

typedef struct distil_plan distil_plan;

/* Bytes of workspace a plan over these configurations needs: the largest
 * configuration's elementals plus the largest elementals / correlator
 * workspace.  No device needed. */
int distil_plan_workspace(const distil_batch_shape* shape, const distil_batch_cfg* cfgs, int ncfg,
                          size_t* bytes);

/* Build a plan: optionally autotune (autotune != 0: run the correlator of
 * the first configuration on its first timeslice once per candidate vector
 * of kernel variants (six, covering every variant of every site),
 * with event timing, and keep the faster variant of every site; this runs
 * eagerly on `stream`, synchronises it and resets the context's kernel
 * statistics), then capture, on `stream`, the whole ensemble (per
 * configuration: elementals, correlator with the source at t = 0, GEVP)
 * into one CUDA graph.  The workspace is used by every run of the plan and
 * must outlive it; the cfgs pointers are captured into the graph.  The
 * plan sets ctx's tuning table to the variants it chose. */
int distil_plan_create(distil_ctx* ctx, const distil_batch_shape* shape, const distil_batch_cfg* cfgs, int ncfg,
                       int autotune, void* workspace, size_t ws_bytes, distil_stream stream, distil_plan** out);

/* Launch the captured graph on `stream` (asynchronous).  Plans of one
 * context share the context's device error word. */
int distil_plan_run(distil_plan* plan, distil_stream stream);

/* The variants the plan was captured with, variants[3] as in
 * distil_set_tuning, and the number of kernel launches in its graph. */
int distil_plan_info(const distil_plan* plan, int* variants, int* kernels);

void distil_plan_destroy(distil_plan* plan);

/* ------------------------------------------------------------------ */
/* Introspection                                                       */
/* ------------------------------------------------------------------ */

/* Device-side status of ctx.  Kernels record in a device word the first
 * bounded wait that expired (a tensor-core pipeline stage that never
 * arrived); once set, later tensor-core launches of ctx return at once and
 * leave their outputs unwritten.  This call synchronises the device, stores
 * the code in *code (0 = no expired wait; 1 = MMA waiting for a copied stage,
 * 2 = copy producer waiting for a free stage, 3 = epilogue waiting for the
 * accumulator, 4 = teardown waiting for copies in flight) and returns
 * DISTIL_ETIMEOUT with a message when it is nonzero.  reset != 0 clears
 * the word afterwards.  code may be NULL. */
int distil_device_status(distil_ctx* ctx, int reset, unsigned* code);

/* Limit, in SM clock cycles, of the bounded waits inside the tensor-core
 * pipelines of ctx (a copied stage, a free stage, the accumulator); cycles <= 0
 * restores the default of 2^31 (about a second at 2 GHz).  On expiry a
 * kernel records the code read by distil_device_status and returns; the
 * teardown waits for copies and MMAs still in flight keep the default limit.
 * A short limit makes the next tensor-core call fail on purpose (failure
 * detection without a device fault).  Host only. */
int distil_set_wait_limit(distil_ctx* ctx, long long cycles);

/* Scan count values of x (f64, or f32 when is_f32) for NaN or Inf;
 * synchronises `stream`.  Returns DISTIL_OK with *first_bad = -1 when all
 * are finite, else DISTIL_EINVAL with *first_bad = the lowest index of a
 * non-finite value (a complex array is scanned as 2 count reals).
 * first_bad may be NULL.  For validating inputs before a call. */
int distil_scan_finite(distil_ctx* ctx, const void* x, long long count, int is_f32,
                       long long* first_bad, distil_stream stream);

/* 1 if the library implements `mode`, else 0 (no device needed). */
int distil_mode_supported(int mode);

/* Per-kernel statistics of the library's own launches. */
typedef struct {
  char name[64];       /* kernel family, e.g. "simt_gemm_f64"            */
  long long launches;  /* launches since the last distil_profile_enable  */
  double ms;           /* summed event-timed duration (0 if not timing)  */
} distil_kernel_stat;

/* Reset the per-kernel counters of ctx (synchronises the device first).
 * timing != 0 additionally brackets every later launch with a pair of CUDA
 * events recorded on the launching stream.  Launch counting is always on.
 * Do not enable timing while a stream of ctx is being captured into a
 * CUDA graph. */
int distil_profile_enable(distil_ctx* ctx, int timing);

/* Copy up to `max` kernel statistics into out[] and the number of kernel
 * families seen into *count.  Waits for the recorded events to complete. */
int distil_profile_read(distil_ctx* ctx, distil_kernel_stat* out, int max, int* count);

/* ------------------------------------------------------------------ */
/* One-meson operators with distillation profiles                      */
/* ------------------------------------------------------------------ */
/* Paper Sec. 2.3 ("Improved charmonium operators"): operators qbar Gamma q
 * with Gamma in {gamma_0 gamma_5, gamma_0 gamma_5 gamma_i nabla_i,
 * gamma_i BB_i}, N_B Gaussian distillation profiles for each, the
 * 3 N_B x 3 N_B correlation matrix pruned by the singular vectors of its
 * largest singular values at one time separation, then the GEVP
 * (distil_gevp on the pruned matrix).  Only DISTIL_MIXED_FP16X6 is built
 * (other modes: DISTIL_ENOTSUP).  gamma_0 is the Euclidean gamma_4 of the
 * Dirac-Pauli basis above, gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4. */

int distil_meson_elementals_workspace(int L, int nt, int nv, int np, int mode, size_t* bytes);

/* phi[t][q][d][i][j] = sum_x exp(-i p_q.x) v_i(x)^dagger (D_d v_j)(x), the
 * colour inner product of v_i with the displaced D_d v_j, d = 0..6 for
 * 1, nabla_x, nabla_y, nabla_z, BB_x, BB_y, BB_z:
 *   (nabla_k f)(x) = 1/2 [U_k(x) f(x+k) - U_k(x-k)^dagger f(x-k)]
 *   (the symmetric gauge-covariant difference, periodic in space) and
 *   BB_i = eps_ijk nabla_j nabla_k = nabla_j nabla_k - nabla_k nabla_j for
 *   (i, j, k) cyclic, the right derivative acting first.
 *   v    [nt][nv][L^3][3]        c64 device (distillation vectors)
 *   U    [nt][3][L^3][3][3]      c64 device: U[t][k][s][a][b] = row a,
 *                                column b of the link from s in direction k
 *   mom  [np][3] int32           HOST, read during the call
 *   phi  [nt][np][7][nv][nv]     c128 device, fully overwritten
 * The products are formed exactly in double-float and contracted on the
 * tensor cores in 4032-long K chunks (the elementals scheme of FP16X6).
 * Sizes: 1 <= L <= 128, nt >= 1, 1 <= nv <= 1024, 1 <= np <= 16. */
int distil_meson_elementals(distil_ctx* ctx, const void* v, const void* U, int L, int nt, int nv,
                            const int32_t* mom, int np, int mode, void* phi, void* workspace,
                            size_t ws_bytes, distil_stream stream);

int distil_meson_correlate_workspace(int nv, int np, int nb, int mode, size_t* bytes);

/* C[q][a][b][t] = -Tr[Phi_a(q, t) tau(t) Phibar_b(q, 0) gamma_5 tau(t)^dagger gamma_5]
 * (the isovector connected correlator, source at t0 = 0, backward
 * propagator from gamma_5-hermiticity) for operators a = 7 type + sigma
 * (nb profiles sigma per type; 3 nb operators):
 *   Phi_a    = sum_c Gamma_c (x) g Phi^(d_c) g      spin-major [4nv][4nv]
 *   Phibar_b = sum_c gamma_4 Gamma_c^dagger gamma_4 (x) (g Phi^(d_c)(0) g)^dagger
 *   type 0: Gamma = gamma_4 gamma_5, d = 0;  type 1: gamma_4 gamma_5 gamma_k,
 *   d = 1 + k;  type 2: gamma_k, d = 4 + k  (k = x, y, z summed);
 *   g = diag(prof[sigma]) multiplies both quark indices.
 *   phi_snk [nt][np][7][nv][nv]  c128 device: sink elementals at t
 *   phi_src [np][7][nv][nv]      c128 device: source elementals at t0 = 0
 *   tau     [nt][4nv][4nv]       c64 device: tau(t, 0), spin-major
 *   prof    [nb][nv]             f64 device
 *   C       [np][3nb][3nb][nt]   c128 device, fully overwritten
 * Two tensor-core GEMMs per (t, q) with K = 4 nv (Q_b = Phibar_b g5 tau^dagger
 * g5, then X_b = tau Q_b) and a double-float reduction with the profiles.
 * Sizes: nt >= 1, 1 <= nv <= 1024, 1 <= np <= 16, 1 <= nb <= 10. */
int distil_meson_correlate(distil_ctx* ctx, const void* phi_snk, const void* phi_src, const void* tau,
                           int nt, int nv, int np, const double* prof, int nb, int mode, void* C,
                           void* workspace, size_t ws_bytes, distil_stream stream);

/* Pruning (Sec. 2.3: the singular vectors of the n largest singular values
 * of C at one time separation):  C(t_prune) = U S V^dagger,
 *   Un[q][a][m]   = column m of U (m < nkeep), scaled so that its
 *                   largest-modulus component (the first of equal ones) is
 *                   real and positive                     c128 device
 *   Ct[q][m][n][t] = (Un^dagger C(t) Un)[m][n]           c128 device
 *   sv[q][a]       = the singular values, descending     f64 device or NULL
 *   C [np][nops][nops][nt] c128 device.  One-sided Jacobi SVD in FP64.
 * Sizes: 1 <= nops <= 32, 1 <= nkeep <= min(nops, 16), 0 <= t_prune < nt. */
int distil_meson_prune(distil_ctx* ctx, const void* C, int np, int nops, int nt, int t_prune, int nkeep,
                       void* Ct, void* Un, double* sv, distil_stream stream);

/* ------------------------------------------------------------------ */
/* A1^{-+} glueball operators                                          */
/* ------------------------------------------------------------------ */
/* Paper Sec. 2.2 ("Improved glueball operators"): operators built from the
 * chromo-magnetic field B_i = eps_ijk F_jk (clover discretisation of the
 * field strength) and adjoint gauge-covariant symmetric differences D_j. */

int distil_glueball_workspace(int L, int nt, size_t* bytes);

/* O[t][n], n = 0..4, the five A1^{-+} operators of timeslice t at zero
 * momentum (repeated indices summed, eps the Levi-Civita symbol):
 *   O_1 = sum_x Tr(eps_ijk B_i D_j B_k)
 *   O_2 = sum_x Tr(eps_ijk eps_ilm B_j B_k D_l B_m)
 *   O_3 = sum_x Tr(eps_ijk B_i D_j^3 B_k)
 *   O_4 = sum_x Tr(eps_ijk B_i D_j^2 D_k B_j)
 *   O_5 = sum_x Tr(eps_ijk B_i D_j D_i^2 B_k)
 * with F_{mu nu}(x) = (Q - Q^dagger) / (8 i) minus a third of its trace, Q
 * the sum of the four counter-clockwise plaquettes of the (mu, nu) plane
 * that start and end at x; B_i = 2 F_jk for (i, j, k) cyclic; (D_j X)(x) =
 * 1/2 [U_j(x) X(x+j) U_j(x)^dagger - U_j(x-j)^dagger X(x-j) U_j(x-j)],
 * D_j^2 = D_j D_j (lattice units, periodic space).
 *   U  [nt][3][L^3][3][3]  c64 device: U[t][k][s][a][b], as for the mesons
 *   O  [nt][5]             c128 device, fully overwritten
 * FP64 on CUDA cores (deterministic sums).  Sizes: 2 <= L <= 128, nt >= 1. */
int distil_glueball_operators(distil_ctx* ctx, const void* U, int L, int nt, void* O, void* workspace,
                              size_t ws_bytes, distil_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* DISTIL_H */
