/* lqcd.h — C ABI of the GB300 (sm_103a) Wilson-Dirac library.
 *
 * Operator (paper arXiv:1112.5280, Section 3: the even-odd preconditioned
 * Wilson hopping term "dslash" and the inversion of the fermion matrix are
 * the hot path; the operator is not written out there, this is the textbook
 * Wilson form with r = 1 in the kappa normalisation):
 *
 *   M psi(x) = psi(x) - kappa sum_mu [ eta (1 - g_mu) U_mu(x) psi(x+mu)
 *                                     + eta (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ]
 *
 * chiral gamma matrices g_k = [[0, -i s_k], [i s_k, 0]] (mu = 0,1,2 = x,y,z),
 * g_t = [[0, 1], [1, 0]] (mu = 3), g5 = diag(1, 1, -1, -1); eta = t_bc on
 * hops across the t boundary (t_bc = -1: antiperiodic), else 1.
 * Even-odd (Section 3 "even-odd preconditioned"): with D_pq the hop from
 * parity q to parity p, Mhat = 1 - kappa^2 D_eo D_oe on even sites,
 * bhat_e = b_e + kappa D_eo b_o and x_o = b_o + kappa D_oe x_e.
 *
 * Host layout (borrowed for the duration of a call, never retained):
 *   site s = x + Lx*(y + Ly*(z + Lz*t)), x fastest; parity (x+y+z+t) mod 2, 0 = even
 *   links   double[V][4][3][3][2]  (mu, row, col, re/im)
 *   spinors double[V][4][3][2]     (spin, colour, re/im)
 * All extents must be even and >= 2; V/2 < 2^31.
 *
 * Return values: LQCD_OK (0) or a negative LQCD_E* code; lqcd_last_error()
 * gives a message for the calling thread. Handles are owned by the library
 * and released with the matching *_destroy; destroying NULL is a no-op.
 * All device work of a context runs on its stream; calls that return host
 * data synchronise that stream. A context is used by one host thread at a time.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>

#if defined(__GNUC__)
#define LQCD_API __attribute__((visibility("default")))
#else
#define LQCD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LQCD_OK 0
#define LQCD_EINVAL (-1)       /* bad argument (sizes, parities, precisions, NULL) */
#define LQCD_ENOMEM (-2)       /* device allocation failed, or request beyond the engine budget */
#define LQCD_ENOCONV (-3)      /* solver hit maxiter before the tolerance */
#define LQCD_EBREAKDOWN (-4)   /* Krylov breakdown (zero denominator) */
#define LQCD_ENONFINITE (-5)   /* NaN or Inf in a residual */
#define LQCD_ETIMEOUT (-6)     /* engine deadline passed */
#define LQCD_ECUDA (-7)        /* CUDA runtime error (message in lqcd_last_error) */
#define LQCD_EBUSY (-8)        /* engine cannot admit the request now (slots or memory in use) */

/* storage precisions */
#define LQCD_F64 0
#define LQCD_F32 1
#define LQCD_F16 2
#define LQCD_BF16 3
/* FP64-class: each real stored as an (hi, lo) pair of floats (8 bytes) and computed in
 * double-float arithmetic (48-bit significand) on the FP32 pipes, which on GB300 run far
 * faster than its FP64 pipe. Links of LQCD_DF64 fields are stored the same way. */
#define LQCD_DF64 4

/* field subsets */
#define LQCD_EVEN 0
#define LQCD_ODD 1
#define LQCD_FULL 2

/* solvers */
#define LQCD_CG 0        /* CG on Mhat^dag Mhat (normal equations of the Schur system) */
#define LQCD_BICGSTAB 1  /* BiCGStab on Mhat */

typedef struct lqcd_ctx lqcd_ctx;
typedef struct lqcd_gauge lqcd_gauge;
typedef struct lqcd_field lqcd_field;
typedef struct lqcd_mom lqcd_mom;
typedef struct lqcd_engine lqcd_engine;
typedef struct lqcd_dslash_batch lqcd_dslash_batch;

LQCD_API const char* lqcd_status_string(int status);
/* Message of the last failing call on this host thread ("" if none). */
LQCD_API const char* lqcd_last_error(void);
/* Library version string. */
LQCD_API const char* lqcd_version(void);

/* ---------------------------------------------------------------- context */

/* Binds CUDA device `device`. cuda_stream: a cudaStream_t borrowed by the
 * context (it must stay valid until the context and every object made from it
 * are destroyed), or NULL to create an owned non-blocking stream.
 * lqcd_ctx_destroy releases the handle; the context's device resources are
 * freed once its last gauge field, spinor field and engine are destroyed too. */
LQCD_API int lqcd_ctx_create(lqcd_ctx** out, int device, void* cuda_stream);
LQCD_API void lqcd_ctx_destroy(lqcd_ctx* ctx);
/* Replaces the stream (borrowed; NULL restores the owned stream). */
LQCD_API int lqcd_ctx_set_stream(lqcd_ctx* ctx, void* cuda_stream);
LQCD_API void* lqcd_ctx_stream(const lqcd_ctx* ctx);
LQCD_API int lqcd_ctx_sync(lqcd_ctx* ctx);
/* Number of batched-kernel launches this context has issued (instrumentation). */
LQCD_API long long lqcd_ctx_launch_count(const lqcd_ctx* ctx);
/* The one-shot solves keep their device buffers on the context between calls
 * (the Krylov engine of lqcd_solve*, lqcd_solve_normal and the HMC driver; the
 * BiCGStab vectors; operator and upload temporaries), so repeated solves
 * allocate nothing. This waits for the context's stream and frees them; the
 * next call allocates again. Objects the caller created are untouched. */
LQCD_API int lqcd_ctx_release_cache(lqcd_ctx* ctx);

/* ---------------------------------------------------------------- gauge field (A1) */

/* Uploads an SU(3) gauge field (host layout above) and converts it on the
 * device to the structure-of-arrays even-odd layout. An FP64 18-real copy is
 * always kept (true residuals); `prec` / `compress` (18 or 12 reals, row 2
 * rebuilt from rows 0-1 as conj(row0 x row1), the RECONSTRUCT TWELVE of
 * Section 3) choose the default copy used for fields of that precision.
 * prec LQCD_F16 and LQCD_BF16 both store FP16 links; LQCD_DF64 links always keep
 * 18 reals (compress is ignored for them). t_bc: +1 or -1.
 * The 12-real form assumes det U = 1 (true for the seeded generator). */
LQCD_API int lqcd_gauge_upload(lqcd_ctx* ctx, const int dims[4], const double* host_U, int prec,
                      int compress, int t_bc, lqcd_gauge** out);
/* Same from a device pointer (e.g. a torch tensor) in the host layout. */
LQCD_API int lqcd_gauge_upload_dev(lqcd_ctx* ctx, const int dims[4], const double* dev_U, int prec,
                          int compress, int t_bc, lqcd_gauge** out);
/* Adds a resident copy in another precision / compression (from the FP64 copy). */
LQCD_API int lqcd_gauge_add_copy(lqcd_gauge* g, int prec, int compress);
/* Copies the FP64 master copy back to the host layout above (V x 4 x 3 x 3 complex). */
LQCD_API int lqcd_gauge_download(const lqcd_gauge* g, double* host_U);
/* Device bytes held by the gauge field (all copies). */
LQCD_API size_t lqcd_gauge_bytes(const lqcd_gauge* g);
LQCD_API void lqcd_gauge_destroy(lqcd_gauge* g);

/* ---------------------------------------------------------------- spinor fields (A2) */

/* Allocates a spinor field of the gauge's lattice: subset LQCD_EVEN, LQCD_ODD
 * (one checkerboard, V/2 sites) or LQCD_FULL (both). Contents are zero. */
LQCD_API int lqcd_field_create(lqcd_ctx* ctx, const int dims[4], int prec, int subset, lqcd_field** out);
/* host_psi: full-lattice host spinor; sites outside the field's subset are ignored. */
LQCD_API int lqcd_field_upload(lqcd_field* f, const double* host_psi);
/* Writes the field's sites into host_psi (full-lattice array); other sites untouched. */
LQCD_API int lqcd_field_download(const lqcd_field* f, double* host_psi);
/* Device-pointer variants (full-lattice FP64 array in the host layout, on the device). */
LQCD_API int lqcd_field_upload_dev(lqcd_field* f, const double* dev_psi);
LQCD_API int lqcd_field_download_dev(const lqcd_field* f, double* dev_psi);
/* dst = scale * src on the common subset, converting precision. */
LQCD_API int lqcd_field_copy(lqcd_field* dst, const lqcd_field* src, double scale);
/* ||f||^2 over the field's sites (FP64 accumulation). */
LQCD_API int lqcd_field_norm2(const lqcd_field* f, double* out);
LQCD_API int lqcd_field_zero(lqcd_field* f);
LQCD_API size_t lqcd_field_bytes(const lqcd_field* f);
LQCD_API void lqcd_field_destroy(lqcd_field* f);

/* ---------------------------------------------------------------- operators (A3-A5) */

/* out_{p} = D_{p,1-p} in_{1-p} (hopping term alone; dagger != 0 gives (D^dag)_{p,1-p}
 * = g5 D_{p,1-p} g5). in must hold parity 1-p (subset 1-p or FULL); out must hold
 * parity p. Both fields have the same precision; the gauge copy of that precision
 * (with the gauge's compression) is used. Asynchronous on the context stream. */
LQCD_API int lqcd_dslash_eo(const lqcd_gauge* g, const lqcd_field* in, lqcd_field* out, int out_parity,
                   int dagger);
/* A reusable batch of n independent applications out_i = D_{p,1-p} in_i (as
 * lqcd_dslash_eo), each with its own gauge field and lattice size, all fields of
 * one precision and one context, executed in a single kernel launch by
 * lqcd_dslash_batch_apply. Small lattices leave most of the GPU idle in a launch of
 * their own; batching fills it. The gauges and fields are borrowed and must
 * outlive the batch. Creation uploads the batch description (synchronous); apply
 * is asynchronous on the context stream and allocates nothing. */
LQCD_API int lqcd_dslash_batch_create(int n, const lqcd_gauge* const* g,
                                      const lqcd_field* const* in, lqcd_field* const* out,
                                      int out_parity, int dagger, lqcd_dslash_batch** batch);
LQCD_API int lqcd_dslash_batch_apply(lqcd_dslash_batch* batch);
LQCD_API void lqcd_dslash_batch_destroy(lqcd_dslash_batch* batch);
/* out_e = in_e - kappa^2 D_eo D_oe in_e (or Mhat^dag = g5 Mhat g5 when dagger).
 * in and out hold the even parity (EVEN or FULL); uses an odd temporary of the context. */
LQCD_API int lqcd_apply_Mhat(const lqcd_gauge* g, double kappa, const lqcd_field* in, lqcd_field* out,
                    int dagger);
/* out = M in (full, unpreconditioned); both fields FULL. */
LQCD_API int lqcd_apply_M(const lqcd_gauge* g, double kappa, const lqcd_field* in, lqcd_field* out,
                 int dagger);
/* Twisted-mass operators (paper Section 3): M = A - kappa D with the site-diagonal
 * A = 1 + i a g5, a = 2 kappa mu, and its even-odd Schur complement
 * Mhat = A - kappa^2 D_eo A^-1 D_oe, A^-1 = (1 - i a g5) / (1 + a^2). dagger gives the
 * adjoint (M(mu)^dag = g5 M(-mu) g5). Arguments, layouts and errors as for lqcd_apply_M
 * and lqcd_apply_Mhat; mu = 0 is exactly the Wilson operator. */
LQCD_API int lqcd_apply_M_tm(const lqcd_gauge* g, double kappa, double mu, const lqcd_field* in,
                             lqcd_field* out, int dagger);
LQCD_API int lqcd_apply_Mhat_tm(const lqcd_gauge* g, double kappa, double mu, const lqcd_field* in,
                                lqcd_field* out, int dagger);

/* Mhat exactly as lqcd_apply_Mhat, for callers that cannot let the library
 * allocate device memory: applications whose device memory belongs to their
 * own pool (a caching allocator such as PyTorch's, or a fixed-budget arena),
 * where a library cudaMalloc can fail while the pool still holds free blocks,
 * and latency-sensitive callers that cannot accept the device-wide
 * synchronisation of cudaMalloc / cudaFree. The paper has no counterpart; this
 * is an interface addition of the library.
 * The odd-parity temporary lives in a fixed 16 MiB device array that is part of
 * the library image (every GPU that loads the library holds it until the process
 * exits). Lattices whose half spinor exceeds it (FP32 beyond V/2 = 174762 sites,
 * FP64 and double-float beyond V/2 = 87381) are rejected with LQCD_EINVAL, and so are
 * a non-finite kappa and a gauge field without the resident link copy that
 * lqcd_apply_Mhat would use for the fields' precision (the gauge's compression; 18
 * reals for LQCD_DF64): make it first with lqcd_gauge_add_copy. The call never calls
 * cudaMalloc, cudaFree or an allocating routine. Its first call on a device looks the
 * array's device address up with cudaGetSymbolAddress while that device is current
 * (and again after the device's context was destroyed and made anew, e.g. by
 * cudaDeviceReset); make that first call before any stream capture. Every call uses the same array: calls whose GPU work can
 * overlap (different streams or contexts on one device without ordering between
 * them) race on it. The temporary is fully written before it is read, so a call
 * never sees what an earlier call left there. */
LQCD_API int lqcd_apply_Mhat_noalloc(const lqcd_gauge* g, double kappa, const lqcd_field* in,
                                     lqcd_field* out, int dagger);

/* ---------------------------------------------------------------- solvers (A6-A9) */

typedef struct lqcd_solve_opts {
  int solver;           /* LQCD_CG or LQCD_BICGSTAB */
  int sloppy_prec;      /* LQCD_F64: plain FP64 solve; LQCD_DF64: double-float solve;
                           LQCD_F32 / F16 / BF16: mixed precision */
  int sloppy_compress;  /* 18 or 12 reals per link of the sloppy operator */
  int maxiter;          /* iteration limit (default 50000) */
  double delta;         /* reliable-update threshold on |r| (<= 0: 0.01 for FP16 / BF16 sloppy,
                           0.001 for FP32 sloppy, none for FP64 and double-float) */
  int chunk;            /* iterations per CUDA-graph replay / host poll (default 8) */
  int use_graph;        /* 1: capture iteration chunks as CUDA graphs (default 1) */
  int ru_interval;      /* iterations between reliable-update blocks in a CUDA-graph chunk
                           (0: default 4) */
  int true_prec;        /* FP64-class true residual, solution and outer correction: LQCD_F64
                           (native) or LQCD_DF64 (double-float); -1 (default): LQCD_F64 for an
                           FP64 solve, LQCD_DF64 otherwise */
  int multi_rhs_links;  /* solves that share one gauge field in a batch (lqcd_solve_multi,
                           lqcd_solve_batch, engines), sloppy FP32 / FP16 / BF16 Wilson: 0
                           (default) the sloppy Dslash loads each site block's links once for
                           a group of those solves when the autotuner measured that faster
                           (lqcd_autotune_dslash), else each solve loads its own; 1 always
                           shares them (the tuned group size if there is one, else groups as
                           large as leave 8 tiles per SM); -1 never shares. The results are
                           the same bit for bit in every case. */
  double mu;            /* twisted mass (paper Section 3: M = 1 - kappa D + 2 i kappa mu g5,
                           one flavour of the N_f = 2 doublet; the other is -mu). 0 (default):
                           the Wilson operator. Any finite value. */
} lqcd_solve_opts;

typedef struct lqcd_solve_info {
  int status;            /* LQCD_OK, LQCD_ENOCONV, LQCD_EBREAKDOWN, LQCD_ENONFINITE */
  int iters;             /* Krylov iterations (sloppy) */
  int reliable_updates;  /* FP64 true-residual recomputations */
  int pad;
  double true_resid;     /* ||b - M x|| / ||b|| with the full FP64 operator */
  double ms;             /* wall time of the call */
} lqcd_solve_info;

LQCD_API void lqcd_solve_opts_default(lqcd_solve_opts* opts);

/* Solves M x = b (full lattice) through the even-odd Schur system to
 * ||b - M x|| <= tol ||b||, checked in FP64 on the full operator. host_src and
 * host_x are full-lattice host spinors. info (may be NULL) is filled even on
 * failure; the return value equals info->status. */
LQCD_API int lqcd_solve(const lqcd_gauge* g, const double* host_src, double kappa, double tol,
               const lqcd_solve_opts* opts, double* host_x, lqcd_solve_info* info);
/* Same with device fields: src and x are FULL FP64 fields. */
LQCD_API int lqcd_solve_fields(const lqcd_gauge* g, const lqcd_field* src, double kappa, double tol,
                      const lqcd_solve_opts* opts, lqcd_field* x, lqcd_solve_info* info);
/* Multi-right-hand-side solve (A10): n sources on one gauge field, one batched
 * Krylov recurrence per source, links streamed once per site block for all
 * sources. srcs[i], xs[i]: FULL FP64 fields. infos: n entries (may be NULL).
 * Returns LQCD_OK if every solve converged, else the first failing status. */
LQCD_API int lqcd_solve_multi(const lqcd_gauge* g, int n, const lqcd_field* const* srcs, double kappa,
                     double tol, const lqcd_solve_opts* opts, lqcd_field* const* xs,
                     lqcd_solve_info* infos);
/* Batched one-shot solve (A10, A11): n independent systems M(kappas[i], mu) x_i = b_i,
 * each on its own gauge field gauges[i] (any lattice sizes; all of one context), to its
 * own tolerance tols[i], advanced together in the batched engine's launches. Gauges that
 * are the same object share their link reads (multi-RHS); different ones form a
 * multi-lattice batch. srcs[i], xs[i]: FULL FP64 fields of gauges[i]'s lattice. Each
 * result equals the solve of that system alone, bit for bit. opts->solver LQCD_BICGSTAB
 * runs the systems one after another. infos: n entries (may be NULL). Returns LQCD_OK if
 * every solve converged, else the first failing status; LQCD_EINVAL for n outside
 * 1..1024, a NULL entry, or gauges of different contexts. */
LQCD_API int lqcd_solve_batch(int n, const lqcd_gauge* const* gauges, const lqcd_field* const* srcs,
                              const double* kappas, const double* tols, const lqcd_solve_opts* opts,
                              lqcd_field* const* xs, lqcd_solve_info* infos);

/* ---------------------------------------------------------------- pure gauge */

/* SU(3) heatbath of the Wilson plaquette action S = beta sum_P (1 - Re Tr U_P / 3)
 * (paper Section 3: the pure-gauge side needs an SU(3) heatbath, citing Creutz), in
 * place. The sweeps run on the gauge field's double-float copy (matrix algebra in
 * double-float, the draws in FP64); the FP64 master and every other copy of g are
 * rebuilt from it afterwards, so the links carry a 48-bit significand. nsweeps sweeps, numbered sweep0, sweep0 + 1, ...; a sweep updates the
 * links class by class (mu = 0..3, parity even then odd), each link by Cabibbo-Marinari
 * over the SU(2) subgroups (0,1), (1,2), (0,2) with Creutz's SU(2) draw. Random numbers
 * are Philox4x64-10 with key (seed, 0) and counter (4 s + mu, sweep, subgroup, attempt),
 * s the lexicographic site index, so the result depends only on the links, beta, seed
 * and sweep numbers. reunit != 0: reunitarise every link after each sweep. A draw that
 * is not accepted within 1000 attempts leaves its subgroup unchanged; *fails (may be
 * NULL) counts them. beta must be finite and >= 0. Synchronous. */
LQCD_API int lqcd_heatbath(lqcd_gauge* g, double beta, int nsweeps, unsigned long long seed,
                           unsigned long long sweep0, int reunit, long long* fails);
/* Average plaquette sum_{x, mu<nu} Re Tr U_munu(x) / (18 V) of the FP64 master copy,
 * summed in a fixed order (deterministic). Synchronous. */
LQCD_API int lqcd_plaquette(const lqcd_gauge* g, double* plaq);

/* ---------------------------------------------------------------- HMC */

/* Hybrid Monte Carlo for N_f = 2 (twisted-mass) Wilson fermions with even-odd
 * preconditioning (paper Section 3: HMC with even-odd preconditioning, the 2MN integrator
 * and multiple integration timescales). Conventions:
 *   S = beta sum_P (1 - Re Tr U_P / 3) + phi^dag (Mhat^dag Mhat)^-1 phi (even sites),
 *   Mhat as lqcd_apply_Mhat_tm; momenta P traceless anti-Hermitian per link, kinetic energy
 *   -sum Tr(P^2) / 2; dU/dt = P U, dP/dt = -G with G the su(3) gradient of S
 *   (dS/de = -sum Tr(H G) for U -> exp(e H) U).
 * A momentum field (lqcd_mom) holds one traceless anti-Hermitian 3x3 per link in FP64; its
 * host layout is that of the links, V x 4 x 3 x 3 complex. */
LQCD_API int lqcd_mom_create(lqcd_ctx* ctx, const int dims[4], lqcd_mom** out);  /* zeroed */
LQCD_API int lqcd_mom_upload(lqcd_mom* m, const double* host);
LQCD_API int lqcd_mom_download(const lqcd_mom* m, double* host);
LQCD_API int lqcd_mom_zero(lqcd_mom* m);
/* -sum Tr(P^2) / 2, summed in a fixed order. Synchronous. */
LQCD_API int lqcd_mom_kinetic(const lqcd_mom* m, double* energy);
LQCD_API void lqcd_mom_destroy(lqcd_mom* m);
/* m += coeff G_g, G_g = (beta/3) TA(U W) (W the staple sum, TA the traceless
 * anti-Hermitian part). Asynchronous. */
LQCD_API int lqcd_gauge_force(const lqcd_gauge* g, double beta, double coeff, lqcd_mom* m);
/* m += coeff G_f for the solution x = (Mhat^dag Mhat)^-1 phi (FULL FP64 field, even half
 * used): with Y = Mhat x, Phi = x_e + A^-1 D_oe x_e, Psi = Y + A^-dag (D^dag)_oe Y,
 * G_f = -2 kappa^2 eta TA(U [((1 - g_mu) Phi(x+mu))^T conj(Psi(x)) + Psi(x+mu)^T
 * conj((1 + g_mu) Phi(x))]) (spin summed; eta the t-boundary sign), computed in
 * double-float. x is not modified. *s_f (may be NULL) receives S_f = |Y|^2 = phi^dag x.
 * Synchronous. */
LQCD_API int lqcd_fermion_force(const lqcd_gauge* g, double kappa, double mu, const lqcd_field* x,
                                double coeff, lqcd_mom* m, double* s_f);
/* U_mu(x) <- exp(eps P_mu(x)) U_mu(x) in double-float (the Taylor polynomial, to a tail
 * below 2^-50, after scaling |eps P| below 1/2, reduced by Cayley-Hamilton to one matrix
 * product; then squaring). The FP64 master and the derived link copies are rebuilt. */
LQCD_API int lqcd_gauge_update(lqcd_gauge* g, const lqcd_mom* m, double eps);
/* Solves (Mhat^dag Mhat) x_e = src_e by the CG engine (mixed precision with reliable
 * updates as lqcd_solve; opts->mu the twisted mass; CG only) to
 * |src_e - Mhat^dag Mhat x_e| <= tol |src_e| in FP64-class arithmetic. src, x: FULL FP64
 * fields; the odd half of src is ignored and that of x is zeroed. */
LQCD_API int lqcd_solve_normal(const lqcd_gauge* g, const lqcd_field* src, double kappa, double tol,
                               const lqcd_solve_opts* opts, lqcd_field* x, lqcd_solve_info* info);

#define LQCD_LEAPFROG 0
#define LQCD_2MN 1   /* second-order minimum norm (Omelyan, Mryglod, Folk), lambda 0.1931833275 */

typedef struct lqcd_hmc_params {
  double beta, kappa, mu;  /* gauge coupling, hopping parameter, twisted mass */
  double tau;              /* trajectory length */
  int nsteps;              /* outer (fermion force) steps */
  int ngauge;              /* inner (gauge force) steps per outer step, >= 1 */
  int scheme;              /* LQCD_LEAPFROG or LQCD_2MN, on both levels */
  int chrono;              /* initial guess of each force solve after the first: 0 (default) x = 0;
                              1 the last solution; 2 the linear extrapolation 2 X_last - X_before.
                              The solves still converge to tol, so the trajectory changes only at
                              the level of tol (and is reversible only to that level) */
  double tol;              /* residual of the force solves (normal equations) */
  double accept_u;         /* uniform in (0, 1] for the Metropolis test; <= 0: no test, links kept */
} lqcd_hmc_params;

typedef struct lqcd_hmc_info {
  double dH, H0, H1;                 /* H1 - H0 */
  double kinetic0, kinetic1, gauge0, gauge1, fermion0, fermion1;
  double plaquette;                  /* of the links left in g */
  int accepted, force_evals, solver_iters, pad;
  double ms;
} lqcd_hmc_info;

LQCD_API void lqcd_hmc_params_default(lqcd_hmc_params* p);
/* One molecular-dynamics trajectory from (g, m) with pseudofermion phi (FULL FP64, even half
 * used; S_f at the start = phi^dag (Mhat^dag Mhat)^-1 phi, evaluated from each force solve's X
 * as 2 Re <phi, X> - |Mhat X|^2, whose error is quadratic in the solve's). Updates g and m in place. The
 * gauge force runs ngauge inner steps per outer step; kicks at the same links are merged,
 * so a trajectory takes nsteps + 1 fermion solves (leapfrog) or 2 nsteps + 1 (2MN). With
 * accept_u > 0 the links are restored when accept_u > exp(-dH). opts: the solver (CG;
 * sloppy precision, reliable updates); opts->mu is replaced by p->mu. Synchronous. */
LQCD_API int lqcd_hmc_trajectory(lqcd_gauge* g, const lqcd_hmc_params* p, lqcd_mom* m,
                                 const lqcd_field* phi, const lqcd_solve_opts* opts, lqcd_hmc_info* info);

/* ---------------------------------------------------------------- meson correlators */

/* Dirac structures Gamma of lqcd_meson_correlator (chiral basis above) */
#define LQCD_G_1 0    /* scalar */
#define LQCD_G_5 1    /* pseudoscalar g5 */
#define LQCD_G_X 2    /* vector g_x, g_y, g_z, g_t: 2..5 */
#define LQCD_G_5X 6   /* axial g5 g_x, ..., g5 g_t: 6..9 */

/* Meson two-point functions from a point-source propagator (paper Section 4, eq. 4.1):
 *   C_Gamma(t) = sum over spatial x of  - Tr[ S^dag(x) g5 Gamma S(x) Gamma g5 ],
 * trace over spin and colour, where S(x) is the 12 x 12 matrix whose column 3*beta+b
 * is props[3*beta+b] (the solution for the point source of spin beta, colour b) at
 * site x. props: 12 FULL FP64 fields of one lattice. gammas: ngamma (<= 16) codes.
 * host_corr: ngamma x Lt complex values (re, im), t the absolute time coordinate.
 * Synchronous; the per-slice sum is in a fixed order (deterministic). */
LQCD_API int lqcd_meson_correlator(const lqcd_field* const* props, int ngamma, const int* gammas,
                                   double* host_corr);

/* ---------------------------------------------------------------- batched engine (A11, A12) */

/* A Krylov engine that advances many independent solves (any lattice sizes,
 * own gauge field and kappa each) in the same kernel launches. hbm_budget:
 * device bytes the engine may hold for solver state (0: no limit); max_slots:
 * concurrent solves (<= 1024). opts: as for lqcd_solve (CG only). */
LQCD_API int lqcd_engine_create(lqcd_ctx* ctx, const lqcd_solve_opts* opts, size_t hbm_budget,
                       int max_slots, lqcd_engine** out);
/* Device bytes one request on this lattice holds while active. */
LQCD_API size_t lqcd_engine_request_bytes(const lqcd_engine* e, const int dims[4]);
/* Admits a solve of M x = src (src: FULL FP64 field, copied at submit). Returns
 * LQCD_EBUSY when no slot or not enough budget is free now (the caller retries
 * after results are collected), LQCD_ENOMEM when the request can never fit. */
LQCD_API int lqcd_engine_submit(lqcd_engine* e, const lqcd_gauge* g, const lqcd_field* src, double kappa,
                       double tol, long long* request_id);
/* The same for the twisted-mass operator with this request's mu (lqcd_engine_submit
 * takes mu from the engine's options); requests with different kappa and mu share
 * the engine's launches. LQCD_EINVAL for a non-finite kappa or mu. */
LQCD_API int lqcd_engine_submit_tm(lqcd_engine* e, const lqcd_gauge* g, const lqcd_field* src,
                                   double kappa, double mu, double tol, long long* request_id);
/* Admits a solve of the even-odd normal equations (Mhat^dag Mhat) x_e = src_e (the HMC
 * force solve): src FULL FP64 with its odd half ignored; converged when
 * |src_e - Mhat^dag Mhat x_e| <= tol |src_e| (FP64-class); the result's odd half is zero. */
LQCD_API int lqcd_engine_submit_normal(lqcd_engine* e, const lqcd_gauge* g, const lqcd_field* src,
                                       double kappa, double mu, double tol, long long* request_id);
/* Runs one chunk of iterations for every active solve; *n_active: solves still running. */
LQCD_API int lqcd_engine_step(lqcd_engine* e, int* n_active);
/* Ids of solves finished since the last call (up to max). */
LQCD_API int lqcd_engine_completed(lqcd_engine* e, long long* ids, int max, int* n);
/* Copies the solution of a finished request into x (FULL FP64) and frees its slot. */
LQCD_API int lqcd_engine_result(lqcd_engine* e, long long request_id, lqcd_field* x, lqcd_solve_info* info);
/* Stops a running request: it finishes at the next step with `status` (a negative
 * LQCD_E* code, e.g. LQCD_ETIMEOUT) and its best iterate so far. */
LQCD_API int lqcd_engine_cancel(lqcd_engine* e, long long request_id, int status);
/* Active solves and device bytes in use. */
LQCD_API int lqcd_engine_stats(const lqcd_engine* e, int* active, size_t* bytes_in_use);
LQCD_API void lqcd_engine_destroy(lqcd_engine* e);

/* ---------------------------------------------------------------- instrumentation */

/* Measured fused multiply-add throughput of the context's device in TFLOP/s (2 flop per
 * FMA): kind 0 FP64, kind 1 FP32, kind 2 FP32 issued as packed pairs (fma.rn.f32x2, two
 * FMAs per lane and instruction). The FP64 Dslash and the double-float kernels are bound
 * by these rates rather than by HBM on GB300, whose FP64 pipe runs at a small fraction of
 * its FP32 rate; the paper has no counterpart (it reports FP64 GFLOP/s on an AMD GPU).
 * Runs a probe kernel of independent FMA chains on every SM six times on the context
 * stream (the first as warm-up) and reports the fastest; about 0.1 s. Synchronous;
 * allocates and frees a few bytes. LQCD_EINVAL for another kind. */
LQCD_API int lqcd_alu_peak(lqcd_ctx* ctx, int kind, double* tflops);

/* Debug build (compiled with -DLQCD_DEBUG_BOUNDS; lqcd.py loads it when the environment
 * variable LQCD_DEBUG_BOUNDS=1): every spinor and link access of the batched kernels checks
 * its site index against the field; the first index outside is recorded and replaced by 0,
 * so that the kernel stays inside its buffers (no trap). This waits for the context's stream
 * and returns in *word the first record since the last call, (1 << 63) | (Vh << 32) | index,
 * or 0, and clears the records. LQCD_EINVAL in the normal build. */
LQCD_API int lqcd_debug_bounds(lqcd_ctx* ctx, unsigned long long* word);

/* ---------------------------------------------------------------- tuning */

/* Caps the persistent grid of batched kernel family (0 Dslash, 1 BLAS) at
 * mult CTAs per SM (0: occupancy limit). */
LQCD_API void lqcd_set_grid_multiplier(int family, int mult);
/* Dslash kernel form for LQCD_DF64 fields: 0 = one thread per output site, 1 = three
 * threads per site, one per output colour (default). Results agree to rounding. */
LQCD_API int lqcd_set_dslash_form(int prec, int form);

/* Launch autotuner: the persistent batched Dslash takes its grid shape and kernel form
 * from measurement on this device. lqcd_autotune_dslash times one batched Dslash launch
 * over n slots (slot i on gauge g[i], which may repeat; fields of precision prec, zero
 * valued scratch allocated and freed by the call) for every distinct persistent grid,
 * 1 .. occupancy-limit CTAs per SM, of every compiled kernel form (for LQCD_F32 also the
 * one-thread-per-site Dslash compiled for 8 CTAs per SM, a second register budget), and
 * records the fastest. The default (occupancy limit, default form) is kept unless another choice is
 * more than 2% faster. The record applies to every later Dslash launch (lqcd_dslash_eo,
 * batches, operators, solves, engines) of the same precision and link reals whose tile
 * count (64 output sites a tile) has the same floor(log2).
 * When all n > 1 slots are on the same gauge field (n right-hand sides, as in
 * lqcd_solve_multi) and prec is LQCD_F32, LQCD_F16 or LQCD_BF16, it also times the
 * shared-link form, in which a CTA loads a site block's links once and applies them to a
 * group of slots, for every group size ceil(n / d) >= 2 and every grid, and records, under
 * (prec, link reals, n, floor(log2) of the site blocks), the group size of the fastest
 * (kept only when more than 2% faster than the slots loading their own links; else 0).
 * Engines with n slots on one gauge field take that group size in their sloppy steps.
 * Synchronous; not to be run while another thread launches on the same device. The table
 * is process-wide. */
typedef struct lqcd_tune_result {
  int prec;         /* spinor precision of the key */
  int nr;           /* link reals of the key (12 or 18) */
  int ntiles;       /* tiles of the tuned launch */
  int ctas_per_sm;  /* chosen persistent grid, CTAs per SM (0: occupancy limit) */
  int form;         /* chosen kernel form: 0 one thread per site, 1 colour split (DF64),
                       2 shared-link multi-RHS, 3 one thread per site compiled for 8 CTAs
                       per SM (FP32: 128 registers, more warps with fewer loads each) */
  int candidates;   /* configurations timed */
  double us_best;   /* per launch, chosen configuration */
  double us_default;/* per launch, untuned default (shared-link entries: the own-link launch) */
  int nrhs;         /* 0: launch-shape entry; n >= 2: shared-link entry for n slots on one gauge */
  int group;        /* shared-link entries: slots per group (0: own links faster) */
} lqcd_tune_result;
LQCD_API int lqcd_autotune_dslash(int n, const lqcd_gauge* const* g, int prec, int compress,
                                  lqcd_tune_result* out);
/* Copies up to max table entries into out; *n = entries in the table. */
LQCD_API int lqcd_tune_entries(lqcd_tune_result* out, int max, int* n);
LQCD_API void lqcd_tune_clear(void);
/* JSON file of the table ({"format": "lqcd-tune", "version": 2, "device": name_smN,
 * "entries": [{prec, nr, nrhs, bucket, ntiles, ctas_per_sm, form, group, candidates,
 * us_best, us_default}, ...]}); loading a file made on another device model, or a malformed
 * file or entry, gives LQCD_EINVAL and loads nothing. */
LQCD_API int lqcd_tune_save(const char* path);
LQCD_API int lqcd_tune_load(const char* path);

#ifdef __cplusplus
}
#endif
#endif /* LQCD_H */
