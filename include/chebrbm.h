/*
 * chebrbm.h -- C ABI of the GB300 (sm_103a) hot path of the RBM-Chebyshev
 * method for spin spectral functions: Hendry, Chen, Weinberg, Feiguin,
 * "Chebyshev expansion of spectral functions using restricted Boltzmann
 * machines", arXiv:2103.08804.
 *
 * One projection step of the Chebyshev recursion fits a complex RBM psi_n to
 * the target phi_n = 2 beta_{n-1} H' t~_{n-1} - beta_{n-2} t~_{n-2}
 * (Sec. III, last paragraph) by the natural-gradient update of Sec. III,
 * with every expectation sampled from |psi_n|^2.  The calls below are the
 * steps of that projection in the paper's order:
 *
 *   rbm_logpsi        theta and log psi of the RBM ansatz           (Sec. I)
 *   mc_sweep          Metropolis sampling of |psi_s|^2              (Sec. III)
 *   cheb_local_target R(s) = phi_s / psi_s over Heisenberg bonds    (Secs. III, V)
 *   logderiv          O_k(s) = d log psi_s / d alpha_k              (Sec. III)
 *   logpsi_backward   sum_s g_s conj(O_k(s)), the VJP of log psi    (Sec. III)
 *   sr_step           <R>, <|R|^2>, <O*>, <O* R>, gamma, F, S and the
 *                     shifted solve (S + lambda I) dalpha = F      (Sec. III)
 *   cheb_moment       beta_n, mu_n and the Krylov columns           (Secs. II, IV)
 *   cheb_gram         sigma_nm = <t_n|t_m>, H_nm = <t_n|H'|t_m>     (Sec. IV)
 *   cheb_krylov       moment correction and projected eigenproblem  (Secs. IV, V)
 *   cheb_extrapolate  higher moments by linear prediction           (Sec. VI)
 *
 * CONVENTIONS
 *   Memory. Every array argument is a DEVICE pointer owned by the caller,
 *     unless a comment says "host". The library never frees caller memory.
 *     The context owns only its workspace, allocated once in cr_create, so
 *     the hot calls allocate nothing and can be captured in a CUDA graph.
 *     The exceptions are cheb_krylov, cheb_extrapolate and, in CR_MIXED
 *     contexts, cheb_gram (called once per sequence or momentum), which
 *     size their scratch on first use (and grow it for larger inputs).
 *   Streams. Every call is asynchronous on the context's stream; results
 *     are valid after that stream is synchronised.
 *   Precision. "complex" arrays are interleaved (re, im) in the context's
 *     storage precision: complex128 for CR_FP64, complex64 for CR_FP32 and
 *     CR_MIXED. Results documented as complex128 (beta, mu, F, stats, G, H)
 *     are complex128 in every mode.
 *   Parameters. An RBM with N visible and M hidden units is one complex
 *     vector alpha = [a (N) | b (M) | W (N x M, row-major, W[i*M + j])];
 *     its index is the k of O_k, S_kk' and F_k. P = N + M + N*M.
 *   Spins. int8 [B][N], entries +1 / -1, site r = x + Lx*y.
 *   Lattice. Periodic; bonds are all (r, r + x-hat) in increasing r and
 *     then, when Ly > 1, all (r, r + y-hat) in increasing r.
 *   Hamiltonian. H = J sum_b S_i . S_j with S^z = sigma/2 (Sec. V);
 *     H' = (H - E0)/a - W' (Sec. II).
 *   Errors. Argument checks return a status synchronously and set the text
 *     returned by cr_last_error. Failures detected on the device (a
 *     non-positive Cholesky pivot, non-finite estimators or parameters, a
 *     bounded device wait that gave up) set a device status word that
 *     cr_sync_status reads and clears. CG that stops at its iteration limit
 *     above tolerance is an error (CR_ENOTCONV) only when the caller asks for
 *     it (cr_sr_opts.cg_strict); sr_step always reports the iteration count
 *     and residual in its stats, so a fixed CG budget can be run and its
 *     truncation measured.
 *   B == 0 is valid for every call and launches nothing.
 */
#ifndef CHEBRBM_H
#define CHEBRBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cr_ctx cr_ctx;

typedef enum {
    CR_OK = 0,
    CR_EINVAL = 1,      /* bad argument */
    CR_ENOMEM = 2,      /* workspace allocation failed (cr_create only) */
    CR_ECUDA = 3,       /* a CUDA runtime call or launch failed */
    CR_ETIMEOUT = 4,    /* a bounded device wait gave up */
    CR_ENOTCONV = 5,    /* CG reached its iteration limit above tolerance */
    CR_ESINGULAR = 6,   /* Cholesky met a non-positive pivot */
    CR_ENONFINITE = 7   /* NaN or Inf in an estimator */
} cr_status;

typedef enum {
    CR_FP64 = 0,        /* everything in float64 */
    CR_FP32 = 1,        /* float32 storage and arithmetic, float64 sums and solve */
    CR_MIXED = 2        /* float32 storage; contractions on the tensor cores in
                           split bf16 (3 terms) with float32 accumulation;
                           float64 sums and solve */
} cr_prec;

/* Context flags. */
#define CR_CTX_EXPLICIT_S 1 /* allocate the explicit P x P complex128 S for
                               Cholesky solves */
#define CR_CTX_S_BF16X3 2   /* mixed contexts: build the explicit S from two-term
                               bf16 splits (three products, about 2^-16 relative
                               per product) instead of the default three-term
                               splits (six products, about float32 accuracy).
                               Cheaper, but its error can make S + shift I
                               indefinite at small shifts (CR_ESINGULAR). */

/* Modes of sr_step.  CR_SR_FIT: the projection fit of Sec. III (R = phi/psi,
   F = dgamma gamma cot gamma (<O* R>/<R> - <O*>)).  CR_SR_ENERGY: ground-state
   preparation (Sec. I: minimise <H>), R = the local energy (H psi)/psi in any
   affine units (e.g. cheb_local_target with n = 1, prev = psi, beta = 1 gives
   the local H'), F = -dgamma (<O* R> - <O*> <R>), dgamma the learning rate;
   stats [0] is then 0. */
#define CR_SR_FIT 0
#define CR_SR_ENERGY 1

/* Solvers for sr_step. */
#define CR_SOLVE_CHOLESKY 0 /* explicit S and a direct solve (needs CR_CTX_EXPLICIT_S):
                               float64 contexts with P <= 2048 factor S in float64 in one
                               CTA; every other context factors S blocked (64 x 64
                               blocks, many CTAs) in the factor precision (float64 for
                               float64 contexts, float32 otherwise) and refines the
                               solution in float64 against S until |r| <= 1e-12 |F|,
                               the residual stops halving, or min(cg_maxit, 10) steps
                               (stats [5] steps, [6] relative residual).  Mixed
                               contexts build S on the tensor cores (bf16 splits of
                               both operands, float32 accumulation; see
                               CR_CTX_S_BF16X3); the others accumulate it in
                               float64. */
#define CR_SOLVE_CG 1       /* matrix-free S v = O^dag (O v) / Ns, float64 CG */

/* Length of the stats array written by sr_step (complex128 / float64 slots). */
#define CR_STATS_LEN 8
/* stats layout (float64): [0] gamma, [1] Re <R>, [2] Im <R>, [3] <|R|^2>,
   [4] c = dgamma * gamma cot gamma, [5] CG iterations, [6] CG relative
   residual, [7] |F|_2 */

typedef struct {
    int Lx, Ly;         /* Ly == 1: chain of Lx sites. Needs Lx >= 3 and
                           Ly == 1 or Ly >= 3. */
    double J;           /* exchange constant */
} cr_lattice;

/* A variational state: an RBM, optionally times the probe factor.
   probe != 0 means t~(sigma) = f_q(sigma) RBM(sigma) with
   f_q(sigma) = N^{-1/2} sum_r e^{-i q.r} sigma_r / 2, i.e. the exact
   t_0 = S^z_q psi of Sec. II / Appendix B. */
typedef struct {
    const void* params; /* device, complex [P], context precision */
    int probe;
    double qx, qy;
} cr_state;

/* Counter-based random stream (Philox4x32-10, Salmon et al. SC'11).
   key = seed; counter = (walker, step lo, step hi, 0). Host struct; calls
   that draw from it advance `counter` on the host, synchronously.  When
   device_counter is non-NULL the stream position lives on the device
   instead (one uint64): kernels read it there and the library advances it
   on the context stream, so the calls can be captured in a CUDA graph and
   replayed; `counter` is then ignored. */
typedef struct {
    uint64_t seed;
    uint64_t counter;
    uint64_t* device_counter;
} cr_philox;

/* The target of projection step n (Sec. III, last paragraph). */
typedef struct {
    int n;                  /* state being fitted, n >= 1 */
    cr_state prev;          /* t~_{n-1} */
    cr_state prev2;         /* t~_{n-2}; ignored when n == 1 */
    const double* beta_prev;  /* device complex128 [1]: beta_{n-1}; beta_0 = 1 */
    const double* beta_prev2; /* device complex128 [1]: beta_{n-2}; ignored when n == 1 */
    double E0, a, Wp;       /* H' = (H - E0)/a - W' */
} cr_target;

typedef struct {
    double dgamma;          /* rotation fraction delta-gamma of Sec. III */
    double shift;           /* additive diagonal shift lambda > 0 */
    int solver;             /* CR_SOLVE_CHOLESKY or CR_SOLVE_CG */
    int cg_maxit;           /* CG iteration limit (CG only) */
    double cg_tol;          /* CG stops when |r| <= cg_tol |F| */
    int cg_precond;         /* 0: plain CG; 1: Jacobi preconditioner diag(S) + shift */
    int mode;               /* CR_SR_FIT (Sec. III fit) or CR_SR_ENERGY (ground state) */
    int cg_strict;          /* 1: CG ending at cg_maxit with |r| > cg_tol |F| sets CR_ENOTCONV
                               in the device status word; 0: it does not (the update
                               is still applied in both cases) */
} cr_sr_opts;

/* ---------------------------------------------------------------- context */

/* Create a context for one lattice and hidden-layer width M.
   max_walkers bounds B in every later call. flags: CR_CTX_EXPLICIT_S.
   stream: a cudaStream_t (NULL = legacy default stream).
   Allocates all workspace; returns CR_ENOMEM / CR_ECUDA on failure. */
cr_status cr_create(cr_ctx** out, const cr_lattice* lattice, int M, int max_walkers,
                    cr_prec prec, int flags, void* stream);
cr_status cr_destroy(cr_ctx* ctx);
/* Rebind the context to another stream (e.g. a graph-capture stream). */
cr_status cr_set_stream(cr_ctx* ctx, void* stream);
/* Walker chunks of the split-K reductions (the sums over walkers in F, the
   O averages and O^dag u are formed per chunk, then combined in float64 in
   chunk order).  cr_create picks ceil(max_walkers / 128), at most 128, which
   is also the largest value cr_set_chunks accepts (cr_max_chunks).  Fewer
   chunks launch fewer CTAs, which pays when several contexts run
   concurrently on one GPU; the results change only by the summation order.
   Returns CR_EINVAL outside [1, cr_max_chunks]. */
cr_status cr_set_chunks(cr_ctx* ctx, int n_chunks);
int cr_max_chunks(const cr_ctx* ctx);
/* Text of the last error of this context (static storage in the context). */
const char* cr_last_error(const cr_ctx* ctx);
/* Synchronise the context stream, then read and clear the device status
   word: returns the first device-side error since the last call, or CR_OK. */
cr_status cr_sync_status(cr_ctx* ctx);
/* Instrumentation.  cr_n_launches: kernels this context has launched so far
   (host counter).  cr_time_kernel arms CUDA-event timing of one kernel
   family (CR_KERNEL_*; -1 disarms): every later launch of it records a
   start/stop event pair on the context stream, up to `capacity` launches
   (events are created here, outside any hot call).  cr_kernel_times
   synchronises the stream and writes the recorded durations in ms (host
   float [capacity]); returns their count, or -1 on error. */
#define CR_KERNEL_SWEEP 0   /* Metropolis sweep */
#define CR_KERNEL_TARGET 1  /* H' application: local target and moment columns */
#define CR_KERNEL_THETA 2   /* theta = b + sigma W and log psi */
#define CR_KERNEL_OV 3      /* u = O v (matrix-free S, first half) */
#define CR_KERNEL_REDUCE 4  /* sum_s op(O_k(s)) g_s (F, Obar, S v second half, VJP) */
#define CR_KERNEL_CG 5      /* CG vector update */
#define CR_KERNEL_SBUILD 6  /* explicit S: Gram matrix of O */
#define CR_KERNEL_CHOL 7    /* blocked Cholesky factor (potrf, trsm, syrk) */
#define CR_KERNEL_TRSV 8    /* triangular solves of the refinement */
#define CR_KERNEL_FCG 9     /* fused CG solve (mixed contexts: one launch per solve) */
#define CR_KERNEL_GRAM 10   /* Krylov Gram G, H on the tensor cores (mixed contexts) */
long long cr_n_launches(const cr_ctx* ctx);
cr_status cr_time_kernel(cr_ctx* ctx, int kernel_id, int capacity);
int cr_kernel_times(cr_ctx* ctx, float* ms_out, int capacity);

/* CTAs of the fused CG kernel (its walker-block shape: walkers per CTA =
   ceil(B / n_ctas)).  0 (the default) takes one CTA per SM; a smaller count
   leaves SMs to other sequences' kernels running at the same time (the
   batch autotuner's knob).  Clamped below to what the kernel's per-CTA
   limits need (512 walkers and 512 parameters per CTA); CR_EINVAL above the
   SM count or for a context without the fused CG. */
cr_status cr_set_fcg_ctas(cr_ctx* ctx, int n_ctas);

/* 1 when sr_step's CG runs as one fused persistent kernel in this context
   (CR_MIXED contexts with N, M <= 256 whose walker and parameter counts fit
   the kernel's per-CTA limits), else 0. */
int cr_fused_cg(const cr_ctx* ctx);

/* Sizes: N, M, P, number of bonds. */
int cr_n_sites(const cr_ctx* ctx);
int cr_n_hidden(const cr_ctx* ctx);
int cr_n_params(const cr_ctx* ctx);
int cr_n_bonds(const cr_ctx* ctx);

/* ------------------------------------------------------------- hot path */

/* Sec. I: theta_j = b_j + sum_i W_ij sigma_i and
   log psi = sum_i a_i sigma_i + sum_j log(2 cosh theta_j) (principal log per
   term, so log psi is defined mod 2 pi i). The probe flag of `state` is
   ignored: this is the RBM factor alone.
   spins [B][N]; theta_out complex [B][M] or NULL; logpsi_out complex [B]. */
cr_status rbm_logpsi(cr_ctx* ctx, const cr_state* state, const int8_t* spins, int B,
                     void* theta_out, void* logpsi_out);

/* Sec. III: Metropolis sampling of |psi_s|^2 / <psi|psi>. Each walker makes
   n_sweeps * N proposals; a proposal picks a bond uniformly
   (floor(u0 * N_b / 2^32)) and, if its spins are antiparallel, exchanges them
   with probability min(1, |psi(s')/psi(s)|^2), accepting iff
   ((u1 >> 9) + 1/2) / 2^23 < |psi(s')/psi(s)|^2. Proposal p of walker w uses
   Philox call counter + p/2, words (2(p%2), 2(p%2)+1). The stream position
   (rng->counter, or *rng->device_counter) advances by ceil(n_sweeps * N / 2).
   Total S^z is conserved.
   spins [B][N] in/out. theta [B][M] in/out: on entry it must equal
   b + sigma W for `state` (as written by rbm_logpsi); on exit it matches the
   new spins. logpsi_out [B] (NULL allowed), tanh_out [B][M] = tanh(theta)
   (NULL allowed), n_accepted [B] int32 accepted moves in this call (NULL
   allowed). The probe flag of `state` must be 0. */
cr_status mc_sweep(cr_ctx* ctx, const cr_state* state, int8_t* spins, void* theta, int B,
                   int n_sweeps, cr_philox* rng, void* logpsi_out, void* tanh_out,
                   int32_t* n_accepted);

/* Secs. III and V: R(s) = phi_n(s) / psi_n(s) with
   phi_1 = beta_0 H' t~_0 and phi_n = 2 beta_{n-1} H' t~_{n-1} - beta_{n-2} t~_{n-2},
   (H v)(s) = sum_b [(J/4) s_i s_j v(s) + (J/2)[s_i != s_j] v(s^{ij})].
   spins [B][N] samples of |psi_n|^2, logpsi_n [B] log psi_n at those
   samples (from mc_sweep or rbm_logpsi), R_out complex [B].  mean_out:
   device complex128 [1] receiving <R> summed in float64 (this is
   beta_n = <psi|phi>/<psi|psi> of Sec. III once the fit has converged), or
   NULL. */
cr_status cheb_local_target(cr_ctx* ctx, const cr_target* target, const int8_t* spins,
                            const void* logpsi_n, int B, void* R_out, double* mean_out);

/* Sec. III: O_{a_i} = sigma_i, O_{b_j} = tanh theta_j, O_{W_ij} = sigma_i tanh theta_j.
   theta [B][M] (from rbm_logpsi / mc_sweep). tanh_out [B][M] (NULL allowed);
   O_out complex [B][P] explicit log-derivatives (NULL allowed). */
cr_status logderiv(cr_ctx* ctx, const cr_state* state, const int8_t* spins, const void* theta,
                   int B, void* tanh_out, void* O_out);

/* Backward of log psi: grad_params[k] = sum_s g_s conj(O_k(s)), i.e. the
   vector-Jacobian product that gives d L / d conj(alpha) for a real loss L
   with d L / d conj(log psi_s) = g_s. tanh_theta [B][M], grad_logpsi
   complex [B], grad_params complex [P] (overwritten). */
cr_status logpsi_backward(cr_ctx* ctx, const cr_state* state, const int8_t* spins,
                          const void* tanh_theta, int B, const void* grad_logpsi,
                          void* grad_params);

/* logpsi_backward without any allocation.  The paper has no counterpart:
   this entry point exists for callers that cannot allocate device memory
   themselves -- code inside a framework whose caching allocator owns the
   device's memory, plugins or services held to a fixed footprint, or callers
   that must avoid the device-wide synchronisation a cudaFree brings -- and
   so cannot create a context.  It computes the same
   grad_params[k] = sum_s g_s conj(O_k(s)) as logpsi_backward, with no context:
   N, M and the precision (complex128 for CR_FP64, complex64 otherwise) are
   arguments, and the work runs on `stream` (a cudaStream_t, NULL = legacy
   default stream).  Its reduction scratch is a fixed 4 MiB float64 array in
   the library's device image, which bounds the size: N + M + N*M up to about
   131,000 parameters (2 <= N <= 1024, 1 <= M <= 512); larger sizes return
   CR_EINVAL.  The array exists on a device once the CUDA module holding it
   is loaded there, which the CUDA runtime may do lazily, at the first use of
   any of that module's symbols on that device (possibly this call's first
   call); from then on the device holds it until the process exits.  The call
   itself allocates nothing and calls no allocating routine.  The first call
   on each device looks up the scratch array's device address for that device
   (cudaGetSymbolAddress, which may trigger that module load), so make that
   first call before any stream capture; doing so also keeps every later call
   free of driver-side allocation.  Walker sums are accumulated in float32
   over blocks of 32 walkers and carried in float64, so the result stays as
   accurate as logpsi_backward's at any walker count.  All calls share the
   one array and it keeps the last call's contents (every entry a call reads
   is written by that call first, so nothing needs clearing); calls whose
   work overlaps on the GPU race on it, so serialise them (one stream, or
   events).  errbuf (host, errbuf_len bytes, or NULL) receives the reason for
   a non-CR_OK status. */
cr_status logpsi_backward_noalloc(int N, int M, cr_prec prec, const int8_t* spins,
                                  const void* tanh_theta, int B, const void* grad_logpsi,
                                  void* grad_params, void* stream, char* errbuf, int errbuf_len);

/* The starting point of projection step n (Sec. III, last paragraph; the
   paper leaves it open): n == 1: out = psi with a_0 += i pi/2 (exactly
   2i S^z_0 psi, since e^{i pi sigma/2} = i sigma), so that the first fit starts
   with weight on H' S^z_q psi; n >= 2: out = prev (RBM_{n-1}, warm start).
   psi, prev, out: device complex [P] in the context precision (prev ignored
   for n == 1, psi for n >= 2; out may alias the source). */
cr_status cheb_init_params(cr_ctx* ctx, int n, const void* psi, const void* prev, void* out);

/* Sec. III natural-gradient update, on samples of |psi|^2:
     gamma = arccos sqrt(min(1, |<R>|^2 / <|R|^2>)),
     F_k   = dgamma * gamma cot gamma * (<O_k* R>/<R> - <O_k*>)   (gamma cot gamma = 1 below 1e-8),
     S_kk' = <O_k* O_k'> - <O_k>* <O_k'>,
   then solves (S + shift I) dalpha = F in float64 and sets
   params += dalpha. params complex [P] in/out (context precision);
   tanh_theta [B][M] at the samples; R complex [B]; stats_out float64
   [CR_STATS_LEN] (device) or NULL.  shift >= 0 (shift 0 needs S itself
   positive definite: a rank-deficient S then gives CR_ESINGULAR on the
   Cholesky path).  Walker sums of the estimators: float64 in CR_FP64;
   compensated float32 chunk sums combined in float64 in CR_FP32, and in
   CR_MIXED for Cholesky and Jacobi-preconditioned solves; in CR_MIXED with
   plain CG both sums are one tensor-core launch (three-term bf16 splits,
   float32 accumulation over K segments, float64 across them). */
cr_status sr_step(cr_ctx* ctx, void* params, const int8_t* spins, const void* tanh_theta,
                  const void* R, int B, const cr_sr_opts* opts, double* stats_out);

/* Sec. III, the matrix-free product of the CG solve on its own:
     out = (S + shift I) v,  S v = O^dag (O v) / B - <O>^* (<O> . v),
   computed by the same kernels as the CG of sr_step (in CR_MIXED contexts
   the O v and O^dag u contractions on the tensor cores, from bf16 splits),
   with <O> summed over the same samples first.  spins [B][N], tanh_theta
   [B][M] at the samples; v, out: device complex128 [P]; u_out: context
   precision complex [B] receiving u = O v (NULL allowed).  For parity
   checks of the products against an explicit O. */
cr_status sr_sv(cr_ctx* ctx, const int8_t* spins, const void* tanh_theta, int B, const double* v,
                double shift, void* u_out, double* out);

/* Appendix A: symmetry projection of one Chebyshev sequence, computed for
   the local probe S^z_00, onto every momentum of the L x L square lattice
   (the context's lattice must be square).  For each sample s of |psi|^2 and
   each stored state t_n (plain RBM states, no probe factor):
     B~_nk(s) = L^-1 sum_m e^{-i 2 pi k.m / L} (1/4) sum_{r=0..3}
                t_n(s'_{m,r}) / psi(s),   s'_{m,r}(x) = s(Q^r x + m),
   Q (x, y) = (-y, x) mod L the quarter turn about the probe site, i.e. the
   amplitude ratio of L P_k^(T) P^(R) |t_n>: each term T_{d_r} R^r of the
   rotation projector (d_r = (0,0), (1,0), (1,1), (0,1), R a quarter turn
   about a plaquette centre) returns the probe to the origin, so it is Q^r
   and P^(R) leaves a probe-site-symmetric state unchanged.  states: host array of Nm cr_state;
   spins int8 [B][N]; logpsi_ref: log psi at the samples (context precision
   complex [B]); Bt_out: context precision complex [L*L][Nm][B], momentum
   index k1 + L k2, so that row block k is the Bmat of cheb_gram for that
   momentum (G^(k)_nn' = <conj(B~_nk) B~_n'k>; mu_nk = G^(k)_0n).
   workspace: caller-owned device memory of sym_workspace_bytes(ctx, B)
   bytes (4 N B N bytes of transformed configurations and two complex
   arrays); the call allocates nothing. */
size_t sym_workspace_bytes(const cr_ctx* ctx, int B);
cr_status sym_btilde(cr_ctx* ctx, const cr_state* states, int Nm, const int8_t* spins,
                     const void* logpsi_ref, int B, void* workspace, size_t workspace_bytes,
                     void* Bt_out);

/* Appendix A, the projected Hamiltonian H^(k)_nn' = <t~_nk|H'|t~_n'k> /
   <psi|psi>: sym_btilde plus
     HB~_nk(s) = <s|H'|t~_nk> / psi(s)
               = L^-1 sum_m e^{-i 2 pi k.m / L} (1/4) sum_r
                 (H' t_n)(s'_{m,r}) / psi(s)   (Sec. V bonds),
   which holds because H' commutes with every translation and rotation of
   the periodic square lattice.  (H' t_n)(s') is formed from the amplitudes
   t_n(s'^{ij}) of the exchanged configurations, never as a ratio to
   t_n(s'), which may vanish: the s' are not samples of |t_n|^2.  hprime: host float64 {E0, a, W'} (a != 0).
   Bt_out and HBt_out: context precision complex [L*L][Nm][B]; row block k
   of the two is the (Bmat, HBmat) pair of cheb_gram for momentum k, which
   then gives G^(k) and H^(k) for cheb_krylov.  workspace: caller-owned
   device memory of sym_h_workspace_bytes(ctx, B) bytes (sym_workspace_bytes
   plus theta at the 4 N B transformed configurations, 4 N B M complex
   values, and two more complex arrays); the call allocates nothing.
   Errors as sym_btilde; a == 0 or a NULL hprime / HBt_out is CR_EINVAL. */
size_t sym_h_workspace_bytes(const cr_ctx* ctx, int B);
cr_status sym_hbtilde(cr_ctx* ctx, const cr_state* states, int Nm, const int8_t* spins,
                      const void* logpsi_ref, int B, const double* hprime, void* workspace,
                      size_t workspace_bytes, void* Bt_out, void* HBt_out);

/* Sec. II, Eq. (Aw), with the Jackson damping of Sec. V: the spectral
   function on a frequency grid from the moments mu_n, n = 0 .. Nm - 1,
     A(omega) = [g_0 mu_0 + 2 sum_{n>=1} g_n mu_n T_n(omega')]
                / (a pi sqrt(1 - omega'^2)),   omega' = omega / a - W',
   (the paper's prefactor 2 W'/W_* is 1/a), and 0 where |omega'| >= 1.
   g_n = ((Nm - n + 1) cos(pi n/(Nm+1)) + sin(pi n/(Nm+1)) cot(pi/(Nm+1)))
   / (Nm + 1) when jackson = 1, else 1.  mu: device complex128 [Nm]
   (1 <= Nm <= 12800); omega: device float64 [n_omega] (excitation energies
   E - E0); A_out: device complex128 [n_omega].  Float64 throughout. */
cr_status cheb_spectrum(cr_ctx* ctx, const double* mu, int Nm, double a, double Wp,
                        int jackson, const double* omega, int n_omega, double* A_out);

/* Sec. IV: the spectral function of the Krylov projection, broadened by
   eta, from its poles lambda_k (H' units) and weights w_k (cheb_krylov):
     A(omega) = -Im sum_k w_k / (omega' + i eta/a - lambda_k) / (pi a),
   the same function the continued fraction of the Lanczos tridiagonal form
   evaluates.  poles, weights: device float64 [K]; omega, A_out: device
   float64 [n_omega].  Needs a > 0, eta > 0. */
cr_status cheb_lorentzian(cr_ctx* ctx, const double* poles, const double* weights, int K,
                          double a, double Wp, double eta, const double* omega, int n_omega,
                          double* A_out);

/* Sec. VI (higher moments by extrapolation; the paper cites the method and
   gives no algorithm): linear prediction of Chebyshev moments (Ganahl et
   al., Phys. Rev. B 90, 045144 (2014)) with the growing-mode treatment of
   Barthel, Schollwoeck and White (Phys. Rev. B 79, 245101 (2009)).  For
   each of n_seq sequences of n_known moments mu_0 .. mu_{N-1}:
     a = argmin sum_{n=n0}^{N-1} |mu_n + sum_{i=1}^{order} a_i mu_{n-i}|^2
       (normal equations with a Tikhonov term reg * max_i R_ii, Cholesky);
     z_k = roots of z^p + a_1 z^{p-1} + ... + a_p (Aberth-Ehrlich);
     c_k from sum_k c_k z_k^m = mu_{N-p+m}, m < p (LU, partial pivoting);
     w_k = z_k / |z_k| where |z_k| > 1, else z_k;
     mu_{N-p+m} = sum_k c_k w_k^m for m >= p.
   mu: device complex128 [n_seq][n_known]; mu_out: device complex128
   [n_seq][n_out], the known moments followed by the prediction;
   roots_out: device complex128 [n_seq][order] (the fitted z_k) or NULL;
   info_out: device int [n_seq] or NULL: root iterations used, -1 when the
   root iteration stopped at its limit (500), -2 when a system was
   singular.  Needs 1 <= order <= 512 and order <= n0 < n_known <= n_out,
   reg >= 0.  A non-positive Cholesky pivot (reg = 0 on a rank-deficient
   window) or a singular amplitude system sets CR_ESINGULAR on the device
   and NaN in that sequence's prediction.  Float64 throughout; sizes its
   scratch (2 order^2 complex128 per sequence) on first use. */
cr_status cheb_extrapolate(cr_ctx* ctx, const double* mu, int n_seq, int n_known, int order,
                           int n0, double reg, int n_out, double* mu_out, double* roots_out,
                           int* info_out);

/* One sequence's part of a batched run (cr_batch_run): its context and
   device buffers, the target of the projection step being fitted and the
   update options. */
typedef struct {
    cr_ctx* ctx;            /* the sequence's context; its stream runs the sequence */
    void* params;           /* RBM_n being fitted, complex [P], in/out */
    int8_t* spins;          /* fit walkers [B][N], in/out */
    void* theta;            /* complex [B][M], in/out: theta of params at spins */
    void* tanh_theta;       /* complex [B][M], out (workspace) */
    void* logpsi;           /* complex [B], in/out: log psi_n at spins */
    void* R;                /* complex [B], out (workspace) */
    int B;
    int n_sweeps;           /* Metropolis sweeps per natural-gradient iteration */
    cr_target target;       /* the target of projection step n (Sec. III) */
    cr_sr_opts opts;
    cr_philox* rng;         /* host struct (device_counter for graph replays) */
    double* stats;          /* device float64 [CR_STATS_LEN] of the last iteration, or NULL */
} cr_seq_iter;

/* Secs. III and V: n_iter natural-gradient iterations of n_seqs
   independent Chebyshev sequences (probe momenta, lattices of different
   sizes), each iteration per sequence
     mc_sweep (n_sweeps sweeps, giving log psi_n and tanh theta),
     cheb_local_target (R), sr_step (the update), rbm_logpsi (theta, log psi_n
     of the updated RBM),
   each sequence on its own context's stream: the work is forked from
   `stream` (a cudaStream_t, NULL = legacy default) and joined back into it
   through events the contexts own, the sequences' launches interleaved
   iteration by iteration so that they run side by side.  Nothing is
   exchanged between sequences.  The whole call can be captured into one
   CUDA graph on `stream`.  The contexts must be distinct.  Returns the first
   failing call's status (its text in that context's cr_last_error). */
cr_status cr_batch_run(const cr_seq_iter* seqs, int n_seqs, int n_iter, void* stream);

/* Sec. III: the explicit S + shift I of sr_step's Cholesky path, built by
   the same kernels on samples of |psi|^2 (Obar from the same samples), copied
   to S_out: device complex128 [P][P], the full Hermitian matrix.  For
   inspection and accuracy checks (mixed contexts: the tensor-core S against
   a float64 context's).  Needs CR_CTX_EXPLICIT_S. */
cr_status sr_smatrix(cr_ctx* ctx, const int8_t* spins, const void* tanh_theta, int B,
                     double shift, double* S_out);

/* Secs. II and IV, on samples s of |psi|^2 of the reference state psi:
     Bcol[s]  = beta t~(s) / psi(s)              (B_n of the Gram estimator)
     HBcol[s] = beta (H' t~)(s) / psi(s)          (needs hprime, else NULL)
     mu[0:2]  = < conj(f_q(s)) Bcol[s] >          complex128, mu_n of Sec. II
   with f_q the probe factor at momentum (qx, qy). state: t~_n; beta: device
   complex128 [1]; logpsi_ref [B] log psi at the samples; hprime: host
   float64 {E0, a, Wp} or NULL. Bcol, HBcol: complex [B] or NULL; mu_out:
   device complex128 [1] or NULL. */
cr_status cheb_moment(cr_ctx* ctx, const cr_state* state, const double* beta, double qx,
                      double qy, const int8_t* spins, const void* logpsi_ref, int B,
                      const double* hprime, void* Bcol, void* HBcol, double* mu_out);

/* Sec. IV estimators: G_nm = <conj(B_n) B_m>, H_nm = <conj(B_n) HB_m>, then
   H <- (H + H^dag)/2. Bmat, HBmat complex [Nm][ld] (row n = column B_n over
   the B samples, leading dimension ld >= B); G_out, H_out complex128
   [Nm][Nm] (device).  HBmat and H_out may both be NULL (G only).
   CR_FP64 / CR_FP32: products in the storage precision, sums in float64.
   CR_MIXED: both contractions on the tensor cores (tcgen05) from three-term
   bf16 splits of the float32 values with float32 accumulation over walker
   chunks and K segments, float64 across segments (about float32 accuracy);
   G is Hermitian by construction (upper triangle mirrored, real diagonal).
   The mixed path sizes its device scratch on first use: bf16 planes of
   6 * 2 Nm (padded to 256) * B bytes per matrix and the per-segment sums;
   a failed allocation is CR_ENOMEM. */
cr_status cheb_gram(cr_ctx* ctx, const void* Bmat, const void* HBmat, int Nm, int B, int ld,
                    double* G_out, double* H_out);

/* Secs. IV and V in float64 on the device: with G^+ the pseudo-inverse of G
   (eigenvalues below cutoff * max dropped), c_0 = e_0, c_1 = G^+ H c_0,
   c_{n+1} = G^+ (2 H c_n - G c_{n-1}), mu'_n = (G c_n)_0 for n < n_out; and
   the projected eigenproblem H c = lambda G c by canonical
   orthogonalisation, with weights w_k = |<v_k| X^dag G e_0>|^2.
   G, H complex128 [Nm][Nm]; mu_corr_out complex128 [n_out]; poles_out,
   weights_out float64 [Nm] (entries past the kept rank are 0); rank_out int32
   [1] (device) or NULL. Nm <= 512. */
cr_status cheb_krylov(cr_ctx* ctx, const double* G, const double* H, int Nm, double cutoff,
                      int n_out, double* mu_corr_out, double* poles_out, double* weights_out,
                      int32_t* rank_out);

#ifdef __cplusplus
}
#endif

#endif /* CHEBRBM_H */
