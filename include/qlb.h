/*
 * qlb.h -- C-ABI of the GB300 purified quantics-MPS Lindblad stepper (libqlb.so).
 *
 * What the library computes (Moulinas & Waintal, "A multilevel tensor network
 * compression technique for simulating Lindblad dynamics in superconducting
 * circuits"):
 *   * the Lindblad equation, Eq. 1, with hbar = 1, for a few bosonic modes;
 *   * the density matrix is kept as a global purification rho = Psi Psi^dag
 *     (Sec. IV.A) whose Psi is a matrix product state over the quantics sites of
 *     all modes (Sec. IV.B-C): mode m of N_m = 2^R_m Fock levels is split into
 *     R_m binary sites, sigma_1 (most significant bit) first (Sec. II.A);
 *   * one step is the first-order Kraus map K = U + h L of Sec. V.B with
 *     U_1 = 1 - i h H_eff, H_eff = H - (i/2) sum_k L_k^dag L_k, the jump
 *     branches sqrt(h) L_k stacked on the purification index (matrix addition,
 *     Sec. V.A), every bond recompressed, the purification rank truncated
 *     (Sec. IV.A) and rho renormalised to unit trace (Sec. V.B, last paragraph).
 *
 * Conventions common to every call:
 *   * Complex numbers are passed as interleaved (re, im) doubles (the layout of
 *     C99 double _Complex and numpy complex128).
 *   * Dense per-mode matrices are N_m x N_m, row-major, complex128.
 *   * Inputs are copied during the call; the caller keeps ownership of every
 *     buffer it passes.  Every handle is created and destroyed by the caller;
 *     destroying a system invalidates the ops and states made from it.
 *   * All device memory is owned by the library; state tensors stay resident on
 *     the GPU.  Host pointers are plain host memory (pageable or pinned).
 *   * Every call returns a qlb_status: 0 on success, > 0 a warning (the call
 *     did its work), < 0 an error (the call did nothing that the caller can
 *     observe, except where a call says otherwise).  No call aborts the process.
 *     qlb_last_error() returns a thread-local message for the last failing call.
 *   * Calls are synchronous unless qlb_options.stream_ordered is set, in which
 *     case qlb_step returns after enqueueing work on the context's stream.
 *   * A context serialises its work on one CUDA stream; handles of one context
 *     must not be used from several host threads at once.
 */
#ifndef QLB_H
#define QLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t qlb_status;

#define QLB_OK 0
#define QLB_WUNSTABLE 1    /* warning: the explicit U_1 = 1 - i h H_eff has a spectral
                              bound above 1 at this dt (Sec. III.A stiffness remark) */
#define QLB_EINVAL (-1)     /* bad argument (null handle, size, mode index ...) */
#define QLB_ENOMEM (-2)     /* device allocation failed or the HBM budget is exceeded */
#define QLB_ENOTCONV (-3)   /* a Jacobi eigen/SVD solve hit its sweep limit */
#define QLB_ETIMEOUT (-4)   /* a bounded device wait gave up */
#define QLB_ENONFINITE (-5) /* NaN/Inf met in the state or a trace */
#define QLB_EDEVICE (-6)    /* CUDA error or no usable device */
#define QLB_ESTATE (-7)     /* handle not ready for this call (e.g. no Hamiltonian) */

typedef struct qlb_ctx qlb_ctx;
typedef struct qlb_system qlb_system;
typedef struct qlb_op qlb_op;
typedef struct qlb_state qlb_state;

/* Arithmetic of the step. */
#define QLB_PREC_F64 0   /* every operation in FP64 (the parity form) */
#define QLB_PREC_MIXED 1 /* the truncation solves and the GEMMs chosen by mixed_gemm in
                            double-float (pairs of FP32, ~48-bit significands) on the FP32
                            pipes, with FP64 operands and results; truncation decisions,
                            weights and renormalisation in FP64 */
#define QLB_PREC_TC 2    /* QLB_PREC_MIXED with the MPO application (the two zip-up
                            contractions of every site) on the tensor cores in 3xTF32
                            (operands split into two TF32 parts, FP32 accumulation);
                            Gram matrices, truncation decisions and renormalisation stay
                            FP64 (Sec. V.A MPO.MPS product; precision split of the
                            contractions only) */

typedef struct {
  int device;            /* CUDA device ordinal */
  int precision;         /* QLB_PREC_* */
  double tol;            /* relative discarded-weight cutoff: keep the smallest k with
                            sum_{i>=k} s_i^2 <= tol * sum_i s_i^2 (default 1e-12) */
  int chi_max;           /* cap on every inter-site bond (default 64) */
  int chi_mu_max;        /* cap on the purification rank chi_mu (default 16) */
  double zip_tol_factor; /* the on-the-fly truncation inside the MPO application uses
                            tol * zip_tol_factor (default 1e-6: the zip-up truncates in a
                            frame that is not orthonormal, so it must cut far below tol) */
  double degeneracy_gap; /* singular values within this relative gap are one cluster and
                            are never split by a cut (default 1e-10) */
  int max_sweeps;        /* Jacobi sweep limit before QLB_ENOTCONV (default 40); below 60
                            it also caps the QL iterations per eigenvalue */
  size_t hbm_budget;     /* bytes of device memory the context may hold; 0 = no limit */
  int stream_ordered;    /* 1: qlb_step only enqueues; 0 (default): it synchronises */
  int zip_solver;        /* how a zip-up bond finds the range of M: 1 (default) column-
                            pivoted Gram-Schmidt on G = M M^dag with one
                            re-orthogonalisation, stopping at the weight cutoff or at the
                            working precision's rounding level, and the Jacobi eigen-solve
                            only when the cap is reached first; 0 the Jacobi eigen-solve
                            on every zip-up bond */
  int zip_chi_max;       /* cap on the zip-up bonds, in [chi_max, 256]; 0 (default) = chi_max.
                            The zip-up truncates in a frame that is not orthonormal, so a
                            cap that binds there costs accuracy that the final sweep cannot
                            recover */
  int mixed_gemm;        /* GEMMs of the mixed forms (QLB_PREC_MIXED, QLB_PREC_TC) that multiply
                            and sum in double-float (~48-bit significands, FP32 pipes) with FP64
                            operands and results: 0 none (all FP64), 1 (default) the MPO
                            application and the products of the truncation sweep, 2 also the
                            Gram matrices the truncations are decided on.  Ignored in QLB_PREC_F64;
                            in QLB_PREC_TC the MPO application stays on the tensor cores */
} qlb_options;

/* Fills *opt with the defaults listed above. */
void qlb_default_options(qlb_options* opt);

/* Creates a context on opt->device (opt may be NULL for defaults). */
qlb_status qlb_create(const qlb_options* opt, qlb_ctx** out);
void qlb_destroy(qlb_ctx* ctx);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* qlb_last_error(void);

/* The cudaStream_t the context runs its setup work on (operator builds). */
qlb_status qlb_ctx_stream(qlb_ctx* ctx, void** stream);
/* Waits for all work of the context and of its states (device-wide). */
qlb_status qlb_synchronize(qlb_ctx* ctx);
/* Device bytes currently held by the context. */
qlb_status qlb_ctx_memory(qlb_ctx* ctx, size_t* bytes);
/* Number of device allocations the context has made since it was created (every
 * buffer of its systems, ops and states, and per-call temporaries).  Lets a caller
 * check that a call allocated nothing.  The paper has no counterpart. */
qlb_status qlb_ctx_alloc_count(qlb_ctx* ctx, int64_t* n);

/* ------------------------------------------------------------------ systems */

/* A system of n_modes bosonic modes; mode m has N_m = 2^R[m] levels (1 <= R[m] <= 12,
 * sum R[m] <= 64).  Sec. II.A (quantics encoding), Sec. IV.C (one quantics chain
 * per mode, modes joined by compressed bonds). */
qlb_status qlb_system_create(qlb_ctx* ctx, int n_modes, const int* R, qlb_system** out);
void qlb_system_destroy(qlb_system* sys);

/* ------------------------------------------------------------------ operators */

/* Built-in single-mode factors (Sec. II.B; Sec. VII for the charge basis). */
#define QLB_F_ID 0     /* identity */
#define QLB_F_A 1      /* a: <n|a|n'> = delta_{n+1,n'} sqrt(n'), open at n = 0 */
#define QLB_F_ADAG 2   /* a^dag, the conjugate transpose of the truncated a */
#define QLB_F_NUM 3    /* n = diag(0..N-1) */
#define QLB_F_PARITY 4 /* (-1)^n */
#define QLB_F_CHARGE 5 /* diag(j - param): charge operator with charge offset param */
#define QLB_F_COSPHI 6 /* (|j><j+1| + |j+1><j|)/2, open ends (charge-basis cos phi) */
#define QLB_F_DENSE 7  /* caller's dense N_m x N_m complex128 row-major matrix */

typedef struct {
  int mode;            /* 0 <= mode < n_modes */
  int kind;            /* QLB_F_* */
  int power;           /* factor raised to this power (>= 1; 0 is treated as 1) */
  double param;        /* QLB_F_CHARGE offset; ignored otherwise */
  const double* dense; /* QLB_F_DENSE: 2*N_m*N_m doubles; ignored otherwise */
} qlb_factor;

/* One term: (re + i im) times the ordered product of its factors.  Factors on
 * the same mode multiply as matrices in the order given (products of the
 * truncated matrices, Sec. II.B); factors on different modes are tensored. */
typedef struct {
  double re, im;
  const qlb_factor* factors;
  int n_factors;
} qlb_term;

/* Builds sum_t term_t as a quantics MPO (Sec. II.B): each term's per-mode dense
 * matrix is TT-SVD'd on the device into an MPO of R_m sites, the modes are
 * joined, the terms are summed and the sum is recompressed.  tol is the relative
 * discarded weight per bond (<= 0 selects 1e-30, i.e. only numerical zeros are
 * dropped); chi_max caps every MPO bond (<= 0: no cap).  The op keeps its dense
 * per-mode factors on the device so that L^dag L can be formed exactly. */
qlb_status qlb_op_build(qlb_system* sys, const qlb_term* terms, int n_terms, double tol, int chi_max,
                        qlb_op** out);
void qlb_op_destroy(qlb_op* op);
/* Bond dimensions D_1..D_{L-1} of the op's MPO (n_out = L-1; cap = size of out). */
qlb_status qlb_op_bond_dims(const qlb_op* op, int* out, int cap, int* n_out);
/* Dense matrix of the op's MPO (for small systems, 2^L <= 4096): out holds 2*4^L doubles. */
qlb_status qlb_op_to_dense(const qlb_op* op, double* out, size_t n_doubles);

/* H(t) = H0 + f(t_n) H1 (Sec. III.A, coefficient form H0 + f(t) H1).  H1 may be NULL.
 * f_table[n] is f at the left end t_n of the n-th step since the state was made
 * (first-order step, left endpoint); steps past the end of the table use f = 0.
 * The ops are referenced, not copied: keep them alive while the system is used. */
qlb_status qlb_set_hamiltonian(qlb_system* sys, const qlb_op* H0, const qlb_op* H1, const double* f_table,
                               int64_t n_f);
/* Adds a Lindblad operator L_k (Eq. 1).  Referenced, not copied. */
qlb_status qlb_add_jump(qlb_system* sys, const qlb_op* L);
/* Selects the Kraus scheme used by qlb_step (Sec. V.B).
 *   order 1 (default): K = U + h L, Kraus operators U_1 = 1 - i h H_eff and
 *     sqrt(h) L_k, local error O(h^2).
 *   order 2: K = U' + (h/2)(U L + L U) + (h^2/2) L^2, Kraus operators
 *     U_1' = 1 - i h H_eff - (h^2/2) H_eff^2, sqrt(h/2) U_1 L_k, sqrt(h/2) L_k U_1
 *     and (h/sqrt 2) L_j L_k: 1 + 2l + l^2 branches on the purification leg,
 *     local error O(h^3).
 * Order 2 needs a time-independent Hamiltonian (H1 == NULL) and at most 6 jump
 * operators; otherwise QLB_EINVAL (here, or from qlb_step if the system changes
 * afterwards).  States rebuild their Kraus MPO on their next step. */
qlb_status qlb_set_scheme(qlb_system* sys, int order);

/* ------------------------------------------------------------------ states */

/* Pure separable start, chi_mu = chi_e = 1 (Sec. V, first paragraph): mode_vecs[m]
 * holds N_m complex128 amplitudes (normalised by the call). */
qlb_status qlb_state_init_product(qlb_system* sys, const double* const* mode_vecs, qlb_state** out);
void qlb_state_destroy(qlb_state* st);
/* The cudaStream_t of the state: every launch that touches the state (steps,
 * observables) goes there, so states of one context step concurrently.  With
 * stream_ordered set, callers time qlb_step with events on this stream. */
qlb_status qlb_state_stream(qlb_state* st, void** stream);
/* Non-blocking completion check of the state's enqueued work: QLB_OK when its
 * stream is idle, 2 (a positive status, nothing done) while work is pending. */
#define QLB_BUSY 2
qlb_status qlb_state_poll(qlb_state* st);

/* Sets the truncation parameters used by every later step of this state and
 * recompresses the state once with them (Sec. V.A compression, Sec. IV.A
 * purification truncation).  tol <= 0 keeps the current value; chi caps <= 0 keep
 * theirs.  Caps may not exceed the values the state was allocated for (the
 * context's chi_max / chi_mu_max at init). */
qlb_status qlb_truncate(qlb_state* st, double tol, int chi_max, int chi_mu_max);

/* n steps of size dt of the first-order Kraus map (Sec. V.B), each followed by
 * recompression and renormalisation.  Returns QLB_WUNSTABLE (after doing the
 * work) if the Gershgorin bound of |U_1| exceeds 1 + 1e-12 at this dt. */
qlb_status qlb_step(qlb_state* st, double dt, int64_t n);

/* Tr(O rho) for the unit-trace rho of the state; out = (re, im). */
qlb_status qlb_expectation(qlb_state* st, const qlb_op* O, double* out);
/* <psi|rho|psi> for the product target psi = (x)_m target_mode_vecs[m] (normalised by the call). */
qlb_status qlb_fidelity(qlb_state* st, const double* const* target_mode_vecs, double* out);
/* Tr rho of the stored purification (1 after every step, up to rounding). */
qlb_status qlb_trace(qlb_state* st, double* out);
/* Tr rho^2 (Sec. IV.A). */
qlb_status qlb_purity(qlb_state* st, double* out);
/* Tr rho^2 like qlb_purity, but allocating no device memory.  The paper has no
 * counterpart: this call exists for callers that must not allocate while they
 * ask, e.g. code whose device memory belongs to another allocator with a fixed
 * budget, or monitoring loops that cannot pay for the device-wide
 * synchronisation of cudaFree.  The Gram matrix and the sums live in a fixed
 * scratch array inside the library's device image (about 256 KB, held by every
 * GPU that loads the library until the process exits); it serves purification
 * ranks chi_mu <= 128 and returns QLB_EINVAL with a message for larger ones
 * (qlb_create caps chi_mu_max at 128, so no state of this library reaches that
 * branch today).  The first call on a device looks up that array's device
 * address with that device current (no allocation).  All calls share the one
 * array, so calls that overlap on the GPU (other host threads, other streams)
 * race; results are written, never accumulated, so a previous call's contents do
 * not matter.  The call is synchronous: it reads the bond dimensions back and
 * waits for the state's stream, so it cannot run inside CUDA stream capture.
 * out receives the purity. */
qlb_status qlb_purity_noalloc(qlb_state* st, double* out);
/* [chi_mu, chi_1, ..., chi_{L-1}] (n_out = L). */
qlb_status qlb_bond_dims(qlb_state* st, int* out, int cap, int* n_out);
/* Diagnostics of the last step: out[0] = Tr rho before renormalisation,
 * out[1] = largest relative discarded weight over the bonds, out[2] = the
 * Gershgorin bound of |U_1|, out[3] = steps taken since init. */
qlb_status qlb_step_stats(qlb_state* st, double* out4);

/* Dense purification Psi of a small state (2^L <= 4096) as a 2^L x chi_mu
 * row-major complex128 matrix, rho = Psi Psi^dag (Sec. IV.A); *chi_mu_out gets
 * chi_mu.  out must hold 2 * 2^L * chi_mu doubles (n_doubles). */
qlb_status qlb_state_to_dense(qlb_state* st, double* out, size_t n_doubles, int* chi_mu_out);
/* Dense matrix of the Kraus operator of branch k (0: U_1 = 1 - i dt H_eff(t_n)
 * at the state's current step n, k >= 1: sqrt(dt) L_k) exactly as the step
 * applies it (Sec. V.B), for 2^L <= 2048; out holds 2 * 4^L doubles. */
qlb_status qlb_kraus_to_dense(qlb_state* st, double dt, int k, double* out, size_t n_doubles);

/* Host copy of the state (checkpoint / preemption): bond dims and site tensors.
 * qlb_state_export with out == NULL stores the needed size in *n_bytes. */
qlb_status qlb_state_export(qlb_state* st, void* out, size_t cap, size_t* n_bytes);
qlb_status qlb_state_import(qlb_state* st, const void* in, size_t n_bytes);

/* ------------------------------------------------------------------ groups */

/* Many independent states stepped together.  The method's step (Sec. V.B with
 * the zip-up of Sec. V.A and the purification truncation of Sec. IV.A) is a chain
 * of small dependent launches per state: apart, one state keeps only a few SMs
 * busy.  A group runs each launch of the step once for all of its members (one
 * CTA, cluster or GEMM grid slice per member, blockIdx.y = member), captured as
 * one CUDA graph on the group's own stream, so n_states states cost one chain of
 * launches.  A member's numbers are the ones its own qlb_step computes: the same
 * kernels, shapes, K splits and reduction orders, bit for bit when the members
 * share one planned shape.  When planned sizes differ, an eigen-solve may run on
 * the kernel the largest co-member's size needs (the same rotations, thresholds
 * and truncation rule: results agree to rounding).  The per-class timings of
 * qlb_profile_* do not cover group steps; the solver counters do.
 *
 * The members must belong to ctx, be distinct, and step the same launch sequence:
 * the same number of sites, the same precision form and Kraus scheme (their mode
 * sizes, operators, caps and bond dimensions may differ; each is planned for its
 * own).  The group holds the handles, not their ownership: destroy the group
 * before any of its states.  Between group steps the members stay usable one by
 * one (observables, qlb_step, qlb_truncate); their own streams are ordered before
 * and after the group's work.  n_states in 1..4096. */
typedef struct qlb_group qlb_group;
qlb_status qlb_group_create(qlb_ctx* ctx, qlb_state* const* states, int n_states, qlb_group** out);
void qlb_group_destroy(qlb_group* g);
/* n steps of size dt for every member (qlb_step's semantics and return codes;
 * QLB_WUNSTABLE if any member's map is unstable at dt; the first member error
 * otherwise).  Synchronous unless the context is stream_ordered. */
qlb_status qlb_group_step(qlb_group* g, double dt, int64_t n);
/* Kernel launches of one captured group step (0 before the first step). */
qlb_status qlb_group_launches(qlb_group* g, int* per_step);
/* The cudaStream_t the group's steps run on. */
qlb_status qlb_group_stream(qlb_group* g, void** stream);

/* ------------------------------------------------------------------ serving */

/* Continuous-batching service of independent solves on one GPU (the serving
 * workload: requests of differing mode counts, Fock sizes and bond caps arriving
 * over time).  A server takes over its context: while it exists only its worker
 * thread issues device work on that context (the caller must not use the context,
 * its systems or states meanwhile).  The worker admits pending requests in
 * arrival order while fewer than max_live are running and the request's
 * estimated device memory fits hbm_budget (0: no limit) next to the running ones;
 * it builds the request's system and state, and steps the running states in
 * chunks of at most `chunk` steps: running requests whose step plans have the
 * same shape (sites, precision form, Kraus MPO bonds, bond capacities) step
 * together as one group (see "groups"), each group on its own stream, so the
 * groups overlap on the GPU.  It evaluates a request's observables when its
 * steps are done, and releases its memory and slot.  The context must be created
 * with stream_ordered = 1. */
typedef struct qlb_server qlb_server;

/* One solve.  Every array is copied at qlb_submit (dense factors included). */
typedef struct {
  int n_modes;                     /* 1..16 */
  const int* R;                    /* N_m = 2^R[m] */
  const qlb_term* H;               /* time-independent Hamiltonian terms (n_H may be 0) */
  int n_H;
  const qlb_term* const* jumps;    /* jumps[k]: the n_jump_terms[k] terms of L_k */
  const int* n_jump_terms;
  int n_jumps;
  const double* const* mode_vecs;  /* product start: N_m complex128 per mode */
  double dt;                       /* first-order Kraus step (Sec. V.B) */
  int64_t steps;
  double tol;                      /* truncation of this request; <= 0: the context's */
  int chi_max;                     /* <= the context's chi_max; <= 0: the context's */
  int chi_mu_max;                  /* <= the context's chi_mu_max; <= 0: the context's */
  const qlb_term* const* obs;      /* observables: Tr(O rho) at completion */
  const int* n_obs_terms;
  int n_obs;
} qlb_request;

qlb_status qlb_server_create(qlb_ctx* ctx, size_t hbm_budget, int max_live, int chunk, qlb_server** out);
/* Stops the worker (running requests are dropped) and frees the server. */
void qlb_server_destroy(qlb_server* srv);
/* Queues a request; *ticket identifies it.  QLB_EINVAL for malformed requests. */
qlb_status qlb_submit(qlb_server* srv, const qlb_request* req, int64_t* ticket);
/* QLB_BUSY while the request is pending or running.  Once done: QLB_OK with
 * results = (re, im) of each observable (cap doubles at most) and times3 = seconds
 * since the server was created at arrival, admission and completion; a failed
 * request returns its error status, a cancelled one QLB_ESTATE. */
qlb_status qlb_poll(qlb_server* srv, int64_t ticket, double* results, int cap, double* times3);
/* Cancels a pending or running request (a running one stops between two chunks). */
qlb_status qlb_cancel(qlb_server* srv, int64_t ticket);
/* out6 = [running, peak running, peak device bytes of the context, completed,
 * steps taken, pending]. */
qlb_status qlb_server_stats(qlb_server* srv, double* out6);

/* ------------------------------------------------------------------ profiling */

/* Kernel classes for qlb_profile_read. */
#define QLB_K_CONTRACT 0 /* zip-up site contraction (carry x site x MPO) */
#define QLB_K_GRAM 1     /* Gram matrices of the truncations */
#define QLB_K_EIG 2      /* Jacobi eigen solves + truncation select */
#define QLB_K_APPLY 3    /* projections / absorptions after a truncation */
#define QLB_K_OTHER 4
#define QLB_K_COUNT 5

/* When enabled, every launch of the step is bracketed by CUDA events on the
 * context stream and its duration accumulated per kernel class. */
qlb_status qlb_profile_enable(qlb_ctx* ctx, int on);
/* Total milliseconds and launches per class since the last reset; flops and
 * bytes are the algorithmic counts of those launches (device-side shapes). */
qlb_status qlb_profile_read(qlb_ctx* ctx, int kclass, double* ms, int64_t* launches, double* flops,
                            double* bytes);
qlb_status qlb_profile_reset(qlb_ctx* ctx);
/* Eigen-solver counters of the context since the last qlb_profile_reset, kept
 * whether or not profiling is on (also inside captured step graphs); the first
 * min(n_out, 9) of: out[0] solves, out[1] Jacobi sweeps plus QL passes, out[2] sum
 * of the runtime matrix sizes n, out[3] sum of the kept counts k, out[4] solves
 * that reached the sweep (or QL iteration) limit, out[5] solves whose matrices did
 * not fit in one CTA's shared memory (spread over a thread-block cluster, or in a
 * global-memory workspace), out[6] the largest runtime size n, out[7] zip-up range
 * bases built by pivoted Gram-Schmidt (zip_solver = 1), out[8] of those, the ones
 * that reached the zip-up cap and left the bond to the Jacobi solve.  A bond the
 * range basis served counts in out[0], out[2] and out[3] like a solve.
 * Synchronises the device. */
qlb_status qlb_profile_solver_stats(qlb_ctx* ctx, double* out, int n_out);

/* Autotuner of the step's launch shapes: times the zip-up Gram GEMM at split-K
 * factors 1, 2, 4, 8, 16 for every (rows, inner size) bucket with CUDA events on
 * random data, installs the fastest in the context (used by every state planned
 * afterwards) and, when path is non-NULL, writes the table as lines "m K ksplit".
 * Allocates scratch for the duration of the call.  The paper has no counterpart. */
qlb_status qlb_autotune(qlb_ctx* ctx, const char* path);
/* Installs a table written by qlb_autotune (QLB_EINVAL if unreadable or empty). */
qlb_status qlb_load_tuning(qlb_ctx* ctx, const char* path);

/* Measured fused multiply-add throughput of device `device` in TFLOP/s:
 * kind 0 = FP64, kind 1 = FP32 (independent FMA chains over every SM, timed with
 * CUDA events, best of three ~20 ms launches).  The denominators of the
 * truncation solvers' roofline.  Allocates a few KB for the duration of the call. */
qlb_status qlb_measure_peak(int device, int kind, double* tflops);

/* C = A B for host row-major complex128 matrices (A m x k, B k x n, C m x n) through
 * the tensor-core engine of QLB_PREC_TC: the same 3xTF32 tcgen05 GEMM the mixed form
 * applies the Kraus MPO with (Sec. V.A), exposed so that its numerics can be checked
 * against an FP64 product.  Copies the operands to device `device`, allocating for the
 * duration of the call.  QLB_ETIMEOUT if a bounded wait of the kernel gave up. */
qlb_status qlb_tc_zgemm(int device, int m, int n, int k, const double* A, const double* B, double* C);

/* C = A B as above through one of the step's GEMM engines: engine 0 the FP64
 * work-distributed GEMM, 1 the same GEMM multiplying and summing in double-float
 * (the mixed forms), 2 the tensor-core 3xTF32 GEMM (as qlb_tc_zgemm).  ms: device
 * time of one launch (CUDA events, after one untimed launch).  Allocates device
 * memory for the duration of the call. */
qlb_status qlb_zgemm_check(int device, int engine, int m, int n, int k, const double* A, const double* B,
                           double* C, double* ms);

/* One truncation solve of the step, by a named kernel, on a host Hermitian matrix:
 * exposed so that each solver's numerics and device time can be checked on its
 * own (Sec. V.A truncated factorisation of a bond through its Gram matrix G).
 *   precision  QLB_PREC_F64 (FP64 arithmetic) or QLB_PREC_MIXED (double-float)
 *   solver     0 the kernel the step takes for a planned size n, 1 one-CTA Jacobi,
 *              2 Jacobi over a cluster of 8 CTAs (n <= 128), 3 over 16 CTAs
 *              (n <= 256), 4 Householder + implicit QL (FP64 only, n <= 64),
 *              5 the zip-up range basis (pivoted Gram-Schmidt)
 *   G          n x n row-major complex128 (2 n^2 doubles), Hermitian, 1 <= n <= 512
 *   tol, cap   the truncation: relative discarded weight and the cap on k
 *   lam        n doubles: the eigenvalues, descending, clamped at 0 (solvers 0-4;
 *              zeros for 5)
 *   V          n x k kept vectors as columns, row-major complex128 (2 n k doubles
 *              written, room for 2 n n)
 *   k_out      the kept count; -1 when solver 5 reached the cap first (the step
 *              then runs the Jacobi solve)
 *   ms         device time of one launch (CUDA events, after one untimed launch)
 * QLB_EINVAL for a solver that does not take this size or precision, QLB_ENOTCONV
 * at the sweep limit, QLB_ENONFINITE for non-finite input.  Allocates device memory
 * for the duration of the call. */
qlb_status qlb_eig_check(int device, int precision, int solver, int n, const double* G, double tol, int cap,
                         double* lam, double* V, int* k_out, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* QLB_H */
