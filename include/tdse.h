/*
 * tdse.h — C ABI of the GB300 (sm_103a) propagator for the laser-driven
 * hydrogen time-dependent Schrödinger equation in a field-free eigenstate
 * basis (Ó Broin & Nikolopoulos, "An OpenCL implementation for the solution
 * of TDSE on GPU and CPU architectures", arXiv:1201.6062).
 *
 * The ODE (paper Sec. 3, Eq. "tdse_ode_c"; Sec. 4, Eq. "ode"):
 *     dc/dt = -i H(t) c,   H(t) = diag(E) + f(t) D,
 * with c the complex amplitudes of N = (lmax+1)*n eigenstates, grouped into
 * angular-momentum blocks l = 0..lmax of n states each (block l holds
 * amplitudes [l*n, (l+1)*n)).  By the dipole selection rule (Sec. 3.1,
 * Fig. "Matrix") D couples only neighbouring blocks: D_{l,l+1} = U_l is a
 * dense real n x n block and D_{l+1,l} = U_l^T (Sec. 5: only the upper blocks
 * are stored).  f(t) is the electric-field sample (length gauge, Sec. 5);
 * tdse_set_gauge selects the velocity gauge instead (f(t) = A(t), D = i K).
 *
 * Entry points: contexts (tdse_create / tdse_destroy), one product
 * (tdse_hmatvec), propagation (tdse_propagate: RK4, Taylor, Lanczos;
 * tdse_propagate_host; tdse_propagate_rkf45: adaptive), pulse batches
 * (tdse_propagate_batch), uneven batches (tdse_group_*), the adjoint
 * (tdse_adjoint), norms and populations, the velocity-gauge field
 * (tdse_vector_potential_sin2), tracing (tdse_profile_*).
 *
 * Common conventions
 *  - Complex vectors are interleaved (re, im) FP64 pairs, i.e. the memory of
 *    a complex128 array.  c[2*a] = Re c_a, c[2*a+1] = Im c_a.
 *  - Pointers documented "device" must be CUDA device memory of the current
 *    device, 16-byte aligned; "host" pointers are ordinary host memory.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it and the call returns without waiting, except where noted.
 *  - Field samples (the paper does not fix this; the reading used here):
 *      samples_per_step = 1: field[k] = f(t0 + k dt), k = 0..nsteps; the
 *        value at a half step is the mean of its two neighbours;
 *      samples_per_step = 2: field[h] = f(t0 + h dt/2), h = 0..2*nsteps.
 *  - Every call returns a tdse_status and never throws.  On failure the
 *    output buffers are unspecified and tdse_last_error() describes the cause
 *    (thread-local string, valid until the next call on the same thread).
 *  - A context is not thread-safe; distinct contexts may be used from
 *    distinct threads.
 */
#ifndef TDSE_H
#define TDSE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TDSE_OK = 0,
    TDSE_EINVAL = 1,    /* bad argument (NULL, size, enum, misaligned pointer) */
    TDSE_ENOMEM = 2,    /* device or host allocation failed                    */
    TDSE_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed         */
    TDSE_ETIMEOUT = 4,  /* a bounded device-side wait gave up                  */
    TDSE_ENOTSUP = 5    /* valid request this build does not support           */
} tdse_status;

typedef enum {
    TDSE_RK4 = 0,       /* classic 4-stage Runge-Kutta (App. B, "RKFinal"/"RKDeriv") */
    TDSE_TAYLOR = 1,    /* truncated Taylor series (App. B, Eq. "taylor")             */
    TDSE_LANCZOS = 2    /* short-iterative Lanczos, the method Sec. 5.2 proposes next:
                           `taylor_order` = Krylov dimension m (1..32) products per
                           step, H frozen at the time `taylor_hold` selects, then
                           c <- |c| V exp(-i T dt) e_1 with T the Lanczos tridiagonal.
                           A step whose |dt| times the half-width of T's
                           Gershgorin interval exceeds 4096 is not formed: the
                           state becomes invalid and the next tdse_sync fails.
                           tdse_propagate / tdse_propagate_host only.              */
} tdse_scheme;

typedef enum {
    TDSE_HOLD_LEFT = 0, /* Taylor: H frozen at t_k (the paper's "known time t")  */
    TDSE_HOLD_MID = 1   /* Taylor: H frozen at t_k + dt/2                        */
} tdse_hold;

/*
 * Arithmetic of the dipole-block products.  The state, the diagonal part
 * E o c, the stage/term updates, norms and populations are FP64 in every
 * mode.
 *   TDSE_FP64   U stored FP64, products and sums in FP64.
 *   TDSE_FP32   U stored FP32 (half the bytes), products and sums in FP32,
 *               each block result rounded into the FP64 state.
 *   TDSE_DF32   U stored as an FP32 (hi, lo) pair, products and sums in
 *               float-float arithmetic (about 44 significant bits) on the
 *               FP32 pipe; FP64-class accuracy without FP64 multiplies.
 *   TDSE_BF16X3 tdse_propagate_batch only (other entry points return
 *               TDSE_ENOTSUP, tdse_populations/tdse_norm excepted): U, U^T
 *               and the batched states split into bf16 (hi, lo) pairs, three
 *               tcgen05 tensor-core products (hh + hl + lh) with FP32
 *               accumulation; the batched state between stages is
 *               float-float (FP32 hi + lo) instead of FP64, because the FP64
 *               pipe of this GPU would cost more than the products.
 */
typedef enum {
    TDSE_FP64 = 0,
    TDSE_FP32 = 1,
    TDSE_DF32 = 2,
    TDSE_BF16X3 = 3
} tdse_precision;

typedef struct tdse_ctx tdse_ctx;            /* one Hamiltonian (E, U) resident on the GPU */

/* Version of this ABI (major*10000 + minor*100 + patch). */
int tdse_version(void);

/* Thread-local description of the last failure on this thread ("" if none). */
const char *tdse_last_error(void);

/*
 * tdse_create — upload one Hamiltonian (paper Sec. 5, storage: each diagonal
 * block E_L followed by the superdiagonal block D_L, lower blocks implicit).
 *   energies       host, FP64 [(lmax+1)*n], block l contiguous.
 *   dipole_blocks  host, FP64 [lmax][n][n], row-major U_l = D_{l,l+1};
 *                  may be NULL when lmax == 0.
 *   lmax           >= 0; n >= 1; n <= 4096.
 *   prec           arithmetic of the dipole products (see tdse_precision).
 *   out            receives the new context; the caller owns it and frees it
 *                  with tdse_destroy.
 * The host arrays are copied (and converted to the storage format of `prec`)
 * into device memory owned by the context; they may be freed on return.
 * Synchronous.  Errors: EINVAL, ENOMEM, ECUDA.
 */
tdse_status tdse_create(const double *energies, const double *dipole_blocks,
                        int lmax, int n, tdse_precision prec, tdse_ctx **out);

/* Frees the context and its device memory (after synchronising its work). */
void tdse_destroy(tdse_ctx *ctx);

/* Number of amplitudes N = (lmax+1)*n of the context (0 if ctx is NULL). */
long tdse_size(const tdse_ctx *ctx);

/*
 * tdse_hmatvec — one Hamiltonian-vector product (paper Sec. 4, the block
 * form of H C): y = -i H(f) x  (scale_by_minus_i != 0) or y = H(f) x.
 *   x, y   device, complex [N]; must not alias.
 * Asynchronous on `stream`.  Errors: EINVAL, ECUDA.
 */
tdse_status tdse_hmatvec(tdse_ctx *ctx, double f, const double *x, double *y,
                         int scale_by_minus_i, void *stream);

/*
 * tdse_propagate — advance c over nsteps steps of dt (paper Sec. 4 and
 * App. B): each RK4 stage or Taylor term is one Hamiltonian-vector product
 * fused with its stage update.
 *   c               device, complex [N], in: c(t0), out: c(t0 + nsteps dt).
 *   field           device, FP64 [samples_per_step*nsteps + 1] (see above).
 *   samples_per_step 1 or 2.
 *   dt              step (> 0 or < 0, finite); nsteps >= 0.
 *   scheme          TDSE_RK4 or TDSE_TAYLOR.
 *   taylor_order    K >= 1 (Taylor only; ignored for RK4).
 *   taylor_hold     tdse_hold (Taylor only).
 * Systems whose dipole blocks fit in one CTA's shared memory (at most 1024
 * amplitudes; FP64 also lmax*n^2 <= 16384) run every step in a single
 * launch of one CTA; larger ones take a product launch and an update launch
 * per stage.  Block-product tracing (tdse_profile_*) sees only the latter.
 * Scratch vectors live in the context.  Asynchronous on `stream`; the
 * context must not be used on another stream concurrently.
 * Errors: EINVAL, ECUDA.
 */
tdse_status tdse_propagate(tdse_ctx *ctx, double *c, const double *field,
                           int samples_per_step, double dt, long nsteps,
                           tdse_scheme scheme, int taylor_order, int taylor_hold,
                           void *stream);

/*
 * tdse_propagate_host — tdse_propagate on HOST buffers: copies c and field
 * to the device, propagates, copies c back and synchronises `stream`.
 *   c_host      host, complex [N], in/out.
 *   field_host  host, FP64 [samples_per_step*nsteps + 1].
 * Errors: as tdse_propagate, plus ENOMEM.
 */
tdse_status tdse_propagate_host(tdse_ctx *ctx, double *c_host, const double *field_host,
                                int samples_per_step, double dt, long nsteps,
                                tdse_scheme scheme, int taylor_order, int taylor_hold,
                                void *stream);

/*
 * tdse_sync — waits for the work enqueued on `stream` and reports device-side
 * failures of this context's kernels since the last check: TDSE_ETIMEOUT if a
 * bounded wait inside a kernel gave up (every such wait stops after 2 s; the
 * kernel then finishes without further waiting, and the results of the calls
 * since the last check are invalid); TDSE_EINVAL if a TDSE_LANCZOS step was
 * out of range (see tdse_scheme; that state is invalid).  Clears the device
 * status word.
 * Errors: EINVAL, ECUDA, ETIMEOUT.
 */
tdse_status tdse_sync(tdse_ctx *ctx, void *stream);

/*
 * tdse_norm — out[b] = sum_a |c[b][a]|^2 for b < B, FP64 with a fixed
 * reduction order (bitwise reproducible).  Unitarity is the error measure of
 * paper Sec. 5.1.
 *   c    device, complex [B][N];  out  device, FP64 [B].
 * Errors: EINVAL, ECUDA.
 */
tdse_status tdse_norm(tdse_ctx *ctx, const double *c, int B, double *out, void *stream);

/*
 * tdse_populations — populations after the pulse (paper Sec. 5: the
 * continuum population is the ionisation).  For each of B states:
 *   per_state [B][N]   |c_a|^2                     (device, may be NULL)
 *   per_l     [B][lmax+1] sum over each block      (device, may be NULL)
 *   bound     [B]  sum over E_a <  0               (device, may be NULL)
 *   ionised   [B]  sum over E_a >= 0               (device, may be NULL)
 * FP64, fixed reduction order.  Errors: EINVAL, ECUDA.
 */
tdse_status tdse_populations(tdse_ctx *ctx, const double *c, int B, double *per_state,
                             double *per_l, double *bound, double *ionised, void *stream);

/*
 * tdse_propagate_batch — B independent pulses sharing the context's
 * Hamiltonian (a pulse sweep).  The B states are advanced together so that
 * each dipole block is read once per stage for all of them (block GEMMs
 * U_l [X_{l+1}] and U_l^T [X_l] with X the n x 2B real matrix of the states'
 * real and imaginary parts).  By precision of the context:
 *   FP32    FP32 block GEMM on the FMA pipe.
 *   DF32    float-float block GEMM (every operand an FP32 hi/lo pair,
 *           chunked offset accumulators folded into float-float sums): FP64-
 *           class products for all pulses from FP32 instructions.
 *   BF16X3  tcgen05 tensor-core GEMM of bf16 hi/lo splits (3 products).
 *   FP64    the pulses run one after the other on the single-system path
 *           (as does TDSE_LANCZOS on FP64 and DF32 contexts; FP32 and
 *           BF16X3 contexts return ENOTSUP for it).
 *   c      device, complex [B][N], in/out.
 *   field  device, FP64 [B][samples_per_step*nsteps + 1].
 * Other arguments as tdse_propagate.  Errors: EINVAL, ENOMEM, ENOTSUP, ECUDA.
 */
tdse_status tdse_propagate_batch(tdse_ctx *ctx, double *c, const double *field, int B,
                                 int samples_per_step, double dt, long nsteps,
                                 tdse_scheme scheme, int taylor_order, int taylor_hold,
                                 void *stream);

/*
 * tdse_adjoint — gradient of L = sum_a w_a |c_a(T)|^2 with respect to every
 * field sample, by the exact discrete adjoint of tdse_propagate (the paper
 * has no adjoint; discretise-then-differentiate).  The forward pass stores
 * c every `checkpoint_every` steps; the backward pass recomputes each
 * segment's stage vectors from its checkpoint and runs the costate
 * recursion g_x = (-i H)^dagger g_k backwards.
 *   c0         device, complex [N] (not modified).
 *   field      device, FP64 [samples_per_step*nsteps + 1].
 *   weights    device, FP64 [N] (w_a).
 *   checkpoint_every  >= 1.
 *   grad_field device, FP64, same length as field (overwritten).
 *   c_final    device, complex [N] or NULL: receives c(T).
 *   loss       device, FP64 [1] or NULL: receives L.
 * Errors: EINVAL, ENOMEM, ECUDA, ENOTSUP (TDSE_LANCZOS, BF16X3 contexts).
 */
tdse_status tdse_adjoint(tdse_ctx *ctx, const double *c0, const double *field,
                         int samples_per_step, double dt, long nsteps, tdse_scheme scheme,
                         int taylor_order, int taylor_hold, const double *weights,
                         int checkpoint_every, double *grad_field, double *c_final,
                         double *loss, void *stream);

/*
 * Gauge of the coupling (paper Sec. 5).  In the length gauge (the default)
 * the field factor f(t) is the electric field E(t) and D is real symmetric:
 * upper blocks U_l, lower blocks U_l^T.  In the velocity gauge f(t) is the
 * vector potential A(t) and D = i K is Hermitian with K real antisymmetric:
 * upper blocks i U_l, lower blocks -i U_l^T (the same stored U_l; the
 * momentum matrix elements and the 1/c factor are folded into them).
 */
typedef enum {
    TDSE_LENGTH = 0,
    TDSE_VELOCITY = 1
} tdse_gauge;

/*
 * tdse_set_gauge — select the gauge of every later call on ctx (products,
 * propagation, Lanczos, the adjoint and batches).  Groups take the gauge
 * each member had when tdse_group_create was called.  Synchronises the
 * device; must not be called while work of ctx is in flight.  For a BF16X3
 * context the stored transposed dipole planes change sign (exact).
 * Errors: EINVAL (NULL ctx, unknown gauge), ECUDA.
 */
tdse_status tdse_set_gauge(tdse_ctx *ctx, tdse_gauge gauge);

/*
 * tdse_vector_potential_sin2 — velocity-gauge field samples for the sin^2
 * pulse E(t) = E0 sin^2(pi t / T) sin(omega t) on [0, T], T = 2 pi cycles /
 * omega, zero elsewhere (paper Sec. 5): A[k] = -int_0^{t0 + k h} E(t') dt'
 * for k < nsamples, each interval of length h integrated by the five-point
 * Gauss-Legendre rule (the integral up to t0 over the intervals [j h,
 * (j+1) h] below t0 and the remainder), summed in a fixed order.  For
 * tdse_propagate on the grid t0 + j dt/samples_per_step pass h =
 * dt/samples_per_step and nsamples = samples_per_step*nsteps + 1.
 *   A   device, FP64 [nsamples], 8-byte aligned.
 * Requires omega > 0, cycles > 0, h > 0, t0 >= 0 (all finite),
 * 1 <= nsamples < 2^31 and t0/h < 2^24.  Asynchronous on `stream`.
 * Errors: EINVAL, ECUDA.
 */
tdse_status tdse_vector_potential_sin2(double E0, double omega, double cycles, double t0, double h,
                                       long nsamples, double *A, void *stream);

/*
 * Field given as a function of time, for propagators that choose their own
 * stage times (tdse_propagate_rkf45).
 *   TDSE_FIELD_SIN2   the sin^2 pulse of Sec. 5: E(t) = E0 sin^2(pi t/T)
 *                     sin(omega t) on [0, T], T = 2 pi cycles/omega, zero
 *                     elsewhere.  Length gauge: f(t) = E(t).  Velocity gauge:
 *                     f(t) = A(t), A(t0) = a0 and A advanced over each
 *                     accepted step (and to each stage time) by the
 *                     five-point Gauss-Legendre rule.
 *   TDSE_FIELD_CONST  f(t) = E0 (omega, cycles, a0 unused).
 */
typedef enum {
    TDSE_FIELD_SIN2 = 0,
    TDSE_FIELD_CONST = 1
} tdse_field_kind;

typedef struct {
    int kind;               /* tdse_field_kind */
    double E0, omega, cycles;
    double a0;              /* velocity gauge, sin^2: A(t0) */
} tdse_field_fn;

typedef struct {
    long accepted, rejected, forced;   /* forced: accepted at h <= dt_min with err > tol */
    double t;               /* time reached (t1 unless max_attempts ran out) */
    double dt;              /* step the controller proposes next */
    double err;             /* error estimate of the last attempt */
    double a;               /* velocity gauge, sin^2: A(t) */
} tdse_rkf_stats;

/*
 * tdse_propagate_rkf45 — adaptive Runge-Kutta-Fehlberg 4(5) from t0 to t1
 * (App. B names the embedded pair; Fehlberg's 1969 coefficients).  Each
 * attempt takes six products; the 5th-order combination advances c (as in
 * the paper) and e = h sum (b5_i - b4_i) k_i estimates the local error.
 * Controller: err = |e|_2 / |c|_2; accept when err <= tol, or (forced)
 * when the step is at dt_min;
 * next step h * clamp(0.9 (tol/err)^(1/5), 0.2, 5) within [dt_min, dt_max];
 * no attempt passes t1, and one that would leave less than 1e-12 of the
 * remaining interval takes all of it.  The decisions are taken on the device; the host
 * reads the controller between chunks of attempts, so the call returns with
 * the stream synchronised.
 *   c             device, complex [N], in: c(t0), out: c(t reached).
 *   field         host, the field function (copied).
 *   t0 <= t1, dt0 > 0, tol > 0, 0 <= dt_min <= dt_max (dt_max > 0): finite.
 *   max_attempts  >= 0: bound on accepted plus rejected attempts.
 *   stats         host or NULL.
 * Errors: EINVAL (also when the step underflows: tol unattainable with
 * dt_min = 0; c then holds the last accepted state), ENOTSUP (BF16X3
 * context), ECUDA, ETIMEOUT.
 */
tdse_status tdse_propagate_rkf45(tdse_ctx *ctx, double *c, const tdse_field_fn *field,
                                 double t0, double t1, double dt0, double tol, double dt_min,
                                 double dt_max, long max_attempts, tdse_rkf_stats *stats,
                                 void *stream);

/*
 * Kernel tracing.  While enabled, every block-product launch of the context
 * is bracketed by a pair of CUDA events on its stream, and every kernel the
 * context launches is counted.  tdse_profile_read waits for the recorded
 * events, returns the summed device time of the block-product launches (ms),
 * their number and the number of all kernels launched since the last read,
 * and resets the counters.  Any output pointer may be NULL.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
tdse_status tdse_profile_enable(tdse_ctx *ctx, int on);
tdse_status tdse_profile_read(tdse_ctx *ctx, double *mv_ms, long *mv_launches, long *kernel_launches);

/*
 * Launch shape of the block product (Sec. 4.1: the rows of all stored blocks
 * are split into one balanced contiguous range per work-group).  Reports the
 * CTAs of one product launch, the ring CTAs the plan places on each SM (1:
 * every CTA holds an SM alone; more when short rows of dipole blocks that
 * stream from HBM leave shared memory for several rings), the threads per
 * CTA, whether rows stream through the bulk-copy ring (1) or per-thread
 * loads (0), and whether RK4 / Taylor propagations run all their stages in
 * persistent launches (1) or one product and one update launch per stage
 * (0).  Any output pointer may be NULL.  A bf16x3 context has no
 * single-system product: ENOTSUP.  Errors: EINVAL, ENOTSUP.
 */
tdse_status tdse_plan_info(tdse_ctx *ctx, int *ctas, int *ctas_per_sm, int *threads, int *ring, int *persistent);

/*
 * tdse_populations_noalloc — the populations of tdse_populations for callers
 * that cannot allocate device memory when they need them (for example when
 * another framework's allocator already holds all device memory, or inside a
 * latency-critical loop where an allocation would synchronise the device).
 * It needs no context and calls no allocator; the paper has no counterpart
 * (it is a deployment convenience of this library).
 *   c          device, complex [B][N], N = (lmax+1)*n, 16-byte aligned.
 *   energies   device, FP64 [N] (decides bound E < 0 vs ionised E >= 0).
 *   per_state, per_l, bound, ionised: device outputs as in tdse_populations,
 *              any may be NULL.
 * Limit: B*(lmax+1) <= 16384; larger requests fail with TDSE_EINVAL.
 * Scratch: one fixed 384 KB device array per GPU, held until the process
 * exits and shared by every call; each call writes every entry it later
 * reads, but calls whose kernels overlap on the GPU (different streams, no
 * ordering between them) race on it and must be serialised by the caller.
 * The first call on each device resolves the array's device address with
 * that device current.  CUDA loads device code lazily by default, so that
 * first call is also when the 384 KB array is placed in device memory: make
 * it while the device still has that much free (before another allocator
 * reserves the rest) and before any stream capture.  After cudaDeviceReset
 * the next call on that device is a first call again.
 * Asynchronous on `stream`.  Errors: EINVAL, ECUDA.
 */
tdse_status tdse_populations_noalloc(const double *c, const double *energies, int lmax, int n, int B,
                                     double *per_state, double *per_l, double *bound, double *ionised,
                                     void *stream);

/*
 * Uneven batches: several contexts of different (lmax, n) advanced together
 * (paper Sec. 4 products and App. B RK4 for each system; Sec. 4.1 work
 * split over all of them).  Two ways to run them, chosen by tdse_group_tune
 * or tdse_group_set_persistent:
 *  - bucketed (the default): the systems are bucketed by the thread layout
 *    their row length takes (a handful of classes); each stage is one
 *    block-product launch per bucket (the bucket's rows split evenly over the
 *    GPU's SMs) and its members' stage update;
 *  - one persistent launch: every stage of every step of every system in
 *    one cooperative launch with one thread layout, the rows of all systems
 *    split over all SMs; each stage is the block product, a bounded grid
 *    barrier, the stage update of each CTA's equal slice of all systems'
 *    amplitudes, and a second barrier.
 * All contexts must share one precision.
 */
typedef struct tdse_group tdse_group;

/* systems: host array of `count` contexts (borrowed: they must outlive the
 * group).  Errors: EINVAL, ENOMEM, ECUDA. */
tdse_status tdse_group_create(tdse_ctx *const *systems, int count, tdse_group **out);
void tdse_group_destroy(tdse_group *g);

/*
 * c_ptrs[s]      device, complex [N_s] state of system s (in/out).
 * field_ptrs[s]  device, FP64 [samples_per_step*nsteps + 1] field of system s.
 * Both arrays are host arrays of `count` device pointers.  RK4 only.  One
 * step is captured once into a CUDA graph (re-captured when dt,
 * samples_per_step or the buckets' plans change) and replayed nsteps times;
 * in it every bucket runs its four stages (block product, then its members'
 * stage update) on a stream of its own, the buckets side by side, joined at
 * the end of the step.  The systems' own
 * scratch vectors are used, so a context must not be propagated on its own
 * while its group runs.  Errors: EINVAL, ECUDA.
 */
tdse_status tdse_group_propagate(tdse_group *g, double *const *c_ptrs,
                                 const double *const *field_ptrs, int samples_per_step,
                                 double dt, long nsteps, void *stream);

/*
 * tdse_group_set_persistent — on = 1: later propagations run as one
 * persistent launch (per 2^18 steps) for all systems.  layout: index of the
 * thread layout (0 .. the library's layout count - 1; -1: the one the
 * group's largest n takes alone); rows_per_stage: 1, 2, 4 or 8 rows per bulk
 * copy (0: the plan's own).  Plans the launch (work split, the systems'
 * column-partial slots) and synchronises the device.  on = 0: back to the
 * buckets.  Not while a propagation of the group is in flight.
 * Errors: EINVAL (argument out of range, a depth that does not fit the
 * layout's stage), ENOTSUP (rows too short for the bulk-copy ring, or the
 * launch's CTAs cannot all be resident), ENOMEM, ECUDA; on error the group
 * keeps its previous mode.
 *
 * tdse_group_persistent_info — whether the group runs as one launch, and
 * that launch's CTAs, CTAs per SM, threads per CTA and rows per ring stage
 * (zeros when it does not).  Any output pointer may be NULL.  Errors: EINVAL.
 */
tdse_status tdse_group_set_persistent(tdse_group *g, int on, int layout, int rows_per_stage);
tdse_status tdse_group_persistent_info(const tdse_group *g, int *on, int *ctas, int *ctas_per_sm, int *threads,
                                       int *rows_per_stage);

/* As tdse_sync, for a group (also reports the member kernels' timeouts). */
tdse_status tdse_group_sync(tdse_group *g, void *stream);

/*
 * tdse_group_tune — autotuner of the block product's tile shape per bucket
 * (Sec. 4.1 leaves the work-group size to the device; the paper tuned it by
 * hand per GPU): for every thread layout from the members' own to the next
 * two wider ones (more column groups per row per CTA) and every valid ring
 * depth (1, 2, 4, 8 rows per bulk copy) it re-plans the bucket, times `reps`
 * launches, and keeps the fastest for later tdse_group_propagate calls.
 * Then it times max(reps, 2) whole RK4 steps with the tuned buckets against
 * one persistent launch (tdse_group_set_persistent) for the thread layout of
 * the group's largest n and the next two wider ones at every valid depth,
 * all on zero states and a zero field, and keeps the faster way.
 * Reports the depth chosen for the bucket with the most dipole bytes and the
 * summed best time of one product of every system (either pointer may be
 * NULL).  Clobbers the members' scratch vectors; synchronises `stream`.
 * Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT.
 */
tdse_status tdse_group_tune(tdse_group *g, int reps, int *chosen_rs, double *best_ms, void *stream);

/*
 * Tuning cache.  tdse_group_tuning_save writes, to the text file `path`, one
 * line per bucket: its precision and members' (lmax, n), then the thread
 * layout and rows per stage it uses; and one line for the whole group: its
 * systems' (lmax, n) and whether it runs as one persistent launch, with that
 * launch's layout and depth.  tdse_group_tuning_load applies every
 * line whose bucket (or group) matches g's (same precision and members, in
 * order) and still fits, re-planning those buckets, and reports how many
 * lines it applied (may be NULL); other lines are ignored.  Host file I/O only; a
 * re-planned bucket's next propagation captures a new step graph.
 * Errors: EINVAL (NULL argument, unreadable or unwritable file, not a tuning
 * file), ENOMEM, ECUDA.
 */
tdse_status tdse_group_tuning_save(const tdse_group *g, const char *path);
tdse_status tdse_group_tuning_load(tdse_group *g, const char *path, int *applied);

/*
 * tdse_set_batch_persistent — bf16x3 contexts: on = 1 (the default) runs
 * every stage of a tdse_propagate_batch call in one cooperative launch (per
 * 2^20 stages), the output tiles of all stages dealt round-robin over the
 * CTAs; a tile of the next stage loads the state planes of blocks l-1 and
 * l+1 once every tile of those blocks (for its pulse columns) has written
 * them in the previous stage, and updates its own state once block l's
 * tiles have (per-(block, column tile) counters with bounded waits; the
 * planes alternate between two buffers).  on = 0: one launch per stage.  Both
 * give the same results bit for bit.  Errors: EINVAL, ENOTSUP (not a bf16x3
 * context).
 */
tdse_status tdse_set_batch_persistent(tdse_ctx *ctx, int on);

/*
 * Failure detection.
 *
 * tdse_set_device_memory_limit caps the device memory that all contexts and
 * groups of this library hold together (bytes; 0 removes the cap).  A call
 * that would allocate beyond it fails with TDSE_ENOMEM, as when cudaMalloc
 * itself fails, and leaves what it allocated before to its context.  It lets
 * a caller bound the library's footprint beside another framework's
 * allocator, and lets tests make an allocation fail without filling the GPU.
 * tdse_device_memory_in_use reports the bytes held now.  The fixed scratch of
 * tdse_populations_noalloc is not counted.  Errors: EINVAL.
 *
 * Every propagating call (tdse_propagate, _host, _batch, tdse_adjoint,
 * tdse_group_propagate) scans its field samples on the device; a NaN or
 * infinite sample sets a bit of the status word, and the next tdse_sync
 * (tdse_group_sync) reports TDSE_EINVAL (the host-buffer entry point checks
 * on the host and fails at once).
 *
 * tdse_inject_wait_timeout is a test hook for the timeout path: it runs, on
 * `stream`, one CTA that streams a few bulk copies of the context's energies
 * through a two-stage ring with the same bounded waits the product kernels
 * use, then waits for one stage that nothing arms.  That wait gives up after
 * timeout_ns (1e3..1e9), the CTA lets its copies in flight land, and the
 * next tdse_sync reports TDSE_ETIMEOUT; the context stays usable.
 * Errors: EINVAL, ENOTSUP (bf16x3), ECUDA.
 */
tdse_status tdse_set_device_memory_limit(long long bytes);
long long tdse_device_memory_in_use(void);
tdse_status tdse_inject_wait_timeout(tdse_ctx *ctx, long timeout_ns, void *stream);

/*
 * tdse_group_plan_info — as tdse_plan_info, for bucket `bucket` of a group
 * (0 <= bucket < *buckets); also reports the number of buckets, its members
 * and the rows per ring stage its launches use.  Any output pointer may be
 * NULL; with bucket = -1 only *buckets is written.  Errors: EINVAL.
 */
tdse_status tdse_group_plan_info(const tdse_group *g, int bucket, int *buckets, int *members, int *ctas,
                                 int *ctas_per_sm, int *threads, int *ring, int *rows_per_stage);

#ifdef __cplusplus
}
#endif
#endif /* TDSE_H */
