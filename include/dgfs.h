/*
 * dgfs.h -- C ABI of the GB300 (sm_103a) fast spectral collision library.
 *
 * Computes the multi-species fast Fourier spectral collision operator
 * Q^(pq)(f_p, f_q) of Jaiswal, Hu, Brillon & Alexeenko (PASC'19, arXiv
 * 1903.04670) for every spatial point and every species pair: "given f_p, f_q
 * on N^3 uniform points, produce Q^(pq) at the same grid" (Sec. 2.1).
 *
 * Conventions shared by every entry point
 *  - Velocity grid: N points per dimension on [-L, L]^3, cell centred
 *    (c_j = -L + (j + 1/2) h, h = 2L/N), flattened as (ix*N + iy)*N + iz with
 *    x slowest.  n = N^3.
 *  - Distribution layout f[P][S][n]; operator layout Q[P][S][S][n] with the
 *    pair index p-major, q-minor: Q[pt][p][q] = Q^(pq)(f[pt][p], f[pt][q]).
 *  - Element type: double for a DGFS_FP64 plan, float for every other plan.
 *  - Pointers named *_dev are device pointers on the plan's device; *_host are
 *    host pointers (pageable or pinned).  The caller owns every buffer it
 *    passes; the plan owns its tables and workspace.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued asynchronously unless stated otherwise.
 *  - Errors are returned as dgfs_status codes and never thrown across the
 *    ABI.  A failed call leaves caller buffers in an unspecified state.
 *    dgfs_last_error() gives a human-readable detail of the last failure in
 *    the calling thread.  Asynchronous device faults surface as DGFS_ECUDA on
 *    a later call.
 *  - A plan is immutable after creation and owns one workspace: calls on the
 *    same plan must not overlap (same stream or externally ordered).
 */
#ifndef DGFS_H
#define DGFS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgfs_plan_s *dgfs_plan;
typedef struct dgfs_graph_s *dgfs_graph;
typedef struct dgfs_batch_s *dgfs_batch;
typedef struct dgfs_dg_s *dgfs_dg;

typedef enum {
    DGFS_OK = 0,
    DGFS_EINVAL = 1,       /* bad argument: size, shape, pointer, range      */
    DGFS_ENOMEM = 2,       /* device or host allocation failed               */
    DGFS_ECUDA = 3,        /* CUDA runtime error (launch, copy, async fault) */
    DGFS_ETIMEOUT = 4,     /* a bounded device wait gave up                  */
    DGFS_EUNSUPPORTED = 5  /* valid request this build does not implement    */
} dgfs_status;

typedef enum {
    DGFS_FP64 = 0,     /* FP64 SIMT FFT path (parity anchor)                  */
    DGFS_FP32_TC = 1,  /* tcgen05 DFT-GEMM, 3xTF32 compensated, FP32 accum.   */
    DGFS_TF32 = 2,     /* tcgen05 DFT-GEMM, single TF32 product, FP32 accum.  */
    DGFS_BF16X3 = 3    /* tcgen05 DFT-GEMM, 3-term split BF16, FP32 accum.    */
} dgfs_precision;

/* Parameters of one species pair (p, q): VSS kernel of Eq. (3) with viscosity
 * index omega, scattering parameter alpha and non-dimensional reference
 * diameter d (Kn of Eq. (4) with n0 = H0 = 1, T_ref = T0).  beta_override:
 * NaN = beta^(pq) from Eq. (4) and the beta^(pq) definition (Sec. 2);
 * otherwise the constant used as beta (e.g. the constant Krook-Wu kernel of
 * Sec. 3.2 with omega = alpha = 1). */
typedef struct {
    double omega;
    double alpha;
    double d;
    double beta_override;
} dgfs_pair;

/* Create a plan and its tables (Algorithm 1, Sec. 2.2).
 *   out        : receives the plan handle (set to NULL on failure).
 *   N          : grid points per dimension; 2^a 3^b with 4 <= N <= 48.
 *   L          : half-width of the velocity domain [-L, L]^3 (> 0).
 *   M          : spherical-design size on the full sphere: 6 (octahedron) or
 *                12 (icosahedron), weights 4 pi / M.
 *   N_rho      : Gauss-Legendre points on [0, R_pq] (1 <= N_rho <= 64).
 *   S          : number of species (1 <= S <= 4).
 *   masses     : host array [S] of non-dimensional masses (> 0).
 *   pairs      : host array [S*S], p-major.
 *   prec       : arithmetic of the collision path (see dgfs_precision).
 *   max_points : largest P any later call may pass (1 <= max_points <= 65535,
 *                the points are one grid dimension of the per-point passes);
 *                sizes the workspace.
 *   device     : CUDA device ordinal.
 * Tables are generated on the device in FP64 (per pair: R_pq, quadratures,
 * phase vectors, b^(pq) with N_rho*M*n entries and c^(pq) with n entries).
 * Synchronous.  Errors: EINVAL, ENOMEM, ECUDA, EUNSUPPORTED. */
dgfs_status dgfs_plan_create(dgfs_plan *out, int N, double L, int M, int N_rho, int S,
                             const double *masses, const dgfs_pair *pairs,
                             dgfs_precision prec, int max_points, int device);

/* Declared fast variant (no counterpart in the paper's algorithm): when every
 * pair has alpha = 1 (VHS, so the angular integral is 4 pi sinc(theta |k|)
 * and b_rs does not depend on the design direction s) and the design weights
 * are equal, sum_{r,s} w_r w_s b_rs fft(A_rs B_rs) = sum_r w_r w_s b_r
 * fft(sum_s A_rs B_rs): the forward transforms and the accumulation run once
 * per radial node instead of once per (r, s).  Exact in exact arithmetic;
 * results differ from Algorithm 2's order only by rounding.  It is on by
 * default for plans that qualify (FP64 plans); enable = 0 restores the
 * literal Algorithm 2 order.  Errors: EINVAL, EUNSUPPORTED (enable != 0 on a
 * plan that does not qualify). */
dgfs_status dgfs_plan_set_collapse(dgfs_plan plan, int enable);

/* ---- Dealiased operator (declared variant) ------------------------------
 * Algorithm 2 forms the translate product on the N-point grid, so its Fourier
 * coefficients are the cyclic sum over l + m = k (mod N); the Galerkin form of
 * Eq. (7) sums over l + m = k without wrap-around.  These entry points give
 * the latter by the 3/2 rule, on a plan created at N' = 3N/2 (same L):
 *   1. f' = spectral interpolant of f on the N' grid: the coefficients of f
 *      at its N wavenumbers with the planes carrying -N/2 zeroed (their +N/2
 *      partner is not on the N grid, so only then is the interpolant real);
 *   2. Q' = dgfs_collide on the N' plan (its precision form);
 *   3. Q = the N original wavenumbers of Q', -N/2 planes zeroed, on the N grid.
 * The resampling is FP64.  f_dev [P][S][N^3] and Q_dev [P][S][S][N^3] in the
 * plan's element type; work_dev: caller-owned device scratch, 256-byte
 * aligned, at least dgfs_dealias_work_bytes bytes.  No allocation.
 * Asynchronous.  Errors: EINVAL (also when the plan's N is not 3N/2), ECUDA. */
dgfs_status dgfs_dealias_work_bytes(dgfs_plan plan, int P, int N, size_t *bytes);
dgfs_status dgfs_collide_dealiased(dgfs_plan plan, int P, int N, const void *f_dev, void *Q_dev, void *work_dev,
                                   size_t work_bytes, void *stream);

/* Release a plan and everything it owns.  NULL is accepted.  Synchronous. */
dgfs_status dgfs_plan_destroy(dgfs_plan plan);

/* Collision operator, Algorithm 2 (Sec. 2.2) for all P*S*S (point, pair)
 * evaluations:
 *   Q^(pq) = beta^(pq) Re( ifft( sum_{r,s} w_r w_s b_rs . fft( ifft(t1) ifft(t2) ) )
 *                          - f_p . ifft( c . fft(f_q) ) )
 *   t1 = exp(+i m_q/(m_p+m_q) a_rs) fft(f_p), t2 = exp(-i m_p/(m_p+m_q) a_rs) fft(f_q).
 *   f_dev : device [P][S][n] input (16-byte aligned for tensor-core plans).
 *   Q_dev : device [P][S][S][n] output.
 *   1 <= P <= max_points.  No allocation.  Errors: EINVAL, ECUDA. */
dgfs_status dgfs_collide(dgfs_plan plan, int P, const void *f_dev, void *Q_dev, void *stream);

/* Same operator with host buffers: copies f to the device, evaluates, copies
 * Q back.  Synchronous with respect to the host (returns when Q_host is
 * written).  Uses the plan's staging buffers; no allocation. */
dgfs_status dgfs_collide_host(dgfs_plan plan, int P, const void *f_host, void *Q_host, void *stream);

/* Allocation-free variant of dgfs_collide for DGFS_FP64 plans.  The paper has
 * no counterpart: this entry point exists for callers that may not allocate
 * device memory while they evaluate (a host framework that owns the device
 * memory budget, or a latency-critical loop where an allocation and the
 * synchronisation it can cause are not acceptable).  It computes exactly what
 * dgfs_collide computes, with the same arguments and layouts, but takes its
 * scratch from a 32 MiB array built into the library (every GPU that loads the
 * library holds that array until the process exits) and calls no allocation
 * routine.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is kept per device together with
 *    the id of the context it was found in; after cudaDeviceReset the next
 *    call runs in a new context and looks the address up again (make that
 *    call, too, outside a stream capture).
 *  - All calls on a device share the one array: calls that may overlap on the
 *    GPU (other streams, other host threads) race and must be serialised by the
 *    caller.  Nothing in the array needs to start at zero.
 *  - P is bounded by the array: if even one evaluation per pass does not fit,
 *    the call returns DGFS_EINVAL with the required size in dgfs_last_error().
 *  - Errors: EINVAL (bad argument, P too large), EUNSUPPORTED (not an FP64
 *    plan), ECUDA. */
dgfs_status dgfs_collide_noalloc(dgfs_plan plan, int P, const void *f_dev, void *Q_dev, void *stream);

/* Synchronise the plan's device and report deferred device-side conditions:
 * DGFS_ETIMEOUT if a bounded wait inside a tensor-core kernel expired since
 * the last check (the flag is cleared), DGFS_ECUDA for an asynchronous fault.
 * dgfs_collide_host performs this check itself. */
dgfs_status dgfs_plan_check(dgfs_plan plan);

/* Self-test of the fault path (instrumentation, no counterpart in the paper):
 * enqueue a one-block kernel that performs the same bounded mbarrier wait the
 * tensor-core kernels use, on a barrier that nothing completes (expire != 0)
 * or that the kernel completes itself (expire == 0).  The expired wait raises
 * the plan's flag, so the next dgfs_plan_check returns DGFS_ETIMEOUT; the
 * context stays usable.  Errors: EINVAL, EUNSUPPORTED (FP64 plans have no
 * device waits), ECUDA. */
dgfs_status dgfs_plan_selftest_wait(dgfs_plan plan, int expire, void *stream);

/* Adjoint of the bilinear map (f_p, f_q) -> Q^(pq) (bilinearity of Eq. (7)):
 * for an upstream gradient dQ = dL/dQ [P][S][S][n] returns
 *   df[P][S][n]   = sum over pairs of the f_p- and f_q-gradients,
 *   domega[S*S]   = dL/d omega_pq (host or device pointer, see domega_on_host),
 * recomputing the per-(rho, sigma) translates instead of storing them.
 * f_dev, dQ_dev and df_dev have the plan's element type (double for FP64
 * plans, float otherwise).  FP64 plans run the adjoint in FP64; the other
 * plans run its (rho, sigma) loop on the tensor cores in their operand format
 * and the parts outside it (the transforms of dQ and dQ f_p, the loss-term
 * adjoint, the final inverse transforms, the omega reduction) in FP64; they
 * allocate their FP64 scratch per call, stream-ordered.
 * df_dev is overwritten.  domega may be NULL.  Errors: EINVAL, ECUDA, ENOMEM,
 * ETIMEOUT (a bounded device wait expired), EUNSUPPORTED (the Hermitian
 * form, or N outside 8, 16, 24, 32, 48 on a tensor-core plan). */
dgfs_status dgfs_collide_backward(dgfs_plan plan, int P, const void *f_dev, const void *dQ_dev,
                                  void *df_dev, double *domega, int domega_on_host, void *stream);

/* FP64 moments of Q on the cell-centred grid (conservation, Sec. 2 Eq. (2)):
 *   out[pt][p][q][0..4] = h^3 sum_j Q_j * {1, m_p c_x, m_p c_y, m_p c_z, m_p |c|^2}
 *   Q_dev : device [P][S][S][n] (the plan's element type).
 *   out_dev : device double [P][S][S][5].  Errors: EINVAL, ECUDA. */
dgfs_status dgfs_moments(dgfs_plan plan, int P, const void *Q_dev, double *out_dev, void *stream);

/* Plan introspection.  info (host, 16 doubles):
 *  [0] N [1] L [2] M [3] N_rho [4] S [5] precision [6] max_points
 *  [7] workspace bytes [8] table bytes [9] chunk (evaluations per launch)
 *  [10] (r, s) blocks of the accumulation stage (tensor-core plans)
 *  [11] split products per contraction (tensor-core plans)
 *  [12], [13] CTA groups per (r, s) of the plane and pencil stages (tensor-core plans)
 *  [14] 1 if dgfs_plan_autotune chose the launch parameters
 *  [15] 1 if the sigma collapse is on (dgfs_plan_set_collapse). */
dgfs_status dgfs_plan_info(dgfs_plan plan, double *info);

/* Copy pair (p, q)'s tables to host FP64 buffers for verification:
 *   scalars[8] = {R, beta, gamma, eta, dlogbeta/domega, m_q/mu, m_p/mu, overridden}
 *   rho[N_rho], w_rho[N_rho], sigma[3*M], w_sigma[M],
 *   b[N_rho][M][n] complex (interleaved re, im), c[n] complex.
 * Any output pointer may be NULL.  Synchronous. */
dgfs_status dgfs_plan_pair_tables(dgfs_plan plan, int p, int q, double *scalars, double *rho,
                                  double *w_rho, double *sigma, double *w_sigma, double *b, double *c);

/* Homogeneous relaxation step f_p += dt sum_q Q^(pq) at every point (the
 * spatially homogeneous form of Eq. (1) with explicit Euler time stepping, as
 * in Table 2): f_dev [P][S][n] is updated in place from Q_dev [P][S][S][n].
 * Element type of the plan.  Errors: EINVAL, ECUDA. */
dgfs_status dgfs_relax_step(dgfs_plan plan, int P, void *f_dev, const void *Q_dev, double dt, void *stream);

/* Capture a batch of uneven instances into one CUDA graph: `steps` repetitions
 * of, for each i < count, dgfs_collide(plans[i], P[i], f_dev[i], Q_dev[i]) and,
 * if dt != 0, dgfs_relax_step(plans[i], P[i], f_dev[i], Q_dev[i], dt).  Plans
 * may differ in N, S, M, N_rho and precision but must share one device; an
 * instance's plan must not be used elsewhere while its graph runs (one
 * workspace per plan).  The buffers are bound at capture time.  Synchronous
 * capture; *out receives the graph.  Errors: EINVAL, ECUDA and those of the
 * captured calls. */
dgfs_status dgfs_graph_capture(int count, const dgfs_plan *plans, const int *P, void *const *f_dev,
                               void *const *Q_dev, double dt, int steps, dgfs_graph *out);

/* Replay a captured batch on `stream` (asynchronous). */
dgfs_status dgfs_graph_launch(dgfs_graph graph, void *stream);

/* Number of library kernels one replay of the graph runs. */
dgfs_status dgfs_graph_kernel_count(dgfs_graph graph, long long *count);

/* Release a graph (synchronises its device).  NULL is accepted. */
dgfs_status dgfs_graph_destroy(dgfs_graph graph);

/* Batched work list over uneven instances (several plans with their own N,
 * S, M, N_rho, precision and point counts), the launch-level form of the
 * batching over independent problems (Sec. 3.3: every spatial point and
 * species pair is one evaluation of Algorithm 2).  Instance i evaluates
 * Q^(pq) of f_dev[i] ([P[i]][S][N^3] on the plan's device, 16-byte aligned for
 * tensor-core plans) into Q_dev[i] ([P[i]][S][S][N^3]) exactly as
 * dgfs_collide would; with dt != 0 each launch then applies
 * dgfs_relax_step(plans[i], P[i], f_dev[i], Q_dev[i], dt).  The tensor-core
 * instances that share N and the operand format run their stages together.
 * Their jobs (species pair, chunk of points) form rounds: round k holds the
 * k-th job of every such instance.  By default each stage is launched once
 * per round over all its jobs, each CTA finding its job in a device table;
 * with dgfs_batch_set_schedule(batch, 1) a group of N = 24, 32 or 48 runs all
 * its rounds in one work-list launch instead (see dgfs_plan_set_schedule).
 * FP64 instances run their own collision call.  The pointers are fixed
 * at creation (their contents may change between launches); plans must be
 * distinct, on one device, not used elsewhere while the batch runs, and
 * destroyed only after the batch.  A plan
 * whose launch configuration changes afterwards (dgfs_plan_autotune,
 * dgfs_plan_set_kernel_variant, dgfs_plan_set_collapse) makes the batch stale:
 * dgfs_batch_launch then returns EINVAL and a new batch is needed.  Stage A
 * runs its default kernel variant in a batch.  *out receives the batch.
 * Errors: EINVAL (bad or repeated instance, misaligned f), ENOMEM, ECUDA,
 * EUNSUPPORTED. */
dgfs_status dgfs_batch_create(int count, const dgfs_plan *plans, const int *P, void *const *f_dev,
                              void *const *Q_dev, double dt, dgfs_batch *out);

/* Enqueue one pass of the batch on `stream` (asynchronous; capturable into a
 * CUDA graph).  Errors: EINVAL (NULL or stale batch), ECUDA. */
dgfs_status dgfs_batch_launch(dgfs_batch batch, void *stream);

/* How the batch's tensor-core groups run (Sec. 2.2 batches the M N_rho
 * transforms of a point; Sec. 3.3 makes every (point, pair) evaluation
 * independent, so any order of the jobs is the same computation):
 *   0  per-stage launches, one round of jobs at a time (two streams; default);
 *   1  one work-list launch per group of N = 24, 32, 48.
 * Both give the same bits.  Takes effect at the next dgfs_batch_launch.
 * Errors: EINVAL (NULL batch or mode not 0 or 1). */
dgfs_status dgfs_batch_set_schedule(dgfs_batch batch, int mode);

/* Release a batch (synchronises its device).  NULL is accepted. */
dgfs_status dgfs_batch_destroy(dgfs_batch batch);

/* Autotuner for tensor-core plans: times candidate launch configurations
 * (points per launch, (r, s) blocks of the accumulation stage, CTA counts of
 * the plane and pencil stages) with CUDA events on the caller's f_dev / Q_dev
 * (P points; Q_dev is overwritten) and keeps the fastest; *best_ms (may be
 * NULL) receives its time per call.  Synchronous.  Errors: EINVAL,
 * EUNSUPPORTED (FP64 plans have no tunable launch parameters), ECUDA,
 * ETIMEOUT. */
dgfs_status dgfs_plan_autotune(dgfs_plan plan, int P, const void *f_dev, void *Q_dev, void *stream,
                               double *best_ms);

/* Tensor-core plans: choose the kernel of the first plane stage (T_z, T_y),
 * the one contraction stage with alternative implementations:
 *   0  two 128-thread pipelines per CTA, each thread one operand row (default);
 *   1  warp-specialised: load, transpose and store warpgroups hand items on
 *      through double-buffered shared memory and TMEM (N = 16, 24, 32);
 *   2  256-thread pipelines, two threads per operand row (N = 16, 32, 48).
 * All give the same results to rounding; dgfs_plan_autotune times those that
 * fit and keeps the fastest.  Errors: EINVAL, EUNSUPPORTED (FP64 plan, or the
 * variant does not fit N). */
dgfs_status dgfs_plan_set_kernel_variant(dgfs_plan plan, int variant);

/* Tensor-core plans: how dgfs_collide runs the stages of Algorithm 2's
 * (r, s) loop for its jobs (a job: one species pair and chunk of points):
 *   0  one launch per stage and job; the next job's first stage overlaps the
 *      current job's last on a second stream (default);
 *   1  one work-list launch per call (N = 24, 32, 48): CTAs claim tasks (one
 *      CTA's share of a stage for a job, or a slice of the partial sums) from
 *      a device-side queue in which every task comes after the tasks it reads
 *      from, wait (bounded) on per-job counters for them, run the stage body
 *      and publish their completion; a CTA keeps claiming while the tasks are
 *      of its stage and hands a task of another stage on to a fresh CTA.
 *      Uses the default first-stage kernel variant.
 * Both give the same bits (the same stage bodies on the same data).
 * dgfs_plan_autotune also times mode 1 and keeps it where it is faster.
 * Changing the schedule makes batches built on the plan stale.  The plan's
 * mode is read back with dgfs_plan_get_schedule.  Errors: EINVAL (mode not 0
 * or 1), EUNSUPPORTED (FP64 plan, or mode 1 with another N). */
dgfs_status dgfs_plan_set_schedule(dgfs_plan plan, int mode);
dgfs_status dgfs_plan_get_schedule(dgfs_plan plan, int *mode);

/* Instrumentation of the work-list schedule (no counterpart in the paper):
 * while trace_dev (device memory of `bytes` bytes, caller-owned) is set,
 * every work-list launch records per task four 64-bit words at
 * trace_dev[4 * task]: the global timer (ns) when a CTA took the task, when
 * its dependencies were met and when it ended, and (SM id << 8 | stage, 0-3 =
 * A, B, C, partial sums).  Tasks past bytes / 32 are not recorded; each launch
 * overwrites the buffer from task 0.  NULL switches the trace off.  Process-wide,
 * not thread-safe.  Always returns OK. */
dgfs_status dgfs_debug_worklist_trace(void *trace_dev, size_t bytes);

/* Instrumentation of the work-list schedule: the (r, s) per wave of its queue
 * (rounded up to whole radial nodes; default 12), for the work lists built
 * afterwards (every call in plan mode, at creation for batches).
 * Process-wide.  Errors: EINVAL (rs_per_wave < 1). */
dgfs_status dgfs_debug_worklist_chunk(int rs_per_wave);

/* Declared variant (not the paper's literal Algorithm 2): the Hermitian form.
 * Algorithm 1's wavenumber map gives index N/2 the wavenumber -N/2, which has
 * no +N/2 partner, so a translate of a real f is not exactly real.  With
 * enable != 0, dgfs_collide evaluates
 *   F~ = P fft(f),  f~ = ifft(F~),
 *   QG = sum_rs w_r w_s b_rs . fft( ifft(e^{+i m_q/mu a_rs} F~_p) . ifft(e^{-i m_p/mu a_rs} F~_q) ),
 *   Q  = beta ( ifft(P QG) - f~_p . ifft(c . F~_q) ),
 * P removing every Fourier mode with an index equal to N/2 (the Nyquist
 * planes, of the inputs and of the gain).  Every translate is then real, so
 * the library carries two spatial points in one complex grid (point 2e as
 * the real part, 2e+1 as the imaginary part): the (r, s) work per evaluation
 * halves.  Results differ from the literal form by the Nyquist content (small
 * for resolved distributions).  Enabling allocates the form's workspace
 * (about max_points/2 packed spectra, plus the tensor-core forms' z-pass
 * images); disabling frees it.  dgfs_collide and dgfs_collide_host (and graphs
 * captured from them) follow the setting; dgfs_collide_backward,
 * dgfs_collide_noalloc, dgfs_collide_dealiased and dgfs_batch_create refuse a
 * plan in this form (EUNSUPPORTED).  Errors: EINVAL, EUNSUPPORTED (odd N, or
 * N = 48 on a tensor-core plan), ENOMEM, ECUDA. */
dgfs_status dgfs_plan_set_hermitian(dgfs_plan plan, int enable);

/* Number of the library's kernels launched since the plan was created
 * (host-side counter of launches enqueued by dgfs_* calls on this plan). */
dgfs_status dgfs_plan_launch_count(dgfs_plan plan, long long *count);

/* Profiling hooks (instrumentation, no counterpart in the paper).  With
 * enable != 0 every later kernel launch on the plan is bracketed by a pair of
 * CUDA events recorded on the launch's own stream (16384 pairs, reset on each
 * enable call); enable == 0 synchronises and frees them.  Asynchronous. */
dgfs_status dgfs_plan_profile(dgfs_plan plan, int enable);

/* Aggregate the recorded launches per kernel class.  Synchronises the device.
 *   names     : host char[max_classes][64] (may be NULL), NUL-terminated class names
 *   counts    : host long long[max_classes] launches per class (may be NULL)
 *   total_ms  : host double[max_classes] summed event durations (may be NULL)
 *   n_classes : receives the number of classes written.
 * Returns EINVAL if slots ran out (the totals then cover the first 16384). */
dgfs_status dgfs_plan_profile_read(dgfs_plan plan, int max_classes, char *names, long long *counts,
                                   double *total_ms, int *n_classes);

/* ---- 1-D DG transport around the operator (Eq. (1); Sec. 3.3) ------------
 * Eq. (1), df_p/dt + c . grad_x f_p = sum_q Q^(pq)(f_p, f_q), is solved in the
 * paper by Runge-Kutta discontinuous Galerkin in one space dimension with
 * purely diffuse walls (Sec. 3.3, Couette case of Table 2); the paper defers the
 * formulas to its references, and these entry points implement the textbook
 * nodal scheme:
 *  - Ne equal elements on [x0, x1], K Gauss-Legendre nodes per element (DG
 *    order K); point index e*K + j (element-major), so f[P][S][n] with
 *    P = Ne*K uses the collision layout;
 *  - weak form with the nodes as quadrature and the upwind flux c_x f:
 *      J w_i df_i/dt = c_x sum_j w_j phi_i'(xi_j) f_j - phi_i(+1) F_R + phi_i(-1) F_L,
 *    J = (x1 - x0) / (2 Ne);
 *  - diffuse walls: velocities entering the domain see n_w M_w(c), with
 *    M_w = (m_p/(pi T_w))^{3/2} exp(-m_p |c - u_w|^2 / T_w) and n_w set so
 *    that the discrete net mass flux sum_c c_x f(c) through the wall is zero;
 *  - time: three-stage SSP Runge-Kutta (Shu-Osher form).
 * The DG object keeps a non-owning reference to its plan (which must outlive
 * it), its stage buffers and its wall tables; calls on one DG object or on
 * its plan must not overlap. */

/* Create the DG discretisation for a plan.
 *   walls : host double[8] = {T, ux, uy, uz} of the left wall (x = x0), then
 *           of the right wall (x = x1); T > 0.
 *   1 <= K <= 5, Ne >= 1, Ne*K <= the plan's max_points, x1 > x0, S <= 4.
 * Allocates the stage buffers (two of [P][S][n] and one of [P][S][S][n], in
 * the plan's element type).  Synchronous.  Errors: EINVAL, ENOMEM, ECUDA. */
dgfs_status dgfs_dg_create(dgfs_dg *out, dgfs_plan plan, int Ne, int K, double x0, double x1,
                           const double *walls);

/* Release a DG object (NULL accepted).  Synchronises its device. */
dgfs_status dgfs_dg_destroy(dgfs_dg dg);

/* Physical positions of the P = Ne*K points: host double[P]. */
dgfs_status dgfs_dg_nodes(dgfs_dg dg, double *x_host);

/* Right-hand side of Eq. (1) in the DG weak form:
 *   rhs = -c_x df/dx (upwind DG, diffuse walls) + sum_q Q[pt][p][q]
 *   f_dev   : device [P][S][n] (P = Ne*K), the plan's element type.
 *   Q_dev   : device [P][S][S][n] collision results, or NULL for transport only.
 *   rhs_dev : device [P][S][n] output; must not alias f_dev.
 * Two kernels (wall-flux reduction, nodal right-hand sides), accumulated in
 * FP64.  Asynchronous.  Errors: EINVAL, ECUDA. */
dgfs_status dgfs_dg_rhs(dgfs_dg dg, const void *f_dev, const void *Q_dev, void *rhs_dev, void *stream);

/* One SSP-RK3 step of Eq. (1) in place on f_dev [P][S][n]:
 *   f1 = f + dt L(f); f2 = 3/4 f + 1/4 (f1 + dt L(f1)); f = 1/3 f + 2/3 (f2 + dt L(f2)),
 * L(g) = dgfs_dg_rhs(g, with_collisions ? dgfs_collide(g) : NULL).
 * With collisions, each stage calls the plan's collision operator on all P
 * points (the step then takes the plan's precision form).  No allocation;
 * graph-capturable.  Asynchronous.  Errors: EINVAL, ECUDA, ETIMEOUT. */
dgfs_status dgfs_dg_step(dgfs_dg dg, void *f_dev, double dt, int with_collisions, void *stream);

/* ---- Several slabs side by side (the paper's linear domain decomposition,
 * Sec. 3.3: elements split into contiguous blocks, one per process, sharing
 * O(S N^3) values per interface).  A DG object then covers one block of
 * elements, [x0, x1] being the block's own interval; at an internal
 * interface its neighbour's boundary trace replaces the wall.  Traces are
 * FP64 device arrays [S][n] (n = N^3). */

/* Boundary traces of f_dev [P][S][n]: left_dev = element 0 at xi = -1, the
 * value the left neighbour needs; right_dev = element Ne-1 at xi = +1, the
 * value the right neighbour needs.  Either may be NULL.  Asynchronous.
 * Errors: EINVAL, ECUDA. */
dgfs_status dgfs_dg_traces(dgfs_dg dg, const void *f_dev, double *left_dev, double *right_dev, void *stream);

/* dgfs_dg_rhs with neighbour traces: halo_left_dev is the left neighbour's
 * right trace (used for velocities entering from the left, c_x > 0),
 * halo_right_dev the right neighbour's left trace (c_x < 0); NULL = the wall
 * of dgfs_dg_create at that side.  Asynchronous.  Errors: EINVAL, ECUDA. */
dgfs_status dgfs_dg_rhs_halo(dgfs_dg dg, const void *f_dev, const void *Q_dev, void *rhs_dev,
                             const double *halo_left_dev, const double *halo_right_dev, void *stream);

/* One Runge-Kutta stage, the building block of dgfs_dg_step for
 * decomposed slabs (traces are exchanged between stages):
 *   out = a0 f0 + a1 (f_in + dt L(f_in)),  L as in dgfs_dg_step, halos as in
 *   dgfs_dg_rhs_halo.
 * out may alias f0 but not f_in; f0 may be NULL when a0 = 0.  With
 * collisions, the plan's operator is evaluated on f_in into the DG object's
 * buffer.  Asynchronous.  Errors: EINVAL, ECUDA, ETIMEOUT. */
dgfs_status dgfs_dg_stage(dgfs_dg dg, const void *f_in_dev, const void *f0_dev, void *out_dev, double a0, double a1,
                          double dt, int with_collisions, const double *halo_left_dev,
                          const double *halo_right_dev, void *stream);

/* Peak issue rate of the tensor cores on `device` (instrumentation for the
 * roofline, no counterpart in the paper): one CTA per SM issues `iters`
 * back-to-back tcgen05 MMAs of shape M = 128, N = 256 from zeroed shared-memory
 * operands into TMEM; kind 0 = kind::tf32 (K = 8 per MMA, the peak of the
 * TF32-split forms), kind 1 = kind::f16 with BF16 operands (K = 16, the peak
 * of the split-BF16 form).  *tflops = 2 M N K iters SMs / (best of three
 * timed launches, CUDA events).  Synchronous; allocates 4 bytes.
 * 64 <= iters <= 65536.  Errors: EINVAL, ECUDA, ETIMEOUT. */
dgfs_status dgfs_probe_mma_rate(int device, int kind, int iters, double *tflops);

/* Host-side fault injection for the library's own allocations
 * (instrumentation, no counterpart in the paper).  After
 * dgfs_debug_fail_alloc(n), n > 0, the n-th allocation the library makes from
 * then on -- a device allocation or one of its host objects (plan, tensor-core
 * state, batch, graph, DG object) -- reports failure without allocating; the
 * call that made it returns DGFS_ENOMEM, sets its output handle to NULL and
 * releases what it had allocated.  The hook then switches itself off; n = 0
 * switches it off at once.  Process-wide, not thread-safe against concurrent
 * creation calls.  No GPU fault is involved: the failure is decided on the
 * host before the allocation routine would run.
 * dgfs_debug_live_allocations: device allocations the library holds now
 * (plans, batches, DG objects and per-call workspaces not yet released). */
void dgfs_debug_fail_alloc(int n);
long long dgfs_debug_live_allocations(void);

/* Static strings; never NULL. */
const char *dgfs_status_string(dgfs_status s);
const char *dgfs_last_error(void);
const char *dgfs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DGFS_H */
