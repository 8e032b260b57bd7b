/*
 * ntu.h -- C ABI of the GB300 neighbourhood tensor update (NTU) library.
 *
 * The library implements one NTU bond update of an infinite PEPS on the
 * two-site checkerboard cell (Dziarmaga, arXiv:2107.06635, Sec. II and
 * Figs. 2-5): split the Trotter gate (Fig. 2(a)), apply it and QR-reduce the
 * two site tensors to R_A, R_B without physical/ancilla index (Fig. 2(b)),
 * contract the exact eight-site neighbourhood into the Hermitian,
 * non-negative bond metric g (Fig. 3(b), Fig. 4), and truncate the bond back
 * to D by alternating least squares with a tolerance-selected pseudo-inverse,
 * starting from the local SVD truncation (Fig. 2(c,d), Fig. 5, Eqs. 2-5).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - complex numbers are complex128: interleaved (re, im) doubles, i.e. the
 *    layout of C99 `double _Complex`;
 *  - site tensor T[p][l][u][r][dn], row-major, dn fastest, with
 *    p = s_phys * d_anc + s_anc (d_p = d_phys * d_anc);
 *  - two-site gate G[sA'][sB'][sA][sB] (d_phys^4 complex);
 *  - bond b of the cell is A's leg b in the order (r, u, l, dn):
 *    0: A.r-B.l, 1: A.u-B.dn, 2: A.l-B.r, 3: A.dn-B.u;
 *  - K = D * r is the bond dimension after the gate; n_g = K*K;
 *  - reduced matrices R are K x K row-major; isometries Q are (d_p D^3) x K
 *    row-major with rows (p, e, u, dn), e = the horizontal leg pointing away
 *    from the bond (l for the left-role site, r for the right-role site);
 *  - metric g is n_g x n_g row-major, rows = bra pair (kA', kB'), columns =
 *    ket pair (kA, kB), kA slow (Fig. 4(d,e): eps = x^H g x, Eq. 2);
 *  - truncated matrices M_A, M_B are K x D row-major.
 *
 * Ownership and errors
 * --------------------
 *  - The caller owns every array it passes and keeps it alive until the call
 *    returns (host pointers) or until the context's stream has passed the
 *    work (device pointers, "_dev" calls); the library copies what it keeps.
 *  - The context owns all device memory it allocates (ntu_init) and frees it
 *    in ntu_destroy.
 *  - Every call returns an ntu_status; none aborts the process or traps the
 *    GPU.  Numeric failures found on the device (non-finite values,
 *    non-convergence of an eigen-solver) are raised through a status word
 *    read back at the next synchronising call (ntu_sync, or any call taking
 *    host pointers).  ntu_last_error() gives a one-line description.
 *  - A context is used by one host thread at a time.
 */
#ifndef NTU_H
#define NTU_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ntu_ctx ntu_ctx;

typedef enum {
  NTU_OK = 0,
  NTU_EINVAL = 1,        /* bad argument (shape, index, NULL pointer)        */
  NTU_ENOMEM = 2,        /* device allocation failed                         */
  NTU_ECUDA = 3,         /* CUDA runtime error                               */
  NTU_ENUMERIC = 4,      /* non-finite value or solver non-convergence        */
  NTU_ETIMEOUT = 5,      /* a bounded device-side wait ran out                */
  NTU_EUNSUPPORTED = 6,  /* valid request this build does not support        */
  NTU_ESTATE = 7         /* calls made out of order (apply -> env -> als)     */
} ntu_status;

typedef enum {
  NTU_FP64 = 0,          /* every step in FP64                                */
  NTU_MIXED_FP32 = 1,    /* environment contraction (Fig. 4) in FP32,         */
                         /* solvers in FP64                                   */
  NTU_MIXED_BF16X3 = 2   /* environment contraction with split-BF16 tensor-  */
                         /* core products, FP32 accumulation; solvers FP64   */
} ntu_precision;

typedef struct {
  int D;            /* bond dimension, 1 <= D <= 8                           */
  int d_phys;       /* physical dimension, 2 <= d_phys <= 4                  */
  int d_anc;        /* ancilla dimension (1: none, 2: purification)         */
  int r;            /* gate rank kept by the split, 1 <= r <= d_phys^2      */
  int als_sweeps;   /* fixed number of ALS sweeps (Fig. 5, Eq. 5), 0..1000; */
                    /*   0: the SVDU truncation of Fig. 2(c,d) only          */
  int precision;    /* ntu_precision                                         */
  int tau_kmin;     /* candidate pseudo-inverse tolerances are 10^-k,       */
  int tau_kmax;     /*   k = tau_kmin..tau_kmax (Eq. 4)                      */
  int max_batch;    /* largest n accepted by the ntu_batch_* calls          */
  int wait_budget;  /* polls (about 0.25 us each) a device-side rendezvous  */
                    /*   between the CTAs of one item may wait before it     */
                    /*   gives up and raises NTU_ETIMEOUT; 0: 2^23 (~2 s).   */
                    /*   The tensor-core kernels' internal pipeline waits    */
                    /*   keep a fixed limit of 2^28 polls: a short budget    */
                    /*   there would end a CTA with copies in flight.        */
} ntu_config;

/* Create a context for one (D, d, r) configuration.  `stream` is a
 * cudaStream_t (NULL: the context creates its own non-blocking stream).
 * The context belongs to the device current at this call: its memory, the
 * SM count that sizes its persistent grids and the kernels' shared-memory
 * limits are that device's, so make it current for every later call on the
 * context.  Without a usable device the call returns NTU_ECUDA.
 * Requires d_p * D^2 >= r so that the gated site matrix has at least K rows,
 * and D * r <= 32.  NTU_MIXED_BF16X3 needs a compute capability 10.x GPU and
 * 2 * d_p * D <= 64 (else NTU_EUNSUPPORTED, before any device work).
 * Allocates all device memory the calls below need for up to max_batch items.
 * On the mixed contexts a max_batch of at most 3 * SMs / 2 (228 on 152 SMs)
 * lets each item's ALS run on a cluster of 2 CTAs, at most 3 * SMs / 4 on
 * 4 (same results, bit for bit); its ALS scratch is then allocated that many
 * times. */
int ntu_init(const ntu_config* cfg, void* stream, ntu_ctx** out);
int ntu_destroy(ntu_ctx* ctx);
/* The last error message of `ctx`; with ctx == NULL, of the calling thread's
 * last failed call that had no context (ntu_init, ntu_gate_qr_noalloc). */
const char* ntu_last_error(const ntu_ctx* ctx);
/* Wait for the context's stream; returns the first device-raised status. */
int ntu_sync(ntu_ctx* ctx);

/* ---- two-site unit cell held by the context (host pointers) ------------ */

/* Load / read the iPEPS tensors A and B (each d_p*D^4 complex). */
int ntu_set_state(ntu_ctx* ctx, const double* A, const double* B);
int ntu_get_state(ntu_ctx* ctx, double* A, double* B);

/* Fig. 2(a,b): split `gate` (d_phys^4 complex) at rank r, apply its halves to
 * the two sites of `bond`, and QR-reduce them.  Keeps Q and R on the device
 * for the next two calls.  RA_out / RB_out (K x K complex each) may be NULL. */
int ntu_apply_gate(ntu_ctx* ctx, int bond, const double* gate,
                   double* RA_out, double* RB_out);

/* Fig. 4: the exact eight-site metric of the bond prepared by
 * ntu_apply_gate, Hermitised, non-negativity repaired and normalised to unit
 * trace.  g_out (n_g x n_g complex) may be NULL; diag_out (3 doubles, may be
 * NULL) receives [||g - g^H|| / ||g|| before repair, lambda_min / lambda_max
 * (NaN when a Cholesky factorisation certified g positive definite and no
 * repair was needed), log(trace) removed by the normalisation]. */
int ntu_env_metric(ntu_ctx* ctx, int bond, double* g_out, double* diag_out);

/* Fig. 5, Eqs. 2-5: SVDU start, als_sweeps ALS sweeps with the tolerance
 * chosen to minimise eps, balancing, then A' = Q_A M_A, B' = Q_B M_B written
 * back into the context's state (unit Frobenius norm each).  Outputs (may be
 * NULL): eps, delta = eps / eps0, and the last selected tolerance (NaN when
 * als_sweeps = 0: the result is then the SVDU truncation of Fig. 2(c,d)). */
int ntu_als_truncate(ntu_ctx* ctx, int bond, double* eps_out, double* delta_out,
                     double* tau_out);

/* One second-order Trotter step: single-site gate `gate1_half` (d_phys x
 * d_phys complex, NULL for none) on both sites, then the four bond updates
 * in the order 0,1,2,3 with gates2[b] (4 x d_phys^4 complex), then
 * gate1_half again.  delta_out (4 doubles) may be NULL. */
int ntu_step(ntu_ctx* ctx, const double* gates2, const double* gate1_half,
             double* delta_out);

/* Cluster estimator <O> on site 0 (A) or 1 (B): the site with `op` (d_phys x
 * d_phys complex) on its physical factor, closed by the leaf edge tensors of
 * its four neighbours, over the same network with the identity.  value_out:
 * one complex. */
int ntu_measure(ntu_ctx* ctx, int site, const double* op, double* value_out);

/* ---- simple update of the cell (Sec. II) ------------------------------- */
/* The simple update (SU) keeps a diagonal bond tensor lambda_b (D
 * non-negative values) on each of the cell's four bonds and uses the metric
 * g_SU = 1_d (x) 1_d (x) prod_j lambda_j over the six outer bonds of the
 * updated pair (Sec. II), whose minimiser is a truncated SVD (cost ~D^5, no
 * environment contraction).  Convention: the state tensors A, B set by
 * ntu_set_state are in the symmetric gauge, each leg carrying sqrt(lambda)
 * of its bond.  ntu_init sets every lambda to 1; ntu_set_state leaves the
 * lambdas alone.
 * ntu_su_set_lambdas / ntu_su_get_lambdas: lam is 4 x D doubles, row b =
 *   lambda of bond b (finite, >= 0; else NTU_EINVAL).
 * ntu_su_update: one SU bond update of `bond` with `gate` (d_phys^4
 *   complex): the outer legs of both sites are weighted by sqrt(lambda),
 *   gate + QR (Fig. 2(a,b)), truncation of R_A R_B^T to its D largest
 *   singular values with sqrt(S) on both sides (Fig. 2(c,d)), recompose,
 *   the outer weights removed again (values at or below 1e-14 x the bond's
 *   largest give 0), each tensor normalised; lambda_bond becomes the kept
 *   singular values normalised to unit 2-norm.  delta_out (may be NULL):
 *   the discarded weight sum_{i>D} s_i^2 / sum_i s_i^2, the relative error
 *   in the metric g_SU.
 * ntu_su_step: the second-order Trotter step of ntu_step with SU bond
 *   updates (gates2 4 x d_phys^4, gate1_half d_phys x d_phys or NULL);
 *   delta_out 4 doubles or NULL. */
int ntu_su_set_lambdas(ntu_ctx* ctx, const double* lam);
int ntu_su_get_lambdas(ntu_ctx* ctx, double* lam);
int ntu_su_update(ntu_ctx* ctx, int bond, const double* gate, double* delta_out);
int ntu_su_step(ntu_ctx* ctx, const double* gates2, const double* gate1_half,
                double* delta_out);

/* ---- batches of independent bond updates (device pointers) ------------- */
/* Item i is the bond Ta[i].r - Tb[i].l (bond-0 orientation) of its own
 * two-site cell with gate gates[i].  All arrays are contiguous stacks of n
 * items; work is queued on the context's stream and the call returns at once. */

/* The whole update: Ta_out / Tb_out receive A', B'; info (n x 4 doubles)
 * receives [eps, delta, eps0, tau] per item (tau NaN when als_sweeps = 0). */
int ntu_batch_update_dev(ntu_ctx* ctx, int n, const double* Ta, const double* Tb,
                         const double* gates, double* Ta_out, double* Tb_out,
                         double* info);

/* Same with host pointers: host-to-device copies, the update and the
 * device-to-host copies, synchronised before return.  A batch of at least
 * 6 x SMs items runs as two halves whose copies overlap the other half's
 * compute (a second stream of the context, created on first use); the
 * outputs equal those of one ntu_batch_update_dev call bit for bit, and
 * ntu_stage_times then reports the second half.  Pinned host buffers let
 * the copies run asynchronously. */
int ntu_batch_update_host(ntu_ctx* ctx, int n, const double* Ta, const double* Tb,
                          const double* gates, double* Ta_out, double* Tb_out,
                          double* info);

/* ---- uneven batches ------------------------------------------------------
 * Independent bond updates whose bond dimension D and gate rank r differ from
 * item to item (the batch form of the step driver, Sec. II, run over many
 * independent bonds).  An ntu_uneven holds one context per kind (D, r) --
 * each with its own plan, work space and stream -- and pinned host staging.
 * Every call forks the kinds' work from the uneven's stream onto the kind
 * streams and joins it back, so the kinds run concurrently on the GPU.
 *
 * ntu_uneven_init: n_kinds distinct kinds (D[k], r[k]), at most max_items[k]
 *   items of kind k per call; d_phys, d_anc, als_sweeps, precision, tau_kmin,
 *   tau_kmax as in ntu_config (shared by every kind); stream NULL creates a
 *   private stream.  Errors: NTU_EINVAL (repeated kind, bad sizes), and the
 *   errors of ntu_init for any kind.
 * ntu_uneven_update_host: n items (host pointers); item i is of kind
 *   kind[i]; Ta, Tb, Ta_out, Tb_out are the items' site tensors concatenated
 *   in item order (item i takes d_p * D^4 complex of its kind); gates n x
 *   d_phys^4 complex; info n x 4 ([eps, delta, eps0, tau] as in
 *   ntu_batch_update_dev).  The items of each kind go through that kind's
 *   batched update; with use_graph = 1 the device part of the call (copies
 *   in, every kind's update, copies out) is captured as one CUDA graph the
 *   first time a given set of per-kind counts is seen, and replayed by later
 *   calls with the same counts.  Synchronises before return; afterwards the
 *   items count as staged (below).  Errors: NTU_EINVAL (unknown kind, more
 *   items of a kind than max_items), device status of any kind as in
 *   ntu_sync.
 * ntu_uneven_stage: copy n items (same layout) to the device and keep them
 *   there as the staged items; synchronises.
 * ntu_uneven_run: enqueue the update of the staged items on the uneven's
 *   stream and return without synchronising; results stay on the device.
 *   mode NTU_UNEVEN_GROUPED: one batched update per kind; NTU_UNEVEN_GRAPH:
 *   the same captured as a CUDA graph on first use for the staged per-kind
 *   counts and replayed afterwards; NTU_UNEVEN_PER_ITEM: one update launch
 *   sequence per item (the per-bond form, for comparison).  All modes give
 *   the same results.  Errors: NTU_EINVAL (mode).
 * ntu_uneven_sync: wait for the uneven's stream; device status of every kind
 *   with staged items, as in ntu_sync.
 * ntu_uneven_fetch: copy the results of the staged items back (kind[] must
 *   give the staged per-kind counts, else NTU_ESTATE); synchronises.
 * ntu_uneven_last_launch_count: kernels launched by the last update or run
 *   (for a graph replay: the kernels of the graph).
 * ntu_uneven_last_error: description of the last failure (uneven == NULL:
 *   of the last failed ntu_uneven_init). */
typedef struct ntu_uneven ntu_uneven;
enum { NTU_UNEVEN_GROUPED = 0, NTU_UNEVEN_GRAPH = 1, NTU_UNEVEN_PER_ITEM = 2 };
int ntu_uneven_init(int d_phys, int d_anc, int als_sweeps, int precision, int tau_kmin,
                    int tau_kmax, int n_kinds, const int* D, const int* r, const int* max_items,
                    void* stream, ntu_uneven** out);
int ntu_uneven_update_host(ntu_uneven* uneven, int n, const int* kind, const double* Ta,
                           const double* Tb, const double* gates, double* Ta_out,
                           double* Tb_out, double* info, int use_graph);
int ntu_uneven_stage(ntu_uneven* uneven, int n, const int* kind, const double* Ta,
                     const double* Tb, const double* gates);
int ntu_uneven_run(ntu_uneven* uneven, int mode);
int ntu_uneven_sync(ntu_uneven* uneven);
int ntu_uneven_fetch(ntu_uneven* uneven, int n, const int* kind, double* Ta_out,
                     double* Tb_out, double* info);
int ntu_uneven_last_launch_count(const ntu_uneven* uneven);
int ntu_uneven_destroy(ntu_uneven* uneven);
const char* ntu_uneven_last_error(const ntu_uneven* uneven);

/* Stage calls (device pointers), for testing and for callers that chain
 * their own pipeline.
 *   gate_qr : Fig. 2(a,b)   -> QA, QB ((d_p D^3) x K), RA, RB (K x K)
 *   env     : Fig. 4        -> raw g (n_g x n_g), no Hermitisation/repair
 *   repair  : Sec. II       -> g Hermitised, repaired, unit trace; diag n x 3
 *   als     : Fig. 5        -> MA, MB (K x D), info n x 4
 *   recompose: Fig. 2(e)    -> Ta_out, Tb_out                              */
int ntu_batch_gate_qr_dev(ntu_ctx* ctx, int n, const double* Ta, const double* Tb,
                          const double* gates, double* QA, double* RA, double* QB,
                          double* RB);
int ntu_batch_env_dev(ntu_ctx* ctx, int n, const double* Ta, const double* Tb,
                      const double* QA, const double* QB, double* g);
int ntu_batch_repair_dev(ntu_ctx* ctx, int n, double* g, double* diag);
int ntu_batch_als_dev(ntu_ctx* ctx, int n, const double* g, const double* RA,
                      const double* RB, double* MA, double* MB, double* info);
int ntu_batch_recompose_dev(ntu_ctx* ctx, int n, const double* QA, const double* QB,
                            const double* MA, const double* MB, double* Ta_out,
                            double* Tb_out);

/* Failure-detection test hook.  With `on` = 1 every later ALS rendezvous of
 * the context waits for one arrival more than the CTAs of an item make, so
 * each such wait runs out after wait_budget polls and the next synchronising
 * call returns NTU_ETIMEOUT (the results of that call are invalid); `on` = 0
 * restores normal operation.  Only contexts whose ALS runs on CTA clusters
 * have this rendezvous (mixed precision and max_batch <= 3 * SMs / 2);
 * others return NTU_EUNSUPPORTED.  No wait is unbounded, nothing faults, and
 * the context stays usable. */
int ntu_inject_wait_timeout(ntu_ctx* ctx, int on);

/* ---- launch tuning ------------------------------------------------------
 * Schedule and arithmetic choices of a context's kernels.  Fields:
 *   t12_pair        -1: automatic (pair at D = 8); 0: the fused t1 -> t2
 *                   kernel runs one (k, k') unit per GEMM2; 1: pairs of units
 *                   (k, k'), (k, k'+1) share one N = 128 GEMM2 (D = 8 only);
 *   als_ctas_per_sm 0: automatic (3 when a batch has more than 2 x SMs items,
 *                   else 2); 2 or 3: the ALS kernel's register budget for
 *                   that many CTAs per SM;
 *   als_split       0: automatic (the split chosen at ntu_init, reduced
 *                   while items x split exceeds the SMs, 1.5 x SMs at
 *                   D <= 4); 1, 2 or 4 CTAs per item's ALS, at most the
 *                   split ntu_init allocated for (mixed contexts only;
 *                   FP64 contexts take 0 or 1);
 *   als_build       how the mixed contexts build the ALS reduced metric
 *                   (Fig. 5(b)): 0 automatic (2 where possible), 1 in
 *                   double-FP32 on the FP32 lanes, 2 its first stage on the
 *                   tensor cores with exact BF16 slicing (K = D r = 16 or
 *                   32, on one CTA or on a cluster of als_split CTAs that
 *                   divide its tiles; else the lanes).  The two builds
 *                   agree to ~2^-48 relative, not bit for bit.
 * The schedule fields change speed only: with the same als_build every
 * combination gives the same numbers bit for bit.
 * ntu_set_tuning rejects out-of-range values with NTU_EINVAL and drops the
 * CUDA graphs the context captured.  ntu_get_tuning reads the settings and,
 * in split_max, the largest als_split this context accepts.
 * ntu_uneven_set_tuning / ntu_uneven_get_tuning do the same for one kind
 * (index into the kinds of ntu_uneven_init) of an uneven batch; setting
 * drops the uneven's captured graphs. */
typedef struct {
  int t12_pair;
  int als_ctas_per_sm;
  int als_split;
  int als_build;
} ntu_tuning;
int ntu_set_tuning(ntu_ctx* ctx, const ntu_tuning* t);
int ntu_get_tuning(const ntu_ctx* ctx, ntu_tuning* t, int* split_max);
int ntu_uneven_set_tuning(ntu_uneven* uneven, int kind, const ntu_tuning* t);
int ntu_uneven_get_tuning(const ntu_uneven* uneven, int kind, ntu_tuning* t, int* split_max);

/* CUDA graphs of the unit-cell step.  With graphs on (the default), the
 * device work of ntu_step and ntu_su_step -- the single-site gates and the
 * four bond updates, some 90 launches -- is captured as one CUDA graph on
 * the first call (one graph per call form: with or without gate1_half) and
 * replayed by later calls; the gates are copied in before the replay and
 * the deltas read back after it.  Off: the same launches are issued one by
 * one.  Results are identical.  Capture needs the context's own or a
 * non-legacy stream; where capture fails the call runs the launches
 * directly. */
int ntu_set_graphs(ntu_ctx* ctx, int on);

/* Number of kernel launches the last ntu_batch_update_* call queued. */
int ntu_last_launch_count(const ntu_ctx* ctx);

/* Stage timing of ntu_batch_update_dev / _host.  With profiling on (flag 1),
 * the context records CUDA events on its stream between the stages of each
 * update; ntu_stage_times then synchronises and writes the durations in ms of
 * the last update's five stages into ms_out[5]: gate+QR (Fig. 2(a,b)),
 * environment (Fig. 4), repair (Sec. II), ALS (Fig. 5), recompose
 * (Fig. 2(e)).  The ALS stage is exactly one kernel launch. */
int ntu_set_profiling(ntu_ctx* ctx, int on);
int ntu_stage_times(ntu_ctx* ctx, double* ms_out);

/* Which solver path the device took, counted since the previous call (then
 * reset), into counts[8]: counts[0] ALS solves whose tolerance selection
 * (Eq. 4) was decided by Gershgorin discs (every candidate tolerance keeps
 * every eigenpair of g_A) and solved by conjugate gradients, counts[1] ALS
 * solves decided by a shifted Cholesky factorisation and solved by
 * iterative refinement, counts[2] ALS solves through the eigendecomposition
 * and the full selection, counts[3] metrics certified positive definite by
 * Gershgorin discs, counts[4] by Cholesky, counts[5] metrics repaired
 * through the eigendecomposition (Sec. II), counts[6] QRs of gated matrices
 * (Fig. 2(b)) by double-FP32 CholeskyQR2 (mixed contexts), counts[7] by
 * Householder (FP64 contexts, and matrices too ill-conditioned for
 * CholeskyQR2).  Synchronises the context's stream. */
int ntu_solver_paths(ntu_ctx* ctx, int* counts);

/* ---- a stage for callers that cannot allocate device memory ----------- */
/* The paper has no counterpart to this call; it exists for callers that
 * cannot call cudaMalloc (a framework that owns all device memory through
 * its own pool, or code that must not trigger the device-wide
 * synchronisation of cudaMalloc/cudaFree), and so cannot create an ntu_ctx.
 * It computes exactly what ntu_batch_gate_qr_dev computes for one item
 * (gate split, gate application, QR with positive diag(R)) from device
 * pointers Ta, Tb (d_p D^4 complex each), gate (d_phys^4 complex) into
 * QA, QB ((d_p D^3) x K) and RA, RB (K x K), queued on `stream` (NULL: the
 * legacy default stream), and allocates nothing: its scratch is one fixed
 * 4 MiB array in device memory, held by every GPU that loads the library
 * until the process exits.  Sizes needing more than 4 MiB of scratch
 * (16 * (2 d^2 r + 4 (d_p D^3)(D r)) bytes) are rejected with NTU_EINVAL.
 * The first call on a device looks up the array's device address and sets a
 * kernel's shared-memory limit there, so make that first call before any
 * stream capture; under lazy module loading (the CUDA default) that first
 * call, or the first launch of its kernels, may also load the module, which
 * places the array and may synchronise the device, so make a warm-up call
 * outside latency-critical code.  The looked-up address is kept for the
 * life of the process: no cudaDeviceReset may come between calls.  Every
 * call reuses the same array: calls that overlap on the GPU (different
 * streams, or several host threads) race on it and must be serialised by
 * the caller.  Errors are reported through ntu_last_error(NULL), whose
 * message belongs to the calling host thread.  No device status is kept:
 * a non-finite input gives non-finite outputs and still returns NTU_OK, so
 * check the outputs where that matters. */
int ntu_gate_qr_noalloc(int D, int d_phys, int d_anc, int r, const double* Ta,
                        const double* Tb, const double* gate, double* QA, double* RA,
                        double* QB, double* RB, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NTU_H */
