/*
 * qxd.h -- C ABI of the GB300 library for the openQ*D Dirac operator with
 * C* boundary conditions (arXiv:1710.08839).
 *
 * The library applies D = m0 + Dw + dDsw for one quark of integer charge
 * qhat (Sec. 2.3, Eqs. (16)-(23); periodic time, so dDb = 0) on the extended
 * lattice of Sec. 2.1 (Eq. (1)): x1 is doubled to 2 L1, the mirror half of
 * the gauge field is the complex conjugate of the physical half (Eq. (4a)),
 * and crossing the x2 or x3 boundary of a C* direction lands in the mirror
 * copy (shifted boundary, Eq. (11), Fig. 1). It also solves D x = b.
 *
 * Conventions shared by every entry point:
 *  - Return value: QXD_OK (0) or a negative qxd_status. No entry point
 *    throws, exits or aborts; qxd_last_error() gives a message for the
 *    calling thread's last failure.
 *  - Ownership: the caller owns every pointer passed in; the library copies
 *    what it keeps (gauge field, parameters) into its own device storage and
 *    never frees or retains caller memory. A qxd_lattice is owned by the
 *    library between qxd_lattice_create and qxd_lattice_destroy.
 *  - Streams: `stream` arguments are cudaStream_t values (NULL = the stream
 *    given at create time). Calls are asynchronous on that stream unless
 *    stated otherwise; calls that return a device-side status (set_gauge,
 *    sw_build, solve) synchronise that stream.
 *  - Threads: one lattice must not be used by two host threads at once, nor
 *    by calls on two streams whose work may overlap on the GPU: a lattice's
 *    calls share its conversion scratch and work fields (Schwarz, solver,
 *    deflation). The engine and server keep the work fields of every request
 *    apart, so their requests may share an operator.
 *  - Site order ("lexicographic"): x = (x0, x1, x2, x3) over the simulated
 *    lattice N = (T, N1, L2, L3), N1 = 2 L1 when direction 1 is C*, else L1;
 *    index ((x0 N1 + x1) L2 + x2) L3 + x3 (x3 fastest).
 *  - Spinor, lexicographic layout: [site][spin 4][colour 3][re, im], FP64
 *    (double) or FP32 (float) by the precision flag. Spin basis: chiral,
 *    gamma5 = diag(1, 1, -1, -1), gamma0 = [[0, -1], [-1, 0]],
 *    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] (the paper fixes no basis).
 *  - Spinor, native layout: the library's even-odd structure-of-arrays
 *    layout; qxd_spinor_bytes gives its size, qxd_spinor_pack/unpack convert.
 */
#ifndef QXD_H
#define QXD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qxd_lattice qxd_lattice;

typedef enum {
    QXD_OK = 0,
    QXD_ERR_ARG = -1,            /* invalid argument (sizes, flags, NULL)          */
    QXD_ERR_OOM = -2,            /* device or host allocation failed               */
    QXD_ERR_CUDA = -3,           /* a CUDA runtime call or kernel launch failed    */
    QXD_ERR_NOT_ADMISSIBLE = -4, /* gauge field violates the orbifold constraint   */
    QXD_ERR_SW_SINGULAR = -5,    /* a clover block is singular or non-finite       */
    QXD_ERR_NOT_CONVERGED = -6,  /* solver hit max_iter (x and info still written) */
    QXD_ERR_NUMERIC = -7,        /* NaN/Inf met in a solver                        */
    QXD_ERR_STATE = -8,          /* call out of order (e.g. Dw before sw_build)    */
    QXD_ERR_TIMEOUT = -9         /* a bounded device-side wait ran out             */
} qxd_status;

/* precision of spinors passed to qxd_Dw and friends */
#define QXD_FP64 0x0
#define QXD_FP32 0x1
/* where caller spinor buffers live */
#define QXD_DEVICE 0x0
#define QXD_HOST 0x10
/* spinor layout of caller buffers */
#define QXD_LAYOUT_LEX 0x0
#define QXD_LAYOUT_NATIVE 0x100

/* qxd_set_gauge flags */
#define QXD_GAUGE_PHYSICAL_HALF 0x0      /* arrays over x1 < L1; mirror built by Eq. (4a) */
#define QXD_GAUGE_EXTENDED_CHECKED 0x1   /* arrays over the whole simulated lattice;      */
                                         /* rejected unless they obey Eq. (4a)            */
#define QXD_GAUGE_EXTENDED_UNCHECKED 0x2 /* whole simulated lattice, taken as is          */
#define QXD_GAUGE_HOST 0x10              /* su3/u1 pointers are host memory               */

/*
 * Create a lattice: physical extents T x L1 x L2 x L3 (Sec. 2.1, Eq. (1)).
 * cstar_mask: bit k (k = 1, 2, 3) makes direction k a C* direction. Any C*
 * direction needs bit 1 (the orbifold doubles x1). Time is periodic.
 * Requirements (else QXD_ERR_ARG): T, L1, L2, L3 even and >= 2, so that the
 * even-odd parity x0 + x1 + x2 + x3 mod 2 is well defined on the shifted
 * torus; the simulated volume below 2^30 sites.
 * stream: the default cudaStream_t for this lattice (NULL = legacy default).
 * Allocates the device storage of the gauge field and the clover term.
 */
int qxd_lattice_create(qxd_lattice** out, int T, int L1, int L2, int L3,
                       unsigned cstar_mask, void* stream);

/* Free all storage of the lattice (NULL is accepted). Synchronises its stream. */
int qxd_lattice_destroy(qxd_lattice* lat);

/*
 * A view shares the gauge field (and clover field tensors) of `parent` (or of
 * parent's own parent) and owns its own quark parameters, clover term,
 * scratch and solver work: one view per (m0, csw, cswqed, qhat) lets several
 * quarks use one resident gauge field. Every entry point that takes a
 * lattice accepts a view, except qxd_set_gauge (QXD_ERR_STATE). A new gauge
 * field on the parent makes each view's clover term stale: the view returns
 * QXD_ERR_STATE until it calls qxd_sw_build again. The parent cannot be
 * destroyed while views exist (QXD_ERR_STATE). stream: NULL = the parent's.
 */
int qxd_lattice_view(qxd_lattice** out, qxd_lattice* parent, void* stream);

/* Simulated extents N[4] and volume (number of sites) of the lattice. */
int qxd_lattice_dims(const qxd_lattice* lat, int* N4, long long* volume);

/*
 * Set the gauge field (Sec. 2.1, Eqs. (3)-(4a)).
 * su3:       SU(3) links U(x, mu), layout [site][mu 4][row 3][col 3][re, im]
 *            double; u1_angle: photon field A(x, mu), layout [site][mu 4]
 *            double (z = exp(i A)).
 * With QXD_GAUGE_PHYSICAL_HALF the site range is the physical lattice
 * x1 < L1 in lexicographic order of (T, L1, L2, L3); the mirror half is set
 * to U^* and -A (Eq. (4a)). Without C* the physical lattice is the whole
 * lattice. With QXD_GAUGE_EXTENDED_* the arrays cover the simulated lattice.
 * Links must be SU(3) to 1e-10 (the FP32 path stores two rows and rebuilds
 * the third): otherwise QXD_ERR_ARG. CHECKED rejects fields that violate
 * Eq. (4a) beyond 1e-12 with QXD_ERR_NOT_ADMISSIBLE. The field tensors of
 * the clover term are computed here (FP64). Invalidates the clover term.
 * Synchronises the lattice stream.
 */
int qxd_set_gauge(qxd_lattice* lat, const double* su3, const double* u1_angle, int flags);

/*
 * Set the quark parameters of Sec. 2.3 (Eq. (16), (17), (21)): bare mass m0,
 * SU(3) and U(1) SW coefficients csw, cswqed, and the integer charge
 * qhat = q / q_el (the U(1) links enter as z^qhat; q_el cancels from D).
 * Invalidates the clover term (call qxd_sw_build next).
 */
int qxd_set_params(qxd_lattice* lat, double m0, double csw, double cswqed, int qhat);

/*
 * Build the site-diagonal part M(x) = (4 + m0) + dDsw(x) of D (Eq. (21)-(23))
 * as two 6x6 Hermitian blocks per site (spins {0,1} and {2,3} in the chiral
 * basis), in FP64 and FP32, and their inverses (used by the even-odd and
 * SAP paths; Sec. 2.4, Doo^-1). Needs qxd_set_gauge and qxd_set_params
 * (else QXD_ERR_STATE). Returns QXD_ERR_SW_SINGULAR if any block is
 * singular to working precision or non-finite (inverse pivots below
 * 1e-12 of the block norm). Synchronises the lattice stream.
 */
int qxd_sw_build(qxd_lattice* lat);

/*
 * out = D in (Sec. 2.3): (D psi)(x) = M(x) psi(x)
 *   - 1/2 sum_mu [ (1 - gamma_mu) U(x,mu) z(x,mu)^qhat psi(x + mu)
 *                + (1 + gamma_mu) U(x-mu,mu)^+ z(x-mu,mu)^-qhat psi(x - mu) ].
 * flags: QXD_FP64 | QXD_FP32, QXD_DEVICE | QXD_HOST, QXD_LAYOUT_LEX |
 * QXD_LAYOUT_NATIVE. FP32 computes in single precision with SU(3) links
 * stored as two rows plus the U(1) angle; FP64 uses full links.
 * in/out: caller buffers of one spinor field each; must not overlap.
 * Host buffers (QXD_HOST, lexicographic layout only) are copied through
 * library scratch on the device; that call synchronises the stream.
 * Needs qxd_sw_build (else QXD_ERR_STATE).
 */
int qxd_Dw(qxd_lattice* lat, void* out, const void* in, int flags, void* stream);

/*
 * Even-odd form (Sec. 2.4, Eqs. (29)-(30)). Sites are even when
 * x0 + x1 + x2 + x3 is even. With D = M + H (M site-diagonal, H the hopping
 * term, which connects only opposite parities):
 *   qxd_Dhat:            out_e = D_hat in_e = (M_ee - H_eo M_oo^-1 H_oe) in_e
 *   qxd_eo_prepare:      out_e = b_e - H_eo M_oo^-1 b_o   (source of D_hat x_e = out_e)
 *   qxd_eo_reconstruct:  x_o   = M_oo^-1 (b_o - H_oe x_e) (x_e read from x, x_o written)
 * All buffers are full-lattice spinor fields (flags as for qxd_Dw, device
 * memory only); Dhat and prepare read the even sites of their input and
 * write zeros on the odd sites of their output. Needs qxd_sw_build.
 */
int qxd_Dhat(qxd_lattice* lat, void* out, const void* in, int flags, void* stream);
int qxd_eo_prepare(qxd_lattice* lat, void* out, const void* b, int flags, void* stream);
int qxd_eo_reconstruct(qxd_lattice* lat, void* x, const void* b, int flags, void* stream);

/*
 * Schwarz alternating procedure (the preconditioner of the GCR solver; the
 * paper names it, Sec. 1-2, without giving it): out = SAP(in), ncy cycles of
 * the multiplicative Schwarz method on 4^4 blocks coloured by the parity of
 * the block coordinates (blocks of colour 0, then colour 1); per block the
 * residual in - D out is computed over the whole lattice and out += the
 * result of nmr minimal-residual steps on the even-odd form of D restricted
 * to the block (hops leaving the block dropped). Starts from out = 0.
 * flags: precision and layout as for qxd_Dw, device buffers only. The
 * lattice needs every extent a multiple of 8 and, with C* boundaries,
 * L1 a multiple of 4 with L_k/4 + L1/4 even (else QXD_ERR_ARG). The first
 * FP32 application on a lattice (here or inside qxd_solve) allocates two
 * FP32 work fields (the last block corrections of every site and the block
 * residuals of the even sites: 144 bytes per site), kept with the lattice
 * until qxd_lattice_destroy. In FP32 the residual of a block visit is
 * carried from the previous visits (the block solve's own residual plus the
 * face-crossing hops of the other colour's corrections), which equals
 * in - D out up to rounding.
 */
int qxd_sap(qxd_lattice* lat, void* out, const void* in, int ncy, int nmr, int flags, void* stream);

/* out[i] = SAP(in[i]), i < nrhs: the FP32 Schwarz method of qxd_sap for
 * nrhs right-hand sides of the same operator, solved together: each thread
 * block stages the links of its block once and solves the block for each
 * right-hand side in turn (the operator's links and clover blocks are read
 * from DRAM once for all of them). Each out[i] is bit for bit the result of
 * qxd_sap(lat, out[i], in[i], ncy, nmr, QXD_FP32 | QXD_LAYOUT_NATIVE).
 * out and in: host arrays of nrhs device pointers to FP32 fields in the
 * native layout (qxd_spinor_pack); every out[i] distinct and different from
 * every in[j] (else QXD_ERR_ARG). The library keeps the work fields of nrhs
 * right-hand sides (144 bytes per site each) with the lattice, reallocated
 * when a call needs more, until qxd_lattice_destroy. Errors as for qxd_sap. */
int qxd_sap_multi(qxd_lattice* lat, int nrhs, void* const* out, const void* const* in, int ncy, int nmr,
                  void* stream);

/* ---------------------------------------------------------------------------
 * Solver: D x = b to a true FP64 relative residual |b - D x| / |b| <= tol.
 * Flexible GCR (the paper names GCR with SAP preconditioning, Sec. 1-2, but
 * does not specify either): Krylov directions phi_k = P(r_k) from the
 * preconditioner P, chi_k = A phi_k made orthonormal by Gram-Schmidt with
 * FP64-accumulated inner products, x updated in FP64 at each restart,
 * where the residual is recomputed as b - D x in FP64 (reliable update; also
 * triggered when the inner residual falls below delta times the last true one).
 * system QXD_SOLVE_FULL: GCR on D over the whole lattice.
 * system QXD_SOLVE_EO:   GCR on D_hat for x_e, then x_o by reconstruction.
 * precond QXD_PRECOND_SAP: Schwarz alternating procedure on 4^4 blocks
 * (full system only; inner_prec FP32 or FP64).
 * precond QXD_PRECOND_DFL_SAP: local deflation plus SAP (full system,
 * inner_prec FP32; needs qxd_dfl_subspace, or qxd_dfl_refresh after the
 * operator changed): phi = chi + SAP(r - D chi), chi = P A^-1 P^dag r with the
 * little system A solved by GCR to a relative residual dfl_tol (at most
 * dfl_max_iter steps). For ns = 8, 16 or 32 the GCR runs on the Schur
 * complement of the even blocks (blocks coloured as in SAP), A_ee - A_eo
 * A_oo^-1 A_oe, whose residual and source dfl_tol then refers to, and the
 * odd blocks follow; for other ns on A itself.
 * ------------------------------------------------------------------------- */
#define QXD_PRECOND_NONE 0
#define QXD_PRECOND_SAP 1
#define QXD_PRECOND_DFL_SAP 2
#define QXD_SOLVE_FULL 0
#define QXD_SOLVE_EO 1

typedef struct {
    double tol;       /* target true FP64 relative residual                          */
    int max_iter;     /* limit on Krylov steps over all restarts                     */
    int nkv;          /* Krylov vectors kept before a restart, 1..16                 */
    int precond;      /* QXD_PRECOND_NONE | QXD_PRECOND_SAP                          */
    int system;       /* QXD_SOLVE_FULL | QXD_SOLVE_EO                               */
    int inner_prec;   /* QXD_FP64 | QXD_FP32: Krylov vectors, inner D, preconditioner */
    int sap_ncy;      /* SAP cycles per preconditioner call                          */
    int sap_nmr;      /* minimal-residual steps per block solve                      */
    double delta;     /* reliable update when |r_inner| < delta |r_true| (0: off)    */
    int flags;        /* x and b: QXD_DEVICE | QXD_HOST, QXD_LAYOUT_LEX | _NATIVE     */
    double dfl_tol;   /* QXD_PRECOND_DFL_SAP: relative residual of the little solves */
    int dfl_max_iter; /* QXD_PRECOND_DFL_SAP: step limit of one little solve         */
} qxd_solver_params;

typedef struct {
    int status;            /* QXD_OK, QXD_ERR_NOT_CONVERGED, QXD_ERR_NUMERIC        */
    int iterations;        /* Krylov steps                                          */
    int restarts;          /* true-residual recomputations (reliable updates)       */
    double true_relres;    /* |b - D x| / |b| in FP64 at return                     */
    double time_ms;        /* wall time of the call                                 */
    int dw64_calls;        /* FP64 applications of D (or D_hat)                     */
    int inner_calls;       /* applications of the inner operator                    */
    int little_iters;      /* little-solver steps over all preconditioner calls     */
} qxd_solve_info;

/* Defaults: tol 1e-10, max_iter 2000, nkv 16, no preconditioner, full system,
 * FP64, ncy 5, nmr 5, delta 1e-4, device lexicographic buffers, dfl_tol 1e-2,
 * dfl_max_iter 64. */
void qxd_solver_defaults(qxd_solver_params* p);

/*
 * Solve D x = b (FP64 fields, layout and location by params->flags; x is
 * output only, the initial guess is zero). info may be NULL. Returns QXD_OK,
 * QXD_ERR_NOT_CONVERGED (x and info still written), QXD_ERR_NUMERIC, or an
 * argument/state error. Work vectors are allocated on the first call and
 * kept with the lattice. Synchronises the stream.
 */
int qxd_solve(qxd_lattice* lat, void* x, const void* b, const qxd_solver_params* params,
              qxd_solve_info* info, void* stream);

/*
 * out = D in, like qxd_Dw with device buffers in the lexicographic layout,
 * but without allocating device memory. The paper has no counterpart: this
 * entry point exists for callers that cannot let a library allocate during a
 * call (frameworks that hand out all device memory from their own pool,
 * latency-bound paths where a cudaMalloc and the device synchronisation it
 * may imply are not acceptable, jobs that hold nearly all device memory).
 * The layout conversion goes through a fixed scratch array in the library's
 * device memory (2 x 12 MiB) instead of the scratch qxd_Dw allocates.
 * - flags: QXD_FP64 or QXD_FP32 only (device buffers, lexicographic layout).
 * - Lattices above 65536 simulated sites are rejected with QXD_ERR_ARG.
 * - The first call on a device is its set-up: it looks up the scratch
 *   array's device address (cudaGetSymbolAddress) and keeps it. Under CUDA's
 *   lazy module loading (the default) that lookup is also what loads the
 *   array onto the device, so the first call reserves the 24 MiB, and it
 *   can fail with QXD_ERR_CUDA (out of memory) on a nearly full device.
 *   Make the first call at set-up, while memory is available and before any
 *   stream capture; the array then stays reserved until the process exits,
 *   and later calls allocate nothing.
 * - Every call on a device shares the one scratch array, which keeps the
 *   last call's contents (each call overwrites all it reads): calls that
 *   overlap on the GPU (other streams, other threads) race and must be
 *   serialised by the caller.
 */
int qxd_Dw_noalloc(qxd_lattice* lat, void* out, const void* in, int flags, void* stream);

/*
 * out[i] = D_i in[i] for i < n in one kernel launch, where D_i is the operator
 * of lats[i] (lattices or views, possibly of different sizes; the same
 * lattice may appear many times). Native-layout device buffers, precision
 * QXD_FP64 or QXD_FP32 in flags. Right-hand sides of one operator share each
 * site's link, angle and clover loads (rhs_per_site of them per site: 1, 2,
 * 4 or 8, or 0 to let the library time the choices on the first batch of a
 * given size class and keep the fastest). Same numbers as qxd_Dw per
 * right-hand side. The paper applies one operator at a time (Sec. 2.3); this
 * is the batched form of the same operator.
 */
int qxd_Dw_batch(int n, qxd_lattice* const* lats, void* const* out, const void* const* in, int flags,
                 int rhs_per_site, void* stream);

/* ---------------------------------------------------------------------------
 * Batched solve engine (continuous batching of independent solves).
 * Every submitted request is a solve D x = b with its own operator (lattice
 * or view; views let requests with different m0, qhat share one resident
 * gauge field). qxd_engine_step advances every active request by one flexible
 * GCR step (as qxd_solve with system QXD_SOLVE_FULL, inner_prec QXD_FP32),
 * with one kernel launch per SAP half-cycle, one batched D and one launch
 * per vector operation for all active requests together; it then retires
 * finished requests and admits queued ones while the device memory of the
 * active requests stays within hbm_budget_bytes (a request larger than the
 * budget runs alone) and their number within max_active. Each request is
 * charged its largest footprint at admission: four FP64 fields, one FP32
 * residual and params->nkv FP32 Krylov pairs, 24 V (4 * 8 + (1 + 2 nkv) * 4)
 * bytes on a lattice of V sites. Work vectors come from the engine's caching
 * device allocator, which keeps the bytes it holds (in use plus cached)
 * within the budget by releasing cached blocks before it allocates more. A
 * request whose work vectors cannot be allocated fails alone (its status is
 * the error); the other requests go on. A request's result does not depend
 * on the other requests in the batch (same kernels, grids and reduction
 * orders as alone).
 * Buffers x and b (FP64, device; lexicographic unless params->flags has
 * QXD_LAYOUT_NATIVE) and the operator must stay valid until the request is
 * done (qxd_engine_poll). The paper solves one system at a time; this
 * engine is a design choice of this library.
 * ------------------------------------------------------------------------- */
typedef struct qxd_engine qxd_engine;

int qxd_engine_create(qxd_engine** out, size_t hbm_budget_bytes, int max_active, void* stream);
int qxd_engine_destroy(qxd_engine* e);
/* queue a request; id receives its handle */
int qxd_engine_submit(qxd_engine* e, qxd_lattice* op, void* x, const void* b, const qxd_solver_params* params,
                      long long* id);
/* one step for all active requests; counts after the step (n_done: retired by this step) */
int qxd_engine_step(qxd_engine* e, int* n_active, int* n_pending, int* n_done);
/* request status; done = 1 once x is written (info.status: QXD_OK, QXD_ERR_NOT_CONVERGED, ...) */
int qxd_engine_poll(qxd_engine* e, long long id, qxd_solve_info* info, int* done);
/* drop the record of a finished request */
int qxd_engine_forget(qxd_engine* e, long long id);
/* step until no request is active or queued */
int qxd_engine_run(qxd_engine* e);
/* device bytes of active requests, bytes held by the allocator, steps so far */
int qxd_engine_stats(const qxd_engine* e, size_t* bytes_in_use, size_t* bytes_held, long long* steps);
/* CUDA graphs of the batched Schwarz launch sets (lattices under 2^20 sites):
 * captures made and replays of a captured graph so far. A set is captured on
 * its first use and replayed while the job table, job count, CTA count, ncy
 * and nmr stay the same. Either pointer may be NULL. */
int qxd_engine_graph_stats(const qxd_engine* e, long long* captures, long long* replays);

/* ---------------------------------------------------------------------------
 * Serving runtime: lanes of the solve engine by lattice size. The paper has
 * no counterpart. Lane i takes the requests on lattices of fewer than
 * lane_sites[i] simulated sites (not taken by an earlier lane; the last lane
 * takes the rest) and has its own CUDA stream, its own engine
 * (qxd_engine_create with lane_budget[i] bytes and max_active) and its own
 * host worker thread, which admits, steps and retires that lane's requests
 * without waiting for the other lanes: a request on a small lattice does not
 * wait for the steps of large ones. The lanes' streams have graded CUDA
 * priorities, the lane of the smallest lattices the highest, so that the GPU
 * schedules a small request's thread blocks ahead of those still queued for
 * large lattices. A request's result is the engine's (the
 * same, bit for bit, as the request solved alone). submit, poll, forget and
 * stats may be called from any thread. Buffers x and b and the operator must
 * stay valid and unchanged until the request is done. qxd_server_destroy
 * waits until every submitted request is done, then stops the workers.
 * ------------------------------------------------------------------------- */
typedef struct qxd_server qxd_server;

/* nlanes >= 1; lane_sites: nlanes - 1 positive increasing bounds (may be
 * NULL if nlanes = 1); lane_budget: nlanes byte budgets; max_active >= 1 */
int qxd_server_create(qxd_server** out, int nlanes, const long long* lane_sites, const size_t* lane_budget,
                      int max_active);
int qxd_server_destroy(qxd_server* s);
/* queue a request (checked as by qxd_engine_submit); id receives its handle */
int qxd_server_submit(qxd_server* s, qxd_lattice* op, void* x, const void* b, const qxd_solver_params* params,
                      long long* id);
/* done = 1 once x is written; info.status as for qxd_engine_poll */
int qxd_server_poll(qxd_server* s, long long id, qxd_solve_info* info, int* done);
/* drop the record of a finished request */
int qxd_server_forget(qxd_server* s, long long id);
/* requests submitted to and completed by lane `lane`, and its engine steps */
int qxd_server_stats(const qxd_server* s, int lane, long long* submitted, long long* completed, long long* steps);

/* ---------------------------------------------------------------------------
 * Pseudofermion action of the RHMC (Sec. 2.4):
 *   S_pf = -1/2 ln|Det D_oo| + sum_k phi_k^dag P_k phi_k,
 *   P_k  = prod_j (D_hat^dag D_hat + nu_j^2) / (D_hat^dag D_hat + mu_j^2),
 * with D_hat = D_ee - D_eo D_oo^-1 D_oe the even-odd operator and phi_k
 * fields on the even sites. D_hat^dag = gamma5 D_hat gamma5 (gamma5
 * hermiticity of D). All of this is FP64.
 * ------------------------------------------------------------------------- */
#define QXD_SITES_EVEN 0
#define QXD_SITES_ODD 1
#define QXD_SITES_ALL 2

/*
 * *out = sum over the sites x of the selected parity of ln|det M(x)|, with
 * M(x) the 12x12 site-diagonal block of D (4 + m0 plus the SW term, the two
 * 6x6 chirality blocks of qxd_sw_build). sites = QXD_SITES_ODD gives
 * ln|Det D_oo|, the exact term of S_pf (Sec. 2.4: D_oo is diagonal in the
 * lattice index, so its determinant is computed exactly). Each block's
 * determinant is taken by Gaussian elimination with partial pivoting; the
 * sum is reduced in a fixed order (same result on every call). Returns
 * QXD_ERR_SW_SINGULAR if a block is exactly singular or the result is not
 * finite, QXD_ERR_STATE before qxd_sw_build. Synchronises the lattice's stream.
 */
int qxd_sw_logdet(qxd_lattice* lat, int sites, double* out);

typedef struct {
    double tol;       /* stop when each shift's residual is <= tol |b|             */
    int max_iter;     /* limit on CG steps (all passes together)                   */
    int flags;        /* x and b: QXD_DEVICE | QXD_HOST, QXD_LAYOUT_LEX | _NATIVE  */
    int prec;         /* QXD_FP64: FP64 throughout. QXD_FP32: the operator in FP32 */
                      /* (vectors and scalars FP64), the base residual replaced by */
                      /* the true FP64 residual whenever it fell by delta, then    */
                      /* each shift checked in FP64 and refined by FP32-operator   */
                      /* CG on its residual until it meets tol                     */
    double delta;     /* QXD_FP32: reliable-update factor, 0 < delta < 1           */
} qxd_mscg_params;

typedef struct {
    int status;             /* QXD_OK, QXD_ERR_NOT_CONVERGED, QXD_ERR_NUMERIC       */
    int iterations;         /* CG steps                                             */
    double true_relres;     /* max over shifts of |b - (A + s_j) x_j| / |b| (FP64)   */
    double action;          /* qxd_rational_apply: Re <phi, P phi>; else 0           */
    double time_ms;         /* wall time of the call                                */
    int dhat_calls;         /* applications of D_hat (A costs two)                  */
} qxd_mscg_info;

/* Defaults: tol 1e-10, max_iter 10000, device lexicographic buffers, FP64,
 * delta 0.01. */
void qxd_mscg_defaults(qxd_mscg_params* p);

/*
 * Multi-shift CG: x[j] = (D_hat^dag D_hat + sigma[j])^-1 b for j < nshift
 * (1 <= nshift <= 16, sigma[j] >= 0, any order), all from one Krylov space
 * (the paper solves its rational factors with multi-shift CG, Sec. 2.4 and
 * App. A, without giving the method; this is the standard shifted CG, whose
 * residuals of all shifts stay collinear with the base residual).
 * b and x[j]: full-lattice FP64 spinor fields (layout and location by
 * params->flags); only the even sites of b are read, the odd sites of each
 * x[j] are set to zero. The smallest shift is the base system; a shift stops
 * updating once its residual is below tol |b|. At the end each shift's
 * true residual is recomputed in FP64 (relres[j] if relres is not NULL;
 * the largest in info->true_relres). Returns QXD_ERR_NOT_CONVERGED (x and
 * info still written) when a true residual exceeds tol. Work vectors are
 * allocated on the first call and kept with the lattice. Synchronises.
 */
int qxd_mscg(qxd_lattice* lat, int nshift, const double* sigma, void* const* x, const void* b,
             const qxd_mscg_params* params, qxd_mscg_info* info, double* relres, void* stream);

/*
 * out = P phi with P = prod_{j<n} (A + nu[j]^2) / (A + mu[j]^2),
 * A = D_hat^dag D_hat (one frequency-splitting factor P_k of Sec. 2.4, or a
 * Hasenbusch ratio), computed as phi + sum_j rho_j (A + mu[j]^2)^-1 phi with
 * the partial-fraction residues rho_j = prod_l (nu_l^2 - mu_j^2) /
 * prod_{l != j} (mu_l^2 - mu_j^2) and one qxd_mscg over the shifts mu[j]^2.
 * info->action = Re <phi, P phi> (the factor's term of S_pf). The mu[j]
 * must be distinct and 1 <= n <= 16. Fields and flags as qxd_mscg (odd sites
 * of out set to zero). The tolerance applies to each shifted solve.
 */
int qxd_rational_apply(qxd_lattice* lat, int n, const double* nu, const double* mu, void* out, const void* phi,
                       const qxd_mscg_params* params, qxd_mscg_info* info, void* stream);

/* ---------------------------------------------------------------------------
 * Gauge observables and the Wilson flow (App. A; the paper defines its
 * action densities and topological charge at positive flow time of the
 * Wilson flow of Luscher (2010), Sec. 3). FP64.
 * ------------------------------------------------------------------------- */

/*
 * out[0] = E_SU(3) = -1/(2V) sum_x sum_{mu,nu} tr{F_munu(x) F_munu(x)}
 * out[1] = E_U(1)  = -1/(2V) sum_x sum_{mu,nu} A_munu(x)^2
 * out[2] = Q_top   = 1/(32 pi^2) sum_x sum eps_{mu nu rho sigma} tr{F_munu F_rhosigma}
 * with the clover tensors of the SW term: F = (Q_munu - Q_numu)/8 and
 * A_munu = i/(4 q_el) Im{four U(1) plaquettes} (Sec. 2.3). Both tensors are
 * anti-Hermitian, so the minus signs (not printed in the paper) make the E
 * non-negative. Sums run over the physical lattice of volume V: with C*
 * boundaries the mirror half holds the conjugate field with the same
 * densities, so E is the mean over the simulated lattice and Q half its sum.
 * q_el > 0 is the elementary charge of the U(1) normalisation (1/6 with C*
 * boundaries in the paper, Sec. 2.2). Works on a lattice or a view (the
 * gauge field of the owner). Synchronises the lattice's stream.
 */
int qxd_gauge_observables(qxd_lattice* lat, double q_el, double* out);

/*
 * Flows the lattice's gauge field in place by nsteps steps of size eps
 * (flow time t = nsteps eps): SU(3) by dV/dt = Z(V) V with
 * Z(x,mu) = -1/2 (W - W^dag) + 1/6 tr(W - W^dag), W = U(x,mu) times the sum
 * of the six staples (Luscher's Wilson flow), integrated with his
 * third-order Runge-Kutta scheme; the U(1) angles by the same scheme with
 * dA(x,mu)/dt = -sum_{nu != mu} [sin theta_munu(x) - sin theta_munu(x-nu)]
 * (compact plaquette action), kept in [-pi, pi). With C* boundaries only the
 * physical links are integrated and the mirror links are set to their
 * complex conjugates (-A), so the field stays admissible exactly.
 * Afterwards the FP32 copies and the field tensors are refreshed, and every
 * clover term built from the old field (this lattice's and its views') is
 * stale: qxd_Dw and the solvers return QXD_ERR_STATE until qxd_sw_build.
 * Views cannot flow (QXD_ERR_STATE): flow the lattice that owns the field.
 * Allocates its work fields (about 0.9 KB per site) for the call; if that
 * fails (QXD_ERR_OOM) the field is unchanged. A failure after the first step
 * started leaves the field unusable (QXD_ERR_STATE until qxd_set_gauge).
 * Synchronises the lattice's stream.
 */
int qxd_wflow(qxd_lattice* lat, double eps, int nsteps);

/* ---------------------------------------------------------------------------
 * Local deflation (openQ*D's deflation-accelerated solver, named in Sec. 1
 * and Table 2 without details; Luscher's local deflation). The deflation
 * subspace S is spanned by block-local fields phi_{b,k}, k < ns, on the
 * 4^4 blocks of the Schwarz method: ns global fields restricted to each
 * block and orthonormalised there in order (Gram-Schmidt). The little
 * operator A_{(b,k),(b',l)} = <phi_{b,k}, D phi_{b',l}> couples each block to
 * itself and its 8 neighbours. Subspace and little operator belong to the
 * lattice (or view) they were built on; FP32 storage. The lattice must admit
 * the SAP blocks (as qxd_sap).
 * ------------------------------------------------------------------------- */

/*
 * Builds S from ns seeded Gaussian fields, each passed niter times through
 * the Schwarz method (ncy cycles, 4 MR steps: inverse iteration towards the
 * low modes) with a block orthonormalisation after every pass, then the
 * little operator of the current D. 1 <= ns <= 64. Needs qxd_sw_build.
 * Returns QXD_ERR_NUMERIC if a block's fields became linearly dependent.
 * Memory: ns * 96 + 600 bytes per site, plus the little operator
 * (9 ns^2 * 8 bytes per block). Synchronises the lattice's stream.
 */
int qxd_dfl_subspace(qxd_lattice* lat, int ns, int niter, int ncy, unsigned long long seed);

/*
 * Builds S from ns given fields psi[k] (FP64 device fields, lexicographic
 * layout; they are block-orthonormalised, not modified) and the little
 * operator of the current D. Errors as qxd_dfl_subspace.
 */
int qxd_dfl_set_basis(qxd_lattice* lat, int ns, const void* const* psi);

/*
 * Recomputes the little operator for the lattice's current operator (after
 * qxd_set_params + qxd_sw_build with a new mass or charge, or a new gauge
 * field) keeping the subspace. QXD_ERR_STATE without a subspace or clover.
 */
int qxd_dfl_refresh(qxd_lattice* lat);

/*
 * Copies the little operator to host memory: A_out[((b * 9 + j) * ns + k) * ns
 * + l] (complex, re/im pairs of doubles) = <phi_{b,k}, D phi_{n_j(b),l}>,
 * n_0(b) = b, n_{1+2mu}(b) = b + mu, n_{2+2mu}(b) = b - mu, blocks numbered
 * lexicographically in block coordinates (b3 fastest). A_out may be NULL to
 * query *ns_out and *nblk_out only.
 */
int qxd_dfl_little(qxd_lattice* lat, double* A_out, int* ns_out, int* nblk_out);

/* Writes sum_b phi_{b,k} (FP64 device field, lexicographic layout) to out. */
int qxd_dfl_basis(qxd_lattice* lat, int k, void* out);

/* Bytes of one spinor field in the native layout for precision `prec`. */
size_t qxd_spinor_bytes(const qxd_lattice* lat, int prec);

/* Lexicographic (device) -> native (device) and back, precision `prec`. */
int qxd_spinor_pack(qxd_lattice* lat, void* native_out, const void* lex_in, int prec, void* stream);
int qxd_spinor_unpack(qxd_lattice* lat, void* lex_out, const void* native_in, int prec, void* stream);

/* ---------------------------------------------------------------------------
 * Launch-shape autotuning of D (qxd_Dw and every internal full-lattice D, as
 * in the solvers). The paper has no counterpart. A shape is the hop order
 * (software-pipelined: the loads of the next hop issued before the
 * arithmetic of this one, 128 registers, FP32 only; or plain), the threads
 * per block (64 or 128) and the sweep window (rows of x2 per chunk of the
 * tiled site order, a divisor of L2). With the autotuner on (the default),
 * the first D on a lattice shape (extents, C* mask, precision, qhat != 0)
 * times every candidate shape on that call's input (three launches each,
 * CUDA events, synchronising the stream once) and keeps the fastest for the
 * shape, process-wide; with it off, the first call takes the default shape
 * (pipelined in FP32, 128 threads, the largest window up to 64K sites). The
 * output of every call comes from the chosen shape; all shapes compute the
 * same per-site sums in the same order. A first call inside a stream
 * capture must not tune: pin the shape (qxd_dw_set_shape) or make a first
 * call before the capture.
 * ------------------------------------------------------------------------- */
/* enable = 0 or 1; returns the previous setting */
int qxd_set_autotune(int enable);
/* the shape chosen for lat's lattice shape and precision; ms = the time of
 * one application when tuned (0 otherwise). QXD_ERR_STATE if none yet. Any
 * output pointer may be NULL. */
int qxd_dw_shape(const qxd_lattice* lat, int prec, int* pipelined, int* threads, int* rows, float* ms);
/* pin a shape for lat's lattice shape and precision (QXD_ERR_ARG: pipelined
 * not 0/1 or set with FP64, threads not 64/128, rows not dividing L2) */
int qxd_dw_set_shape(const qxd_lattice* lat, int prec, int pipelined, int threads, int rows);
/* every choice made so far (D shapes and the batched D's right-hand sides
 * per site), one per line, as text in buf (truncated to len - 1 characters,
 * NUL-terminated); *needed = the full length + 1. buf may be NULL. */
int qxd_tune_report(char* buf, size_t len, size_t* needed);

/* ---------------------------------------------------------------------------
 * Measurement aid: arithmetic throughput of the current GPU, the denominator
 * of the rooflines of the kernels bound by FP64 or FP32 arithmetic (the FP64
 * operator, the multi-shift CG and the Wilson flow; the FP32 Schwarz block
 * solves). The paper has no counterpart.
 * *flop_per_s = the fused multiply-add rate (2 flops per FMA) of a kernel in
 * which every thread runs 16 independent chains of `iters` FMAs, 8 blocks of
 * 256 threads per SM; best of three timed launches (CUDA events) after one
 * untimed launch, on `stream` (NULL: the default stream). Synchronises.
 * kind: QXD_PROBE_FMA64 (FP64 fma), QXD_PROBE_FMA32 (FP32 fmaf),
 * QXD_PROBE_FMA32X2 (paired FP32 FMA on float2, two per instruction).
 * QXD_ERR_ARG for an unknown kind, iters < 1 or a NULL result.
 * ------------------------------------------------------------------------- */
#define QXD_PROBE_FMA64 0
#define QXD_PROBE_FMA32 1
#define QXD_PROBE_FMA32X2 2
int qxd_fma_rate(int kind, int iters, double* flop_per_s, void* stream);

/* Message of the calling thread's last failure ("" if none). */
const char* qxd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QXD_H */
