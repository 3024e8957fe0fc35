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
 *  - Threads: one lattice must not be used by two host threads at once.
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

/* Bytes of one spinor field in the native layout for precision `prec`. */
size_t qxd_spinor_bytes(const qxd_lattice* lat, int prec);

/* Lexicographic (device) -> native (device) and back, precision `prec`. */
int qxd_spinor_pack(qxd_lattice* lat, void* native_out, const void* lex_in, int prec, void* stream);
int qxd_spinor_unpack(qxd_lattice* lat, void* lex_out, const void* native_in, int prec, void* stream);

/* Message of the calling thread's last failure ("" if none). */
const char* qxd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QXD_H */
