// Internal definitions of the qxd library: lattice object, geometry of the
// extended lattice with shifted C* boundaries, native device layouts and
// complex arithmetic shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "qxd.h"

namespace qxd {

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define QXD_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return ::qxd::cuda_fail(e_, #call); \
    } while (0)

#define QXD_LAUNCHED(what)                               \
    do {                                                 \
        cudaError_t e_ = cudaGetLastError();             \
        if (e_ != cudaSuccess) return ::qxd::cuda_fail(e_, what); \
    } while (0)

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
// Simulated lattice N = (T, N1, L2, L3); N1 = 2 L1 with C* in direction 1.
// A C* direction k = 2, 3 has the shifted boundary of Eq. (11): the site
// beyond x_k = L_k - 1 is (x1 + L1 mod 2 L1, x_k = 0) and vice versa.
//
// Native site order: even sites (x0+x1+x2+x3 even) first, then odd; inside a
// parity, lexicographic order (x3 fastest). Because N3 is even, the two sites
// of lexicographic index 2h and 2h + 1 have opposite parities, so a site of
// lexicographic index i and parity p has native index p * Vh + i / 2.
//
// Kernels that sweep the whole lattice visit sites in a tiled order: the x2
// extent is cut into chunks of R rows, and the chunk index is the slowest
// coordinate of the sweep (chunk, x0, x1, row, x3). Neighbours in x0 are then
// N1 * R * N3 sites apart in the sweep instead of N1 * N2 * N3, which keeps
// their reuse inside L2.
struct Geom {
    int N0, N1, N2, N3;
    int L1;      // physical x1 extent (shift of the C* boundary)
    int cs2, cs3;  // 1 if direction 2 / 3 has the shifted C* boundary
    int V, Vh;
    int R;       // x2 rows per sweep chunk (divides N2)
};

__host__ __device__ __forceinline__ int lex_index(const Geom& g, int x0, int x1, int x2, int x3) {
    return ((x0 * g.N1 + x1) * g.N2 + x2) * g.N3 + x3;
}

// native (even-odd) index of a site from its lexicographic index and parity
__host__ __device__ __forceinline__ int native_index(const Geom& g, int lex, int parity) {
    return parity * g.Vh + (lex >> 1);
}

// sweep position -> coordinates (tiled order, see above)
__host__ __device__ __forceinline__ void sweep_coords(const Geom& g, int tau, int& x0, int& x1, int& x2, int& x3) {
    const int rowlen = g.R * g.N3;
    int within = tau % rowlen;
    int rest = tau / rowlen;
    x1 = rest % g.N1;
    rest /= g.N1;
    x0 = rest % g.N0;
    int chunk = rest / g.N0;
    int r = within / g.N3;
    x3 = within - r * g.N3;
    x2 = chunk * g.R + r;
}

// the same tiled order restricted to the x0 planes [x0b, x0b + nx0) (tau <
// nx0 N1 N2 N3); with x0b = 0 and nx0 = N0 it is sweep_coords
__host__ __device__ __forceinline__ void sweep_coords_slab(const Geom& g, int x0b, int nx0, int tau, int& x0, int& x1,
                                                           int& x2, int& x3) {
    const int rowlen = g.R * g.N3;
    int within = tau % rowlen;
    int rest = tau / rowlen;
    x1 = rest % g.N1;
    rest /= g.N1;
    x0 = x0b + rest % nx0;
    int chunk = rest / nx0;
    int r = within / g.N3;
    x3 = within - r * g.N3;
    x2 = chunk * g.R + r;
}

// sweep over the sites of one parity p (tau < Vh), same tiled order
__host__ __device__ __forceinline__ void sweep_coords_parity(const Geom& g, int p, int tau, int& x0, int& x1,
                                                             int& x2, int& x3) {
    const int half = g.N3 >> 1;
    const int rowlen = g.R * half;
    int within = tau % rowlen;
    int rest = tau / rowlen;
    x1 = rest % g.N1;
    rest /= g.N1;
    x0 = rest % g.N0;
    int chunk = rest / g.N0;
    int r = within / half;
    int j = within - r * half;
    x2 = chunk * g.R + r;
    x3 = 2 * j + ((x0 + x1 + x2 + p) & 1);
}

// coordinates of the site with native index s
__host__ __device__ __forceinline__ void native_coords(const Geom& g, int s, int& x0, int& x1, int& x2, int& x3) {
    int p = s >= g.Vh;
    int h = s - p * g.Vh;
    int lex2 = 2 * h;  // lexicographic index with x3 rounded down to even
    int x3e = lex2 % g.N3;
    int rest = lex2 / g.N3;
    x2 = rest % g.N2;
    rest /= g.N2;
    x1 = rest % g.N1;
    x0 = rest / g.N1;
    x3 = x3e + ((x0 + x1 + x2 + x3e + p) & 1);
}

// neighbour coordinates x + mu (dir = +1) or x - mu (dir = -1), Eq. (10)-(11)
template <int MU, int DIR>
__host__ __device__ __forceinline__ int neighbour_lex(const Geom& g, int x0, int x1, int x2, int x3) {
    if (MU == 0) {
        if (DIR > 0) x0 = (x0 + 1 == g.N0) ? 0 : x0 + 1;
        else x0 = (x0 == 0) ? g.N0 - 1 : x0 - 1;
    } else if (MU == 1) {
        if (DIR > 0) x1 = (x1 + 1 == g.N1) ? 0 : x1 + 1;
        else x1 = (x1 == 0) ? g.N1 - 1 : x1 - 1;
    } else {
        int& xk = (MU == 2) ? x2 : x3;
        const int Lk = (MU == 2) ? g.N2 : g.N3;
        const int cs = (MU == 2) ? g.cs2 : g.cs3;
        bool crossed;
        if (DIR > 0) {
            crossed = (xk + 1 == Lk);
            xk = crossed ? 0 : xk + 1;
        } else {
            crossed = (xk == 0);
            xk = crossed ? Lk - 1 : xk - 1;
        }
        if (crossed && cs) {
            x1 += g.L1;
            if (x1 >= g.N1) x1 -= g.N1;
        }
    }
    return lex_index(g, x0, x1, x2, x3);
}

// ---------------------------------------------------------------------------
// native layouts (structure of arrays over native site index s, V entries)
// ---------------------------------------------------------------------------
// spinor FP32 : float4  psi[6][V]   float f = (3*spin + colour)*2 + re/im,
//                                   vector k holds f = 4k .. 4k+3
// spinor FP64 : double2 psi[12][V]  vector k holds component k = 3*spin+colour
// links  FP32 : float4  U[4][3][V]  rows 0 and 1 of U(x,mu): 12 floats
//                                   (u00 u01 | u02 u10 | u11 u12), row 2 is
//                                   conj(row0 x row1) (SU(3))
// links  FP64 : double2 U[4][9][V]  full 3x3, row major
// angle  FP32 : float4  A[V]        A(x, mu), mu = 0..3
// angle  FP64 : double  A[4][V]
// phase  FP64 : double2 Z[4][V]    z = exp(i A) as (cos A, sin A); per operator
//                                   also Zq[4][V] = z^qhat (built with the clover)
// clover FP32 : float4  C[18][V]    two Hermitian 6x6 blocks (spins {0,1},
//                                   then {2,3}), 36 floats each: 6 real
//                                   diagonals, then the 15 complex entries
//                                   below the diagonal, row major
//                                   ((1,0),(2,0),(2,1),(3,0),...,(5,4))
// clover FP64 : double  C[72][V]    same 72 reals
// field tensor: double  F[60][V]    per plane (01,02,03,12,13,23): the SU(3)
//                                   anti-Hermitian 3x3 F_hat as 9 reals
//                                   (Im d0, Im d1, Im d2, re/im of the upper
//                                   entries (0,1),(0,2),(1,2)), then
//                                   Im sum of the 4 U(1) plaquettes
constexpr int SPINOR_F4 = 6;
constexpr int SPINOR_D2 = 12;
constexpr int CLOVER_F4 = 18;
constexpr int CLOVER_REALS = 72;
constexpr int FTENS_REALS = 60;

// ---------------------------------------------------------------------------
// complex arithmetic
// ---------------------------------------------------------------------------
template <typename R>
struct cplx {
    R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cplx<R> mk(R a, R b) { return cplx<R>{a, b}; }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator-(cplx<R> a) { return {-a.re, -a.im}; }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator*(cplx<R> a, cplx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator*(R s, cplx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> conj(cplx<R> a) { return {a.re, -a.im}; }
// a * conj(b)
template <typename R>
__host__ __device__ __forceinline__ cplx<R> mulc(cplx<R> a, cplx<R> b) {
    return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
// conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ cplx<R> cmul(cplx<R> a, cplx<R> b) {
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// i * a, -i * a
template <typename R>
__host__ __device__ __forceinline__ cplx<R> times_i(cplx<R> a) { return {-a.im, a.re}; }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> times_mi(cplx<R> a) { return {a.im, -a.re}; }

// ---------------------------------------------------------------------------
// the lattice object
// ---------------------------------------------------------------------------
struct SolverWork;
struct MscgWork;
struct DflWork;
struct HostPipe;
}  // namespace qxd

struct qxd_lattice {
    qxd::Geom g;
    int T, L1, L2, L3;
    unsigned cstar_mask;
    cudaStream_t stream;
    int device;

    // gauge field
    double2* U64 = nullptr;  // [4][9][V]
    float4* U32 = nullptr;   // [4][3][V]
    double* A64 = nullptr;   // [4][V]
    double2* Z64 = nullptr;  // [4][V] exp(i A)
    float4* A32 = nullptr;   // [V]
    double* ftens = nullptr; // [60][V]
    bool has_gauge = false;

    // parameters and clover term
    double m0 = 0, csw = 0, cswqed = 0;
    int qhat = 0;
    bool has_params = false;
    double2* Zq64 = nullptr;   // [4][V] z^qhat for this operator's qhat (FP64 kernels)
    double* C64 = nullptr;     // [72][V]
    float4* C32 = nullptr;     // [18][V]
    double* Cinv64 = nullptr;  // [72][V]
    float4* Cinv32 = nullptr;  // [18][V]
    bool has_clover = false;

    // scratch
    int* d_status = nullptr;   // small device status words
    void* scratch_in = nullptr;   // native spinor FP64-sized
    void* scratch_out = nullptr;  // native spinor FP64-sized
    void* scratch_lex = nullptr;  // lexicographic FP64 spinor
    float4* sap_r = nullptr;      // FP32 work fields of the Schwarz method (delta, rho; first FP32 SAP application)
    float4* sap_multi = nullptr;  // work fields of qxd_sap_multi, sap_multi_n right-hand sides
    int sap_multi_n = 0;
    qxd::HostPipe* hostpipe = nullptr;  // streams and events of the pipelined host-buffer D

    qxd::SolverWork* solver = nullptr;  // Krylov work vectors (first solve)
    qxd::MscgWork* mscg = nullptr;      // multi-shift CG work vectors (first use)
    qxd::DflWork* dfl = nullptr;        // deflation subspace and little operator
    unsigned op_version = 0;            // bumped by every successful qxd_sw_build

    // views: a view shares the gauge field of its parent and owns its own
    // parameters, clover term, scratch and solver work
    qxd_lattice* parent = nullptr;
    int nviews = 0;                    // live views of this lattice
    unsigned gauge_version = 0;        // bumped by every successful set_gauge
    unsigned built_gauge_version = 0;  // gauge version the clover was built from
};

namespace qxd {
// launchers implemented in the .cu files
int launch_gauge_ingest(qxd_lattice* lat, const double* su3, const double* ang, int extended,
                        int* d_bad);
int launch_field_tensor(qxd_lattice* lat);
int launch_clover_build(qxd_lattice* lat, int* d_bad);
int launch_dirac(qxd_lattice* lat, void* out, const void* in, int prec, cudaStream_t st);
int launch_pack(qxd_lattice* lat, void* nat, const void* lex, int prec, cudaStream_t st);
int launch_unpack(qxd_lattice* lat, void* lex, const void* nat, int prec, cudaStream_t st);
// page-locked host buffers: device address of p (false for pageable memory)
bool host_device_view(const void* p, void** dev);
int launch_pack_from_host(qxd_lattice* lat, void* nat, const void* lex_dev, int prec, cudaStream_t st);
int launch_unpack_to_host(qxd_lattice* lat, void* lex_dev, const void* nat, int prec, cudaStream_t st);
// out = D in on the x0 planes [x0b, x0b + nx0) only (native fields; the
// launch shape of the full-lattice D)
int launch_dirac_planes(qxd_lattice* lat, void* out, const void* in, int prec, int x0b, int nx0, cudaStream_t st);
// out = D in for page-locked host buffers in the lexicographic layout,
// pipelined over slabs of x0 planes (qxd_Dw's host path); QXD_ERR_ARG if the
// lattice is too short in x0 to cut into slabs (then use the plain path)
int dw_host_pipelined(qxd_lattice* lat, void* out_dev, const void* in_dev, int prec, cudaStream_t st);
// slabs of the pipelined host path for x0 extent N0 (< 3: no pipeline)
int pick_slabs(int N0);
void release_hostio(qxd_lattice* lat);
int ensure_scratch(qxd_lattice* lat);
// the lattice that owns the gauge field (the lattice itself unless a view)
inline qxd_lattice* gauge_owner(qxd_lattice* lat) { return lat->parent ? lat->parent : lat; }
inline const qxd_lattice* gauge_owner(const qxd_lattice* lat) { return lat->parent ? lat->parent : lat; }
// clover built and still matching the current gauge field
inline bool clover_ready(const qxd_lattice* lat) {
    return lat->has_clover && lat->built_gauge_version == gauge_owner(lat)->gauge_version;
}
void release_solver(qxd_lattice* lat);
void release_mscg(qxd_lattice* lat);
void release_dfl(qxd_lattice* lat);
}  // namespace qxd
