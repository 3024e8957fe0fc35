// Full-lattice application of D (Sec. 2.3, Eqs. (16)-(21)):
//   (D psi)(x) = M(x) psi(x) - 1/2 sum_mu [ (1 - g_mu) W(x,mu) psi(x+mu)
//                                  + (1 + g_mu) W(x-mu,mu)^+ psi(x-mu) ],
//   W(x,mu) = U(x,mu) z(x,mu)^qhat,  M(x) = (4 + m0) + dDsw(x),
// which is Eqs. (18)-(20) expanded (the diagonal 4 of Dw moved into M).
// One thread per site; spin projection to half spinors before the colour
// multiplication (the projectors commute with W). FP32: links as two rows
// plus the U(1) angle, hops software-pipelined (k_dirac32); FP64: full links.
// Both parities in one sweep, in the tiled order of sweep_coords so
// neighbour data is reused from L2.
//
// Chiral basis, psi = (psi0, psi1 | psi2, psi3):
//   (1 -+ g0): h = (psi0 +- psi2, psi1 +- psi3),   lower = (+-h0, +-h1)
//   (1 -+ g1): h = (psi0 +- i psi3, psi1 +- i psi2), lower = (-+i h1, -+i h0)
//   (1 -+ g2): h = (psi0 +- psi3, psi1 -+ psi2),   lower = (-+h1, +-h0)
//   (1 -+ g3): h = (psi0 +- i psi2, psi1 -+ i psi3), lower = (-+i h0, +-i h1)
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "dirac_common.cuh"
#include "tune.cuh"

namespace qxd {

namespace {

// Both kernels apply D on the x0 planes [x0b, x0b + nx0) (all of them for
// x0b = 0, nx0 = N0), nsites = nx0 N1 N2 N3 threads.
// FP32: the pipelined hop order of hops_pipelined (128 registers)
template <bool QNZ>
__global__ void __launch_bounds__(DW_THREADS, DW_PP_MIN_BLOCKS)
    k_dirac32(Geom g, Fields<float> f, float q, int x0b, int nx0, int nsites) {
    const int tau = blockIdx.x * blockDim.x + threadIdx.x;
    if (tau >= nsites) return;
    int x0, x1, x2, x3;
    sweep_coords_slab(g, x0b, nx0, tau, x0, x1, x2, x3);
    const int p = (x0 + x1 + x2 + x3) & 1;
    const int s = native_index(g, lex_index(g, x0, x1, x2, x3), p);
    int nb[8];
    neighbours8(g, x0, x1, x2, x3, 1 - p, nb);
    cplx<float> acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = mk(0.f, 0.f);
    hops_pipelined<QNZ>(f, g.V, s, nb, q, acc);
    cplx<float> v[12], w[12];
    load_spinor(f.psi, g.V, s, v);
    clover_mul<true>(f.C, g.V, s, v, w);
#pragma unroll
    for (int i = 0; i < 12; ++i) w[i] = w[i] - 0.5f * acc[i];
    store_spinor_cs(f.out, g.V, s, w);
}

template <typename R, bool QNZ>
__global__ void __launch_bounds__(DW_THREADS, DwMinBlocks<R>::value)
    k_dirac(Geom g, Fields<R> f, R q, int x0b, int nx0, int nsites) {
    const int tau = blockIdx.x * blockDim.x + threadIdx.x;
    if (tau >= nsites) return;
    int x0, x1, x2, x3;
    sweep_coords_slab(g, x0b, nx0, tau, x0, x1, x2, x3);
    const int p = (x0 + x1 + x2 + x3) & 1;
    const int s = native_index(g, lex_index(g, x0, x1, x2, x3), p);
    const int po = 1 - p;
    cplx<R> acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = mk<R>(0, 0);
    dirac_dir<R, QNZ, 0>(g, f, f.psi, g.V, 0, q, x0, x1, x2, x3, s, po, acc);
    dirac_dir<R, QNZ, 1>(g, f, f.psi, g.V, 0, q, x0, x1, x2, x3, s, po, acc);
    dirac_dir<R, QNZ, 2>(g, f, f.psi, g.V, 0, q, x0, x1, x2, x3, s, po, acc);
    dirac_dir<R, QNZ, 3>(g, f, f.psi, g.V, 0, q, x0, x1, x2, x3, s, po, acc);
    cplx<R> v[12], w[12];
    load_spinor(f.psi, g.V, s, v);
    clover_mul<true>(f.C, g.V, s, v, w);
#pragma unroll
    for (int i = 0; i < 12; ++i) w[i] = w[i] - R(0.5) * acc[i];
    if constexpr (sizeof(R) == 4) store_spinor_cs(f.out, g.V, s, w);
    else store_spinor(f.out, g.V, s, w);
}

// lexicographic [site][spin][colour][re,im] <-> native structure of arrays
template <typename R>
__global__ void k_pack(Geom g, const R* __restrict__ lex, typename Fields<R>::vec* __restrict__ nat) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int x0, x1, x2, x3;
    native_coords(g, s, x0, x1, x2, x3);
    const size_t l = (size_t)lex_index(g, x0, x1, x2, x3);
    cplx<R> v[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) v[i] = mk(lex[l * 24 + 2 * i], lex[l * 24 + 2 * i + 1]);
    store_spinor(nat, g.V, s, v);
}

template <typename R>
__global__ void k_unpack(Geom g, const typename Fields<R>::vec* __restrict__ nat, R* __restrict__ lex) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int x0, x1, x2, x3;
    native_coords(g, s, x0, x1, x2, x3);
    const size_t l = (size_t)lex_index(g, x0, x1, x2, x3);
    cplx<R> v[12];
    load_spinor(nat, g.V, s, v);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        lex[l * 24 + 2 * i] = v[i].re;
        lex[l * 24 + 2 * i + 1] = v[i].im;
    }
}

}  // namespace

namespace {

// D with launch shape sh (hop order, threads per block, sweep window) on the
// x0 planes [x0b, x0b + nx0)
int launch_dirac_shape(qxd_lattice* lat, void* out, const void* in, int prec, const DwShape& sh, cudaStream_t st,
                       int x0b = 0, int nx0 = -1) {
    Geom g = lat->g;
    g.R = sh.rows;
    if (nx0 < 0) nx0 = g.N0;
    const int n = nx0 * g.N1 * g.N2 * g.N3;
    const int blocks = (n + sh.threads - 1) / sh.threads;
    const bool qnz = lat->qhat != 0;
    if (prec == QXD_FP32) {
        Fields<float> f{(const float4*)in, (float4*)out, lat->U32, lat->A32, lat->C32};
        if (sh.pipelined) {
            if (qnz) k_dirac32<true><<<blocks, sh.threads, 0, st>>>(g, f, (float)lat->qhat, x0b, nx0, n);
            else k_dirac32<false><<<blocks, sh.threads, 0, st>>>(g, f, 0.f, x0b, nx0, n);
        } else {
            if (qnz) k_dirac<float, true><<<blocks, sh.threads, 0, st>>>(g, f, (float)lat->qhat, x0b, nx0, n);
            else k_dirac<float, false><<<blocks, sh.threads, 0, st>>>(g, f, 0.f, x0b, nx0, n);
        }
    } else {
        Fields<double> f{(const double2*)in, (double2*)out, lat->U64, lat->Zq64, lat->C64};
        if (qnz) k_dirac<double, true><<<blocks, sh.threads, 0, st>>>(g, f, (double)lat->qhat, x0b, nx0, n);
        else k_dirac<double, false><<<blocks, sh.threads, 0, st>>>(g, f, 0.0, x0b, nx0, n);
    }
    QXD_LAUNCHED("k_dirac");
    return QXD_OK;
}

// candidate sweep windows: divisors R of N2 with a window of N1 R N3 sites
// between 16K and 256K, the default (largest window <= 64K) and its nearest
// neighbours among them
std::vector<int> window_candidates(const Geom& g) {
    std::vector<int> ok;
    for (int R = 1; R <= g.N2; ++R) {
        const long long w = (long long)g.N1 * R * g.N3;
        if (g.N2 % R == 0 && w >= 16384 && w <= 262144) ok.push_back(R);
    }
    std::vector<int> out;
    int at = -1;
    for (int i = 0; i < (int)ok.size(); ++i)
        if (ok[i] == g.R) at = i;
    if (at < 0) return {g.R};
    for (int i = std::max(0, at - 1); i <= std::min((int)ok.size() - 1, at + 1); ++i) out.push_back(ok[i]);
    return out;
}

// time every candidate shape on this call's input (3 launches each after
// one untimed launch) and return the fastest
int tune_dirac(qxd_lattice* lat, void* out, const void* in, int prec, cudaStream_t st, DwShape* best) {
    std::vector<DwShape> cand;
    const std::vector<int> rows = window_candidates(lat->g);
    for (int pl = (prec == QXD_FP32 ? 1 : 0); pl >= 0; --pl)
        for (int th : {128, 64})
            for (int R : rows) cand.push_back(DwShape{pl, th, R, 0.f});
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    QXD_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(QXD_ERR_CUDA, "autotune: cudaEventCreate");
    }
    int rc = QXD_OK;
    best->ms = 0.f;
    for (DwShape& c : cand) {
        if ((rc = launch_dirac_shape(lat, out, in, prec, c, st))) break;
        cudaEventRecord(e0, st);
        for (int rep = 0; rep < 3 && !rc; ++rep) rc = launch_dirac_shape(lat, out, in, prec, c, st);
        if (rc) break;
        cudaEventRecord(e1, st);
        const cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "autotune: cudaEventSynchronize");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        c.ms = ms / 3;
        if (best->ms == 0.f || c.ms < best->ms) *best = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

int launch_dirac(qxd_lattice* lat, void* out, const void* in, int prec, cudaStream_t st) {
    const DwKey key = dw_key(lat, prec);
    DwShape sh;
    if (!dw_shape_get(key, &sh)) {
        if (autotune_enabled()) {
            int rc = tune_dirac(lat, out, in, prec, st, &sh);
            if (rc) return rc;
        } else {
            sh = dw_default_shape(lat, prec);
        }
        dw_shape_put(key, sh, autotune_enabled() ? "tuned" : "default");
    }
    return launch_dirac_shape(lat, out, in, prec, sh, st);
}

int launch_dirac_planes(qxd_lattice* lat, void* out, const void* in, int prec, int x0b, int nx0, cudaStream_t st) {
    DwShape sh;
    if (!dw_shape_get(dw_key(lat, prec), &sh)) sh = dw_default_shape(lat, prec);
    return launch_dirac_shape(lat, out, in, prec, sh, st, x0b, nx0);
}

int launch_pack(qxd_lattice* lat, void* nat, const void* lex, int prec, cudaStream_t st) {
    const Geom& g = lat->g;
    const int blocks = (g.V + 255) / 256;
    if (prec == QXD_FP32) k_pack<float><<<blocks, 256, 0, st>>>(g, (const float*)lex, (float4*)nat);
    else k_pack<double><<<blocks, 256, 0, st>>>(g, (const double*)lex, (double2*)nat);
    QXD_LAUNCHED("k_pack");
    return QXD_OK;
}

int launch_unpack(qxd_lattice* lat, void* lex, const void* nat, int prec, cudaStream_t st) {
    const Geom& g = lat->g;
    const int blocks = (g.V + 255) / 256;
    if (prec == QXD_FP32) k_unpack<float><<<blocks, 256, 0, st>>>(g, (const float4*)nat, (float*)lex);
    else k_unpack<double><<<blocks, 256, 0, st>>>(g, (const double2*)nat, (double*)lex);
    QXD_LAUNCHED("k_unpack");
    return QXD_OK;
}

}  // namespace qxd
