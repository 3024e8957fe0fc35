// Full-lattice application of D (Sec. 2.3, Eqs. (16)-(21)):
//   (D psi)(x) = M(x) psi(x) - 1/2 sum_mu [ (1 - g_mu) W(x,mu) psi(x+mu)
//                                  + (1 + g_mu) W(x-mu,mu)^+ psi(x-mu) ],
//   W(x,mu) = U(x,mu) z(x,mu)^qhat,  M(x) = (4 + m0) + dDsw(x),
// which is Eqs. (18)-(20) expanded (the diagonal 4 of Dw moved into M).
// One thread per site; spin projection to half spinors before the colour
// multiplication (the projectors commute with W). FP32: links as two rows
// plus the U(1) angle; FP64: full links. Both parities in one sweep, in the
// tiled order of sweep_coords so neighbour data is reused from L2.
//
// Chiral basis, psi = (psi0, psi1 | psi2, psi3):
//   (1 -+ g0): h = (psi0 +- psi2, psi1 +- psi3),   lower = (+-h0, +-h1)
//   (1 -+ g1): h = (psi0 +- i psi3, psi1 +- i psi2), lower = (-+i h1, -+i h0)
//   (1 -+ g2): h = (psi0 +- psi3, psi1 -+ psi2),   lower = (-+h1, +-h0)
//   (1 -+ g3): h = (psi0 +- i psi2, psi1 -+ i psi3), lower = (-+i h0, +-i h1)
#include "dirac_common.cuh"

namespace qxd {

namespace {

template <typename R, bool QNZ>
__global__ void __launch_bounds__(DW_THREADS, DwMinBlocks<R>::value) k_dirac(Geom g, Fields<R> f, R q) {
    const int tau = blockIdx.x * blockDim.x + threadIdx.x;
    if (tau >= g.V) return;
    int x0, x1, x2, x3;
    sweep_coords(g, tau, x0, x1, x2, x3);
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

int launch_dirac(qxd_lattice* lat, void* out, const void* in, int prec, cudaStream_t st) {
    const Geom& g = lat->g;
    const int blocks = (g.V + DW_THREADS - 1) / DW_THREADS;
    const bool qnz = lat->qhat != 0;
    if (prec == QXD_FP32) {
        Fields<float> f{(const float4*)in, (float4*)out, lat->U32, lat->A32, lat->C32};
        if (qnz) k_dirac<float, true><<<blocks, DW_THREADS, 0, st>>>(g, f, (float)lat->qhat);
        else k_dirac<float, false><<<blocks, DW_THREADS, 0, st>>>(g, f, 0.f);
    } else {
        Fields<double> f{(const double2*)in, (double2*)out, lat->U64, lat->Zq64, lat->C64};
        if (qnz) k_dirac<double, true><<<blocks, DW_THREADS, 0, st>>>(g, f, (double)lat->qhat);
        else k_dirac<double, false><<<blocks, DW_THREADS, 0, st>>>(g, f, 0.0);
    }
    QXD_LAUNCHED("k_dirac");
    return QXD_OK;
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
