// Even-odd form of D (Sec. 2.4, Eqs. (29)-(30)). D = M + H with M the
// site-diagonal part and H the hopping part, H psi(x) = -1/2 sum_mu [...];
// H connects only sites of opposite parity, so
//   D_ee = M_ee, D_oo = M_oo, D_eo = H_eo, D_oe = H_oe,
//   D_hat = M_ee - H_eo M_oo^-1 H_oe   (on the even sites).
// The kernels below evaluate, for all sites x of one parity p,
//   HOP              out = H psi
//   INV_HOP          out = M^-1 (H psi)
//   CLOVER_AUX_MHOP  out = M aux - H psi
//   AUX_MHOP         out = aux - H psi
//   INV_AUX_MHOP     out = M^-1 (aux - H psi)
//   G5_CLOVER_AUX_MHOP  out = gamma5 (M aux - H psi)
// where psi lives on the other parity. Each field is addressed as
// (pointer, stride, offset): element k of the site with native index s is at
// p[k * stride + s - offset], so full-lattice arrays (stride V, offset 0)
// and half-lattice arrays (stride V/2, offset parity * V/2) both work.
#include <string>

#include "dirac_common.cuh"
#include "eo.cuh"

namespace qxd {

namespace {

template <typename R, bool QNZ, int MODE>
__global__ void __launch_bounds__(DW_THREADS, DwMinBlocksEo<R>::value)
    k_dslash_half(Geom g, int p, Fields<R> f, SpRef<R> in, SpRef<R> aux, SpRefOut<R> out,
                  const typename Fields<R>::cvec* __restrict__ Cl, R q) {
    const int tau = blockIdx.x * blockDim.x + threadIdx.x;
    if (tau >= g.Vh) return;
    int x0, x1, x2, x3;
    sweep_coords_parity(g, p, tau, x0, x1, x2, x3);
    const int s = native_index(g, lex_index(g, x0, x1, x2, x3), p);
    const int po = 1 - p;
    cplx<R> acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = mk<R>(0, 0);
    dirac_dir<R, QNZ, 0>(g, f, in.p, in.stride, in.off, q, x0, x1, x2, x3, s, po, acc);
    dirac_dir<R, QNZ, 1>(g, f, in.p, in.stride, in.off, q, x0, x1, x2, x3, s, po, acc);
    dirac_dir<R, QNZ, 2>(g, f, in.p, in.stride, in.off, q, x0, x1, x2, x3, s, po, acc);
    dirac_dir<R, QNZ, 3>(g, f, in.p, in.stride, in.off, q, x0, x1, x2, x3, s, po, acc);
    cplx<R> w[12];
    if (MODE == EO_HOP) {
#pragma unroll
        for (int i = 0; i < 12; ++i) w[i] = R(-0.5) * acc[i];
    } else if (MODE == EO_INV_HOP) {
        cplx<R> t[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) t[i] = R(-0.5) * acc[i];
        clover_mul<true>(Cl, g.V, s, t, w);
    } else if (MODE == EO_CLOVER_AUX_MHOP || MODE == EO_G5_CLOVER_AUX_MHOP) {
        cplx<R> a[12];
        load_spinor(aux.p, aux.stride, s - aux.off, a);
        clover_mul<true>(Cl, g.V, s, a, w);
#pragma unroll
        for (int i = 0; i < 12; ++i) w[i] = w[i] + R(0.5) * acc[i];
        if (MODE == EO_G5_CLOVER_AUX_MHOP) {
            // gamma5 = diag(1, 1, -1, -1): spins 2 and 3 change sign
#pragma unroll
            for (int i = 6; i < 12; ++i) w[i] = R(-1) * w[i];
        }
    } else if (MODE == EO_AUX_MHOP) {
        load_spinor(aux.p, aux.stride, s - aux.off, w);
#pragma unroll
        for (int i = 0; i < 12; ++i) w[i] = w[i] + R(0.5) * acc[i];
    } else {  // EO_INV_AUX_MHOP
        cplx<R> a[12];
        load_spinor(aux.p, aux.stride, s - aux.off, a);
#pragma unroll
        for (int i = 0; i < 12; ++i) a[i] = a[i] + R(0.5) * acc[i];
        clover_mul<true>(Cl, g.V, s, a, w);
    }
    store_spinor(out.p, out.stride, s - out.off, w);
}

// out = M in (or M^-1 in) on the sites of parity p
template <typename R>
__global__ void k_clover_half(Geom g, int p, SpRef<R> in, SpRefOut<R> out,
                              const typename Fields<R>::cvec* __restrict__ Cl) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    const int s = p * g.Vh + h;
    cplx<R> a[12], w[12];
    load_spinor(in.p, in.stride, s - in.off, a);
    clover_mul<true>(Cl, g.V, s, a, w);
    store_spinor(out.p, out.stride, s - out.off, w);
}

template <typename R, bool QNZ>
int launch_mode(qxd_lattice* lat, int mode, int p, const Fields<R>& f, SpRef<R> in, SpRef<R> aux,
                SpRefOut<R> out, const typename Fields<R>::cvec* Cl, cudaStream_t st) {
    const Geom& g = lat->g;
    const int blocks = (g.Vh + DW_THREADS - 1) / DW_THREADS;
    const R q = (R)lat->qhat;
    switch (mode) {
        case EO_HOP: k_dslash_half<R, QNZ, EO_HOP><<<blocks, DW_THREADS, 0, st>>>(g, p, f, in, aux, out, Cl, q); break;
        case EO_INV_HOP: k_dslash_half<R, QNZ, EO_INV_HOP><<<blocks, DW_THREADS, 0, st>>>(g, p, f, in, aux, out, Cl, q); break;
        case EO_CLOVER_AUX_MHOP: k_dslash_half<R, QNZ, EO_CLOVER_AUX_MHOP><<<blocks, DW_THREADS, 0, st>>>(g, p, f, in, aux, out, Cl, q); break;
        case EO_AUX_MHOP: k_dslash_half<R, QNZ, EO_AUX_MHOP><<<blocks, DW_THREADS, 0, st>>>(g, p, f, in, aux, out, Cl, q); break;
        case EO_G5_CLOVER_AUX_MHOP: k_dslash_half<R, QNZ, EO_G5_CLOVER_AUX_MHOP><<<blocks, DW_THREADS, 0, st>>>(g, p, f, in, aux, out, Cl, q); break;
        default: k_dslash_half<R, QNZ, EO_INV_AUX_MHOP><<<blocks, DW_THREADS, 0, st>>>(g, p, f, in, aux, out, Cl, q); break;
    }
    QXD_LAUNCHED("k_dslash_half");
    return QXD_OK;
}

}  // namespace

template <typename R>
int launch_eo(qxd_lattice* lat, int mode, int p, SpRef<R> in, SpRef<R> aux, SpRefOut<R> out, bool inverse,
              cudaStream_t st) {
    Fields<R> f = fields_of<R>(lat);
    const typename Fields<R>::cvec* Cl = clover_of<R>(lat, inverse);
    if (lat->qhat != 0) return launch_mode<R, true>(lat, mode, p, f, in, aux, out, Cl, st);
    return launch_mode<R, false>(lat, mode, p, f, in, aux, out, Cl, st);
}

template <typename R>
int launch_clover_half(qxd_lattice* lat, int p, SpRef<R> in, SpRefOut<R> out, bool inverse, cudaStream_t st) {
    const Geom& g = lat->g;
    const int blocks = (g.Vh + 255) / 256;
    k_clover_half<R><<<blocks, 256, 0, st>>>(g, p, in, out, clover_of<R>(lat, inverse));
    QXD_LAUNCHED("k_clover_half");
    return QXD_OK;
}

template int launch_eo<float>(qxd_lattice*, int, int, SpRef<float>, SpRef<float>, SpRefOut<float>, bool, cudaStream_t);
template int launch_eo<double>(qxd_lattice*, int, int, SpRef<double>, SpRef<double>, SpRefOut<double>, bool, cudaStream_t);
template int launch_clover_half<float>(qxd_lattice*, int, SpRef<float>, SpRefOut<float>, bool, cudaStream_t);
template int launch_clover_half<double>(qxd_lattice*, int, SpRef<double>, SpRefOut<double>, bool, cudaStream_t);

// D_hat psi_e = M_ee psi_e - H_eo M_oo^-1 H_oe psi_e; tmp is an odd-parity field
template <typename R>
int apply_dhat(qxd_lattice* lat, SpRefOut<R> out_e, SpRef<R> in_e, SpRefOut<R> tmp_o, cudaStream_t st) {
    int rc = launch_eo<R>(lat, EO_INV_HOP, 1, in_e, SpRef<R>{}, tmp_o, true, st);
    if (rc) return rc;
    return launch_eo<R>(lat, EO_CLOVER_AUX_MHOP, 0, as_in(tmp_o), in_e, out_e, false, st);
}
template int apply_dhat<float>(qxd_lattice*, SpRefOut<float>, SpRef<float>, SpRefOut<float>, cudaStream_t);
template int apply_dhat<double>(qxd_lattice*, SpRefOut<double>, SpRef<double>, SpRefOut<double>, cudaStream_t);

template <typename R>
int apply_g5dhat(qxd_lattice* lat, SpRefOut<R> out_e, SpRef<R> in_e, SpRefOut<R> tmp_o, cudaStream_t st) {
    int rc = launch_eo<R>(lat, EO_INV_HOP, 1, in_e, SpRef<R>{}, tmp_o, true, st);
    if (rc) return rc;
    return launch_eo<R>(lat, EO_G5_CLOVER_AUX_MHOP, 0, as_in(tmp_o), in_e, out_e, false, st);
}
template int apply_g5dhat<float>(qxd_lattice*, SpRefOut<float>, SpRef<float>, SpRefOut<float>, cudaStream_t);
template int apply_g5dhat<double>(qxd_lattice*, SpRefOut<double>, SpRef<double>, SpRefOut<double>, cudaStream_t);

namespace {

enum { EOAPI_DHAT, EOAPI_PREPARE, EOAPI_RECONSTRUCT };

// in/out are full-lattice native arrays
template <typename R>
int eo_native(qxd_lattice* lat, int what, void* out, const void* in, void* tmp, cudaStream_t st) {
    const int V = lat->g.V;
    int rc;
    if (what == EOAPI_DHAT) {
        // tmp (odd half of a full array) holds M_oo^-1 H_oe in_e
        if ((rc = apply_dhat<R>(lat, full_out<R>(out, V), full_ref<R>(in, V), full_out<R>(tmp, V), st))) return rc;
    } else if (what == EOAPI_PREPARE) {
        if ((rc = launch_clover_half<R>(lat, 1, full_ref<R>(in, V), full_out<R>(tmp, V), true, st))) return rc;
        if ((rc = launch_eo<R>(lat, EO_AUX_MHOP, 0, full_ref<R>(tmp, V), full_ref<R>(in, V), full_out<R>(out, V),
                               false, st)))
            return rc;
    } else {
        // out holds x (even part read); in holds b
        return launch_eo<R>(lat, EO_INV_AUX_MHOP, 1, full_ref<R>(out, V), full_ref<R>(in, V), full_out<R>(out, V),
                            true, st);
    }
    // zero the odd sites of out: native layout keeps each component's odd
    // sites in one contiguous range
    const size_t comp = sizeof(R) == 4 ? 6 : 12;
    const size_t vb = sizeof(typename Fields<R>::vec);
    for (size_t k = 0; k < comp; ++k)
        QXD_CUDA(cudaMemsetAsync((char*)out + (k * V + lat->g.Vh) * vb, 0, (size_t)lat->g.Vh * vb, st));
    return QXD_OK;
}

int eo_api(qxd_lattice* lat, int what, void* out, const void* in, int flags, void* stream, const char* name) {
    if (!lat || !out || !in) return fail(QXD_ERR_ARG, std::string(name) + ": NULL argument");
    if (flags & ~(0x1 | 0x100)) return fail(QXD_ERR_ARG, std::string(name) + ": bad flags (device buffers only)");
    if (what != EOAPI_RECONSTRUCT && out == in)
        return fail(QXD_ERR_ARG, std::string(name) + ": in and out must not overlap");
    if (!qxd::clover_ready(lat)) return fail(QXD_ERR_STATE, std::string(name) + ": needs qxd_sw_build first");
    const int prec = flags & 0x1;
    cudaStream_t st = stream ? (cudaStream_t)stream : lat->stream;
    int rc = ensure_scratch(lat);
    if (rc) return rc;
    if (flags & QXD_LAYOUT_NATIVE)
        return prec == QXD_FP32 ? eo_native<float>(lat, what, out, in, lat->scratch_lex, st)
                                : eo_native<double>(lat, what, out, in, lat->scratch_lex, st);
    if ((rc = launch_pack(lat, lat->scratch_in, in, prec, st))) return rc;
    if (what == EOAPI_RECONSTRUCT && (rc = launch_pack(lat, lat->scratch_out, out, prec, st))) return rc;
    rc = prec == QXD_FP32 ? eo_native<float>(lat, what, lat->scratch_out, lat->scratch_in, lat->scratch_lex, st)
                          : eo_native<double>(lat, what, lat->scratch_out, lat->scratch_in, lat->scratch_lex, st);
    if (rc) return rc;
    return launch_unpack(lat, out, lat->scratch_out, prec, st);
}

}  // namespace

}  // namespace qxd

extern "C" {

int qxd_Dhat(qxd_lattice* lat, void* out, const void* in, int flags, void* stream) {
    return qxd::eo_api(lat, qxd::EOAPI_DHAT, out, in, flags, stream, "qxd_Dhat");
}

int qxd_eo_prepare(qxd_lattice* lat, void* out, const void* b, int flags, void* stream) {
    return qxd::eo_api(lat, qxd::EOAPI_PREPARE, out, b, flags, stream, "qxd_eo_prepare");
}

int qxd_eo_reconstruct(qxd_lattice* lat, void* x, const void* b, int flags, void* stream) {
    return qxd::eo_api(lat, qxd::EOAPI_RECONSTRUCT, x, b, flags, stream, "qxd_eo_reconstruct");
}

}  // extern "C"
