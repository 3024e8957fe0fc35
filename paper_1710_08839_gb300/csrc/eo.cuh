// Even-odd operator launchers and strided spinor references.
#pragma once

#include "dirac_common.cuh"

namespace qxd {

enum { EO_HOP = 0, EO_INV_HOP = 1, EO_CLOVER_AUX_MHOP = 2, EO_AUX_MHOP = 3, EO_INV_AUX_MHOP = 4,
       EO_G5_CLOVER_AUX_MHOP = 5 };

template <typename R>
using DwMinBlocksEo = DwMinBlocks<R>;

// spinor field reference: element k of native site s at p[k * stride + s - off]
template <typename R>
struct SpRef {
    const typename Fields<R>::vec* p = nullptr;
    int stride = 0;
    int off = 0;
};
template <typename R>
struct SpRefOut {
    typename Fields<R>::vec* p = nullptr;
    int stride = 0;
    int off = 0;
};
template <typename R>
inline SpRef<R> as_in(SpRefOut<R> o) {
    return SpRef<R>{o.p, o.stride, o.off};
}
// full-lattice native array
template <typename R>
inline SpRef<R> full_ref(const void* p, int V) {
    return SpRef<R>{(const typename Fields<R>::vec*)p, V, 0};
}
template <typename R>
inline SpRefOut<R> full_out(void* p, int V) {
    return SpRefOut<R>{(typename Fields<R>::vec*)p, V, 0};
}
// half-lattice native array holding the sites of parity par
template <typename R>
inline SpRef<R> half_ref(const void* p, int Vh, int par) {
    return SpRef<R>{(const typename Fields<R>::vec*)p, Vh, par * Vh};
}
template <typename R>
inline SpRefOut<R> half_out(void* p, int Vh, int par) {
    return SpRefOut<R>{(typename Fields<R>::vec*)p, Vh, par * Vh};
}

template <typename R>
Fields<R> fields_of(qxd_lattice* lat);
template <>
inline Fields<float> fields_of<float>(qxd_lattice* lat) {
    return Fields<float>{nullptr, nullptr, lat->U32, lat->A32, lat->C32};
}
template <>
inline Fields<double> fields_of<double>(qxd_lattice* lat) {
    return Fields<double>{nullptr, nullptr, lat->U64, lat->Zq64, lat->C64};
}
template <typename R>
const typename Fields<R>::cvec* clover_of(qxd_lattice* lat, bool inverse);
template <>
inline const float4* clover_of<float>(qxd_lattice* lat, bool inverse) {
    return inverse ? lat->Cinv32 : lat->C32;
}
template <>
inline const double* clover_of<double>(qxd_lattice* lat, bool inverse) {
    return inverse ? lat->Cinv64 : lat->C64;
}

template <typename R>
int launch_eo(qxd_lattice* lat, int mode, int p, SpRef<R> in, SpRef<R> aux, SpRefOut<R> out, bool inverse,
              cudaStream_t st);
template <typename R>
int launch_clover_half(qxd_lattice* lat, int p, SpRef<R> in, SpRefOut<R> out, bool inverse, cudaStream_t st);
template <typename R>
int apply_dhat(qxd_lattice* lat, SpRefOut<R> out_e, SpRef<R> in_e, SpRefOut<R> tmp_o, cudaStream_t st);
// gamma5 D_hat psi_e (Hermitian: D_hat^dag = gamma5 D_hat gamma5)
template <typename R>
int apply_g5dhat(qxd_lattice* lat, SpRefOut<R> out_e, SpRef<R> in_e, SpRefOut<R> tmp_o, cudaStream_t st);

}  // namespace qxd
