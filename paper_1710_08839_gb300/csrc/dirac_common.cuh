// Device building blocks of the Dirac-operator kernels: native-layout loads
// and stores, SU(3) products, spin projection and reconstruction, U(1)
// phases and the clover-block product. Shared by the full-lattice, even-odd
// and Schwarz-block kernels.
#pragma once

#include "qxd_internal.cuh"

namespace qxd {

constexpr int DW_THREADS = 128;

// Register budget of the stencil kernels in the plain hop order: FP32 at most
// 80 registers (6 blocks of 128 threads per SM); the kernels are latency bound
// and more resident warps keep more loads in flight. FP64 at most 128 (4
// blocks). Blocks of 128 threads measured faster than 256 or 64 at the same
// budget. The pipelined FP32 hop order below (hops_pipelined) runs at 128
// registers instead.
template <typename R>
struct DwMinBlocks {
    static constexpr int value = sizeof(R) == 4 ? 6 : 4;
};

template <typename R>
struct Fields;

template <>
struct Fields<float> {
    using vec = float4;
    using cvec = float4;
    const float4* __restrict__ psi;
    float4* __restrict__ out;
    const float4* __restrict__ U;  // [4][3][V] two rows
    const float4* __restrict__ A;  // [V] four angles
    const float4* __restrict__ C;  // [18][V] clover (or inverse)
};

template <>
struct Fields<double> {
    using vec = double2;
    using cvec = double;
    const double2* __restrict__ psi;
    double2* __restrict__ out;
    const double2* __restrict__ U;  // [4][9][V]
    const double2* __restrict__ A;  // [4][V] z = exp(i A) as (cos A, sin A)
    const double* __restrict__ C;   // [72][V]
};

// ---------------------------------------------------------------------------
// spinors: v[3*spin + colour]
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_spinor(const float4* __restrict__ p, int V, int s, cplx<float> v[12]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float4 t = p[(size_t)k * V + s];
        v[2 * k] = mk(t.x, t.y);
        v[2 * k + 1] = mk(t.z, t.w);
    }
}
__device__ __forceinline__ void load_spinor(const double2* __restrict__ p, int V, int s, cplx<double> v[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double2 t = p[(size_t)k * V + s];
        v[k] = mk(t.x, t.y);
    }
}
__device__ __forceinline__ void store_spinor(float4* __restrict__ p, int V, int s, const cplx<float> v[12]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) p[(size_t)k * V + s] = make_float4(v[2 * k].re, v[2 * k].im, v[2 * k + 1].re, v[2 * k + 1].im);
}
// streaming (evict-first) store, for outputs not read again by the kernel
__device__ __forceinline__ void store_spinor_cs(float4* __restrict__ p, int V, int s, const cplx<float> v[12]) {
#pragma unroll
    for (int k = 0; k < 6; ++k)
        __stcs(&p[(size_t)k * V + s], make_float4(v[2 * k].re, v[2 * k].im, v[2 * k + 1].re, v[2 * k + 1].im));
}
__device__ __forceinline__ void store_spinor(double2* __restrict__ p, int V, int s, const cplx<double> v[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) p[(size_t)k * V + s] = make_double2(v[k].re, v[k].im);
}

// ---------------------------------------------------------------------------
// links
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_link(const float4* __restrict__ U, int V, int mu, int s, cplx<float> u[3][3]) {
    const float4 a = U[((size_t)mu * 3 + 0) * V + s];
    const float4 b = U[((size_t)mu * 3 + 1) * V + s];
    const float4 c = U[((size_t)mu * 3 + 2) * V + s];
    u[0][0] = mk(a.x, a.y);
    u[0][1] = mk(a.z, a.w);
    u[0][2] = mk(b.x, b.y);
    u[1][0] = mk(b.z, b.w);
    u[1][1] = mk(c.x, c.y);
    u[1][2] = mk(c.z, c.w);
    // SU(3): row 2 = conj(row0 x row1)
    u[2][0] = conj(u[0][1] * u[1][2] - u[0][2] * u[1][1]);
    u[2][1] = conj(u[0][2] * u[1][0] - u[0][0] * u[1][2]);
    u[2][2] = conj(u[0][0] * u[1][1] - u[0][1] * u[1][0]);
}
__device__ __forceinline__ void load_link(const double2* __restrict__ U, int V, int mu, int s, cplx<double> u[3][3]) {
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        double2 t = U[((size_t)mu * 9 + e) * V + s];
        u[e / 3][e % 3] = mk(t.x, t.y);
    }
}

// U(1) factor z(x,mu)^qhat of the hopping term.
// FP32: from the stored angle, exp(i qhat A). The argument is reduced to
// [-pi, pi] (|A| <= pi, so only a few periods are removed) and evaluated with
// the hardware approximation __sincosf, whose absolute error there is ~1e-6,
// well inside the FP32 tolerance of the operator.
// FP64: z^qhat stored per operator (built with the clover term from
// z = (cos A, sin A) by binary powering).
__device__ __forceinline__ cplx<float> link_phase(const float4* __restrict__ A, int V, int mu, int s, float q) {
    float t = q * reinterpret_cast<const float*>(A + s)[mu];
    const float k = rintf(t * 0.15915494309189535f);
    t = fmaf(-k, 6.2831853071795865f, t);
    float sn, cs;
    __sincosf(t, &sn, &cs);
    return mk(cs, sn);
}
__device__ __forceinline__ cplx<double> link_phase(const double2* __restrict__ Zq, int V, int mu, int s, double) {
    const double2 z = Zq[(size_t)mu * V + s];
    return mk(z.x, z.y);
}

template <typename R>
__device__ __forceinline__ void times3(cplx<R> ph, cplx<R> v[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = ph * v[c];
}

// g = u h
template <typename R>
__device__ __forceinline__ void su3_mul(const cplx<R> u[3][3], const cplx<R> h[3], cplx<R> g[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) g[a] = u[a][0] * h[0] + u[a][1] * h[1] + u[a][2] * h[2];
}
// g = u^+ h
template <typename R>
__device__ __forceinline__ void su3_dag_mul(const cplx<R> u[3][3], const cplx<R> h[3], cplx<R> g[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) g[a] = cmul(u[0][a], h[0]) + cmul(u[1][a], h[1]) + cmul(u[2][a], h[2]);
}

// ---------------------------------------------------------------------------
// spin projection (1 - DIR g_mu) and its reconstruction, chiral basis
// ---------------------------------------------------------------------------
template <typename R, int MU, int DIR>
__device__ __forceinline__ void project(const cplx<R> p[12], cplx<R> h0[3], cplx<R> h1[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cplx<R> a0 = p[c], a1 = p[3 + c], a2 = p[6 + c], a3 = p[9 + c];
        if (MU == 0) {
            h0[c] = DIR > 0 ? a0 + a2 : a0 - a2;
            h1[c] = DIR > 0 ? a1 + a3 : a1 - a3;
        } else if (MU == 1) {
            h0[c] = DIR > 0 ? a0 + times_i(a3) : a0 - times_i(a3);
            h1[c] = DIR > 0 ? a1 + times_i(a2) : a1 - times_i(a2);
        } else if (MU == 2) {
            h0[c] = DIR > 0 ? a0 + a3 : a0 - a3;
            h1[c] = DIR > 0 ? a1 - a2 : a1 + a2;
        } else {
            h0[c] = DIR > 0 ? a0 + times_i(a2) : a0 - times_i(a2);
            h1[c] = DIR > 0 ? a1 - times_i(a3) : a1 + times_i(a3);
        }
    }
}

template <typename R, int MU, int DIR>
__device__ __forceinline__ void accumulate(cplx<R> acc[12], const cplx<R> g0[3], const cplx<R> g1[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = acc[c] + g0[c];
        acc[3 + c] = acc[3 + c] + g1[c];
        if (MU == 0) {
            acc[6 + c] = DIR > 0 ? acc[6 + c] + g0[c] : acc[6 + c] - g0[c];
            acc[9 + c] = DIR > 0 ? acc[9 + c] + g1[c] : acc[9 + c] - g1[c];
        } else if (MU == 1) {
            acc[6 + c] = DIR > 0 ? acc[6 + c] + times_mi(g1[c]) : acc[6 + c] + times_i(g1[c]);
            acc[9 + c] = DIR > 0 ? acc[9 + c] + times_mi(g0[c]) : acc[9 + c] + times_i(g0[c]);
        } else if (MU == 2) {
            acc[6 + c] = DIR > 0 ? acc[6 + c] - g1[c] : acc[6 + c] + g1[c];
            acc[9 + c] = DIR > 0 ? acc[9 + c] + g0[c] : acc[9 + c] - g0[c];
        } else {
            acc[6 + c] = DIR > 0 ? acc[6 + c] + times_mi(g0[c]) : acc[6 + c] + times_i(g0[c]);
            acc[9 + c] = DIR > 0 ? acc[9 + c] + times_i(g1[c]) : acc[9 + c] + times_mi(g1[c]);
        }
    }
}

// ---------------------------------------------------------------------------
// clover blocks: y = M v, two Hermitian 6x6 blocks, packed (6 real diag,
// 15 complex strictly-lower entries row major)
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void herm6_mul(const R d[6], const cplx<R> L[15], const cplx<R> v[6], cplx<R> y[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) y[i] = d[i] * v[i];
    int k = 0;
#pragma unroll
    for (int i = 1; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j, ++k) {
            y[i] = y[i] + L[k] * v[j];
            y[j] = y[j] + cmul(L[k], v[i]);
        }
}

// STREAM: evict-first loads, for kernels that read each clover block once per
// launch (not the Schwarz block solves, which re-read it every MR step)
template <bool STREAM = false>
__device__ __forceinline__ void clover_mul(const float4* __restrict__ C, int V, int s, const cplx<float> v[12],
                                           cplx<float> w[12]) {
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        float r[36];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            float4 t = STREAM ? __ldcs(&C[(size_t)(9 * blk + q) * V + s]) : C[(size_t)(9 * blk + q) * V + s];
            r[4 * q] = t.x;
            r[4 * q + 1] = t.y;
            r[4 * q + 2] = t.z;
            r[4 * q + 3] = t.w;
        }
        float d[6];
        cplx<float> L[15];
#pragma unroll
        for (int i = 0; i < 6; ++i) d[i] = r[i];
#pragma unroll
        for (int k = 0; k < 15; ++k) L[k] = mk(r[6 + 2 * k], r[7 + 2 * k]);
        herm6_mul(d, L, v + 6 * blk, w + 6 * blk);
    }
}

template <bool STREAM = false>
__device__ __forceinline__ void clover_mul(const double* __restrict__ C, int V, int s, const cplx<double> v[12],
                                           cplx<double> w[12]) {
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        double d[6];
        cplx<double> L[15];
#pragma unroll
        for (int i = 0; i < 6; ++i) d[i] = C[(size_t)(36 * blk + i) * V + s];
#pragma unroll
        for (int k = 0; k < 15; ++k)
            L[k] = mk(C[(size_t)(36 * blk + 6 + 2 * k) * V + s], C[(size_t)(36 * blk + 7 + 2 * k) * V + s]);
        herm6_mul(d, L, v + 6 * blk, w + 6 * blk);
    }
}

// The two hops of direction MU at site x (native index s, parity 1 - po),
// raw sum (without the factor -1/2) added to acc. The neighbour spinors are
// read from psi at index (native index - poff) with stride pstride, so the
// same code serves full-lattice and half-lattice fields.
template <typename R, bool QNZ, int MU>
__device__ __forceinline__ void dirac_dir(const Geom& g, const Fields<R>& f,
                                          const typename Fields<R>::vec* __restrict__ psi, int pstride,
                                          int poff, R q, int x0, int x1, int x2, int x3, int s, int po,
                                          cplx<R> acc[12]) {
    cplx<R> v[12], h0[3], h1[3], g0[3], g1[3], u[3][3];
    // forward hop: (1 - g_mu) U(x,mu) z(x,mu)^q psi(x+mu)
    {
        const int sn = native_index(g, neighbour_lex<MU, +1>(g, x0, x1, x2, x3), po);
        load_spinor(psi, pstride, sn - poff, v);
        project<R, MU, +1>(v, h0, h1);
        load_link(f.U, g.V, MU, s, u);
        su3_mul(u, h0, g0);
        su3_mul(u, h1, g1);
        if (QNZ) {
            cplx<R> ph = link_phase(f.A, g.V, MU, s, q);
            times3(ph, g0);
            times3(ph, g1);
        }
        accumulate<R, MU, +1>(acc, g0, g1);
    }
    // backward hop: (1 + g_mu) U(x-mu,mu)^+ z(x-mu,mu)^-q psi(x-mu)
    {
        const int sb = native_index(g, neighbour_lex<MU, -1>(g, x0, x1, x2, x3), po);
        load_spinor(psi, pstride, sb - poff, v);
        project<R, MU, -1>(v, h0, h1);
        load_link(f.U, g.V, MU, sb, u);
        su3_dag_mul(u, h0, g0);
        su3_dag_mul(u, h1, g1);
        if (QNZ) {
            cplx<R> ph = conj(link_phase(f.A, g.V, MU, sb, q));
            times3(ph, g0);
            times3(ph, g1);
        }
        accumulate<R, MU, -1>(acc, g0, g1);
    }
}

// ---------------------------------------------------------------------------
// FP32 hopping term with software pipelining. The eight hops of a site are
// taken in the order (mu, fwd), (mu, bwd), mu = 0..3; the loads of hop k + 1
// (neighbour spinor, link, angle) are issued before the arithmetic of hop k,
// so that every thread keeps one hop's loads in flight while it computes.
// The stencil is bound by load latency: with 128 registers (4 blocks of 128
// threads per SM) this moves more bytes than the plain order at 80 registers
// and 6 blocks per SM.
// ---------------------------------------------------------------------------
constexpr int DW_PP_MIN_BLOCKS = 4;

struct HopData {
    float4 sp[6];  // neighbour spinor
    float4 lk[3];  // rows 0, 1 of the link
    float ang;     // U(1) angle of the link
};

// neighbour native indices: nb[2 mu] = x + mu, nb[2 mu + 1] = x - mu
__device__ __forceinline__ void neighbours8(const Geom& g, int x0, int x1, int x2, int x3, int po, int nb[8]) {
    nb[0] = native_index(g, neighbour_lex<0, +1>(g, x0, x1, x2, x3), po);
    nb[1] = native_index(g, neighbour_lex<0, -1>(g, x0, x1, x2, x3), po);
    nb[2] = native_index(g, neighbour_lex<1, +1>(g, x0, x1, x2, x3), po);
    nb[3] = native_index(g, neighbour_lex<1, -1>(g, x0, x1, x2, x3), po);
    nb[4] = native_index(g, neighbour_lex<2, +1>(g, x0, x1, x2, x3), po);
    nb[5] = native_index(g, neighbour_lex<2, -1>(g, x0, x1, x2, x3), po);
    nb[6] = native_index(g, neighbour_lex<3, +1>(g, x0, x1, x2, x3), po);
    nb[7] = native_index(g, neighbour_lex<3, -1>(g, x0, x1, x2, x3), po);
}

// loads of hop k at site s (forward: link and angle of s; backward: of the
// neighbour sn); a_own = the four angles of s
__device__ __forceinline__ void hop_load(const Fields<float>& f, int V, int k, int s, int sn, const float4& a_own,
                                         HopData& d) {
    const int mu = k >> 1;
    const bool fwd = (k & 1) == 0;
    const int sl = fwd ? s : sn;
#pragma unroll
    for (int c = 0; c < 6; ++c) d.sp[c] = f.psi[(size_t)c * V + sn];
#pragma unroll
    for (int j = 0; j < 3; ++j) d.lk[j] = f.U[((size_t)mu * 3 + j) * V + sl];
    if (fwd) d.ang = mu == 0 ? a_own.x : mu == 1 ? a_own.y : mu == 2 ? a_own.z : a_own.w;
    else d.ang = reinterpret_cast<const float*>(f.A + sn)[mu];
}

// raw hop (without the factor -1/2) added to acc: (1 - DIR g_mu) W psi(x + DIR mu)
// with W = U z^qhat forwards and its adjoint backwards
template <bool QNZ, int MU, int DIR>
__device__ __forceinline__ void hop_compute(const HopData& d, float q, cplx<float> acc[12]) {
    cplx<float> v[12], h0[3], h1[3], g0[3], g1[3], u[3][3];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        v[2 * c] = mk(d.sp[c].x, d.sp[c].y);
        v[2 * c + 1] = mk(d.sp[c].z, d.sp[c].w);
    }
    project<float, MU, DIR>(v, h0, h1);
    u[0][0] = mk(d.lk[0].x, d.lk[0].y);
    u[0][1] = mk(d.lk[0].z, d.lk[0].w);
    u[0][2] = mk(d.lk[1].x, d.lk[1].y);
    u[1][0] = mk(d.lk[1].z, d.lk[1].w);
    u[1][1] = mk(d.lk[2].x, d.lk[2].y);
    u[1][2] = mk(d.lk[2].z, d.lk[2].w);
    u[2][0] = conj(u[0][1] * u[1][2] - u[0][2] * u[1][1]);
    u[2][1] = conj(u[0][2] * u[1][0] - u[0][0] * u[1][2]);
    u[2][2] = conj(u[0][0] * u[1][1] - u[0][1] * u[1][0]);
    if (DIR > 0) {
        su3_mul(u, h0, g0);
        su3_mul(u, h1, g1);
    } else {
        su3_dag_mul(u, h0, g0);
        su3_dag_mul(u, h1, g1);
    }
    if (QNZ) {
        // exp(i qhat A), argument reduced to [-pi, pi] as in link_phase
        float t = q * d.ang;
        const float kk = rintf(t * 0.15915494309189535f);
        t = fmaf(-kk, 6.2831853071795865f, t);
        float sn, cs;
        __sincosf(t, &sn, &cs);
        const cplx<float> ph = mk(cs, DIR > 0 ? sn : -sn);
        times3(ph, g0);
        times3(ph, g1);
    }
    accumulate<float, MU, DIR>(acc, g0, g1);
}

// acc += raw sum of the eight hops at site s with neighbours nb
template <bool QNZ>
__device__ __forceinline__ void hops_pipelined(const Fields<float>& f, int V, int s, const int nb[8], float q,
                                               cplx<float> acc[12]) {
    const float4 a_own = QNZ ? f.A[s] : make_float4(0.f, 0.f, 0.f, 0.f);
    HopData d[2];
    hop_load(f, V, 0, s, nb[0], a_own, d[0]);
    hop_load(f, V, 1, s, nb[1], a_own, d[1]);
    hop_compute<QNZ, 0, +1>(d[0], q, acc);
    hop_load(f, V, 2, s, nb[2], a_own, d[0]);
    hop_compute<QNZ, 0, -1>(d[1], q, acc);
    hop_load(f, V, 3, s, nb[3], a_own, d[1]);
    hop_compute<QNZ, 1, +1>(d[0], q, acc);
    hop_load(f, V, 4, s, nb[4], a_own, d[0]);
    hop_compute<QNZ, 1, -1>(d[1], q, acc);
    hop_load(f, V, 5, s, nb[5], a_own, d[1]);
    hop_compute<QNZ, 2, +1>(d[0], q, acc);
    hop_load(f, V, 6, s, nb[6], a_own, d[0]);
    hop_compute<QNZ, 2, -1>(d[1], q, acc);
    hop_load(f, V, 7, s, nb[7], a_own, d[1]);
    hop_compute<QNZ, 3, +1>(d[0], q, acc);
    hop_compute<QNZ, 3, -1>(d[1], q, acc);
}

}  // namespace qxd
