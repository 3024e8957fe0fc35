// Gauge observables and the Wilson flow (App. A; Luscher's flow, Sec. 3).
//
// * qxd_gauge_observables reduces the clover field tensors of the gauge
//   field (kept by qxd_set_gauge, one anti-Hermitian F per plane and site plus
//   the U(1) four-plaquette Im sum) to
//     E_SU(3) = 1/V sum_x sum_{mu<nu} |F_munu(x)|^2 = -1/(2V) sum tr{F F},
//     E_U(1)  = 1/V sum_x sum_{mu<nu} (Im sum / (4 q_el))^2,
//     Q_top   = 1/(4 pi^2) sum_x [tr F01 F23 - tr F02 F13 + tr F03 F12]
//   (the 24 terms of the epsilon sum, grouped), with the C* sum halved to
//   the physical lattice (the mirror half carries the conjugate field).
// * qxd_wflow integrates dV/dt = Z(V) V, Z = -1/2 (W - W^dag) +
//   1/6 tr(W - W^dag), W = U(x,mu) (sum of the six staples), with Luscher's
//   third-order Runge-Kutta scheme in its one-accumulator form
//     X <- a eps Z(W_i) + b X,  W_{i+1} = exp(X) W_i,
//     (a, b) = (1/4, 0), (8/9, -17/9), (3/4, -1),
//   and the compact U(1) field by the same scheme with
//     dA(x,mu)/dt = -sum_{nu != mu} [sin theta_munu(x) - sin theta_munu(x - nu)].
//   With C* boundaries only the physical links (x1 < L1) are integrated; each
//   update is written to the mirror link as its complex conjugate (-A for
//   the angle), which keeps the orbifold constraint exact. One thread per
//   link; the stages read one copy of the field and write the other.
#include <cmath>
#include <string>

#include "blas.cuh"
#include "su3.cuh"

namespace qxd {

int launch_field_tensor(qxd_lattice* lat);

namespace {

// ---------------------------------------------------------------------------
// observables
// ---------------------------------------------------------------------------

struct Anti {
    double d[3];  // F_ii = i d_i
    C64 o[3];     // F_01, F_02, F_12
};

__device__ __forceinline__ Anti load_plane(const double* __restrict__ F, size_t V, int plane, int s) {
    const double* f = F + (size_t)plane * 10 * V + s;
    Anti a;
    a.d[0] = f[0];
    a.d[1] = f[V];
    a.d[2] = f[2 * V];
    a.o[0] = mk(f[3 * V], f[4 * V]);
    a.o[1] = mk(f[5 * V], f[6 * V]);
    a.o[2] = mk(f[7 * V], f[8 * V]);
    return a;
}

// tr(A B) for anti-Hermitian A, B: -(sum a_i b_i + 2 Re sum_{i<j} A_ij conj(B_ij))
__device__ __forceinline__ double tr_ab(const Anti& a, const Anti& b) {
    double s = a.d[0] * b.d[0] + a.d[1] * b.d[1] + a.d[2] * b.d[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) s += 2.0 * (a.o[k].re * b.o[k].re + a.o[k].im * b.o[k].im);
    return -s;
}

// planes in the order of the field tensor: 01 02 03 12 13 23
__global__ void __launch_bounds__(RED_THREADS) k_gauge_obs(int V, const double* __restrict__ F, double u1_norm,
                                                          double* __restrict__ partials) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < V; s += gridDim.x * blockDim.x) {
        Anti f[6];
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            f[p] = load_plane(F, (size_t)V, p, s);
            acc[0] -= tr_ab(f[p], f[p]);
            const double im = F[((size_t)p * 10 + 9) * V + s];
            acc[1] += im * im * u1_norm;
        }
        acc[2] += tr_ab(f[0], f[5]) - tr_ab(f[1], f[4]) + tr_ab(f[2], f[3]);
    }
    block_reduce_store<3>(acc, 3, partials);
}

// ---------------------------------------------------------------------------
// Wilson flow
// ---------------------------------------------------------------------------

// exp(X) for traceless X (the flow's X is anti-Hermitian and traceless). By
// the Cayley-Hamilton theorem X^3 = d1 X + d0 with d1 = tr(X^2)/2 and
// d0 = det X, so every power is X^n = a_n + b_n X + c_n X^2 with
//   a_{n+1} = c_n d0,  b_{n+1} = a_n + c_n d1,  c_{n+1} = b_n,
// and exp(X) = A + B X + C X^2 with A, B, C the sums of a_n/n!, b_n/n!,
// c_n/n! (the Taylor series, summed on these scalars). X is first scaled by
// 2^-k to |X|_F <= 1/2, where 24 terms leave a remainder below 1e-30, and
// the result squared k times. One 3x3 product (X^2) instead of one per term.
__device__ M3 expm3(const M3& X0) {
    double n2 = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) n2 += X0.a[i][j].re * X0.a[i][j].re + X0.a[i][j].im * X0.a[i][j].im;
    double nrm = sqrt(n2);
    int k = 0;
    while (nrm > 0.5 && k < 40) {
        nrm *= 0.5;
        ++k;
    }
    const double sc = ldexp(1.0, -k);
    M3 X;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) X.a[i][j] = sc * X0.a[i][j];
    const M3 X2 = mul(X, X);
    const C64 d1 = 0.5 * (X2.a[0][0] + X2.a[1][1] + X2.a[2][2]);
    const C64 d0 = X.a[0][0] * (X.a[1][1] * X.a[2][2] - X.a[1][2] * X.a[2][1]) -
                   X.a[0][1] * (X.a[1][0] * X.a[2][2] - X.a[1][2] * X.a[2][0]) +
                   X.a[0][2] * (X.a[1][0] * X.a[2][1] - X.a[1][1] * X.a[2][0]);
    // term n: (a, b, c) / n!
    C64 a = mk(1.0, 0.0), b = mk(0.0, 0.0), c = mk(0.0, 0.0);
    C64 A = a, B = b, Cc = c;
#pragma unroll 1
    for (int n = 0; n < 24; ++n) {
        const double r = 1.0 / (n + 1);
        const C64 an = r * (c * d0);
        const C64 bn = r * (a + c * d1);
        const C64 cn = r * b;
        a = an;
        b = bn;
        c = cn;
        A = A + a;
        B = B + b;
        Cc = Cc + c;
    }
    M3 E;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) E.a[i][j] = B * X.a[i][j] + Cc * X2.a[i][j] + (i == j ? A : mk(0.0, 0.0));
    for (int i = 0; i < k; ++i) E = mul(E, E);
    return E;
}

struct FlowStage {
    Geom g;
    int cstar1;                 // direction 1 doubled (C*): integrate x1 < L1 only
    int nphys;                  // sites integrated
    const double2* __restrict__ Uin;
    double2* __restrict__ Uout;
    const double* __restrict__ Ain;
    double* __restrict__ Aout;
    double* __restrict__ X;     // SU(3) accumulator, [4][9][V] (anti-Hermitian: 3 Im diag + 3 complex)
    double* __restrict__ Xa;    // U(1) accumulator, [4][V]
    double a, b;                // X <- a Z + b X (a includes eps)
};

__device__ __forceinline__ void store_link(double2* __restrict__ U, size_t V, int mu, int s, const M3& m, bool cj) {
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        const C64 v = m.a[e / 3][e % 3];
        U[((size_t)mu * 9 + e) * V + s] = make_double2(v.re, cj ? -v.im : v.im);
    }
}

__device__ __forceinline__ double wrap_angle(double a) {
    const double two_pi = 6.283185307179586476925286766559;
    a = fmod(a + 3.14159265358979323846264338327950, two_pi);
    if (a < 0.0) a += two_pi;
    return a - 3.14159265358979323846264338327950;
}

__global__ void __launch_bounds__(128) k_wflow_stage(FlowStage f) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * f.nphys) return;
    const Geom& g = f.g;
    const size_t V = (size_t)g.V;
    const int mu = t / f.nphys;
    int p = t - mu * f.nphys;
    // physical site p in lexicographic order of (x0, x1 < N1phys, x2, x3)
    const int n1 = f.cstar1 ? g.L1 : g.N1;
    int x[4];
    x[3] = p % g.N3;
    p /= g.N3;
    x[2] = p % g.N2;
    p /= g.N2;
    x[1] = p % n1;
    x[0] = p / n1;
    const int s = native_of(g, x);
    int c[4];
    auto at = [&](int m1, int d1, int m2, int d2) {
        c[0] = x[0]; c[1] = x[1]; c[2] = x[2]; c[3] = x[3];
        if (d1) shift_coords(g, c, m1, d1);
        if (d2) shift_coords(g, c, m2, d2);
        return native_of(g, c);
    };
    const int sxpm = at(mu, 1, 0, 0);
    // SU(3): staple sum and W = U(x,mu) S
    M3 S;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) S.a[i][j] = mk(0.0, 0.0);
    double zu1 = 0.0;
    const double* A = f.Ain;
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        const int sxpn = at(nu, 1, 0, 0), sxmn = at(nu, -1, 0, 0), sxpmmn = at(mu, 1, nu, -1);
        // U(x+mu,nu) U(x+nu,mu)^dag U(x,nu)^dag
        M3 t1 = mul_nd(mul_nd(load_link64(f.Uin, V, nu, sxpm), load_link64(f.Uin, V, mu, sxpn)),
                       load_link64(f.Uin, V, nu, s));
        // U(x+mu-nu,nu)^dag U(x-nu,mu)^dag U(x-nu,nu)
        M3 t2 = mul(mul_dn(load_link64(f.Uin, V, nu, sxpmmn), dag(load_link64(f.Uin, V, mu, sxmn))),
                    load_link64(f.Uin, V, nu, sxmn));
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) S.a[i][j] = S.a[i][j] + t1.a[i][j] + t2.a[i][j];
        // U(1): theta_munu(x) and theta_munu(x - nu)
        const double th_f = A[(size_t)mu * V + s] + A[(size_t)nu * V + sxpm] - A[(size_t)mu * V + sxpn] -
                            A[(size_t)nu * V + s];
        const double th_b = A[(size_t)mu * V + sxmn] + A[(size_t)nu * V + sxpmmn] - A[(size_t)mu * V + s] -
                            A[(size_t)nu * V + sxmn];
        zu1 -= sin(th_f) - sin(th_b);
    }
    const M3 U = load_link64(f.Uin, V, mu, s);
    const M3 W = mul(U, S);
    // Z = -1/2 (W - W^dag) + 1/6 tr(W - W^dag); tr(W - W^dag) = 2i Im tr W
    const double trim = (W.a[0][0].im + W.a[1][1].im + W.a[2][2].im) * (1.0 / 3.0);
    double* X = f.X;
    M3 Xn;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        // diagonal: Z_ii = -i Im W_ii + i (1/3) Im tr W
        const double zi = -W.a[i][i].im + trim;
        double xi = f.a * zi;
        if (f.b != 0.0) xi += f.b * X[((size_t)mu * 9 + i) * V + s];
        X[((size_t)mu * 9 + i) * V + s] = xi;
        Xn.a[i][i] = mk(0.0, xi);
    }
    const int oi[3] = {0, 0, 1}, oj[3] = {1, 2, 2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int i = oi[k], j = oj[k];
        // Z_ij = -1/2 (W_ij - conj(W_ji))
        const C64 z = mk(-0.5 * (W.a[i][j].re - W.a[j][i].re), -0.5 * (W.a[i][j].im + W.a[j][i].im));
        double re = f.a * z.re, im = f.a * z.im;
        if (f.b != 0.0) {
            re += f.b * X[((size_t)mu * 9 + 3 + 2 * k) * V + s];
            im += f.b * X[((size_t)mu * 9 + 4 + 2 * k) * V + s];
        }
        X[((size_t)mu * 9 + 3 + 2 * k) * V + s] = re;
        X[((size_t)mu * 9 + 4 + 2 * k) * V + s] = im;
        Xn.a[i][j] = mk(re, im);
        Xn.a[j][i] = mk(-re, im);
    }
    const M3 Unew = mul(expm3(Xn), U);
    store_link(f.Uout, V, mu, s, Unew, false);
    double xa = f.a * zu1;
    if (f.b != 0.0) xa += f.b * f.Xa[(size_t)mu * V + s];
    f.Xa[(size_t)mu * V + s] = xa;
    const double anew = wrap_angle(A[(size_t)mu * V + s] + xa);
    f.Aout[(size_t)mu * V + s] = anew;
    if (f.cstar1) {
        int m[4] = {x[0], x[1] + g.L1, x[2], x[3]};
        const int sm = native_of(g, m);
        store_link(f.Uout, V, mu, sm, Unew, true);
        f.Aout[(size_t)mu * V + sm] = -anew;
    }
}

// FP32 two-row links, FP32 angles and z = exp(iA) from the FP64 field
__global__ void k_gauge_derive(Geom g, const double2* __restrict__ U64, const double* __restrict__ A64,
                               float4* __restrict__ U32, double2* __restrict__ Z64, float4* __restrict__ A32) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const size_t V = (size_t)g.V;
    float a32[4];
    for (int mu = 0; mu < 4; ++mu) {
        double2 u[6];
#pragma unroll
        for (int e = 0; e < 6; ++e) u[e] = U64[((size_t)mu * 9 + e) * V + s];
        U32[((size_t)mu * 3 + 0) * V + s] = make_float4((float)u[0].x, (float)u[0].y, (float)u[1].x, (float)u[1].y);
        U32[((size_t)mu * 3 + 1) * V + s] = make_float4((float)u[2].x, (float)u[2].y, (float)u[3].x, (float)u[3].y);
        U32[((size_t)mu * 3 + 2) * V + s] = make_float4((float)u[4].x, (float)u[4].y, (float)u[5].x, (float)u[5].y);
        const double a = A64[(size_t)mu * V + s];
        double sa, ca;
        sincos(a, &sa, &ca);
        Z64[(size_t)mu * V + s] = make_double2(ca, sa);
        a32[mu] = (float)a;
    }
    A32[s] = make_float4(a32[0], a32[1], a32[2], a32[3]);
}

template <typename T>
int dmalloc(T** p, size_t n, const char* what) {
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, what);
    }
    return QXD_OK;
}

}  // namespace

}  // namespace qxd

using namespace qxd;

extern "C" {

int qxd_gauge_observables(qxd_lattice* lat, double q_el, double* out) {
    if (!lat || !out) return fail(QXD_ERR_ARG, "qxd_gauge_observables: NULL argument");
    if (!(q_el > 0.0) || !std::isfinite(q_el)) return fail(QXD_ERR_ARG, "qxd_gauge_observables: q_el > 0 required");
    const qxd_lattice* own = gauge_owner(lat);
    if (!own->has_gauge) return fail(QXD_ERR_STATE, "qxd_gauge_observables: needs qxd_set_gauge first");
    Reducer red;
    int rc = red.init();
    if (rc) return rc;
    const Geom& g = lat->g;
    const double u1_norm = 1.0 / (16.0 * q_el * q_el);
    k_gauge_obs<<<RED_BLOCKS, RED_THREADS, 0, lat->stream>>>(g.V, own->ftens, u1_norm, red.partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        red.release();
        return cuda_fail(e, "k_gauge_obs");
    }
    rc = reduce_finish(red, 3, lat->stream);
    if (!rc) {
        const double V = (double)g.V;
        const double w = (lat->cstar_mask & 2u) ? 0.5 : 1.0;
        const double pi = 3.14159265358979323846264338327950;
        out[0] = red.h_res[0] / V;
        out[1] = red.h_res[1] / V;
        out[2] = w * red.h_res[2] / (4.0 * pi * pi);
    }
    red.release();
    return rc;
}

int qxd_wflow(qxd_lattice* lat, double eps, int nsteps) {
    if (!lat) return fail(QXD_ERR_ARG, "qxd_wflow: lat is NULL");
    if (lat->parent) return fail(QXD_ERR_STATE, "qxd_wflow: a view shares its parent's gauge field; flow the parent");
    if (!lat->has_gauge) return fail(QXD_ERR_STATE, "qxd_wflow: needs qxd_set_gauge first");
    if (!std::isfinite(eps) || nsteps < 0) return fail(QXD_ERR_ARG, "qxd_wflow: finite eps and nsteps >= 0 required");
    if (nsteps == 0) return QXD_OK;
    const Geom& g = lat->g;
    const size_t V = (size_t)g.V;
    const int cstar1 = (lat->cstar_mask & 2u) ? 1 : 0;
    const int nphys = cstar1 ? g.V / 2 : g.V;
    double2* Ubuf = nullptr;
    double *Abuf = nullptr, *X = nullptr, *Xa = nullptr;
    int rc;
    if ((rc = dmalloc(&Ubuf, 36 * V, "cudaMalloc(flow links)")) || (rc = dmalloc(&Abuf, 4 * V, "cudaMalloc(flow angles)")) ||
        (rc = dmalloc(&X, 36 * V, "cudaMalloc(flow accumulator)")) ||
        (rc = dmalloc(&Xa, 4 * V, "cudaMalloc(flow accumulator)"))) {
        cudaFree(Ubuf);
        cudaFree(Abuf);
        cudaFree(X);
        cudaFree(Xa);
        return rc;
    }
    const double coef[3][2] = {{0.25, 0.0}, {8.0 / 9.0, -17.0 / 9.0}, {0.75, -1.0}};
    double2* Ucur = lat->U64;
    double2* Unext = Ubuf;
    double* Acur = lat->A64;
    double* Anext = Abuf;
    const int blocks = (4 * nphys + 127) / 128;
    cudaError_t e = cudaSuccess;
    for (int step = 0; step < nsteps && e == cudaSuccess; ++step)
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            FlowStage f{g, cstar1, nphys, Ucur, Unext, Acur, Anext, X, Xa, coef[k][0] * eps, coef[k][1]};
            k_wflow_stage<<<blocks, 128, 0, lat->stream>>>(f);
            e = cudaGetLastError();
            std::swap(Ucur, Unext);
            std::swap(Acur, Anext);
        }
    if (e == cudaSuccess && Ucur != lat->U64) {
        e = cudaMemcpyAsync(lat->U64, Ucur, 36 * V * sizeof(double2), cudaMemcpyDeviceToDevice, lat->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(lat->A64, Acur, 4 * V * sizeof(double), cudaMemcpyDeviceToDevice, lat->stream);
    }
    if (e == cudaSuccess) {
        k_gauge_derive<<<(g.V + 127) / 128, 128, 0, lat->stream>>>(g, lat->U64, lat->A64, lat->U32, lat->Z64,
                                                                   lat->A32);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    cudaFree(Ubuf);
    cudaFree(Abuf);
    cudaFree(X);
    cudaFree(Xa);
    // the clover terms of this lattice and its views are now stale
    ++lat->gauge_version;
    if (e != cudaSuccess) {
        // the field may be part-way through a step: unusable until set again
        lat->has_gauge = false;
        return cuda_fail(e, "qxd_wflow");
    }
    if ((rc = launch_field_tensor(lat))) {
        lat->has_gauge = false;
        return rc;
    }
    e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess) {
        lat->has_gauge = false;
        return cuda_fail(e, "qxd_wflow: field tensor");
    }
    return QXD_OK;
}

}  // extern "C"
