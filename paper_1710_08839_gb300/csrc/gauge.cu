// Gauge-field ingest (orbifold mirror, Eq. (4a); SU(3) check; FP64 and FP32
// 2-row layouts) and the clover field tensors of the SW term (Eqs. (21)-(23)).
#include "su3.cuh"

namespace qxd {

namespace {

__global__ void k_gauge_ingest(Geom g, int L1phys, int cstar1, const double* __restrict__ su3,
                               const double* __restrict__ ang, int extended, double2* __restrict__ U64,
                               float4* __restrict__ U32, double* __restrict__ A64,
                               double2* __restrict__ Z64, float4* __restrict__ A32,
                               int* __restrict__ bad) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int x0, x1, x2, x3;
    native_coords(g, s, x0, x1, x2, x3);
    bool mirror = false;
    size_t src;
    if (extended) {
        src = (size_t)lex_index(g, x0, x1, x2, x3);
    } else {
        int px1 = x1;
        if (cstar1 && x1 >= g.L1) {  // Eq. (4a): mirror half from the physical half
            px1 = x1 - g.L1;
            mirror = true;
        }
        src = (((size_t)x0 * L1phys + px1) * g.N2 + x2) * g.N3 + x3;
    }
    const size_t V = (size_t)g.V;
    float a32[4];
    int nbad = 0;
    for (int mu = 0; mu < 4; ++mu) {
        const double* p = su3 + (src * 4 + mu) * 18;
        C64 u[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                u[i][j] = mk(p[(i * 3 + j) * 2], p[(i * 3 + j) * 2 + 1]);
                if (mirror) u[i][j] = conj(u[i][j]);
            }
        double a = ang[src * 4 + mu];
        if (mirror) a = -a;
        // SU(3) check: |U U^+ - 1| and |det U - 1|
        double dev = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                C64 s2 = mulc(u[i][0], u[j][0]) + mulc(u[i][1], u[j][1]) + mulc(u[i][2], u[j][2]);
                double re = s2.re - (i == j ? 1.0 : 0.0);
                dev = fmax(dev, fmax(fabs(re), fabs(s2.im)));
            }
        C64 det = u[0][0] * (u[1][1] * u[2][2] - u[1][2] * u[2][1]) -
                  u[0][1] * (u[1][0] * u[2][2] - u[1][2] * u[2][0]) +
                  u[0][2] * (u[1][0] * u[2][1] - u[1][1] * u[2][0]);
        dev = fmax(dev, fmax(fabs(det.re - 1.0), fabs(det.im)));
        if (!(dev <= 1e-10) || !isfinite(a)) ++nbad;
#pragma unroll
        for (int e = 0; e < 9; ++e) U64[((size_t)mu * 9 + e) * V + s] = make_double2(u[e / 3][e % 3].re, u[e / 3][e % 3].im);
        U32[((size_t)mu * 3 + 0) * V + s] =
            make_float4((float)u[0][0].re, (float)u[0][0].im, (float)u[0][1].re, (float)u[0][1].im);
        U32[((size_t)mu * 3 + 1) * V + s] =
            make_float4((float)u[0][2].re, (float)u[0][2].im, (float)u[1][0].re, (float)u[1][0].im);
        U32[((size_t)mu * 3 + 2) * V + s] =
            make_float4((float)u[1][1].re, (float)u[1][1].im, (float)u[1][2].re, (float)u[1][2].im);
        A64[(size_t)mu * V + s] = a;
        double sa, ca;
        sincos(a, &sa, &ca);
        Z64[(size_t)mu * V + s] = make_double2(ca, sa);
        a32[mu] = (float)a;
    }
    A32[s] = make_float4(a32[0], a32[1], a32[2], a32[3]);
    if (nbad) atomicAdd(&bad[0], nbad);
}

// Extended input with the CHECKED flag: mirror site x (x1 >= L1) must hold
// U(x - L1 e1)^* and -A(x - L1 e1) (Eq. (4a)), compared on z = exp(iA).
__global__ void k_check_admissible(Geom g, const double* __restrict__ su3, const double* __restrict__ ang,
                                   int* __restrict__ bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    int x3 = i % g.N3, r = i / g.N3;
    int x2 = r % g.N2;
    r /= g.N2;
    int x1 = r % g.N1, x0 = r / g.N1;
    if (x1 < g.L1) return;
    size_t m = (size_t)i, p = (size_t)lex_index(g, x0, x1 - g.L1, x2, x3);
    int nbad = 0;
    for (int mu = 0; mu < 4; ++mu) {
        double dev = 0.0;
        for (int e = 0; e < 9; ++e) {
            double mre = su3[(m * 4 + mu) * 18 + 2 * e], mim = su3[(m * 4 + mu) * 18 + 2 * e + 1];
            double pre = su3[(p * 4 + mu) * 18 + 2 * e], pim = su3[(p * 4 + mu) * 18 + 2 * e + 1];
            dev = fmax(dev, fmax(fabs(mre - pre), fabs(mim + pim)));
        }
        double am = ang[m * 4 + mu], ap = ang[p * 4 + mu];
        double sm, cm, sp, cp;
        sincos(am, &sm, &cm);
        sincos(ap, &sp, &cp);
        dev = fmax(dev, fmax(fabs(cm - cp), fabs(sm + sp)));
        if (!(dev <= 1e-12)) ++nbad;
    }
    if (nbad) atomicAdd(&bad[1], nbad);
}

// Clover field tensors at one site (FP64): per plane mu < nu the SU(3)
// F_hat = (Q_munu - Q_munu^+)/8 with Q the four leaves through x (Q_numu =
// Q_munu^+), and the imaginary part of the sum of the four U(1) plaquettes
// z_munu(x) + z_munu(x-mu) + z_munu(x-nu) + z_munu(x-mu-nu) (Eqs. (22)-(23)).
__global__ void __launch_bounds__(128) k_field_tensor(Geom g, const double2* __restrict__ U64,
                                                      const double* __restrict__ A64,
                                                      double* __restrict__ F) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const size_t V = (size_t)g.V;
    int x[4];
    native_coords(g, s, x[0], x[1], x[2], x[3]);
    int plane = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
            int c[4];
            auto at = [&](int dm, int dn) {
                c[0] = x[0]; c[1] = x[1]; c[2] = x[2]; c[3] = x[3];
                if (dm) shift_coords(g, c, mu, dm);
                if (dn) shift_coords(g, c, nu, dn);
                return native_of(g, c);
            };
            const int sx = s, sxpm = at(1, 0), sxpn = at(0, 1), sxmm = at(-1, 0), sxmn = at(0, -1),
                      sxmmpn = at(-1, 1), sxpmmn = at(1, -1), sxmmmn = at(-1, -1);
            // leaf 1: U(x,mu) U(x+mu,nu) U(x+nu,mu)^+ U(x,nu)^+
            M3 Q = mul_nd(mul_nd(mul(load_link64(U64, V, mu, sx), load_link64(U64, V, nu, sxpm)),
                                 load_link64(U64, V, mu, sxpn)),
                          load_link64(U64, V, nu, sx));
            // leaf 2: U(x,nu) U(x-mu+nu,mu)^+ U(x-mu,nu)^+ U(x-mu,mu)
            M3 t = mul(mul_nd(mul_nd(load_link64(U64, V, nu, sx), load_link64(U64, V, mu, sxmmpn)),
                              load_link64(U64, V, nu, sxmm)),
                       load_link64(U64, V, mu, sxmm));
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) Q.a[i][j] = Q.a[i][j] + t.a[i][j];
            // leaf 3: U(x-mu,mu)^+ U(x-mu-nu,nu)^+ U(x-mu-nu,mu) U(x-nu,nu)
            t = mul(mul(mul_dn(load_link64(U64, V, mu, sxmm), dag(load_link64(U64, V, nu, sxmmmn))),
                        load_link64(U64, V, mu, sxmmmn)),
                    load_link64(U64, V, nu, sxmn));
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) Q.a[i][j] = Q.a[i][j] + t.a[i][j];
            // leaf 4: U(x-nu,nu)^+ U(x-nu,mu) U(x+mu-nu,nu) U(x,mu)^+
            t = mul_nd(mul(mul_dn(load_link64(U64, V, nu, sxmn), load_link64(U64, V, mu, sxmn)),
                           load_link64(U64, V, nu, sxpmmn)),
                       load_link64(U64, V, mu, sx));
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) Q.a[i][j] = Q.a[i][j] + t.a[i][j];
            // F = (Q - Q^+)/8, anti-Hermitian
            double* f = F + (size_t)plane * 10 * V + s;
            f[0 * V] = (Q.a[0][0].im + Q.a[0][0].im) * 0.125;
            f[1 * V] = (Q.a[1][1].im + Q.a[1][1].im) * 0.125;
            f[2 * V] = (Q.a[2][2].im + Q.a[2][2].im) * 0.125;
            C64 f01 = 0.125 * (Q.a[0][1] - conj(Q.a[1][0]));
            C64 f02 = 0.125 * (Q.a[0][2] - conj(Q.a[2][0]));
            C64 f12 = 0.125 * (Q.a[1][2] - conj(Q.a[2][1]));
            f[3 * V] = f01.re;
            f[4 * V] = f01.im;
            f[5 * V] = f02.re;
            f[6 * V] = f02.im;
            f[7 * V] = f12.re;
            f[8 * V] = f12.im;
            // U(1): z_munu(y) = exp(i (A(y,mu) + A(y+mu,nu) - A(y+nu,mu) - A(y,nu)))
            auto zplaq = [&](int y, int ypm, int ypn) {
                return sin(A64[(size_t)mu * V + y] + A64[(size_t)nu * V + ypm] -
                           A64[(size_t)mu * V + ypn] - A64[(size_t)nu * V + y]);
            };
            double im = zplaq(sx, sxpm, sxpn) + zplaq(sxmm, sx, sxmmpn) + zplaq(sxmn, sxpmmn, sx) +
                        zplaq(sxmmmn, sxmn, sxmm);
            f[9 * V] = im;
        }
}

}  // namespace

int launch_gauge_ingest(qxd_lattice* lat, const double* su3, const double* ang, int kind, int* d_bad) {
    const Geom& g = lat->g;
    QXD_CUDA(cudaMemsetAsync(d_bad, 0, 16, lat->stream));
    const int extended = kind != QXD_GAUGE_PHYSICAL_HALF;
    const int cstar1 = (lat->cstar_mask & 2u) ? 1 : 0;
    int blocks = (g.V + 127) / 128;
    k_gauge_ingest<<<blocks, 128, 0, lat->stream>>>(g, lat->L1, cstar1, su3, ang, extended, lat->U64,
                                                    lat->U32, lat->A64, lat->Z64, lat->A32, d_bad);
    QXD_LAUNCHED("k_gauge_ingest");
    if (kind == QXD_GAUGE_EXTENDED_CHECKED && cstar1) {
        k_check_admissible<<<blocks, 128, 0, lat->stream>>>(g, su3, ang, d_bad);
        QXD_LAUNCHED("k_check_admissible");
    }
    return QXD_OK;
}

int launch_field_tensor(qxd_lattice* lat) {
    const Geom& g = lat->g;
    int blocks = (g.V + 127) / 128;
    k_field_tensor<<<blocks, 128, 0, lat->stream>>>(g, lat->U64, lat->A64, lat->ftens);
    QXD_LAUNCHED("k_field_tensor");
    return QXD_OK;
}

}  // namespace qxd
