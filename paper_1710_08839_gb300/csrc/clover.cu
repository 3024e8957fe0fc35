// Site-diagonal part of D: M(x) = (4 + m0) + dDsw(x) (Eqs. (16), (21)) as two
// Hermitian 6x6 blocks per site, and their inverses (Doo^-1 of Sec. 2.4).
//
// In the chiral basis sigma_0k = diag(s_k, -s_k) and sigma_ij =
// -eps_ijk diag(s_k, s_k), so with X_munu = csw F_hat_munu + cswqed qhat
// (i/4) Im{4 plaquettes} (anti-Hermitian 3x3) the sum over mu, nu of
// (i/4) sigma_munu X_munu is block diagonal:
//   block +/- = (i/2) sum_k s_k (x) Y_k,  Y_k = +/- X_0k - E_k,
//   E_1 = X_23, E_2 = X_31, E_3 = X_12,
// i.e. (1/2) [[ i Y3, i Y1 + Y2 ], [ i Y1 - Y2, -i Y3 ]] on (spin a, colour).
#include "qxd_internal.cuh"

namespace qxd {

namespace {

using C64 = cplx<double>;

struct AH3 {  // anti-Hermitian 3x3
    C64 a[3][3];
};

__device__ __forceinline__ AH3 load_plane(const double* __restrict__ F, size_t V, int s, int plane,
                                          double csw, double u1) {
    const double* f = F + (size_t)plane * 10 * V + s;
    AH3 X;
    double im_u1 = u1 * f[9 * V];
    X.a[0][0] = mk(0.0, csw * f[0] + im_u1);
    X.a[1][1] = mk(0.0, csw * f[1 * V] + im_u1);
    X.a[2][2] = mk(0.0, csw * f[2 * V] + im_u1);
    X.a[0][1] = mk(csw * f[3 * V], csw * f[4 * V]);
    X.a[0][2] = mk(csw * f[5 * V], csw * f[6 * V]);
    X.a[1][2] = mk(csw * f[7 * V], csw * f[8 * V]);
    X.a[1][0] = -conj(X.a[0][1]);
    X.a[2][0] = -conj(X.a[0][2]);
    X.a[2][1] = -conj(X.a[1][2]);
    return X;
}

__device__ __forceinline__ double cabs2(C64 a) { return a.re * a.re + a.im * a.im; }

// Gauss-Jordan inverse with partial pivoting; false if singular/non-finite.
__device__ bool invert6(const C64 H[6][6], C64 B[6][6]) {
    C64 A[6][6];
    double nrm = 0.0;
    for (int i = 0; i < 6; ++i) {
        double rs = 0.0;
        for (int j = 0; j < 6; ++j) {
            A[i][j] = H[i][j];
            B[i][j] = mk(i == j ? 1.0 : 0.0, 0.0);
            rs += sqrt(cabs2(H[i][j]));
        }
        nrm = fmax(nrm, rs);
    }
    if (!isfinite(nrm) || nrm == 0.0) return false;
    for (int k = 0; k < 6; ++k) {
        int piv = k;
        double best = cabs2(A[k][k]);
        for (int i = k + 1; i < 6; ++i) {
            double v = cabs2(A[i][k]);
            if (v > best) {
                best = v;
                piv = i;
            }
        }
        if (!(sqrt(best) >= 1e-12 * nrm)) return false;
        if (piv != k)
            for (int j = 0; j < 6; ++j) {
                C64 t = A[k][j];
                A[k][j] = A[piv][j];
                A[piv][j] = t;
                t = B[k][j];
                B[k][j] = B[piv][j];
                B[piv][j] = t;
            }
        C64 d = A[k][k];
        double id = 1.0 / cabs2(d);
        C64 inv = mk(d.re * id, -d.im * id);
        for (int j = 0; j < 6; ++j) {
            A[k][j] = A[k][j] * inv;
            B[k][j] = B[k][j] * inv;
        }
        for (int i = 0; i < 6; ++i) {
            if (i == k) continue;
            C64 f = A[i][k];
            for (int j = 0; j < 6; ++j) {
                A[i][j] = A[i][j] - f * A[k][j];
                B[i][j] = B[i][j] - f * B[k][j];
            }
        }
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j)
            if (!isfinite(B[i][j].re) || !isfinite(B[i][j].im)) return false;
    return true;
}

// LDL^H factorisation of a Hermitian 6x6 block (packed: real diagonal d,
// strictly lower L row major) and its inverse, all in registers:
// A = L D L^H, A^-1 = M^H D^-1 M with M = L^-1. Returns false when a pivot
// falls below 1e-12 of the block norm (the caller then uses Gauss-Jordan
// with pivoting, which decides singularity).
__device__ __forceinline__ int lidx6(int i, int j) { return i * (i - 1) / 2 + j; }  // i > j

__device__ __forceinline__ bool ldl_inverse6(const double a_d[6], const C64 a_l[15], double nrm, double i_d[6],
                                             C64 i_l[15]) {
    double D[6];
    C64 L[15];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        double dj = a_d[j];
#pragma unroll
        for (int k = 0; k < j; ++k) dj -= cabs2(L[lidx6(j, k)]) * D[k];
        if (!(fabs(dj) >= 1e-12 * nrm)) return false;
        D[j] = dj;
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
            C64 v = a_l[lidx6(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) v = v - D[k] * mulc(L[lidx6(i, k)], L[lidx6(j, k)]);
            L[lidx6(i, j)] = (1.0 / dj) * v;
        }
    }
    // M = L^-1 (unit lower triangular)
    C64 M[15];
#pragma unroll
    for (int j = 0; j < 6; ++j)
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
            C64 v = -L[lidx6(i, j)];
#pragma unroll
            for (int k = j + 1; k < i; ++k) v = v - L[lidx6(i, k)] * M[lidx6(k, j)];
            M[lidx6(i, j)] = v;
        }
    // (A^-1)_ij = sum_{k >= i} conj(M_ki) M_kj / D_k for i >= j (M_kk = 1)
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double v = 1.0 / D[i];
#pragma unroll
        for (int k = i + 1; k < 6; ++k) v += cabs2(M[lidx6(k, i)]) / D[k];
        i_d[i] = v;
#pragma unroll
        for (int j = 0; j < i; ++j) {
            C64 w = (1.0 / D[i]) * M[lidx6(i, j)];
#pragma unroll
            for (int k = i + 1; k < 6; ++k) w = w + (1.0 / D[k]) * cmul(M[lidx6(k, i)], M[lidx6(k, j)]);
            i_l[lidx6(i, j)] = w;
        }
    }
    for (int i = 0; i < 6; ++i)
        if (!isfinite(i_d[i])) return false;
    return true;
}

__device__ __forceinline__ void store_packed(const double d[6], const C64 l[15], int blk, double* __restrict__ C64p,
                                             float4* __restrict__ C32p, size_t V, int s) {
    double v[36];
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = d[i];
#pragma unroll
    for (int k = 0; k < 15; ++k) {
        v[6 + 2 * k] = l[k].re;
        v[7 + 2 * k] = l[k].im;
    }
#pragma unroll
    for (int r = 0; r < 36; ++r) C64p[(size_t)(36 * blk + r) * V + s] = v[r];
#pragma unroll
    for (int q = 0; q < 9; ++q)
        C32p[(size_t)(9 * blk + q) * V + s] =
            make_float4((float)v[4 * q], (float)v[4 * q + 1], (float)v[4 * q + 2], (float)v[4 * q + 3]);
}

// one thread per (site, block): assemble the block from the field tensors,
// store it, invert it (LDL^H, Gauss-Jordan with pivoting as the fallback)
__global__ void __launch_bounds__(128) k_clover_build(Geom g, const double* __restrict__ F, double m0,
                                                      double csw, double u1coef, double* __restrict__ C64p,
                                                      float4* __restrict__ C32p, double* __restrict__ Ci64,
                                                      float4* __restrict__ Ci32, int* __restrict__ bad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * g.V) return;
    const int s = t >> 1, blk = t & 1;
    const size_t V = (size_t)g.V;
    const double sg = blk == 0 ? 1.0 : -1.0;
    // planes: 0:(0,1) 1:(0,2) 2:(0,3) 3:(1,2) 4:(1,3) 5:(2,3)
    AH3 Y1, Y2, Y3;
    {
        AH3 X0 = load_plane(F, V, s, 0, csw, u1coef), X5 = load_plane(F, V, s, 5, csw, u1coef);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) Y1.a[a][b] = sg * X0.a[a][b] - X5.a[a][b];  // E1 = X23
    }
    {
        AH3 X1 = load_plane(F, V, s, 1, csw, u1coef), X4 = load_plane(F, V, s, 4, csw, u1coef);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) Y2.a[a][b] = sg * X1.a[a][b] + X4.a[a][b];  // E2 = X31 = -X13
    }
    {
        AH3 X2 = load_plane(F, V, s, 2, csw, u1coef), X3 = load_plane(F, V, s, 3, csw, u1coef);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) Y3.a[a][b] = sg * X2.a[a][b] - X3.a[a][b];  // E3 = X12
    }
    // packed Hermitian block (1/2) [[ i Y3, i Y1 + Y2 ], [ i Y1 - Y2, -i Y3 ]] + (4 + m0)
    double d[6];
    C64 l[15];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const int a = i % 3, sa = i / 3;
        const C64 yy = sa == 0 ? 0.5 * times_i(Y3.a[a][a]) : 0.5 * times_mi(Y3.a[a][a]);
        d[i] = 4.0 + m0 + yy.re;
#pragma unroll
        for (int j = 0; j < i; ++j) {
            const int b = j % 3, sb = j / 3;
            C64 h;
            if (sa == sb) h = sa == 0 ? 0.5 * times_i(Y3.a[a][b]) : 0.5 * times_mi(Y3.a[a][b]);
            else h = 0.5 * (times_i(Y1.a[a][b]) - Y2.a[a][b]);  // lower-left block (sa = 1, sb = 0)
            l[lidx6(i, j)] = h;
        }
    }
    store_packed(d, l, blk, C64p, C32p, V, s);
    double nrm = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double rs = fabs(d[i]);
#pragma unroll
        for (int j = 0; j < 6; ++j)
            if (j != i) rs += sqrt(cabs2(i > j ? l[lidx6(i, j)] : l[lidx6(j, i)]));
        nrm = fmax(nrm, rs);
    }
    double id[6];
    C64 il[15];
    bool ok = isfinite(nrm) && nrm > 0.0 && ldl_inverse6(d, l, nrm, id, il);
    if (!ok) {
        C64 H[6][6], Hi[6][6];
        for (int i = 0; i < 6; ++i) {
            H[i][i] = mk(d[i], 0.0);
            for (int j = 0; j < i; ++j) {
                H[i][j] = l[lidx6(i, j)];
                H[j][i] = conj(l[lidx6(i, j)]);
            }
        }
        ok = invert6(H, Hi);
        for (int i = 0; i < 6; ++i) {
            id[i] = ok ? Hi[i][i].re : 0.0;
            for (int j = 0; j < i; ++j) il[lidx6(i, j)] = ok ? Hi[i][j] : mk(0.0, 0.0);
        }
        if (!ok) atomicAdd(&bad[0], 1);
    }
    store_packed(id, il, blk, Ci64, Ci32, V, s);
}

// z^qhat per link from z = exp(i A) (binary powering; |z| = 1 so z^-n = conj(z^n))
__global__ void k_link_phases(int n, const double2* __restrict__ Z, int qhat, double2* __restrict__ Zq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    C64 b = mk(Z[i].x, Z[i].y), r = mk(1.0, 0.0);
    int m = qhat < 0 ? -qhat : qhat;
    while (m) {
        if (m & 1) r = r * b;
        b = b * b;
        m >>= 1;
    }
    if (qhat < 0) r = conj(r);
    Zq[i] = make_double2(r.re, r.im);
}

}  // namespace

int launch_clover_build(qxd_lattice* lat, int* d_bad) {
    const Geom& g = lat->g;
    QXD_CUDA(cudaMemsetAsync(d_bad, 0, 16, lat->stream));
    // U(1) part of X: cswqed * qhat * (i/4) Im{sum of 4 plaquettes}
    const double u1coef = lat->cswqed * (double)lat->qhat * 0.25;
    int blocks = (2 * g.V + 127) / 128;
    k_clover_build<<<blocks, 128, 0, lat->stream>>>(g, lat->ftens, lat->m0, lat->csw, u1coef, lat->C64,
                                                    lat->C32, lat->Cinv64, lat->Cinv32, d_bad);
    QXD_LAUNCHED("k_clover_build");
    const int nl = 4 * g.V;
    k_link_phases<<<(nl + 255) / 256, 256, 0, lat->stream>>>(nl, lat->Z64, lat->qhat, lat->Zq64);
    QXD_LAUNCHED("k_link_phases");
    return QXD_OK;
}

}  // namespace qxd
