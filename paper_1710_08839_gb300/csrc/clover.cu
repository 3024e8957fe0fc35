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

__device__ __forceinline__ void build_block(C64 H[6][6], const AH3& Y1, const AH3& Y2, const AH3& Y3,
                                            double diag) {
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            // (1/2) [[ i Y3, i Y1 + Y2 ], [ i Y1 - Y2, -i Y3 ]]
            H[a][b] = 0.5 * times_i(Y3.a[a][b]);
            H[a][3 + b] = 0.5 * (times_i(Y1.a[a][b]) + Y2.a[a][b]);
            H[3 + a][b] = 0.5 * (times_i(Y1.a[a][b]) - Y2.a[a][b]);
            H[3 + a][3 + b] = 0.5 * times_mi(Y3.a[a][b]);
        }
    for (int i = 0; i < 6; ++i) H[i][i] = H[i][i] + mk(diag, 0.0);
}

__device__ __forceinline__ void store_block(const C64 H[6][6], int blk, double* __restrict__ C64p,
                                            float4* __restrict__ C32p, size_t V, int s) {
    float vals[36];
    for (int i = 0; i < 6; ++i) vals[i] = (float)H[i][i].re;
    int k = 0;
    for (int i = 1; i < 6; ++i)
        for (int j = 0; j < i; ++j, ++k) {
            vals[6 + 2 * k] = (float)H[i][j].re;
            vals[6 + 2 * k + 1] = (float)H[i][j].im;
        }
    double dv[36];
    for (int i = 0; i < 6; ++i) dv[i] = H[i][i].re;
    k = 0;
    for (int i = 1; i < 6; ++i)
        for (int j = 0; j < i; ++j, ++k) {
            dv[6 + 2 * k] = H[i][j].re;
            dv[6 + 2 * k + 1] = H[i][j].im;
        }
    for (int r = 0; r < 36; ++r) C64p[(size_t)(36 * blk + r) * V + s] = dv[r];
    for (int q = 0; q < 9; ++q)
        C32p[(size_t)(9 * blk + q) * V + s] =
            make_float4(vals[4 * q], vals[4 * q + 1], vals[4 * q + 2], vals[4 * q + 3]);
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

__global__ void __launch_bounds__(128) k_clover_build(Geom g, const double* __restrict__ F, double m0,
                                                      double csw, double u1coef, double* __restrict__ C64p,
                                                      float4* __restrict__ C32p, double* __restrict__ Ci64,
                                                      float4* __restrict__ Ci32, int* __restrict__ bad) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const size_t V = (size_t)g.V;
    // planes: 0:(0,1) 1:(0,2) 2:(0,3) 3:(1,2) 4:(1,3) 5:(2,3)
    AH3 X[6];
    for (int p = 0; p < 6; ++p) X[p] = load_plane(F, V, s, p, csw, u1coef);
    int nbad = 0;
    for (int blk = 0; blk < 2; ++blk) {
        const double sg = blk == 0 ? 1.0 : -1.0;
        AH3 Y1, Y2, Y3;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                Y1.a[a][b] = sg * X[0].a[a][b] - X[5].a[a][b];  // E1 = X23
                Y2.a[a][b] = sg * X[1].a[a][b] + X[4].a[a][b];  // E2 = X31 = -X13
                Y3.a[a][b] = sg * X[2].a[a][b] - X[3].a[a][b];  // E3 = X12
            }
        C64 H[6][6], Hi[6][6];
        build_block(H, Y1, Y2, Y3, 4.0 + m0);
        store_block(H, blk, C64p, C32p, V, s);
        if (!invert6(H, Hi)) {
            ++nbad;
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) Hi[i][j] = mk(0.0, 0.0);
        }
        store_block(Hi, blk, Ci64, Ci32, V, s);
    }
    if (nbad) atomicAdd(&bad[0], nbad);
}

}  // namespace

int launch_clover_build(qxd_lattice* lat, int* d_bad) {
    const Geom& g = lat->g;
    QXD_CUDA(cudaMemsetAsync(d_bad, 0, 16, lat->stream));
    // U(1) part of X: cswqed * qhat * (i/4) Im{sum of 4 plaquettes}
    const double u1coef = lat->cswqed * (double)lat->qhat * 0.25;
    int blocks = (g.V + 127) / 128;
    k_clover_build<<<blocks, 128, 0, lat->stream>>>(g, lat->ftens, lat->m0, lat->csw, u1coef, lat->C64,
                                                    lat->C32, lat->Cinv64, lat->Cinv32, d_bad);
    QXD_LAUNCHED("k_clover_build");
    return QXD_OK;
}

}  // namespace qxd
