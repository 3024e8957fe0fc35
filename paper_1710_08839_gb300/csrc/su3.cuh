// FP64 3x3 complex matrices and link/neighbour access of the gauge field
// (links in the native layout U64[mu][9][V], site coordinates on the
// simulated lattice with the shifted C* boundaries).
#pragma once

#include "qxd_internal.cuh"

namespace qxd {

namespace {

using C64 = cplx<double>;

struct M3 {
    C64 a[3][3];
};

__device__ __forceinline__ M3 mul(const M3& x, const M3& y) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            C64 s = x.a[i][0] * y.a[0][j];
            s = s + x.a[i][1] * y.a[1][j];
            s = s + x.a[i][2] * y.a[2][j];
            r.a[i][j] = s;
        }
    return r;
}

// x * y^+
__device__ __forceinline__ M3 mul_nd(const M3& x, const M3& y) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            C64 s = mulc(x.a[i][0], y.a[j][0]);
            s = s + mulc(x.a[i][1], y.a[j][1]);
            s = s + mulc(x.a[i][2], y.a[j][2]);
            r.a[i][j] = s;
        }
    return r;
}

// x^+ * y
__device__ __forceinline__ M3 mul_dn(const M3& x, const M3& y) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            C64 s = cmul(x.a[0][i], y.a[0][j]);
            s = s + cmul(x.a[1][i], y.a[1][j]);
            s = s + cmul(x.a[2][i], y.a[2][j]);
            r.a[i][j] = s;
        }
    return r;
}

__device__ __forceinline__ M3 dag(const M3& x) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.a[i][j] = conj(x.a[j][i]);
    return r;
}

__device__ __forceinline__ M3 load_link64(const double2* __restrict__ U64, size_t V, int mu, int s) {
    M3 m;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        double2 v = U64[((size_t)mu * 9 + e) * V + s];
        m.a[e / 3][e % 3] = mk(v.x, v.y);
    }
    return m;
}

__device__ __forceinline__ void shift_coords(const Geom& g, int c[4], int mu, int dir) {
    const int N[4] = {g.N0, g.N1, g.N2, g.N3};
    int v = c[mu] + dir;
    bool crossed = (v == N[mu]) || (v < 0);
    c[mu] = crossed ? (dir > 0 ? 0 : N[mu] - 1) : v;
    if (crossed && ((mu == 2 && g.cs2) || (mu == 3 && g.cs3))) {
        c[1] += g.L1;
        if (c[1] >= g.N1) c[1] -= g.N1;
    }
}

__device__ __forceinline__ int native_of(const Geom& g, const int c[4]) {
    int lex = lex_index(g, c[0], c[1], c[2], c[3]);
    return native_index(g, lex, (c[0] + c[1] + c[2] + c[3]) & 1);
}

}  // namespace

}  // namespace qxd
