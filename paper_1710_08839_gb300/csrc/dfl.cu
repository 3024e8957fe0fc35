// Local deflation of the SAP-preconditioned GCR solver (openQ*D's
// deflation-accelerated solver, named in Sec. 1 and Table 2; Luscher's local
// deflation).
//
// * Subspace: Ns global FP32 fields psi_k, smoothed by SAP applications
//   (inverse iteration on the low modes), each pass followed by block-wise
//   orthonormalisation on the 4^4 blocks of the Schwarz method: the fields
//   restricted to a block are orthonormalised in order (modified
//   Gram-Schmidt), giving phi_{b,k}; phi_k = sum_b phi_{b,k} is stored as one
//   native FP32 field.
// * Little operator: A_{b,j}[k][l] = <phi_{b,k}, D phi_{n_j(b),l}> for
//   n_0(b) = b and n_{1+2mu}(b) = b + mu, n_{2+2mu}(b) = b - mu (block
//   neighbours; across a shifted C* boundary the block coordinate b1 moves by
//   L1/4 like the sites). For each l: T = D phi_l (the FP32 operator) and the
//   hop of every face site out of its block (H_mu), then per block and k the
//   projections <phi_{b,k}, T>_b and <phi_{b,k}, H_mu>_face give
//   A_{b,b+-mu} directly and A_{b,b} = <phi_{b,k}, T>_b - sum of the faces.
// * Preconditioner: M eta = chi + M_SAP(eta - D chi), chi = P A^-1 P^dag eta,
//   with the little system solved by GCR to a relative residual dfl_tol.
//   The little GCR runs on the device: every coefficient (Gram-Schmidt
//   projections, norms, step lengths) goes from the reduction that makes it
//   to the kernels that use it through device memory, a restart cycle of
//   DFL_NKV steps is one CUDA graph, and the host reads the solver state
//   once per cycle.
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "blas.cuh"
#include "dfl.cuh"
#include "dirac_common.cuh"
#include "solver.cuh"

namespace qxd {

namespace {

constexpr int BS = 4;        // block size (the Schwarz blocks)
constexpr int BSITES = 256;  // sites per block = threads per block of the kernels below

// block b (lexicographic in block coordinates, B3 fastest) and local site t
// (lexicographic in the block, x3 fastest) -> global coordinates
__device__ __forceinline__ void block_site(const Geom& g, const DflGeom& d, int b, int t, int x[4]) {
    int B3 = b % d.nb[3];
    int r = b / d.nb[3];
    int B2 = r % d.nb[2];
    r /= d.nb[2];
    int B1 = r % d.nb[1];
    int B0 = r / d.nb[1];
    x[0] = BS * B0 + ((t >> 6) & 3);
    x[1] = BS * B1 + ((t >> 4) & 3);
    x[2] = BS * B2 + ((t >> 2) & 3);
    x[3] = BS * B3 + (t & 3);
}

__device__ __forceinline__ int native_at(const Geom& g, const int x[4]) {
    return native_index(g, lex_index(g, x[0], x[1], x[2], x[3]), (x[0] + x[1] + x[2] + x[3]) & 1);
}

// neighbour block of b in direction mu (dir = +1 or -1)
__device__ __forceinline__ int block_nbr(const Geom& g, const DflGeom& d, int b, int mu, int dir) {
    int B[4];
    B[3] = b % d.nb[3];
    int r = b / d.nb[3];
    B[2] = r % d.nb[2];
    r /= d.nb[2];
    B[1] = r % d.nb[1];
    B[0] = r / d.nb[1];
    int v = B[mu] + dir;
    const bool crossed = v < 0 || v >= d.nb[mu];
    B[mu] = (v + d.nb[mu]) % d.nb[mu];
    if (crossed && ((mu == 2 && g.cs2) || (mu == 3 && g.cs3))) B[1] = (B[1] + g.L1 / BS) % d.nb[1];
    return ((B[0] * d.nb[1] + B[1]) * d.nb[2] + B[2]) * d.nb[3] + B[3];
}

// conj(a) . b over 12 complex numbers
__device__ __forceinline__ void cdot12(const cplx<float> a[12], const cplx<float> b[12], double& re, double& im) {
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        re += (double)a[i].re * b[i].re + (double)a[i].im * b[i].im;
        im += (double)a[i].re * b[i].im - (double)a[i].im * b[i].re;
    }
}

// block-wide sum of NV doubles (BSITES threads); result valid in every thread
template <int NV>
__device__ __forceinline__ void block_sum(double v[NV], double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        double x = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[warp * NV + c] = x;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        double x = 0.0;
        for (int w = 0; w < BSITES / 32; ++w) x += sh[w * NV + c];
        v[c] = x;
    }
    __syncthreads();
}

// Warp sum of 32 FP32 values per lane by recursive halving: at the level
// with lane offset o each lane keeps one half of its values, adds the
// partner's copy of that half and sends the other half, so that after five
// levels (31 shuffles) lane l holds the sum over the warp of value l. The
// tree is fixed, so the sum is deterministic.
__device__ __forceinline__ float warp_reduce_scatter32(float v[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int lev = 0; lev < 5; ++lev) {
        const int o = 16 >> lev, n = 16 >> lev;  // lane offset, values kept
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < n; ++i) {
            const float send = hi ? v[i] : v[i + n];
            const float keep = hi ? v[i + n] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

// ---------------------------------------------------------------------------
// random fields and block orthonormalisation
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Gaussian FP32 entries (Box-Muller on two 24-bit uniforms per complex entry)
__global__ void k_dfl_random(size_t n, unsigned long long seed, float2* __restrict__ out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long h = splitmix64(seed ^ splitmix64(i));
        const float u1 = ((float)(h >> 40) + 1.0f) * (1.0f / 16777217.0f);
        const float u2 = (float)((h >> 16) & 0xFFFFFF) * (1.0f / 16777216.0f);
        const float rr = sqrtf(-2.0f * logf(u1));
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        out[i] = make_float2(rr * cs, rr * sn);
    }
}

// modified Gram-Schmidt of the ns fields restricted to each block; bad[0]
// counts blocks where a field became (numerically) dependent
__global__ void __launch_bounds__(BSITES) k_dfl_orth(Geom g, DflGeom d, int ns, float4* __restrict__ basis,
                                                     int* __restrict__ bad) {
    __shared__ double sh[(BSITES / 32) * 2];
    const int b = blockIdx.x;
    int x[4];
    block_site(g, d, b, threadIdx.x, x);
    const int s = native_at(g, x);
    const size_t V = (size_t)g.V;
    for (int k = 0; k < ns; ++k) {
        cplx<float> v[12];
        load_spinor(basis + (size_t)k * 6 * V, g.V, s, v);
        for (int l = 0; l < k; ++l) {
            cplx<float> u[12];
            load_spinor(basis + (size_t)l * 6 * V, g.V, s, u);
            double c[2] = {0.0, 0.0};
            cdot12(u, v, c[0], c[1]);
            block_sum<2>(c, sh);
            const float cr = (float)c[0], ci = (float)c[1];
#pragma unroll
            for (int i = 0; i < 12; ++i)
                v[i] = mk(v[i].re - (cr * u[i].re - ci * u[i].im), v[i].im - (cr * u[i].im + ci * u[i].re));
        }
        double n2[1] = {0.0};
#pragma unroll
        for (int i = 0; i < 12; ++i) n2[0] += (double)v[i].re * v[i].re + (double)v[i].im * v[i].im;
        block_sum<1>(n2, sh);
        const bool ok = n2[0] > 1e-30 && isfinite(n2[0]);
        const float inv = ok ? (float)(1.0 / sqrt(n2[0])) : 0.0f;
        if (!ok && threadIdx.x == 0) atomicAdd(bad, 1);
#pragma unroll
        for (int i = 0; i < 12; ++i) v[i] = mk(v[i].re * inv, v[i].im * inv);
        store_spinor(basis + (size_t)k * 6 * V, g.V, s, v);
    }
}

// ---------------------------------------------------------------------------
// little operator
// ---------------------------------------------------------------------------

// one hop of direction MU, DIR = +1 (forward) or -1 (backward), raw (without
// the factor -1/2) as a full spinor: (1 -+ g_mu) W psi(x +- mu)
template <bool QNZ, int MU, int DIR>
__device__ __forceinline__ void dfl_hop(const Geom& g, const Fields<float>& f, const float4* __restrict__ psi,
                                        float q, int x0, int x1, int x2, int x3, int s, int po,
                                        cplx<float> out[12]) {
    cplx<float> v[12], h0[3], h1[3], g0[3], g1[3], u[3][3];
#pragma unroll
    for (int i = 0; i < 12; ++i) out[i] = mk(0.f, 0.f);
    const int sn = native_index(g, neighbour_lex<MU, DIR>(g, x0, x1, x2, x3), po);
    load_spinor(psi, g.V, sn, v);
    project<float, MU, DIR>(v, h0, h1);
    if (DIR > 0) {
        load_link(f.U, g.V, MU, s, u);
        su3_mul(u, h0, g0);
        su3_mul(u, h1, g1);
        if (QNZ) {
            cplx<float> ph = link_phase(f.A, g.V, MU, s, q);
            times3(ph, g0);
            times3(ph, g1);
        }
    } else {
        load_link(f.U, g.V, MU, sn, u);
        su3_dag_mul(u, h0, g0);
        su3_dag_mul(u, h1, g1);
        if (QNZ) {
            cplx<float> ph = conj(link_phase(f.A, g.V, MU, sn, q));
            times3(ph, g0);
            times3(ph, g1);
        }
    }
    accumulate<float, MU, DIR>(out, g0, g1);
}

template <bool QNZ, int MU>
__device__ __forceinline__ void face_hop(const Geom& g, const Fields<float>& f, const float4* psi, float q,
                                         const int x[4], int s, int po, float4* __restrict__ H) {
    const int l = x[MU] & (BS - 1);
    cplx<float> h[12];
    if (l == BS - 1) dfl_hop<QNZ, MU, +1>(g, f, psi, q, x[0], x[1], x[2], x[3], s, po, h);
    else if (l == 0) dfl_hop<QNZ, MU, -1>(g, f, psi, q, x[0], x[1], x[2], x[3], s, po, h);
    else {
#pragma unroll
        for (int i = 0; i < 12; ++i) h[i] = mk(0.f, 0.f);
    }
    // the factor -1/2 of the hopping term
#pragma unroll
    for (int i = 0; i < 12; ++i) h[i] = mk(-0.5f * h[i].re, -0.5f * h[i].im);
    store_spinor(H + (size_t)MU * 6 * g.V, g.V, s, h);
}

// H_mu(x) = the hop of direction mu that leaves the block of x (zero when x
// is not on a face of direction mu), for all four mu
template <bool QNZ>
__global__ void __launch_bounds__(256) k_dfl_faces(Geom g, Fields<float> f, const float4* __restrict__ psi, float q,
                                                   float4* __restrict__ H) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int x[4];
    native_coords(g, s, x[0], x[1], x[2], x[3]);
    const int po = 1 - ((x[0] + x[1] + x[2] + x[3]) & 1);
    face_hop<QNZ, 0>(g, f, psi, q, x, s, po, H);
    face_hop<QNZ, 1>(g, f, psi, q, x, s, po, H);
    face_hop<QNZ, 2>(g, f, psi, q, x, s, po, H);
    face_hop<QNZ, 3>(g, f, psi, q, x, s, po, H);
}

// A[b][j][k][l] for one l: projections of T = D phi_l and of the face hops
__global__ void __launch_bounds__(BSITES) k_dfl_project(Geom g, DflGeom d, int ns, int l,
                                                        const float4* __restrict__ basis,
                                                        const float4* __restrict__ T,
                                                        const float4* __restrict__ H, float2* __restrict__ A) {
    __shared__ double sh[(BSITES / 32) * 18];
    const int b = blockIdx.x;
    int x[4];
    block_site(g, d, b, threadIdx.x, x);
    const int s = native_at(g, x);
    const size_t V = (size_t)g.V;
    cplx<float> t[12];
    load_spinor(T, g.V, s, t);
    for (int k = 0; k < ns; ++k) {
        cplx<float> u[12];
        load_spinor(basis + (size_t)k * 6 * V, g.V, s, u);
        double c[18];
#pragma unroll
        for (int i = 0; i < 18; ++i) c[i] = 0.0;
        cdot12(u, t, c[0], c[1]);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const int lm = x[mu] & (BS - 1);
            if (lm == BS - 1 || lm == 0) {
                cplx<float> h[12];
                load_spinor(H + (size_t)mu * 6 * V, g.V, s, h);
                const int j = lm == BS - 1 ? 1 + 2 * mu : 2 + 2 * mu;
                double re = 0.0, im = 0.0;
                cdot12(u, h, re, im);
                c[2 * j] += re;
                c[2 * j + 1] += im;
            }
        }
        block_sum<18>(c, sh);
        if (threadIdx.x == 0) {
            double dre = c[0], dim = c[1];
            for (int j = 1; j < 9; ++j) {
                dre -= c[2 * j];
                dim -= c[2 * j + 1];
                A[(((size_t)b * 9 + j) * ns + k) * ns + l] = make_float2((float)c[2 * j], (float)c[2 * j + 1]);
            }
            A[(((size_t)b * 9 + 0) * ns + k) * ns + l] = make_float2((float)dre, (float)dim);
        }
    }
}

// ---------------------------------------------------------------------------
// restriction, prolongation, little operator
// ---------------------------------------------------------------------------

// c[b][k] = <phi_{b,k}, eta>_b: per site a 12-term dot in FP32, sixteen k
// at a time summed over each warp in FP32 (32 values by recursive halving)
// and over the eight warps of the block in FP64
__global__ void __launch_bounds__(BSITES) k_dfl_restrict(Geom g, DflGeom d, int ns, const float4* __restrict__ basis,
                                                         const float4* __restrict__ eta, double2* __restrict__ c) {
    constexpr int KC = 16;
    __shared__ double sh[(BSITES / 32) * 2 * KC];
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x[4];
    block_site(g, d, b, threadIdx.x, x);
    const int s = native_at(g, x);
    cplx<float> e[12];
    load_spinor(eta, g.V, s, e);
    for (int k0 = 0; k0 < ns; k0 += KC) {
        float v[2 * KC];
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) {
            float re = 0.f, im = 0.f;
            if (k0 + kk < ns) {
                cplx<float> u[12];
                load_spinor(basis + (size_t)(k0 + kk) * 6 * g.V, g.V, s, u);
#pragma unroll
                for (int i = 0; i < 12; ++i) {
                    re = fmaf(u[i].re, e[i].re, fmaf(u[i].im, e[i].im, re));
                    im = fmaf(u[i].re, e[i].im, fmaf(-u[i].im, e[i].re, im));
                }
            }
            v[2 * kk] = re;
            v[2 * kk + 1] = im;
        }
        sh[warp * 2 * KC + lane] = (double)warp_reduce_scatter32(v);  // value `lane` of this warp
        __syncthreads();
        if (threadIdx.x < 2 * KC) {
            double y = 0.0;
            for (int w = 0; w < BSITES / 32; ++w) y += sh[w * 2 * KC + threadIdx.x];
            sh[threadIdx.x] = y;  // row 0 is read only by this thread and the write below
        }
        __syncthreads();
        if (threadIdx.x < KC && k0 + threadIdx.x < ns)
            c[(size_t)b * ns + k0 + threadIdx.x] = make_double2(sh[2 * threadIdx.x], sh[2 * threadIdx.x + 1]);
        __syncthreads();
    }
}

// out(x) = sum_k c[b(x)][k] phi_k(x)
__global__ void __launch_bounds__(BSITES) k_dfl_prolong(Geom g, DflGeom d, int ns, const float4* __restrict__ basis,
                                                        const double2* __restrict__ c, float4* __restrict__ out) {
    const int b = blockIdx.x;
    int x[4];
    block_site(g, d, b, threadIdx.x, x);
    const int s = native_at(g, x);
    float acc[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) acc[i] = 0.f;
    for (int k = 0; k < ns; ++k) {
        const double2 ck = c[(size_t)b * ns + k];
        const float cr = (float)ck.x, ci = (float)ck.y;
        cplx<float> u[12];
        load_spinor(basis + (size_t)k * 6 * g.V, g.V, s, u);
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            acc[2 * i] += cr * u[i].re - ci * u[i].im;
            acc[2 * i + 1] += cr * u[i].im + ci * u[i].re;
        }
    }
    cplx<float> w[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) w[i] = mk(acc[2 * i], acc[2 * i + 1]);
    store_spinor(out, g.V, s, w);
}

__global__ void k_f32_to_f64_native(int V, const float4* __restrict__ in, double2* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    cplx<float> v[12];
    load_spinor(in, V, s, v);
    cplx<double> w[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) w[i] = mk((double)v[i].re, (double)v[i].im);
    store_spinor(out, V, s, w);
}

int dalloc_bytes(void** p, size_t bytes, const char* what) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, what);
    }
    return QXD_OK;
}

}  // namespace

void DflWork::release() {
    if (cycle) cudaGraphExecDestroy(cycle);
    if (cap) cudaStreamDestroy(cap);
    if (h_lstate) cudaFreeHost(h_lstate);
    cycle = nullptr;
    cap = nullptr;
    h_lstate = nullptr;
    void* ps[] = {basis, A, chi, tfield, H, lx, lr, lc, lt, Ainv, d_bad, lstate};
    for (void* p : ps)
        if (p) cudaFree(p);
    lstate = nullptr;
    for (int k = 0; k < DFL_NKV; ++k) {
        if (lp[k]) cudaFree(lp[k]);
        if (lq[k]) cudaFree(lq[k]);
        lp[k] = lq[k] = nullptr;
    }
    basis = nullptr;
    A = nullptr;
    chi = tfield = H = nullptr;
    lx = lc = nullptr;
    lr = lt = Ainv = nullptr;
    eo = false;
    d_bad = nullptr;
    red.release();
    ns = 0;
    ready = false;
}

int DflWork::ensure(const Geom& g, int ns_) {
    if (ns == ns_ && basis) return QXD_OK;
    release();
    d.nb[0] = g.N0 / BS;
    d.nb[1] = g.N1 / BS;
    d.nb[2] = g.N2 / BS;
    d.nb[3] = g.N3 / BS;
    d.nblk = d.nb[0] * d.nb[1] * d.nb[2] * d.nb[3];
    const size_t V = (size_t)g.V;
    const size_t nl = (size_t)d.nblk * ns_;
    int rc;
    if ((rc = dalloc_bytes((void**)&basis, (size_t)ns_ * 6 * V * sizeof(float4), "cudaMalloc(deflation basis)")) ||
        (rc = dalloc_bytes((void**)&A, (size_t)d.nblk * 9 * ns_ * ns_ * sizeof(float2), "cudaMalloc(little operator)")) ||
        (rc = dalloc_bytes((void**)&chi, 6 * V * sizeof(float4), "cudaMalloc(deflation field)")) ||
        (rc = dalloc_bytes((void**)&tfield, 6 * V * sizeof(float4), "cudaMalloc(deflation field)")) ||
        (rc = dalloc_bytes((void**)&H, 4 * 6 * V * sizeof(float4), "cudaMalloc(deflation faces)")) ||
        (rc = dalloc_bytes((void**)&lx, nl * sizeof(double2), "cudaMalloc(little vectors)")) ||
        (rc = dalloc_bytes((void**)&lr, nl * sizeof(float2), "cudaMalloc(little vectors)")) ||

        (rc = dalloc_bytes((void**)&lc, nl * sizeof(double2), "cudaMalloc(little vectors)")) ||
        (rc = dalloc_bytes((void**)&d_bad, sizeof(int), "cudaMalloc(deflation status)")) ||
        (rc = dalloc_bytes((void**)&lstate, sizeof(LittleState), "cudaMalloc(little solver state)")))
        return rc;
    QXD_CUDA(cudaMallocHost(&h_lstate, sizeof(LittleState)));
    for (int k = 0; k < DFL_NKV; ++k)
        if ((rc = dalloc_bytes((void**)&lp[k], nl * sizeof(float2), "cudaMalloc(little vectors)")) ||
            (rc = dalloc_bytes((void**)&lq[k], nl * sizeof(float2), "cudaMalloc(little vectors)")))
            return rc;
    if ((rc = red.init())) return rc;
    eo = ns_ == 8 || ns_ == 16 || ns_ == 32;  // the warp-per-block kernels
    if (eo && ((rc = dalloc_bytes((void**)&lt, nl * sizeof(float2), "cudaMalloc(little vectors)")) ||
               (rc = dalloc_bytes((void**)&Ainv, (size_t)d.nblk * ns_ * ns_ * sizeof(float2),
                                  "cudaMalloc(little operator inverse blocks)"))))
        return rc;
    ns = ns_;
    return QXD_OK;
}

void release_dfl(qxd_lattice* lat) {
    if (!lat->dfl) return;
    lat->dfl->release();
    delete lat->dfl;
    lat->dfl = nullptr;
}

namespace {

int orthonormalise(qxd_lattice* lat, DflWork& W, cudaStream_t st) {
    QXD_CUDA(cudaMemsetAsync(W.d_bad, 0, sizeof(int), st));
    k_dfl_orth<<<W.d.nblk, BSITES, 0, st>>>(lat->g, W.d, W.ns, W.basis, W.d_bad);
    QXD_LAUNCHED("k_dfl_orth");
    int bad = 0;
    QXD_CUDA(cudaMemcpyAsync(&bad, W.d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    QXD_CUDA(cudaStreamSynchronize(st));
    if (bad) return fail(QXD_ERR_NUMERIC, "deflation subspace: " + std::to_string(bad) +
                                             " blocks with linearly dependent fields");
    return QXD_OK;
}

template <int NS>
void launch_invert(DflWork& W, cudaStream_t st);  // A_oo^-1 of the odd blocks (defined with the little solver)

int build_little(qxd_lattice* lat, DflWork& W, cudaStream_t st) {
    const Geom& g = lat->g;
    Fields<float> f{nullptr, nullptr, lat->U32, lat->A32, lat->C32};
    const float q = (float)lat->qhat;
    int rc;
    for (int l = 0; l < W.ns; ++l) {
        const float4* phil = W.basis + (size_t)l * 6 * g.V;
        if ((rc = launch_dirac(lat, W.tfield, phil, QXD_FP32, st))) return rc;
        if (lat->qhat != 0) k_dfl_faces<true><<<(g.V + 255) / 256, 256, 0, st>>>(g, f, phil, q, W.H);
        else k_dfl_faces<false><<<(g.V + 255) / 256, 256, 0, st>>>(g, f, phil, q, W.H);
        QXD_LAUNCHED("k_dfl_faces");
        k_dfl_project<<<W.d.nblk, BSITES, 0, st>>>(g, W.d, W.ns, l, W.basis, W.tfield, W.H, W.A);
        QXD_LAUNCHED("k_dfl_project");
    }
    if (W.eo) {  // inverse self-couplings of the odd blocks
        QXD_CUDA(cudaMemsetAsync(W.d_bad, 0, sizeof(int), st));
        if (W.ns == 16) launch_invert<16>(W, st);
        else if (W.ns == 8) launch_invert<8>(W, st);
        else launch_invert<32>(W, st);
        QXD_LAUNCHED("k_lt_invert");
        int bad = 0;
        QXD_CUDA(cudaMemcpyAsync(&bad, W.d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        QXD_CUDA(cudaStreamSynchronize(st));
        if (bad) return fail(QXD_ERR_NUMERIC, "little operator: singular self-coupling of an odd block");
    }
    QXD_CUDA(cudaStreamSynchronize(st));
    W.op_version = lat->op_version;
    W.ready = true;
    return QXD_OK;
}

// ---------------------------------------------------------------------------
// Little GCR on the device. One step k of a restart cycle is five kernels:
//   apply:     p_k = r, q_k = A r
//   mdot:      a_j = <q_j, q_k>, j < k                      (k > 0)
//   orth:      q_k -= sum a_j q_j, p_k -= sum a_j p_j; qq = |q_k|^2
//   scale_dot: q_k, p_k *= 1/sqrt(qq); al = <q_k, r>
//   update:    x += al p_k, r -= al q_k; rn2 = |r|^2; stop when rn2 <= tol^2 |c|^2
// The reductions write per-block partial sums; the last block to arrive
// (counted with an atomic) adds them in block order, so each coefficient is
// the same on every run, and stores it in the LittleState. Every kernel
// returns at once when the state says done.
// ---------------------------------------------------------------------------

// after block_reduce_store: the last block to arrive sums the nc partials
// in block order into out[0..nc) and returns true (in thread 0 only)
__device__ __forceinline__ bool last_block_finish(const double* __restrict__ partials, int nc, double* out,
                                                  unsigned* count) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(count, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int c = threadIdx.x >> 5; c < nc; c += (int)(blockDim.x >> 5)) {
        const double x = warp_sum_column(partials, c, (int)gridDim.x);
        if ((threadIdx.x & 31) == 0) out[c] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) *count = 0u;
    return threadIdx.x == 0;
}

// Little solver. The Krylov vectors r, p_k, q_k are FP32 and their
// arithmetic is FP32: the little system is solved only to a relative residual
// of dfl_tol (1e-2 by default) as a preconditioner inside the flexible GCR,
// and GB300's FP64 rate (1/63 of FP32, conversions included) made FP64
// vectors the cost of a little step. The solution x and the source c stay
// FP64; inner products are summed in FP32 within a thread and a warp and in
// FP64 across warps and blocks, in a fixed order.

// block-wide sum of NC FP32 values per thread (NC <= 32) into the FP64
// partials of this block (RED_THREADS threads)
template <int NC>
__device__ __forceinline__ void block_reduce_store_f32(const float v[NC], double* __restrict__ partials) {
    __shared__ double sh[RED_THREADS / 32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (NC <= 2) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            float x = v[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) sh[warp][c] = (double)x;
        }
    } else {
        float w[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) w[c] = c < NC ? v[c] : 0.f;
        sh[warp][lane] = (double)warp_reduce_scatter32(w);
    }
    __syncthreads();
    if (threadIdx.x < NC) {
        double y = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) y += sh[w][threadIdx.x];
        partials[(size_t)blockIdx.x * 2 * BLAS_KMAX + threadIdx.x] = y;
    }
}

// q = A r: q[b][k] = sum_j sum_l A[b][j][k][l] r[n_j(b)][l], one thread per
// (b, k); also p = r (A and the products in FP32)
__global__ void k_lt_apply(Geom g, DflGeom d, int ns, const float2* __restrict__ A, const float2* __restrict__ r,
                           float2* __restrict__ p, float2* __restrict__ q, const LittleState* __restrict__ S) {
    if (S->done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.nblk * ns) return;
    const int b = i / ns, k = i - b * ns;
    float re = 0.f, im = 0.f;
    for (int j = 0; j < 9; ++j) {
        const int nb = j == 0 ? b : block_nbr(g, d, b, (j - 1) >> 1, (j & 1) ? +1 : -1);
        const float2* a = A + (((size_t)b * 9 + j) * ns + k) * ns;
        const float2* v = r + (size_t)nb * ns;
        for (int l = 0; l < ns; ++l) {
            const float2 al = a[l], vl = v[l];
            re = fmaf(al.x, vl.x, fmaf(-al.y, vl.y, re));
            im = fmaf(al.x, vl.y, fmaf(al.y, vl.x, im));
        }
    }
    q[i] = make_float2(re, im);
    p[i] = r[i];
}

// the same product with coalesced reads of A, for ns = 8, 16 or 32: one warp
// per block b; G = 32 / ns lanes share a row k, lane g of a row taking the
// ns / G entries l in [g ns / G, (g + 1) ns / G), so that a warp reads
// whole consecutive rows of A[b][j]; the G partial sums of a row are added
// by warp shuffles. A is read once per step and streamed (evict-first), so
// that the Krylov vectors stay in L2.
template <int NS>
__global__ void __launch_bounds__(32) k_lt_apply_warp(Geom g, DflGeom d, const float2* __restrict__ A,
                                                      const float2* __restrict__ r, float2* __restrict__ p,
                                                      float2* __restrict__ q, const LittleState* __restrict__ S) {
    if (S->done) return;
    constexpr int G = 32 / NS, CH = NS / G;
    const int b = blockIdx.x, lane = threadIdx.x;
    const int k = lane / G, part = lane % G;
    float re = 0.f, im = 0.f;
#pragma unroll 3
    for (int j = 0; j < 9; ++j) {
        const int nb = j == 0 ? b : block_nbr(g, d, b, (j - 1) >> 1, (j & 1) ? +1 : -1);
        const float2* a = A + (((size_t)b * 9 + j) * NS + k) * NS + part * CH;
        const float2* v = r + (size_t)nb * NS + part * CH;
#pragma unroll
        for (int l = 0; l < CH; ++l) {
            const float2 al = __ldcs(a + l), vl = v[l];
            re = fmaf(al.x, vl.x, fmaf(-al.y, vl.y, re));
            im = fmaf(al.x, vl.y, fmaf(al.y, vl.x, im));
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (part == 0) {
        const size_t i = (size_t)b * NS + k;
        q[i] = make_float2(re, im);
        p[i] = r[i];
    }
}

// a_j = <q_j, q_k>, j < K
template <int K>
__global__ void __launch_bounds__(RED_THREADS) k_lt_mdot(size_t n, VecList<float2> qs, const float2* __restrict__ qk,
                                                         double* partials, LittleState* S) {
    if (S->done) return;
    float v[2 * K];
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) v[c] = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 y = qk[i];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const float2 x = qs.p[j][i];
            v[2 * j] = fmaf(x.x, y.x, fmaf(x.y, y.y, v[2 * j]));
            v[2 * j + 1] = fmaf(x.x, y.y, fmaf(-x.y, y.x, v[2 * j + 1]));
        }
    }
    block_reduce_store_f32<2 * K>(v, partials);
    last_block_finish(partials, 2 * K, S->a, &S->count);
}

// q_k -= sum_j a_j q_j, p_k -= sum_j a_j p_j; |q_k|^2
template <int K>
__global__ void __launch_bounds__(RED_THREADS) k_lt_orth(size_t n, VecList<float2> qs, VecList<float2> ps,
                                                         float2* __restrict__ qk, float2* __restrict__ pk,
                                                         double* partials, LittleState* S) {
    if (S->done) return;
    float a[2 * K + 1];
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) a[c] = (float)S->a[c];
    float v[1] = {0.f};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float2 y = qk[i], z = pk[i];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const float ar = a[2 * j], ai = a[2 * j + 1];
            const float2 x = qs.p[j][i], w = ps.p[j][i];
            y.x -= ar * x.x - ai * x.y;
            y.y -= ar * x.y + ai * x.x;
            z.x -= ar * w.x - ai * w.y;
            z.y -= ar * w.y + ai * w.x;
        }
        qk[i] = y;
        if (K > 0) pk[i] = z;
        v[0] = fmaf(y.x, y.x, fmaf(y.y, y.y, v[0]));
    }
    block_reduce_store_f32<1>(v, partials);
    double qq;
    if (last_block_finish(partials, 1, &qq, &S->count)) {
        S->qq = qq;
        if (!(qq > 0.0) || !isfinite(qq)) {
            S->status = 1;
            S->done = 1;
        }
    }
}

// q_k, p_k /= |q_k|; al = <q_k, r>
__global__ void __launch_bounds__(RED_THREADS) k_lt_scale_dot(size_t n, float2* __restrict__ qk,
                                                              float2* __restrict__ pk, const float2* __restrict__ r,
                                                              double* partials, LittleState* S) {
    if (S->done) return;
    const float sc = (float)(1.0 / sqrt(S->qq));
    float v[2] = {0.f, 0.f};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float2 x = qk[i], w = pk[i];
        x.x *= sc;
        x.y *= sc;
        w.x *= sc;
        w.y *= sc;
        qk[i] = x;
        pk[i] = w;
        const float2 y = r[i];
        v[0] = fmaf(x.x, y.x, fmaf(x.y, y.y, v[0]));
        v[1] = fmaf(x.x, y.y, fmaf(-x.y, y.x, v[1]));
    }
    block_reduce_store_f32<2>(v, partials);
    last_block_finish(partials, 2, S->al, &S->count);
}

// x += al p_k (FP64), r -= al q_k; |r|^2 and the stopping test
__global__ void __launch_bounds__(RED_THREADS) k_lt_update(size_t n, const float2* __restrict__ pk,
                                                           const float2* __restrict__ qk, double2* __restrict__ x,
                                                           float2* __restrict__ r, double* partials, LittleState* S) {
    if (S->done) return;
    const double ar = S->al[0], ai = S->al[1];
    const float fr = (float)ar, fi = (float)ai;
    float v[1] = {0.f};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 p = pk[i], q = qk[i];
        double2 xi = x[i];
        float2 ri = r[i];
        xi.x += ar * p.x - ai * p.y;
        xi.y += ar * p.y + ai * p.x;
        ri.x -= fr * q.x - fi * q.y;
        ri.y -= fr * q.y + fi * q.x;
        x[i] = xi;
        r[i] = ri;
        v[0] = fmaf(ri.x, ri.x, fmaf(ri.y, ri.y, v[0]));
    }
    block_reduce_store_f32<1>(v, partials);
    double rn2;
    if (last_block_finish(partials, 1, &rn2, &S->count)) {
        S->rn2 = rn2;
        S->it += 1;
        if (!isfinite(rn2)) {
            S->status = 1;
            S->done = 1;
        } else if (rn2 <= S->target2 || S->it >= S->max_iter) {
            S->done = 1;
        }
    }
}

// r = c (FP64 source to the FP32 residual)
__global__ void k_lt_init(size_t n, const double2* __restrict__ c, float2* __restrict__ r) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        r[i] = make_float2((float)c[i].x, (float)c[i].y);
}

// ---------------------------------------------------------------------------
// Even-odd form of the little system. Blocks of one colour (parity of the
// block coordinates, as in the Schwarz method) couple only to blocks of the
// other colour, so with A_ee, A_oo the self-couplings
//   A_hat = A_ee - A_eo A_oo^-1 A_oe   on the even blocks,
//   A_hat y_e = c_e - A_eo A_oo^-1 c_o,  y_o = A_oo^-1 (c_o - A_oe y_e).
// The GCR runs on A_hat (full-length vectors whose odd entries stay zero).
// One warp per block, lanes as in k_lt_apply_warp; A_oo^-1 is formed once per
// little operator by Gauss-Jordan elimination in FP64.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int block_parity(const DflGeom& d, int b) {
    const int B3 = b % d.nb[3];
    int r = b / d.nb[3];
    const int B2 = r % d.nb[2];
    r /= d.nb[2];
    const int B1 = r % d.nb[1];
    const int B0 = r / d.nb[1];
    return (B0 + B1 + B2 + B3) & 1;
}

// block number i of parity p (blocks 2i and 2i + 1 differ only in B3, and
// nb[3] is even, so one of them has each parity)
__device__ __forceinline__ int block_of_parity(const DflGeom& d, int i, int p) {
    const int b = 2 * i;
    return block_parity(d, b) == p ? b : b + 1;
}

__device__ __forceinline__ float2 to_f2(float2 v) { return v; }
__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2((float)v.x, (float)v.y); }

// this lane's share of row k of sum_{j = j0 .. j1} A[b][j] v[n_j(b)]
template <int NS, typename T>
__device__ __forceinline__ void lt_rows(const Geom& g, const DflGeom& d, const float2* __restrict__ A,
                                       const T* __restrict__ v, int b, int j0, int j1, int k, int part, float& re,
                                       float& im) {
    constexpr int G = 32 / NS, CH = NS / G;
#pragma unroll 1
    for (int j = j0; j <= j1; ++j) {
        const int nb = j == 0 ? b : block_nbr(g, d, b, (j - 1) >> 1, (j & 1) ? +1 : -1);
        const float2* a = A + (((size_t)b * 9 + j) * NS + k) * NS + part * CH;
        const T* x = v + (size_t)nb * NS + part * CH;
#pragma unroll
        for (int l = 0; l < CH; ++l) {
            const float2 al = __ldcs(a + l), vl = to_f2(x[l]);
            re = fmaf(al.x, vl.x, fmaf(-al.y, vl.y, re));
            im = fmaf(al.x, vl.y, fmaf(al.y, vl.x, im));
        }
    }
}

// sum of a row over its G lanes (every lane of the row gets it)
template <int NS>
__device__ __forceinline__ void row_sum(float& re, float& im) {
#pragma unroll
    for (int o = (32 / NS) / 2; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
}

// y = A_oo^-1[b] u with u_k given by the lanes of row k (part 0 holds it);
// returns row k of y in every lane of the row
template <int NS>
__device__ __forceinline__ float2 apply_inv(const float2* __restrict__ Ainv, int b, float2 uk, int k, int part,
                                            float2* su) {
    constexpr int G = 32 / NS, CH = NS / G;
    if (part == 0) su[k] = uk;
    __syncwarp();
    const float2* a = Ainv + ((size_t)b * NS + k) * NS + part * CH;
    float re = 0.f, im = 0.f;
#pragma unroll
    for (int l = 0; l < CH; ++l) {
        const float2 al = a[l], vl = su[part * CH + l];
        re = fmaf(al.x, vl.x, fmaf(-al.y, vl.y, re));
        im = fmaf(al.x, vl.y, fmaf(al.y, vl.x, im));
    }
    row_sum<NS>(re, im);
    __syncwarp();
    return make_float2(re, im);
}

// A_oo^-1 for the odd blocks: Gauss-Jordan with partial pivoting on [A_bb | 1]
// in FP64 shared memory, one warp per odd block; a pivot below 1e-12 of the
// largest entry of the block (or not finite) flags the block as singular
template <int NS>
__global__ void __launch_bounds__(32) k_lt_invert(DflGeom d, const float2* __restrict__ A, float2* __restrict__ Ainv,
                                                  int* __restrict__ bad) {
    __shared__ double2 M[NS][2 * NS];
    __shared__ double2 f[NS];
    const int b = block_of_parity(d, blockIdx.x, 1);
    const int lane = threadIdx.x;
    const float2* a = A + (size_t)b * 9 * NS * NS;  // j = 0: the self-coupling
    double amax = 0.0;
    for (int e = lane; e < NS * 2 * NS; e += 32) {
        const int r = e / (2 * NS), c = e % (2 * NS);
        double2 v = make_double2(r == c - NS ? 1.0 : 0.0, 0.0);
        if (c < NS) {
            const float2 x = a[r * NS + c];
            v = make_double2(x.x, x.y);
            amax = fmax(amax, fabs(v.x) + fabs(v.y));
        }
        M[r][c] = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    __syncwarp();
    bool ok = true;
    for (int c = 0; c < NS; ++c) {
        // pivot: largest |M[r][c]| over r >= c (lowest row on ties)
        double best = -1.0;
        int pr = c;
        for (int r = c + lane; r < NS; r += 32) {
            const double m = fabs(M[r][c].x) + fabs(M[r][c].y);
            if (m > best) {
                best = m;
                pr = r;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int opr = __shfl_xor_sync(0xffffffffu, pr, o);
            if (ob > best || (ob == best && opr < pr)) {
                best = ob;
                pr = opr;
            }
        }
        if (!(best > 1e-12 * amax) || !isfinite(best)) {
            ok = false;
            break;
        }
        for (int e = lane; e < 2 * NS; e += 32) {  // swap rows c and pr
            const double2 t = M[c][e];
            M[c][e] = M[pr][e];
            M[pr][e] = t;
        }
        __syncwarp();
        const double2 pv = M[c][c];
        const double den = pv.x * pv.x + pv.y * pv.y;
        const double2 inv = make_double2(pv.x / den, -pv.y / den);
        __syncwarp();
        for (int e = lane; e < 2 * NS; e += 32) {  // row c /= pivot
            const double2 t = M[c][e];
            M[c][e] = make_double2(t.x * inv.x - t.y * inv.y, t.x * inv.y + t.y * inv.x);
        }
        for (int r = lane; r < NS; r += 32) f[r] = M[r][c];
        __syncwarp();
        for (int e = lane; e < NS * 2 * NS; e += 32) {  // row r -= f_r row c, r != c
            const int r = e / (2 * NS), cc = e % (2 * NS);
            if (r == c) continue;
            const double2 fr = f[r], mc = M[c][cc];
            M[r][cc] = make_double2(M[r][cc].x - (fr.x * mc.x - fr.y * mc.y), M[r][cc].y - (fr.x * mc.y + fr.y * mc.x));
        }
        __syncwarp();
    }
    if (!ok) {
        if (lane == 0) atomicAdd(bad, 1);
        return;
    }
    float2* out = Ainv + (size_t)b * NS * NS;
    for (int e = lane; e < NS * NS; e += 32) {
        const double2 v = M[e / NS][NS + e % NS];
        out[e] = make_float2((float)v.x, (float)v.y);
    }
}

// Schur apply, odd half: t_o = A_oo^-1 (A_oe r_e); p_o = q_o = 0
template <int NS>
__global__ void __launch_bounds__(32) k_lt_schur_odd(Geom g, DflGeom d, const float2* __restrict__ A,
                                                     const float2* __restrict__ Ainv, const float2* __restrict__ r,
                                                     float2* __restrict__ t, float2* __restrict__ p,
                                                     float2* __restrict__ q, const LittleState* __restrict__ S) {
    if (S->done) return;
    __shared__ float2 su[NS];
    constexpr int G = 32 / NS;
    const int b = block_of_parity(d, blockIdx.x, 1), lane = threadIdx.x;
    const int k = lane / G, part = lane % G;
    float re = 0.f, im = 0.f;
    lt_rows<NS>(g, d, A, r, b, 1, 8, k, part, re, im);
    row_sum<NS>(re, im);
    const float2 y = apply_inv<NS>(Ainv, b, make_float2(re, im), k, part, su);
    if (part == 0) {
        const size_t i = (size_t)b * NS + k;
        t[i] = y;
        p[i] = make_float2(0.f, 0.f);
        q[i] = make_float2(0.f, 0.f);
    }
}

// Schur apply, even half: q_e = A_ee r_e - A_eo t_o; p_e = r_e
template <int NS>
__global__ void __launch_bounds__(32) k_lt_schur_even(Geom g, DflGeom d, const float2* __restrict__ A,
                                                      const float2* __restrict__ r, const float2* __restrict__ t,
                                                      float2* __restrict__ p, float2* __restrict__ q,
                                                      const LittleState* __restrict__ S) {
    if (S->done) return;
    constexpr int G = 32 / NS;
    const int b = block_of_parity(d, blockIdx.x, 0), lane = threadIdx.x;
    const int k = lane / G, part = lane % G;
    float re = 0.f, im = 0.f, he = 0.f, hm = 0.f;
    lt_rows<NS>(g, d, A, r, b, 0, 0, k, part, re, im);
    lt_rows<NS>(g, d, A, t, b, 1, 8, k, part, he, hm);
    re -= he;
    im -= hm;
    row_sum<NS>(re, im);
    if (part == 0) {
        const size_t i = (size_t)b * NS + k;
        q[i] = make_float2(re, im);
        p[i] = r[i];
    }
}

// source of the Schur system, odd half: t_o = A_oo^-1 c_o, r_o = 0
template <int NS>
__global__ void __launch_bounds__(32) k_lt_prep_odd(DflGeom d, const float2* __restrict__ Ainv,
                                                    const double2* __restrict__ c, float2* __restrict__ t,
                                                    float2* __restrict__ r) {
    __shared__ float2 su[NS];
    constexpr int G = 32 / NS;
    const int b = block_of_parity(d, blockIdx.x, 1), lane = threadIdx.x;
    const int k = lane / G, part = lane % G;
    const size_t i = (size_t)b * NS + k;
    const float2 y = apply_inv<NS>(Ainv, b, to_f2(c[i]), k, part, su);
    if (part == 0) {
        t[i] = y;
        r[i] = make_float2(0.f, 0.f);
    }
}

// even half: r_e = c_e - A_eo t_o
template <int NS>
__global__ void __launch_bounds__(32) k_lt_prep_even(Geom g, DflGeom d, const float2* __restrict__ A,
                                                     const double2* __restrict__ c, const float2* __restrict__ t,
                                                     float2* __restrict__ r) {
    constexpr int G = 32 / NS;
    const int b = block_of_parity(d, blockIdx.x, 0), lane = threadIdx.x;
    const int k = lane / G, part = lane % G;
    float re = 0.f, im = 0.f;
    lt_rows<NS>(g, d, A, t, b, 1, 8, k, part, re, im);
    row_sum<NS>(re, im);
    if (part == 0) {
        const size_t i = (size_t)b * NS + k;
        const float2 ci = to_f2(c[i]);
        r[i] = make_float2(ci.x - re, ci.y - im);
    }
}

// solution on the odd blocks: x_o = A_oo^-1 (c_o - A_oe x_e)
template <int NS>
__global__ void __launch_bounds__(32) k_lt_recon_odd(Geom g, DflGeom d, const float2* __restrict__ A,
                                                     const float2* __restrict__ Ainv, const double2* __restrict__ c,
                                                     double2* __restrict__ x) {
    __shared__ float2 su[NS];
    constexpr int G = 32 / NS;
    const int b = block_of_parity(d, blockIdx.x, 1), lane = threadIdx.x;
    const int k = lane / G, part = lane % G;
    float re = 0.f, im = 0.f;
    lt_rows<NS>(g, d, A, x, b, 1, 8, k, part, re, im);
    row_sum<NS>(re, im);
    const size_t i = (size_t)b * NS + k;
    const float2 ci = to_f2(c[i]);
    const float2 y = apply_inv<NS>(Ainv, b, make_float2(ci.x - re, ci.y - im), k, part, su);
    if (part == 0) x[i] = make_double2(y.x, y.y);
}

template <int NS>
void launch_schur(qxd_lattice* lat, DflWork& W, int k, cudaStream_t st) {
    const int nh = W.d.nblk / 2;
    k_lt_schur_odd<NS><<<nh, 32, 0, st>>>(lat->g, W.d, W.A, W.Ainv, W.lr, W.lt, W.lp[k], W.lq[k], W.lstate);
    k_lt_schur_even<NS><<<nh, 32, 0, st>>>(lat->g, W.d, W.A, W.lr, W.lt, W.lp[k], W.lq[k], W.lstate);
}

template <int NS>
void launch_prep(qxd_lattice* lat, DflWork& W, cudaStream_t st) {
    const int nh = W.d.nblk / 2;
    k_lt_prep_odd<NS><<<nh, 32, 0, st>>>(W.d, W.Ainv, W.lc, W.lt, W.lr);
    k_lt_prep_even<NS><<<nh, 32, 0, st>>>(lat->g, W.d, W.A, W.lc, W.lt, W.lr);
}

template <int NS>
void launch_recon(qxd_lattice* lat, DflWork& W, cudaStream_t st) {
    k_lt_recon_odd<NS><<<W.d.nblk / 2, 32, 0, st>>>(lat->g, W.d, W.A, W.Ainv, W.lc, W.lx);
}

template <int NS>
void launch_invert(DflWork& W, cudaStream_t st) {
    k_lt_invert<NS><<<W.d.nblk / 2, 32, 0, st>>>(W.d, W.A, W.Ainv, W.d_bad);
}

// the launches of one restart cycle (steps k = 0 .. DFL_NKV - 1)
void little_cycle(qxd_lattice* lat, DflWork& W, cudaStream_t st) {
    const size_t n = (size_t)W.d.nblk * W.ns;
    for (int k = 0; k < DFL_NKV; ++k) {
        if (W.eo) {
            if (W.ns == 16) launch_schur<16>(lat, W, k, st);
            else if (W.ns == 8) launch_schur<8>(lat, W, k, st);
            else launch_schur<32>(lat, W, k, st);
        } else if (W.ns == 16)
            k_lt_apply_warp<16><<<W.d.nblk, 32, 0, st>>>(lat->g, W.d, W.A, W.lr, W.lp[k], W.lq[k], W.lstate);
        else if (W.ns == 8)
            k_lt_apply_warp<8><<<W.d.nblk, 32, 0, st>>>(lat->g, W.d, W.A, W.lr, W.lp[k], W.lq[k], W.lstate);
        else if (W.ns == 32)
            k_lt_apply_warp<32><<<W.d.nblk, 32, 0, st>>>(lat->g, W.d, W.A, W.lr, W.lp[k], W.lq[k], W.lstate);
        else
            k_lt_apply<<<(int)((n + 127) / 128), 128, 0, st>>>(lat->g, W.d, W.ns, W.A, W.lr, W.lp[k], W.lq[k],
                                                             W.lstate);
        VecList<float2> qs{}, ps{};
        for (int j = 0; j < k; ++j) {
            qs.p[j] = W.lq[j];
            ps.p[j] = W.lp[j];
        }
        switch (k) {
#define QXD_LT_GS(K)                                                                                         \
    case K:                                                                                                   \
        if (K > 0) k_lt_mdot<(K > 0 ? K : 1)><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, qs, W.lq[k], W.red.partials, \
                                                                                  W.lstate);                  \
        k_lt_orth<K><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, qs, ps, W.lq[k], W.lp[k], W.red.partials, W.lstate); \
        break;
            QXD_LT_GS(0) QXD_LT_GS(1) QXD_LT_GS(2) QXD_LT_GS(3) QXD_LT_GS(4) QXD_LT_GS(5) QXD_LT_GS(6)
            QXD_LT_GS(7) QXD_LT_GS(8) QXD_LT_GS(9) QXD_LT_GS(10) QXD_LT_GS(11) QXD_LT_GS(12) QXD_LT_GS(13)
            QXD_LT_GS(14) QXD_LT_GS(15)
#undef QXD_LT_GS
        }
        k_lt_scale_dot<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, W.lq[k], W.lp[k], W.lr, W.red.partials, W.lstate);
        k_lt_update<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, W.lp[k], W.lq[k], W.lx, W.lr, W.red.partials, W.lstate);
    }
}

// the cycle as a CUDA graph, captured once per work space (its pointers are fixed)
int little_cycle_graph(qxd_lattice* lat, DflWork& W) {
    if (W.cycle) return QXD_OK;
    if (!W.cap) QXD_CUDA(cudaStreamCreateWithFlags(&W.cap, cudaStreamNonBlocking));
    QXD_CUDA(cudaStreamBeginCapture(W.cap, cudaStreamCaptureModeThreadLocal));
    little_cycle(lat, W, W.cap);
    const cudaError_t le = cudaGetLastError();
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(W.cap, &graph);
    if (le != cudaSuccess || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(le != cudaSuccess ? le : ce, "little solver graph capture");
    }
    const cudaError_t ie = cudaGraphInstantiate(&W.cycle, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        W.cycle = nullptr;
        return cuda_fail(ie, "cudaGraphInstantiate (little solver)");
    }
    return QXD_OK;
}

// GCR on the little system A y = c (W.lc) into W.lx, restarted every
// DFL_NKV steps, to |r| <= tol |c| or max_iter steps. With W.eo the GCR runs
// on the Schur complement of the even blocks (|r| and c of that system), and
// the odd blocks follow from the even ones.
int little_gcr(qxd_lattice* lat, DflWork& W, double tol, int max_iter, int* iters, cudaStream_t st) {
    const size_t n = (size_t)W.d.nblk * W.ns;
    const size_t bytes = n * sizeof(double2);
    int rc;
    QXD_CUDA(cudaMemsetAsync(W.lx, 0, bytes, st));
    double cc;
    if (W.eo) {
        if (W.ns == 16) launch_prep<16>(lat, W, st);
        else if (W.ns == 8) launch_prep<8>(lat, W, st);
        else launch_prep<32>(lat, W, st);
        QXD_LAUNCHED("k_lt_prep");
        if ((rc = blas_norm2<float2>(W.red, n, W.lr, &cc, st))) return rc;
    } else {
        if ((rc = blas_norm2<double2>(W.red, n, W.lc, &cc, st))) return rc;
        k_lt_init<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, W.lc, W.lr);
        QXD_LAUNCHED("k_lt_init");
    }
    *iters = 0;
    if (!std::isfinite(cc)) return fail(QXD_ERR_NUMERIC, "little solver: non-finite source");
    if (cc > 0.0) {
        LittleState& h = *W.h_lstate;
        h = LittleState{};
        h.rn2 = cc;
        h.target2 = tol * tol * cc;
        h.max_iter = max_iter;
        h.done = (max_iter < 1 || tol >= 1.0) ? 1 : 0;
        QXD_CUDA(cudaMemcpyAsync(W.lstate, &h, sizeof(LittleState), cudaMemcpyHostToDevice, st));
        if ((rc = little_cycle_graph(lat, W))) return rc;
        while (!h.done) {
            QXD_CUDA(cudaGraphLaunch(W.cycle, st));
            QXD_CUDA(cudaMemcpyAsync(&h, W.lstate, sizeof(LittleState), cudaMemcpyDeviceToHost, st));
            QXD_CUDA(cudaStreamSynchronize(st));
        }
        if (h.status) return fail(QXD_ERR_NUMERIC, "little solver: breakdown or non-finite residual");
        *iters = h.it;
    }
    if (W.eo) {  // x_o = A_oo^-1 (c_o - A_oe x_e)
        if (W.ns == 16) launch_recon<16>(lat, W, st);
        else if (W.ns == 8) launch_recon<8>(lat, W, st);
        else launch_recon<32>(lat, W, st);
        QXD_LAUNCHED("k_lt_recon_odd");
    }
    return QXD_OK;
}

}  // namespace

// out = M_dfl in = chi + SAP(in - D chi), chi = P A^-1 P^dag in (FP32 native)
int dfl_precondition(qxd_lattice* lat, void* out, const void* in, int ncy, int nmr, double tol, int max_iter,
                     int* little_iters, cudaStream_t st) {
    DflWork& W = *lat->dfl;
    const Geom& g = lat->g;
    const size_t n32 = (size_t)12 * g.V;  // complex numbers of a field
    int rc;
    k_dfl_restrict<<<W.d.nblk, BSITES, 0, st>>>(g, W.d, W.ns, W.basis, (const float4*)in, W.lc);
    QXD_LAUNCHED("k_dfl_restrict");
    int it = 0;
    if ((rc = little_gcr(lat, W, tol, max_iter, &it, st))) return rc;
    if (little_iters) *little_iters += it;
    k_dfl_prolong<<<W.d.nblk, BSITES, 0, st>>>(g, W.d, W.ns, W.basis, W.lx, W.chi);
    QXD_LAUNCHED("k_dfl_prolong");
    // rho = in - D chi (into W.tfield)
    if ((rc = launch_dirac(lat, W.tfield, W.chi, QXD_FP32, st))) return rc;
    if ((rc = blas_scale<float2>(n32, -1.0, (float2*)W.tfield, st))) return rc;
    if ((rc = blas_caxpy<float2>(n32, cd(-1.0, 0.0), (const float2*)in, (float2*)W.tfield, st))) return rc;
    if ((rc = sap_apply<float>(lat, W.sap, out, W.tfield, ncy, nmr, st))) return rc;
    return blas_caxpy<float2>(n32, cd(-1.0, 0.0), (const float2*)W.chi, (float2*)out, st);
}

}  // namespace qxd

using namespace qxd;

namespace {

int dfl_checks(qxd_lattice* lat, int ns, const char* name) {
    if (!lat) return fail(QXD_ERR_ARG, std::string(name) + ": lat is NULL");
    if (ns < 1 || ns > 64) return fail(QXD_ERR_ARG, std::string(name) + ": 1 <= ns <= 64");
    if (!qxd::clover_ready(lat)) return fail(QXD_ERR_STATE, std::string(name) + ": needs qxd_sw_build first");
    int rc = sap_check(lat);
    if (rc) return rc;
    if (!lat->dfl) lat->dfl = new DflWork();
    return lat->dfl->ensure(lat->g, ns);
}

}  // namespace

extern "C" {

int qxd_dfl_subspace(qxd_lattice* lat, int ns, int niter, int ncy, unsigned long long seed) {
    int rc = dfl_checks(lat, ns, "qxd_dfl_subspace");
    if (rc) return rc;
    if (niter < 0 || ncy < 1) return fail(QXD_ERR_ARG, "qxd_dfl_subspace: niter >= 0, ncy >= 1");
    DflWork& W = *lat->dfl;
    cudaStream_t st = lat->stream;
    const size_t V = (size_t)lat->g.V;
    W.ready = false;
    const size_t nc = (size_t)ns * 12 * V;
    k_dfl_random<<<4 * 152 * 4, 256, 0, st>>>(nc, seed, (float2*)W.basis);
    QXD_LAUNCHED("k_dfl_random");
    if ((rc = orthonormalise(lat, W, st))) return rc;
    for (int it = 0; it < niter; ++it) {
        for (int k = 0; k < ns; ++k) {
            float4* v = W.basis + (size_t)k * 6 * V;
            if ((rc = sap_apply<float>(lat, W.sap, W.tfield, v, ncy, 4, st))) return rc;
            QXD_CUDA(cudaMemcpyAsync(v, W.tfield, 6 * V * sizeof(float4), cudaMemcpyDeviceToDevice, st));
        }
        if ((rc = orthonormalise(lat, W, st))) return rc;
    }
    return build_little(lat, W, st);
}

int qxd_dfl_set_basis(qxd_lattice* lat, int ns, const void* const* psi) {
    int rc = dfl_checks(lat, ns, "qxd_dfl_set_basis");
    if (rc) return rc;
    if (!psi) return fail(QXD_ERR_ARG, "qxd_dfl_set_basis: NULL fields");
    for (int k = 0; k < ns; ++k)
        if (!psi[k]) return fail(QXD_ERR_ARG, "qxd_dfl_set_basis: NULL field");
    DflWork& W = *lat->dfl;
    cudaStream_t st = lat->stream;
    const size_t V = (size_t)lat->g.V;
    W.ready = false;
    if ((rc = ensure_scratch(lat))) return rc;
    for (int k = 0; k < ns; ++k) {
        // lexicographic FP64 -> native FP64 (scratch) -> native FP32
        if ((rc = launch_pack(lat, lat->scratch_in, psi[k], QXD_FP64, st))) return rc;
        if ((rc = blas_d2f_native(V, (const double2*)lat->scratch_in, (float2*)(W.basis + (size_t)k * 6 * V), st)))
            return rc;
    }
    if ((rc = orthonormalise(lat, W, st))) return rc;
    return build_little(lat, W, st);
}

int qxd_dfl_refresh(qxd_lattice* lat) {
    if (!lat) return fail(QXD_ERR_ARG, "qxd_dfl_refresh: lat is NULL");
    if (!lat->dfl || !lat->dfl->basis || lat->dfl->ns == 0)
        return fail(QXD_ERR_STATE, "qxd_dfl_refresh: no deflation subspace (qxd_dfl_subspace first)");
    if (!qxd::clover_ready(lat)) return fail(QXD_ERR_STATE, "qxd_dfl_refresh: needs qxd_sw_build first");
    return build_little(lat, *lat->dfl, lat->stream);
}

int qxd_dfl_little(qxd_lattice* lat, double* A_out, int* ns_out, int* nblk_out) {
    if (!lat) return fail(QXD_ERR_ARG, "qxd_dfl_little: lat is NULL");
    if (!lat->dfl || !lat->dfl->ready) return fail(QXD_ERR_STATE, "qxd_dfl_little: no little operator");
    DflWork& W = *lat->dfl;
    if (ns_out) *ns_out = W.ns;
    if (nblk_out) *nblk_out = W.d.nblk;
    if (!A_out) return QXD_OK;
    const size_t n = (size_t)W.d.nblk * 9 * W.ns * W.ns;
    std::vector<float2> h(n);
    QXD_CUDA(cudaMemcpyAsync(h.data(), W.A, n * sizeof(float2), cudaMemcpyDeviceToHost, lat->stream));
    QXD_CUDA(cudaStreamSynchronize(lat->stream));
    for (size_t i = 0; i < n; ++i) {
        A_out[2 * i] = h[i].x;
        A_out[2 * i + 1] = h[i].y;
    }
    return QXD_OK;
}

int qxd_dfl_basis(qxd_lattice* lat, int k, void* out) {
    if (!lat || !out) return fail(QXD_ERR_ARG, "qxd_dfl_basis: NULL argument");
    if (!lat->dfl || !lat->dfl->basis || lat->dfl->ns == 0)
        return fail(QXD_ERR_STATE, "qxd_dfl_basis: no deflation subspace");
    if (k < 0 || k >= lat->dfl->ns) return fail(QXD_ERR_ARG, "qxd_dfl_basis: k out of range");
    int rc;
    if ((rc = ensure_scratch(lat))) return rc;
    const size_t V = (size_t)lat->g.V;
    // native FP32 -> native FP64 -> lexicographic
    k_f32_to_f64_native<<<(unsigned)((V + 255) / 256), 256, 0, lat->stream>>>(
        lat->g.V, lat->dfl->basis + (size_t)k * 6 * V, (double2*)lat->scratch_in);
    QXD_LAUNCHED("k_f32_to_f64_native");
    if ((rc = launch_unpack(lat, out, lat->scratch_in, QXD_FP64, lat->stream))) return rc;
    QXD_CUDA(cudaStreamSynchronize(lat->stream));
    return QXD_OK;
}

}  // extern "C"
