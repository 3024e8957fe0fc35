// Vector kernels of the Krylov solvers (see blas.cuh).
//
// FP32 vectors (float2) are combined in FP32 arithmetic; their inner
// products and norms are summed in FP32 over runs of RUN products per
// thread, and each run is added to an FP64 accumulator, which carries the
// long sums over runs, threads and blocks. (GB300 does FP64 at 1/63 of the
// FP32 rate: with every product in FP64, these kernels were bound by the
// FP64 units instead of memory.) FP64 vectors use FP64 throughout.
#include <algorithm>
#include <new>
#include <type_traits>

#include "blas.cuh"

namespace qxd {

namespace {

constexpr int RUN = 16;  // FP32 products summed before they join the FP64 accumulator

template <typename T>
constexpr bool is_f32() { return std::is_same<T, float2>::value; }

__device__ __forceinline__ double2 ld(const float2* p, size_t i) {
    float2 v = p[i];
    return make_double2(v.x, v.y);
}
__device__ __forceinline__ double2 ld(const double2* p, size_t i) { return p[i]; }
__device__ __forceinline__ void st_(double2* p, size_t i, double2 v) { p[i] = v; }

__global__ void __launch_bounds__(RED_FINAL_THREADS) k_reduce_final(const double* __restrict__ partials, int nc,
                                                                     double* __restrict__ res) {
    for (int c = threadIdx.x >> 5; c < nc; c += RED_FINAL_THREADS / 32) {
        const double x = warp_sum_column(partials, c, RED_BLOCKS);
        if ((threadIdx.x & 31) == 0) res[c] = x;
    }
}


template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_mdot(size_t n, int k, VecList<T> xs, const T* __restrict__ y,
                                                      double* __restrict__ partials) {
    // FP64 vectors (the FP32 form is k_mdot32)
    double acc[2 * BLAS_KMAX];
#pragma unroll
    for (int c = 0; c < 2 * BLAS_KMAX; ++c) acc[c] = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 b = ld(y, i);
#pragma unroll
        for (int j = 0; j < BLAS_KMAX; ++j) {
            if (j >= k) break;
            const double2 a = ld(xs.p[j], i);
            acc[2 * j] += a.x * b.x + a.y * b.y;
            acc[2 * j + 1] += a.x * b.y - a.y * b.x;
        }
    }
    block_reduce_store<2 * BLAS_KMAX>(acc, 2 * k, partials);
}

// Elements per loop iteration of the FP32 multi-vector kernels: with few
// vectors a thread has too few loads in flight to cover the DRAM latency
// (one dot product ran at 2.1 TB/s), so it takes U elements at a time.
template <int K>
constexpr int elems_per_iter() { return K <= 1 ? 4 : K <= 3 ? 2 : 1; }

// FP32 multi-dot over K <= 8 vectors with the vector count fixed at compile
// time (K sums in FP32 runs and FP64 registers, K pointers): the general form
// with 16 of each spills and reads at 0.4 of the HBM bandwidth. Partials go to
// columns [col0, col0 + 2K) of each block's row.
template <int K>
__global__ void __launch_bounds__(RED_THREADS) k_mdot32(size_t n, VecList<float2> xs, const float2* __restrict__ y,
                                                        double* __restrict__ partials, int col0) {
    constexpr int U = elems_per_iter<K>();
    float run[2 * K];
    double acc[2 * K];
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) {
        run[c] = 0.f;
        acc[c] = 0.0;
    }
    int cnt = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += U * stride) {
        float2 b[U], a[U][K];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t i = i0 + u * stride;
            b[u] = i < n ? y[i] : make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < K; ++j) a[u][j] = i < n ? xs.p[j][i] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int j = 0; j < K; ++j) {
                run[2 * j] = fmaf(a[u][j].x, b[u].x, fmaf(a[u][j].y, b[u].y, run[2 * j]));
                run[2 * j + 1] = fmaf(a[u][j].x, b[u].y, fmaf(-a[u][j].y, b[u].x, run[2 * j + 1]));
            }
        if ((cnt += U) >= RUN) {
#pragma unroll
            for (int c = 0; c < 2 * K; ++c) {
                acc[c] += run[c];
                run[c] = 0.f;
            }
            cnt = 0;
        }
    }
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) acc[c] += run[c];
    block_reduce_store<2 * K>(acc, 2 * K, partials + col0);
}

// y -= sum_j c_j x_j in FP32 over K <= 16 vectors (count fixed at compile
// time); |y|^2 of the result in FP32 runs added to an FP64 sum
template <int K>
__global__ void __launch_bounds__(RED_THREADS) k_maxpy_norm32(size_t n, CoefList c, VecList<float2> xs,
                                                              float2* __restrict__ y, double* __restrict__ partials) {
    constexpr int U = elems_per_iter<K>();
    float cr[K], ci[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        cr[j] = (float)c.re[j];
        ci[j] = (float)c.im[j];
    }
    float run = 0.f;
    double acc[1] = {0.0};
    int cnt = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += U * stride) {
        float2 b[U], a[U][K];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t i = i0 + u * stride;
            b[u] = i < n ? y[i] : make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < K; ++j) a[u][j] = i < n ? xs.p[j][i] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t i = i0 + u * stride;
            if (i >= n) continue;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                b[u].x = fmaf(-cr[j], a[u][j].x, fmaf(ci[j], a[u][j].y, b[u].x));
                b[u].y = fmaf(-cr[j], a[u][j].y, fmaf(-ci[j], a[u][j].x, b[u].y));
            }
            y[i] = b[u];
            run = fmaf(b[u].x, b[u].x, fmaf(b[u].y, b[u].y, run));
        }
        if ((cnt += U) >= RUN) {
            acc[0] += run;
            run = 0.f;
            cnt = 0;
        }
    }
    acc[0] += run;
    block_reduce_store<1>(acc, 1, partials);
}

// vectors [j0, j0 + kk) of xs, kk <= 8
int launch_mdot32(size_t n, int j0, int kk, const VecList<float2>& xs, const float2* y, double* partials,
                  cudaStream_t st) {
    VecList<float2> sub{};
    for (int j = 0; j < kk; ++j) sub.p[j] = xs.p[j0 + j];
    const int col0 = 2 * j0;
    switch (kk) {
#define QXD_MDOT32(K) \
    case K: k_mdot32<K><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, sub, y, partials, col0); break;
        QXD_MDOT32(1) QXD_MDOT32(2) QXD_MDOT32(3) QXD_MDOT32(4) QXD_MDOT32(5) QXD_MDOT32(6) QXD_MDOT32(7)
        QXD_MDOT32(8)
#undef QXD_MDOT32
        default: return fail(QXD_ERR_ARG, "multi-dot: bad vector count");
    }
    QXD_LAUNCHED("k_mdot32");
    return QXD_OK;
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_norm2(size_t n, const T* __restrict__ x,
                                                       double* __restrict__ partials) {
    double acc[1] = {0.0};
    if constexpr (is_f32<T>()) {
        float run = 0.f;
        int cnt = 0;
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
            const float2 a = x[i];
            run = fmaf(a.x, a.x, fmaf(a.y, a.y, run));
            if (++cnt == RUN) {
                acc[0] += run;
                run = 0.f;
                cnt = 0;
            }
        }
        acc[0] += run;
    } else {
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
            const double2 a = ld(x, i);
            acc[0] += a.x * a.x + a.y * a.y;
        }
    }
    block_reduce_store<1>(acc, 1, partials);
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_maxpy_norm(size_t n, int k, CoefList c, VecList<T> xs,
                                                            T* __restrict__ y, double* __restrict__ partials) {
    // FP64 vectors (the FP32 form is k_maxpy_norm32)
    double acc[1] = {0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double2 b = ld(y, i);
#pragma unroll
        for (int j = 0; j < BLAS_KMAX; ++j) {
            if (j >= k) break;
            const double2 a = ld(xs.p[j], i);
            b.x -= c.re[j] * a.x - c.im[j] * a.y;
            b.y -= c.re[j] * a.y + c.im[j] * a.x;
        }
        st_(y, i, b);
        const double2 r = ld(y, i);  // norm of the stored (rounded) vector
        acc[0] += r.x * r.x + r.y * r.y;
    }
    block_reduce_store<1>(acc, 1, partials);
}

template <typename T>
__global__ void k_caxpy(size_t n, double cre, double cim, const T* __restrict__ x, T* __restrict__ y) {
    if constexpr (is_f32<T>()) {
        const float cr = (float)cre, ci = (float)cim;
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
            const float2 a = x[i];
            float2 b = y[i];
            b.x = fmaf(-cr, a.x, fmaf(ci, a.y, b.x));
            b.y = fmaf(-cr, a.y, fmaf(-ci, a.x, b.y));
            y[i] = b;
        }
    } else {
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
            const double2 a = ld(x, i);
            double2 b = ld(y, i);
            b.x -= cre * a.x - cim * a.y;
            b.y -= cre * a.y + cim * a.x;
            st_(y, i, b);
        }
    }
}

template <typename T>
__global__ void k_scale(size_t n, double s, T* __restrict__ x) {
    if constexpr (is_f32<T>()) {
        const float sf = (float)s;
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
            const float2 a = x[i];
            x[i] = make_float2(a.x * sf, a.y * sf);
        }
    } else {
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
            double2 a = ld(x, i);
            a.x *= s;
            a.y *= s;
            st_(x, i, a);
        }
    }
}

// Native spinor layouts differ between precisions: FP64 keeps component c
// (0..11) of site s at double2 index c * S + s, FP32 keeps it at float2
// index (c / 2) * 2S + 2s + c % 2 (two components per float4). S is the
// number of sites of the array (V, or V/2 for a half-lattice field).
__device__ __forceinline__ size_t f32_index(size_t S, size_t c, size_t s) { return (c >> 1) * 2 * S + 2 * s + (c & 1); }

// x64 += sum_j c_j v_j: the correction summed in FP32 (the v_j are FP32),
// added to x in FP64
__device__ __forceinline__ void update_x32_site(size_t S, size_t s, int k, const double* cre, const double* cim,
                                                const float2* const* vs, double2* __restrict__ x) {
    float cr[BLAS_KMAX], ci[BLAS_KMAX];
#pragma unroll
    for (int j = 0; j < BLAS_KMAX; ++j) {
        cr[j] = j < k ? (float)cre[j] : 0.f;
        ci[j] = j < k ? (float)cim[j] : 0.f;
    }
#pragma unroll
    for (int comp = 0; comp < 12; ++comp) {
        const size_t i32 = f32_index(S, comp, s);
        float dx = 0.f, dy = 0.f;
#pragma unroll
        for (int j = 0; j < BLAS_KMAX; ++j) {
            if (j >= k) break;
            const float2 a = vs[j][i32];
            dx = fmaf(cr[j], a.x, fmaf(-ci[j], a.y, dx));
            dy = fmaf(cr[j], a.y, fmaf(ci[j], a.x, dy));
        }
        double2 b = x[comp * S + s];
        b.x += dx;
        b.y += dy;
        x[comp * S + s] = b;
    }
}

__global__ void k_update_x_native32(size_t S, int k, CoefList c, VecList<float2> vs, double2* __restrict__ x) {
    for (size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (size_t)gridDim.x * blockDim.x)
        update_x32_site(S, s, k, c.re, c.im, vs.p, x);
}

__global__ void k_d2f_native(size_t S, const double2* __restrict__ in, float2* __restrict__ out) {
    for (size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int comp = 0; comp < 12; ++comp) {
            const double2 v = in[comp * S + s];
            out[f32_index(S, comp, s)] = make_float2((float)v.x, (float)v.y);
        }
    }
}

template <typename T>
__global__ void k_update_x(size_t n, int k, CoefList c, VecList<T> vs, double2* __restrict__ x) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double2 b = x[i];
#pragma unroll
        for (int j = 0; j < BLAS_KMAX; ++j) {
            if (j >= k) break;
            const double2 a = ld(vs.p[j], i);
            b.x += c.re[j] * a.x - c.im[j] * a.y;
            b.y += c.re[j] * a.y + c.im[j] * a.x;
        }
        x[i] = b;
    }
}

__global__ void __launch_bounds__(RED_THREADS) k_sub_norm(size_t n, const double2* __restrict__ b,
                                                          const double2* __restrict__ t, double2* __restrict__ r,
                                                          double* __restrict__ partials) {
    double acc[1] = {0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 v = make_double2(b[i].x - t[i].x, b[i].y - t[i].y);
        r[i] = v;
        acc[0] += v.x * v.x + v.y * v.y;
    }
    block_reduce_store<1>(acc, 1, partials);
}

__global__ void k_d2f(size_t n, const double2* __restrict__ in, float2* __restrict__ out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
__global__ void k_f2d(size_t n, const float2* __restrict__ in, double2* __restrict__ out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_double2(in[i].x, in[i].y);
}

inline int ew_blocks(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b < 4 * 152 * 4 ? b : 4 * 152 * 4);
}

}  // namespace

int reduce_finish(Reducer& red, int nc, cudaStream_t st) {
    k_reduce_final<<<1, RED_FINAL_THREADS, 0, st>>>(red.partials, nc, red.d_res);
    QXD_LAUNCHED("k_reduce_final");
    QXD_CUDA(cudaMemcpyAsync(red.h_res, red.d_res, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
    QXD_CUDA(cudaStreamSynchronize(st));
    return QXD_OK;
}

int Reducer::init() {
    if (partials) return QXD_OK;
    QXD_CUDA(cudaMalloc(&partials, sizeof(double) * RED_BLOCKS * 2 * BLAS_KMAX));
    QXD_CUDA(cudaMalloc(&d_res, sizeof(double) * 2 * BLAS_KMAX));
    QXD_CUDA(cudaMallocHost(&h_res, sizeof(double) * 2 * BLAS_KMAX));
    return QXD_OK;
}

void Reducer::release() {
    if (partials) cudaFree(partials);
    if (d_res) cudaFree(d_res);
    if (h_res) cudaFreeHost(h_res);
    partials = d_res = h_res = nullptr;
}

template <typename T>
int blas_mdot(Reducer& red, size_t n, int k, const VecList<T>& xs, const T* y, cd* out, cudaStream_t st) {
    if (k <= 0) return QXD_OK;
    if constexpr (is_f32<T>()) {
        // at most 8 vectors per pass (y read once per pass)
        for (int j0 = 0; j0 < k; j0 += 8) {
            const int rc = launch_mdot32(n, j0, std::min(8, k - j0), xs, y, red.partials, st);
            if (rc) return rc;
        }
    } else {
        k_mdot<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, k, xs, y, red.partials);
        QXD_LAUNCHED("k_mdot");
    }
    int rc = reduce_finish(red, 2 * k, st);
    if (rc) return rc;
    for (int j = 0; j < k; ++j) out[j] = cd(red.h_res[2 * j], red.h_res[2 * j + 1]);
    return QXD_OK;
}

template <typename T>
int blas_norm2(Reducer& red, size_t n, const T* x, double* out, cudaStream_t st) {
    k_norm2<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, x, red.partials);
    QXD_LAUNCHED("k_norm2");
    int rc = reduce_finish(red, 1, st);
    if (rc) return rc;
    *out = red.h_res[0];
    return QXD_OK;
}

template <typename T>
int blas_maxpy_norm(Reducer& red, size_t n, int k, const CoefList& c, const VecList<T>& xs, T* y, double* nrm2,
                    cudaStream_t st) {
    if constexpr (is_f32<T>()) {
        switch (k) {
#define QXD_MAXPY32(K) \
    case K: k_maxpy_norm32<K><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, c, xs, y, red.partials); break;
            QXD_MAXPY32(1) QXD_MAXPY32(2) QXD_MAXPY32(3) QXD_MAXPY32(4) QXD_MAXPY32(5) QXD_MAXPY32(6)
            QXD_MAXPY32(7) QXD_MAXPY32(8) QXD_MAXPY32(9) QXD_MAXPY32(10) QXD_MAXPY32(11) QXD_MAXPY32(12)
            QXD_MAXPY32(13) QXD_MAXPY32(14) QXD_MAXPY32(15) QXD_MAXPY32(16)
#undef QXD_MAXPY32
            case 0: k_norm2<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, y, red.partials); break;  // nothing to subtract
            default: return fail(QXD_ERR_ARG, "multi-axpy: bad vector count");
        }
        QXD_LAUNCHED("k_maxpy_norm32");
    } else {
        k_maxpy_norm<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, k, c, xs, y, red.partials);
        QXD_LAUNCHED("k_maxpy_norm");
    }
    int rc = reduce_finish(red, 1, st);
    if (rc) return rc;
    *nrm2 = red.h_res[0];
    return QXD_OK;
}

template <typename T>
int blas_caxpy(size_t n, cd c, const T* x, T* y, cudaStream_t st) {
    k_caxpy<T><<<ew_blocks(n), 256, 0, st>>>(n, c.real(), c.imag(), x, y);
    QXD_LAUNCHED("k_caxpy");
    return QXD_OK;
}

template <typename T>
int blas_scale(size_t n, double s, T* x, cudaStream_t st) {
    k_scale<T><<<ew_blocks(n), 256, 0, st>>>(n, s, x);
    QXD_LAUNCHED("k_scale");
    return QXD_OK;
}

template <typename T>
int blas_update_x(size_t n, int k, const CoefList& c, const VecList<T>& vs, double2* x, cudaStream_t st) {
    if (k <= 0) return QXD_OK;
    k_update_x<T><<<ew_blocks(n), 256, 0, st>>>(n, k, c, vs, x);
    QXD_LAUNCHED("k_update_x");
    return QXD_OK;
}

int blas_update_x_native32(size_t S, int k, const CoefList& c, const VecList<float2>& vs, double2* x,
                           cudaStream_t st) {
    if (k <= 0) return QXD_OK;
    k_update_x_native32<<<ew_blocks(S), 256, 0, st>>>(S, k, c, vs, x);
    QXD_LAUNCHED("k_update_x_native32");
    return QXD_OK;
}

int blas_d2f_native(size_t S, const double2* in, float2* out, cudaStream_t st) {
    k_d2f_native<<<ew_blocks(S), 256, 0, st>>>(S, in, out);
    QXD_LAUNCHED("k_d2f_native");
    return QXD_OK;
}

int blas_sub_norm(Reducer& red, size_t n, const double2* b, const double2* t, double2* r, double* nrm2,
                  cudaStream_t st) {
    k_sub_norm<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, b, t, r, red.partials);
    QXD_LAUNCHED("k_sub_norm");
    int rc = reduce_finish(red, 1, st);
    if (rc) return rc;
    *nrm2 = red.h_res[0];
    return QXD_OK;
}

int blas_d2f(size_t n, const double2* in, float2* out, cudaStream_t st) {
    k_d2f<<<ew_blocks(n), 256, 0, st>>>(n, in, out);
    QXD_LAUNCHED("k_d2f");
    return QXD_OK;
}

int blas_f2d(size_t n, const float2* in, double2* out, cudaStream_t st) {
    k_f2d<<<ew_blocks(n), 256, 0, st>>>(n, in, out);
    QXD_LAUNCHED("k_f2d");
    return QXD_OK;
}

#define QXD_BLAS_INST(T)                                                                                  \
    template int blas_mdot<T>(Reducer&, size_t, int, const VecList<T>&, const T*, cd*, cudaStream_t);   \
    template int blas_norm2<T>(Reducer&, size_t, const T*, double*, cudaStream_t);                      \
    template int blas_maxpy_norm<T>(Reducer&, size_t, int, const CoefList&, const VecList<T>&, T*,      \
                                    double*, cudaStream_t);                                             \
    template int blas_caxpy<T>(size_t, cd, const T*, T*, cudaStream_t);                                 \
    template int blas_scale<T>(size_t, double, T*, cudaStream_t);                                       \
    template int blas_update_x<T>(size_t, int, const CoefList&, const VecList<T>&, double2*, cudaStream_t);
QXD_BLAS_INST(float2)
QXD_BLAS_INST(double2)

}  // namespace qxd

namespace qxd {

namespace {

__device__ __forceinline__ void block_reduce_store_at(double* v, int nc, double* __restrict__ partials) {
    __shared__ double sh[RED_THREADS / 32][2 * BLAS_KMAX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = 0; c < nc; ++c) {
        double x = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[warp][c] = x;
    }
    __syncthreads();
    if (threadIdx.x < nc) {
        double x = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) x += sh[w][threadIdx.x];
        partials[threadIdx.x] = x;
    }
}

// block-wide sum of NC values per thread into part[0 .. NC) (this block's row)
template <int NC>
__device__ __forceinline__ void block_reduce_row(const double v[NC], double* __restrict__ part,
                                                 double (*sh)[2 * BLAS_KMAX]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        double x = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[warp][c] = x;
    }
    __syncthreads();
    if (threadIdx.x < NC) {
        double x = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) x += sh[w][threadIdx.x];
        part[threadIdx.x] = x;
    }
    __syncthreads();  // sh is reused by the next pass
}

// Batched FP32 multi-dot and multi-axpy. Each job is taken in passes of at
// most 8 vectors with the vector count fixed at compile time, chosen by the
// job's own count: a job's element order and run lengths do not depend on
// the other jobs of the batch, so a request gives the same bits alone and
// in a mix.

// <x_j, y> for K vectors of one job into part[0 .. 2K)
template <int K>
__device__ __forceinline__ void mdot_pass32(size_t n, const void* const* xsv, const float2* __restrict__ y,
                                            double* part, double (*sh)[2 * BLAS_KMAX]) {
    constexpr int U = elems_per_iter<K>();
    const float2* xs[K];
#pragma unroll
    for (int j = 0; j < K; ++j) xs[j] = (const float2*)xsv[j];
    float run[2 * K];
    double acc[2 * K];
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) {
        run[c] = 0.f;
        acc[c] = 0.0;
    }
    int cnt = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += U * stride) {
        float2 b[U], a[U][K];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t i = i0 + u * stride;
            b[u] = i < n ? y[i] : make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < K; ++j) a[u][j] = i < n ? xs[j][i] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int j = 0; j < K; ++j) {
                run[2 * j] = fmaf(a[u][j].x, b[u].x, fmaf(a[u][j].y, b[u].y, run[2 * j]));
                run[2 * j + 1] = fmaf(a[u][j].x, b[u].y, fmaf(-a[u][j].y, b[u].x, run[2 * j + 1]));
            }
        if ((cnt += U) >= RUN) {
#pragma unroll
            for (int c = 0; c < 2 * K; ++c) {
                acc[c] += run[c];
                run[c] = 0.f;
            }
            cnt = 0;
        }
    }
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) acc[c] += run[c];
    block_reduce_row<2 * K>(acc, part, sh);
}

__global__ void __launch_bounds__(RED_THREADS) k_blas_mdot32(const BJob* __restrict__ jobs,
                                                             double* __restrict__ partials) {
    __shared__ double sh[RED_THREADS / 32][2 * BLAS_KMAX];
    const BJob& J = jobs[blockIdx.y];
    double* part = partials + ((size_t)blockIdx.y * RED_BLOCKS + blockIdx.x) * 2 * BLAS_KMAX;
    const float2* y = (const float2*)J.y;
    for (int j0 = 0; j0 < J.k; j0 += 8) {
        const void* const* xs = J.xs + j0;
        double* p = part + 2 * j0;
        switch (J.k - j0 < 8 ? J.k - j0 : 8) {
            case 1: mdot_pass32<1>(J.n, xs, y, p, sh); break;
            case 2: mdot_pass32<2>(J.n, xs, y, p, sh); break;
            case 3: mdot_pass32<3>(J.n, xs, y, p, sh); break;
            case 4: mdot_pass32<4>(J.n, xs, y, p, sh); break;
            case 5: mdot_pass32<5>(J.n, xs, y, p, sh); break;
            case 6: mdot_pass32<6>(J.n, xs, y, p, sh); break;
            case 7: mdot_pass32<7>(J.n, xs, y, p, sh); break;
            default: mdot_pass32<8>(J.n, xs, y, p, sh); break;
        }
    }
}

// y -= sum_j c_j x_j for K vectors of one job; with `norm`, returns this
// thread's |y|^2 (FP32 runs added in FP64)
template <int K>
__device__ __forceinline__ double maxpy_pass32(size_t n, const void* const* xsv, const double* cre,
                                               const double* cim, float2* __restrict__ y, bool norm) {
    constexpr int U = elems_per_iter<K>();
    constexpr int KA = K > 0 ? K : 1;
    const float2* xs[KA];
    float cr[KA], ci[KA];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        xs[j] = (const float2*)xsv[j];
        cr[j] = (float)cre[j];
        ci[j] = (float)cim[j];
    }
    float run = 0.f;
    double acc = 0.0;
    int cnt = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += U * stride) {
        float2 b[U], a[U][KA];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t i = i0 + u * stride;
            b[u] = i < n ? y[i] : make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < K; ++j) a[u][j] = i < n ? xs[j][i] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t i = i0 + u * stride;
            if (i >= n) continue;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                b[u].x = fmaf(-cr[j], a[u][j].x, fmaf(ci[j], a[u][j].y, b[u].x));
                b[u].y = fmaf(-cr[j], a[u][j].y, fmaf(-ci[j], a[u][j].x, b[u].y));
            }
            if (K > 0) y[i] = b[u];
            run = fmaf(b[u].x, b[u].x, fmaf(b[u].y, b[u].y, run));
        }
        if ((cnt += U) >= RUN) {
            acc += run;
            run = 0.f;
            cnt = 0;
        }
    }
    return norm ? acc + run : 0.0;
}

__global__ void __launch_bounds__(RED_THREADS) k_blas_maxpy32(const BJob* __restrict__ jobs,
                                                              double* __restrict__ partials) {
    __shared__ double sh[RED_THREADS / 32][2 * BLAS_KMAX];
    const BJob& J = jobs[blockIdx.y];
    double* part = partials + ((size_t)blockIdx.y * RED_BLOCKS + blockIdx.x) * 2 * BLAS_KMAX;
    float2* y = (float2*)J.out;
    double acc[1] = {0.0};
    for (int j0 = 0;; j0 += 8) {  // passes of up to 8 vectors; |y|^2 in the last
        const int kk = J.k - j0 < 8 ? J.k - j0 : 8;
        const bool last = j0 + kk >= J.k;
        const void* const* xs = J.xs + j0;
        const double *cr = J.cre + j0, *ci = J.cim + j0;
        double a = 0.0;
        switch (kk) {
            case 0: a = maxpy_pass32<0>(J.n, xs, cr, ci, y, last); break;
            case 1: a = maxpy_pass32<1>(J.n, xs, cr, ci, y, last); break;
            case 2: a = maxpy_pass32<2>(J.n, xs, cr, ci, y, last); break;
            case 3: a = maxpy_pass32<3>(J.n, xs, cr, ci, y, last); break;
            case 4: a = maxpy_pass32<4>(J.n, xs, cr, ci, y, last); break;
            case 5: a = maxpy_pass32<5>(J.n, xs, cr, ci, y, last); break;
            case 6: a = maxpy_pass32<6>(J.n, xs, cr, ci, y, last); break;
            case 7: a = maxpy_pass32<7>(J.n, xs, cr, ci, y, last); break;
            default: a = maxpy_pass32<8>(J.n, xs, cr, ci, y, last); break;
        }
        if (last) {
            acc[0] = a;
            break;
        }
    }
    block_reduce_row<1>(acc, part, sh);
}

// one kernel for all batched operations; the switch is uniform per launch
__global__ void __launch_bounds__(RED_THREADS) k_blas_batch(int op, const BJob* __restrict__ jobs,
                                                            double* __restrict__ partials) {
    const BJob& J = jobs[blockIdx.y];
    double* part = partials + ((size_t)blockIdx.y * RED_BLOCKS + blockIdx.x) * 2 * BLAS_KMAX;
    const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t step = (size_t)gridDim.x * blockDim.x;
    if (op == B_NORM2_F64) {
        double acc[1] = {0.0};
        const double2* x = (const double2*)J.y;
        for (size_t i = i0; i < J.n; i += step) acc[0] += x[i].x * x[i].x + x[i].y * x[i].y;
        block_reduce_store_at(acc, 1, part);
    } else if (op == B_SUB_NORM_F64) {
        double acc[1] = {0.0};
        const double2* b = (const double2*)J.b;
        const double2* t = (const double2*)J.y;
        double2* r = (double2*)J.out;
        for (size_t i = i0; i < J.n; i += step) {
            const double2 v = make_double2(b[i].x - t[i].x, b[i].y - t[i].y);
            r[i] = v;
            acc[0] += v.x * v.x + v.y * v.y;
        }
        block_reduce_store_at(acc, 1, part);
    } else if (op == B_SCALE_F32) {
        float2* x = (float2*)J.out;
        const float sf = (float)J.s;
        for (size_t i = i0; i < J.n; i += step) {
            const float2 a = x[i];
            x[i] = make_float2(a.x * sf, a.y * sf);
        }
    } else if (op == B_D2F_NATIVE) {
        const double2* in = (const double2*)J.y;
        float2* out = (float2*)J.out;
        const size_t S = J.n;
        for (size_t s = i0; s < S; s += step) {
#pragma unroll
            for (int comp = 0; comp < 12; ++comp) {
                const double2 v = in[comp * S + s];
                out[f32_index(S, comp, s)] = make_float2((float)v.x, (float)v.y);
            }
        }
    } else if (op == B_UPDATE_X_NATIVE32) {
        for (size_t s = i0; s < J.n; s += step)
            update_x32_site(J.n, s, J.k, J.cre, J.cim, (const float2* const*)J.xs, (double2*)J.out);
    }
}

__global__ void __launch_bounds__(RED_FINAL_THREADS) k_reduce_final_batch(const double* __restrict__ partials,
                                                                           int nc, double* __restrict__ res) {
    const double* p = partials + (size_t)blockIdx.x * RED_BLOCKS * 2 * BLAS_KMAX;
    for (int c = threadIdx.x >> 5; c < nc; c += RED_FINAL_THREADS / 32) {
        const double x = warp_sum_column(p, c, RED_BLOCKS);
        if ((threadIdx.x & 31) == 0) res[(size_t)blockIdx.x * 2 * BLAS_KMAX + c] = x;
    }
}

}  // namespace

int BatchReducer::ensure(int jobs) {
    if (jobs <= cap) return QXD_OK;
    release();
    const int c = jobs < 16 ? 16 : jobs;
    QXD_CUDA(cudaMalloc(&partials, sizeof(double) * (size_t)c * RED_BLOCKS * 2 * BLAS_KMAX));
    QXD_CUDA(cudaMalloc(&d_res, sizeof(double) * (size_t)c * 2 * BLAS_KMAX));
    QXD_CUDA(cudaMallocHost(&h_res, sizeof(double) * (size_t)c * 2 * BLAS_KMAX));
    QXD_CUDA(cudaMalloc(&d_jobs, sizeof(BJob) * (size_t)c));
    // pageable on purpose: a copy from pageable memory returns once the data
    // is staged, so the table can be refilled right after a launch
    h_jobs = new (std::nothrow) BJob[c];
    if (!h_jobs) return fail(QXD_ERR_OOM, "batched BLAS: host allocation failed");
    cap = c;
    return QXD_OK;
}

void BatchReducer::release() {
    if (partials) cudaFree(partials);
    if (d_res) cudaFree(d_res);
    if (h_res) cudaFreeHost(h_res);
    if (d_jobs) cudaFree(d_jobs);
    delete[] h_jobs;
    partials = d_res = h_res = nullptr;
    d_jobs = h_jobs = nullptr;
    cap = 0;
}

int blas_batch(BatchReducer& red, BOp op, int jobs, int nc, cudaStream_t st) {
    if (jobs <= 0) return QXD_OK;
    QXD_CUDA(cudaMemcpyAsync(red.d_jobs, red.h_jobs, sizeof(BJob) * (size_t)jobs, cudaMemcpyHostToDevice, st));
    const bool reduce = op == B_MDOT_F32 || op == B_MAXPY_NORM_F32 || op == B_NORM2_F64 || op == B_SUB_NORM_F64;
    // the elementwise kernels of the single-job path use ew_blocks(n); the
    // reductions use RED_BLOCKS: keep the same grid per job
    dim3 grid(RED_BLOCKS, jobs);
    if (!reduce) {
        size_t nmax = 0;
        for (int j = 0; j < jobs; ++j) nmax = nmax > red.h_jobs[j].n ? nmax : red.h_jobs[j].n;
        grid.x = ew_blocks(nmax);
    }
    if (op == B_MDOT_F32) {
        k_blas_mdot32<<<grid, RED_THREADS, 0, st>>>(red.d_jobs, red.partials);
        QXD_LAUNCHED("k_blas_mdot32");
    } else if (op == B_MAXPY_NORM_F32) {
        k_blas_maxpy32<<<grid, RED_THREADS, 0, st>>>(red.d_jobs, red.partials);
        QXD_LAUNCHED("k_blas_maxpy32");
    } else {
        k_blas_batch<<<grid, RED_THREADS, 0, st>>>((int)op, red.d_jobs, red.partials);
        QXD_LAUNCHED("k_blas_batch");
    }
    if (!reduce) return QXD_OK;
    k_reduce_final_batch<<<jobs, RED_FINAL_THREADS, 0, st>>>(red.partials, nc, red.d_res);
    QXD_LAUNCHED("k_reduce_final_batch");
    QXD_CUDA(cudaMemcpyAsync(red.h_res, red.d_res, sizeof(double) * (size_t)jobs * 2 * BLAS_KMAX,
                             cudaMemcpyDeviceToHost, st));
    QXD_CUDA(cudaStreamSynchronize(st));
    return QXD_OK;
}

}  // namespace qxd
