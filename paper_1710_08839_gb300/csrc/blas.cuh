// Vector kernels of the Krylov solvers on flat complex arrays (FP32 as
// float2, FP64 as double2). Inner products and norms accumulate in FP64 and
// are reduced deterministically: a fixed grid writes per-block partial sums,
// one block adds them in a fixed order (a warp per value), so the result does
// not depend on timing or on other work on the GPU.
#pragma once

#include <complex>

#include "qxd_internal.cuh"

namespace qxd {

constexpr int BLAS_KMAX = 16;       // vectors per multi-vector operation
constexpr int RED_BLOCKS = 608;     // 4 x 152 SMs
constexpr int RED_THREADS = 256;

template <typename T>
struct VecList {
    const T* p[BLAS_KMAX];
};
struct CoefList {
    double re[BLAS_KMAX];
    double im[BLAS_KMAX];
};

// device workspace of the reductions
struct Reducer {
    double* partials = nullptr;  // [RED_BLOCKS][2 * BLAS_KMAX]
    double* d_res = nullptr;     // [2 * BLAS_KMAX]
    double* h_res = nullptr;     // pinned host copy
    int init();
    void release();
};

using cd = std::complex<double>;

// block-wide sum of NC values per thread into partials[blockIdx.x][0..NC)
template <int NC>
__device__ __forceinline__ void block_reduce_store(const double v[NC], int nc, double* __restrict__ partials) {
    __shared__ double sh[RED_THREADS / 32][2 * BLAS_KMAX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        if (c >= nc) break;
        double x = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[warp][c] = x;
    }
    __syncthreads();
    if (threadIdx.x < nc) {
        double x = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) x += sh[w][threadIdx.x];
        partials[(size_t)blockIdx.x * 2 * BLAS_KMAX + threadIdx.x] = x;
    }
}

// Sum of column c of nblocks partial rows (stride 2 BLAS_KMAX) by one warp:
// lane l adds rows l, l + 32, ... in order, then a butterfly of shuffles.
// Every lane ends with the same bits (each level adds the same two values in
// both lanes), and the order is fixed, so the sum is deterministic.
__device__ __forceinline__ double warp_sum_column(const double* __restrict__ partials, int c, int nblocks) {
    const int lane = threadIdx.x & 31;
    double x = 0.0;
    for (int b = lane; b < nblocks; b += 32) x += __ldcg(partials + (size_t)b * 2 * BLAS_KMAX + c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// threads of the final reduction: one warp per column, columns taken in turn
constexpr int RED_FINAL_THREADS = 256;

// sums the RED_BLOCKS partials of the first nc values in a fixed order into
// red.h_res[0..nc) (synchronises the stream)
int reduce_finish(Reducer& red, int nc, cudaStream_t st);

// out[j] = <x_j, y> = sum conj(x_j) y, j < k   (synchronises the stream)
template <typename T>
int blas_mdot(Reducer& red, size_t n, int k, const VecList<T>& xs, const T* y, cd* out, cudaStream_t st);
// |x|^2
template <typename T>
int blas_norm2(Reducer& red, size_t n, const T* x, double* out, cudaStream_t st);
// y -= sum_j c_j x_j ; returns |y|^2
template <typename T>
int blas_maxpy_norm(Reducer& red, size_t n, int k, const CoefList& c, const VecList<T>& xs, T* y, double* nrm2,
                    cudaStream_t st);
// y -= c x (no reduction)
template <typename T>
int blas_caxpy(size_t n, cd c, const T* x, T* y, cudaStream_t st);
// x *= s
template <typename T>
int blas_scale(size_t n, double s, T* x, cudaStream_t st);
// x64 += sum_j c_j v_j  (v_j in precision T)
template <typename T>
int blas_update_x(size_t n, int k, const CoefList& c, const VecList<T>& vs, double2* x, cudaStream_t st);
// r = b - t, returns |r|^2
int blas_sub_norm(Reducer& red, size_t n, const double2* b, const double2* t, double2* r, double* nrm2,
                  cudaStream_t st);
// native FP64 -> native FP32 spinor layout (S sites) and x64 += sum_j c_j v_j
// with v_j native FP32 spinors; the two layouts order components differently
int blas_d2f_native(size_t S, const double2* in, float2* out, cudaStream_t st);
int blas_update_x_native32(size_t S, int k, const CoefList& c, const VecList<float2>& vs, double2* x,
                           cudaStream_t st);
// elementwise precision conversion (same element order)
int blas_d2f(size_t n, const double2* in, float2* out, cudaStream_t st);
int blas_f2d(size_t n, const float2* in, double2* out, cudaStream_t st);

}  // namespace qxd

namespace qxd {

// ---------------------------------------------------------------------------
// Batched forms: one launch serves many independent jobs (grid.y = job). Each
// job's reduction uses exactly the grid and order of the single-job kernel,
// so a job's numbers do not depend on which other jobs share the launch.
// ---------------------------------------------------------------------------
struct BJob {
    size_t n;              // complex numbers (or sites S for the native kernels)
    int k;                 // vectors in xs
    const void* xs[BLAS_KMAX];
    const void* y;         // read operand
    void* out;             // written operand
    const void* b;         // extra operand (sub_norm)
    double cre[BLAS_KMAX], cim[BLAS_KMAX];
    double s;              // scale
};

struct BatchReducer {
    double* partials = nullptr;  // [jobs][RED_BLOCKS][2 KMAX]
    double* d_res = nullptr;     // [jobs][2 KMAX]
    double* h_res = nullptr;     // pinned
    BJob* d_jobs = nullptr;
    BJob* h_jobs = nullptr;      // host copy of the job table (pageable)
    int cap = 0;
    int ensure(int jobs);
    void release();
};

enum BOp { B_MDOT_F32, B_MAXPY_NORM_F32, B_SCALE_F32, B_NORM2_F64, B_SUB_NORM_F64, B_D2F_NATIVE,
           B_UPDATE_X_NATIVE32 };

// run op on the first `jobs` entries of red.h_jobs; reductions return nc
// values per job in red.h_res[job * 2 KMAX + c] (synchronises the stream)
int blas_batch(BatchReducer& red, BOp op, int jobs, int nc, cudaStream_t st);

}  // namespace qxd
