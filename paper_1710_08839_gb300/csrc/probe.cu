// Arithmetic-throughput probe: the FP64 and FP32 fused multiply-add rates of
// the GPU this library runs on. They are the denominators of the ALU-bound
// kernels' rooflines (FP64 D, multi-shift CG and Wilson flow; the FP32
// Schwarz block solves). The paper has no counterpart.
//
// Each thread runs NACC independent multiply-add chains a = a * b + c for
// `iters` rounds, so the issue of one chain never waits on its own previous
// result; the grid holds 8 blocks of 256 threads per SM. Three kinds:
//   QXD_PROBE_FMA64   scalar FP64 fma
//   QXD_PROBE_FMA32   scalar FP32 fma
//   QXD_PROBE_FMA32X2 paired FP32 fma (__ffma2_rn on float2: two FMAs per
//                     instruction, sm_100 and later)
// A flop is one multiply or one add: one FMA counts 2.
#include "qxd_internal.cuh"

namespace qxd {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSM = 8;
constexpr int NACC = 16;

// The accumulators are written out only if their sum equals `never`, a NaN
// passed at run time: never true, but the compiler cannot drop the chains.
__global__ void __launch_bounds__(kProbeThreads) k_fma64(double* sink, int iters, double b, double c, double never) {
    double a[NACC];
#pragma unroll
    for (int i = 0; i < NACC; ++i) a[i] = 1.0 + 1e-3 * i + 1e-6 * threadIdx.x;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < NACC; ++i) a[i] = fma(a[i], b, c);
    double s = 0;
#pragma unroll
    for (int i = 0; i < NACC; ++i) s += a[i];
    if (s == never) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_fma32(float* sink, int iters, float b, float c, float never) {
    float a[NACC];
#pragma unroll
    for (int i = 0; i < NACC; ++i) a[i] = 1.f + 1e-3f * i + 1e-6f * threadIdx.x;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < NACC; ++i) a[i] = fmaf(a[i], b, c);
    float s = 0;
#pragma unroll
    for (int i = 0; i < NACC; ++i) s += a[i];
    if (s == never) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_fma32x2(float* sink, int iters, float b, float c, float never) {
    float2 a[NACC];
#pragma unroll
    for (int i = 0; i < NACC; ++i) a[i] = make_float2(1.f + 1e-3f * i, 1.f - 1e-3f * i + 1e-6f * threadIdx.x);
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < NACC; ++i) a[i] = __ffma2_rn(a[i], bb, cc);
    float s = 0;
#pragma unroll
    for (int i = 0; i < NACC; ++i) s += a[i].x + a[i].y;
    if (s == never) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace qxd

using namespace qxd;

extern "C" int qxd_fma_rate(int kind, int iters, double* flop_per_s, void* stream) {
    if (!flop_per_s || iters < 1) return fail(QXD_ERR_ARG, "qxd_fma_rate: NULL result or iters < 1");
    if (kind != QXD_PROBE_FMA64 && kind != QXD_PROBE_FMA32 && kind != QXD_PROBE_FMA32X2)
        return fail(QXD_ERR_ARG, "qxd_fma_rate: unknown kind");
    int dev = 0, nsm = 0;
    QXD_CUDA(cudaGetDevice(&dev));
    QXD_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = nsm * kProbeBlocksPerSM;
    cudaStream_t st = (cudaStream_t)stream;
    void* sink = nullptr;
    QXD_CUDA(cudaMallocAsync(&sink, (size_t)blocks * sizeof(double), st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = QXD_OK;
    float best_ms = 0.f;
    const double nan = __builtin_nan("");
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = fail(QXD_ERR_CUDA, "qxd_fma_rate: cudaEventCreate");
    }
    // one untimed launch, then the best of three timed ones
    for (int rep = 0; rc == QXD_OK && rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        if (kind == QXD_PROBE_FMA64)
            k_fma64<<<blocks, kProbeThreads, 0, st>>>((double*)sink, iters, 0.999999, 1e-6, nan);
        else if (kind == QXD_PROBE_FMA32)
            k_fma32<<<blocks, kProbeThreads, 0, st>>>((float*)sink, iters, 0.9999f, 1e-4f, (float)nan);
        else
            k_fma32x2<<<blocks, kProbeThreads, 0, st>>>((float*)sink, iters, 0.9999f, 1e-4f, (float)nan);
        cudaEventRecord(e1, st);
        cudaError_t le = cudaGetLastError();
        if (le == cudaSuccess) le = cudaEventSynchronize(e1);
        if (le != cudaSuccess) {
            rc = cuda_fail(le, "qxd_fma_rate: probe kernel");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(sink, st);
    if (rc) return rc;
    const double fmas_per_thread = (double)iters * NACC * (kind == QXD_PROBE_FMA32X2 ? 2 : 1);
    *flop_per_s = 2.0 * fmas_per_thread * blocks * kProbeThreads / (best_ms * 1e-3);
    return QXD_OK;
}
