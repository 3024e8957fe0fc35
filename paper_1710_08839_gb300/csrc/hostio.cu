// Spinor transfer between page-locked host memory and the native device
// layout without a staging copy: the GPU reads (writes) the caller's
// lexicographic host buffer directly over the CPU-GPU link while packing
// (unpacking). One thread per 16-byte element in lexicographic order, so the
// host side is read and written contiguously; the scattered side is device
// memory. Used by qxd_Dw when the host buffers are page-locked (registered
// with or allocated by CUDA); pageable buffers keep the copy path.
//
// qxd_Dw with page-locked buffers is pipelined over slabs of x0 planes: a
// slab is a contiguous range of the lexicographic host buffer, and the D of
// a slab needs the input of the slab and of its two neighbours in x0. Three
// streams overlap copying slab k + 1 in (cudaMemcpyAsync, then the pack
// kernel on the device), applying D to slab k, and unpacking and copying
// slab k - 1 out: the copy engines use the link in both directions at once
// while the SMs compute. (Kernels reading and writing the host buffers
// directly, in the same pipeline, were 8 % slower: they take SMs from D.)
#include <cstdlib>
#include <new>
#include <vector>

#include "dirac_common.cuh"

namespace qxd {

namespace {

// element i of the lexicographic field: site l = i / C, element k = i % C;
// native element k of site s is at k * V + s (C = 6 float4 or 12 double2)
// (elements [i0, i1) of the field)
template <typename T, int C>
__global__ void k_pack_from_host(Geom g, const T* __restrict__ lex, T* __restrict__ nat, size_t i0, size_t i1) {
    for (size_t i = i0 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(i / C), k = (int)(i - (size_t)l * C);
        int r = l;
        const int x3 = r % g.N3;
        r /= g.N3;
        const int x2 = r % g.N2;
        r /= g.N2;
        const int x1 = r % g.N1;
        const int x0 = r / g.N1;
        const int s = native_index(g, l, (x0 + x1 + x2 + x3) & 1);
        nat[(size_t)k * g.V + s] = lex[i];
    }
}

template <typename T, int C>
__global__ void k_unpack_to_host(Geom g, const T* __restrict__ nat, T* __restrict__ lex, size_t i0, size_t i1) {
    for (size_t i = i0 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(i / C), k = (int)(i - (size_t)l * C);
        int r = l;
        const int x3 = r % g.N3;
        r /= g.N3;
        const int x2 = r % g.N2;
        r /= g.N2;
        const int x1 = r % g.N1;
        const int x0 = r / g.N1;
        const int s = native_index(g, l, (x0 + x1 + x2 + x3) & 1);
        lex[i] = nat[(size_t)k * g.V + s];
    }
}

constexpr unsigned kGrid = 152 * 16;  // 16 blocks of 256 threads per SM

}  // namespace

bool host_device_view(const void* p, void** dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the error of an unknown pointer
        return false;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
    *dev = a.devicePointer;
    return true;
}

// sites [s0, s0 + ns) of the lexicographic order (a slab of x0 planes)
int pack_from_host_sites(qxd_lattice* lat, void* nat, const void* lex_dev, int prec, size_t s0, size_t ns,
                         unsigned grid, cudaStream_t st) {
    const Geom& g = lat->g;
    if (prec == QXD_FP32)
        k_pack_from_host<float4, 6><<<grid, 256, 0, st>>>(g, (const float4*)lex_dev, (float4*)nat, 6 * s0, 6 * (s0 + ns));
    else
        k_pack_from_host<double2, 12><<<grid, 256, 0, st>>>(g, (const double2*)lex_dev, (double2*)nat, 12 * s0,
                                                             12 * (s0 + ns));
    QXD_LAUNCHED("k_pack_from_host");
    return QXD_OK;
}

int unpack_to_host_sites(qxd_lattice* lat, void* lex_dev, const void* nat, int prec, size_t s0, size_t ns,
                         unsigned grid, cudaStream_t st) {
    const Geom& g = lat->g;
    if (prec == QXD_FP32)
        k_unpack_to_host<float4, 6><<<grid, 256, 0, st>>>(g, (const float4*)nat, (float4*)lex_dev, 6 * s0, 6 * (s0 + ns));
    else
        k_unpack_to_host<double2, 12><<<grid, 256, 0, st>>>(g, (const double2*)nat, (double2*)lex_dev, 12 * s0,
                                                             12 * (s0 + ns));
    QXD_LAUNCHED("k_unpack_to_host");
    return QXD_OK;
}

int launch_pack_from_host(qxd_lattice* lat, void* nat, const void* lex_dev, int prec, cudaStream_t st) {
    return pack_from_host_sites(lat, nat, lex_dev, prec, 0, (size_t)lat->g.V, kGrid, st);
}

int launch_unpack_to_host(qxd_lattice* lat, void* lex_dev, const void* nat, int prec, cudaStream_t st) {
    return unpack_to_host_sites(lat, lex_dev, nat, prec, 0, (size_t)lat->g.V, kGrid, st);
}

// streams (host reads, host writes) and events of the pipeline
constexpr int kMaxSlabs = 16;
struct HostPipe {
    cudaStream_t rd = nullptr, wr = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    cudaEvent_t in[kMaxSlabs] = {}, out[kMaxSlabs] = {};
    void* stage_out = nullptr;  // device staging of the lexicographic output
    ~HostPipe() {
        if (stage_out) cudaFree(stage_out);
        if (rd) cudaStreamDestroy(rd);
        if (wr) cudaStreamDestroy(wr);
        cudaEvent_t evs[] = {start, done};
        for (cudaEvent_t e : evs)
            if (e) cudaEventDestroy(e);
        for (int k = 0; k < kMaxSlabs; ++k) {
            if (in[k]) cudaEventDestroy(in[k]);
            if (out[k]) cudaEventDestroy(out[k]);
        }
    }
};

int ensure_hostpipe(qxd_lattice* lat) {
    if (lat->hostpipe) return QXD_OK;
    HostPipe* h = new (std::nothrow) HostPipe();
    if (!h) return fail(QXD_ERR_OOM, "qxd_Dw: host allocation failed");
    lat->hostpipe = h;
    QXD_CUDA(cudaStreamCreateWithFlags(&h->rd, cudaStreamNonBlocking));
    QXD_CUDA(cudaStreamCreateWithFlags(&h->wr, cudaStreamNonBlocking));
    QXD_CUDA(cudaEventCreateWithFlags(&h->start, cudaEventDisableTiming));
    QXD_CUDA(cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming));
    for (int k = 0; k < kMaxSlabs; ++k) {
        QXD_CUDA(cudaEventCreateWithFlags(&h->in[k], cudaEventDisableTiming));
        QXD_CUDA(cudaEventCreateWithFlags(&h->out[k], cudaEventDisableTiming));
    }
    return QXD_OK;
}

// slabs: the divisor of N0 nearest to 8 with at least 2 planes per slab
int pick_slabs(int N0) {
    int best = 0;
    for (int S = 3; S <= kMaxSlabs; ++S)
        if (N0 % S == 0 && N0 / S >= 2 && (best == 0 || std::abs(S - 8) < std::abs(best - 8))) best = S;
    return best;
}

void release_hostio(qxd_lattice* lat) {
    delete lat->hostpipe;
    lat->hostpipe = nullptr;
}

int dw_host_pipelined(qxd_lattice* lat, void* out_dev, const void* in_dev, int prec, cudaStream_t st) {
    const Geom& g = lat->g;
    const int S = pick_slabs(g.N0);
    if (S < 3) return fail(QXD_ERR_ARG, "qxd_Dw: lattice too short in x0 for the pipelined host path");
    int rc = ensure_hostpipe(lat);
    if (rc) return rc;
    HostPipe& h = *lat->hostpipe;
    const int planes = g.N0 / S;
    const size_t slab = (size_t)planes * g.N1 * g.N2 * g.N3;
    const unsigned grid = kGrid / 4;  // each transfer kernel takes part of the GPU
    // the pipeline starts after the work already queued on st
    QXD_CUDA(cudaEventRecord(h.start, st));
    QXD_CUDA(cudaStreamWaitEvent(h.rd, h.start, 0));
    QXD_CUDA(cudaStreamWaitEvent(h.wr, h.start, 0));
    const size_t esz = prec == QXD_FP32 ? 24 * sizeof(float) : 24 * sizeof(double);  // bytes per site
    if (!h.stage_out) QXD_CUDA(cudaMalloc(&h.stage_out, (size_t)g.V * 24 * sizeof(double)));
    for (int k = 0; k < S; ++k) {
        QXD_CUDA(cudaMemcpyAsync((char*)lat->scratch_lex + k * slab * esz, (const char*)in_dev + k * slab * esz,
                                 slab * esz, cudaMemcpyDefault, h.rd));
        if ((rc = pack_from_host_sites(lat, lat->scratch_in, lat->scratch_lex, prec, k * slab, slab, grid, h.rd)))
            return rc;
        QXD_CUDA(cudaEventRecord(h.in[k], h.rd));
    }
    // outputs 1 .. S-2 as their inputs arrive, then the two that wrap in x0
    std::vector<int> order;
    for (int k = 1; k + 1 < S; ++k) order.push_back(k);
    order.push_back(S - 1);
    order.push_back(0);
    for (int k : order) {
        QXD_CUDA(cudaStreamWaitEvent(st, h.in[(k + 1) % S], 0));
        QXD_CUDA(cudaStreamWaitEvent(st, h.in[(k + S - 1) % S], 0));
        if ((rc = launch_dirac_planes(lat, lat->scratch_out, lat->scratch_in, prec, k * planes, planes, st))) return rc;
        QXD_CUDA(cudaEventRecord(h.out[k], st));
        QXD_CUDA(cudaStreamWaitEvent(h.wr, h.out[k], 0));
        if ((rc = unpack_to_host_sites(lat, h.stage_out, lat->scratch_out, prec, k * slab, slab, grid, h.wr))) return rc;
        QXD_CUDA(cudaMemcpyAsync((char*)out_dev + k * slab * esz, (const char*)h.stage_out + k * slab * esz,
                                 slab * esz, cudaMemcpyDefault, h.wr));
    }
    QXD_CUDA(cudaEventRecord(h.done, h.wr));
    QXD_CUDA(cudaStreamWaitEvent(st, h.done, 0));
    return QXD_OK;
}

}  // namespace qxd
