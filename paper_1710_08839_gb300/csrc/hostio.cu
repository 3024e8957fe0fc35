// Spinor transfer between page-locked host memory and the native device
// layout without a staging copy: the GPU reads (writes) the caller's
// lexicographic host buffer directly over the CPU-GPU link while packing
// (unpacking). One thread per 16-byte element in lexicographic order, so the
// host side is read and written contiguously; the scattered side is device
// memory. Used by qxd_Dw when the host buffers are page-locked (registered
// with or allocated by CUDA); pageable buffers keep the copy path.
//
// qxd_Dw with page-locked buffers is pipelined over slabs of x0 planes: a
// slab is a contiguous range of the lexicographic host buffer. One stream
// copies the input slabs in (cudaMemcpyAsync, then the pack kernel on the
// device); as soon as slab k is in, D is applied to every output plane whose
// x0 neighbours have arrived (up to the last plane but one of slab k), and
// those planes are unpacked and copied out on a third stream. The two planes
// that wrap around in x0 come last. The copy engines thus use the link in
// both directions at once while the SMs compute, and the output stream
// starts after one input slab. (Kernels reading and writing the host buffers
// directly, in the same pipeline, were 8 % slower: they take SMs from D.)
#include <cstdlib>
#include <new>

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
    cudaEvent_t in[kMaxSlabs] = {}, out[kMaxSlabs + 2] = {};
    void* stage_out = nullptr;  // device staging of the lexicographic output
    ~HostPipe() {
        if (stage_out) cudaFree(stage_out);
        if (rd) cudaStreamDestroy(rd);
        if (wr) cudaStreamDestroy(wr);
        cudaEvent_t evs[] = {start, done};
        for (cudaEvent_t e : evs)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : in)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : out)
            if (e) cudaEventDestroy(e);
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
    for (cudaEvent_t& e : h->in) QXD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (cudaEvent_t& e : h->out) QXD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return QXD_OK;
}

// slabs: the largest divisor of N0 up to 16 with at least 2 planes per slab
// (at least 3 slabs, else 0: no pipeline)
int pick_slabs(int N0) {
    int best = 0;
    for (int S = 3; S <= kMaxSlabs; ++S)
        if (N0 % S == 0 && N0 / S >= 2) best = S;
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
    // output planes [lo, hi) once input slab k is in: up to the last plane but
    // one of slab k (its forward neighbour is in slab k + 1); plane 0 (whose
    // backward neighbour is plane N0 - 1) and plane N0 - 1 come last
    const size_t plane = (size_t)g.N1 * g.N2 * g.N3;
    auto out_range = [&](int lo, int hi, int ev) -> int {
        if (hi <= lo) return QXD_OK;
        int r = launch_dirac_planes(lat, lat->scratch_out, lat->scratch_in, prec, lo, hi - lo, st);
        if (r) return r;
        QXD_CUDA(cudaEventRecord(h.out[ev], st));
        QXD_CUDA(cudaStreamWaitEvent(h.wr, h.out[ev], 0));
        if ((r = unpack_to_host_sites(lat, h.stage_out, lat->scratch_out, prec, lo * plane, (hi - lo) * plane, grid,
                                      h.wr)))
            return r;
        QXD_CUDA(cudaMemcpyAsync((char*)out_dev + lo * plane * esz, (const char*)h.stage_out + lo * plane * esz,
                                 (hi - lo) * plane * esz, cudaMemcpyDefault, h.wr));
        return QXD_OK;
    };
    for (int k = 0; k < S; ++k) {
        QXD_CUDA(cudaStreamWaitEvent(st, h.in[k], 0));  // slabs 0 .. k are in (rd is in order)
        const int lo = k == 0 ? 1 : k * planes - 1;
        const int hi = k == S - 1 ? g.N0 - 1 : (k + 1) * planes - 1;
        if ((rc = out_range(lo, hi, k))) return rc;
    }
    if ((rc = out_range(g.N0 - 1, g.N0, S))) return rc;
    if ((rc = out_range(0, 1, S + 1))) return rc;
    QXD_CUDA(cudaEventRecord(h.done, h.wr));
    QXD_CUDA(cudaStreamWaitEvent(st, h.done, 0));
    return QXD_OK;
}

}  // namespace qxd
