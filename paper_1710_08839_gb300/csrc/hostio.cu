// Spinor transfer between page-locked host memory and the native device
// layout without a staging copy: the GPU reads (writes) the caller's
// lexicographic host buffer directly over the CPU-GPU link while packing
// (unpacking). One thread per 16-byte element in lexicographic order, so the
// host side is read and written contiguously; the scattered side is device
// memory. Used by qxd_Dw when the host buffers are page-locked (registered
// with or allocated by CUDA); pageable buffers keep the copy path.
#include "dirac_common.cuh"

namespace qxd {

namespace {

// element i of the lexicographic field: site l = i / C, element k = i % C;
// native element k of site s is at k * V + s (C = 6 float4 or 12 double2)
template <typename T, int C>
__global__ void k_pack_from_host(Geom g, const T* __restrict__ lex, T* __restrict__ nat) {
    const size_t n = (size_t)C * g.V;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
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
__global__ void k_unpack_to_host(Geom g, const T* __restrict__ nat, T* __restrict__ lex) {
    const size_t n = (size_t)C * g.V;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
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

int launch_pack_from_host(qxd_lattice* lat, void* nat, const void* lex_dev, int prec, cudaStream_t st) {
    const Geom& g = lat->g;
    if (prec == QXD_FP32)
        k_pack_from_host<float4, 6><<<kGrid, 256, 0, st>>>(g, (const float4*)lex_dev, (float4*)nat);
    else
        k_pack_from_host<double2, 12><<<kGrid, 256, 0, st>>>(g, (const double2*)lex_dev, (double2*)nat);
    QXD_LAUNCHED("k_pack_from_host");
    return QXD_OK;
}

int launch_unpack_to_host(qxd_lattice* lat, void* lex_dev, const void* nat, int prec, cudaStream_t st) {
    const Geom& g = lat->g;
    if (prec == QXD_FP32)
        k_unpack_to_host<float4, 6><<<kGrid, 256, 0, st>>>(g, (const float4*)nat, (float4*)lex_dev);
    else
        k_unpack_to_host<double2, 12><<<kGrid, 256, 0, st>>>(g, (const double2*)nat, (double2*)lex_dev);
    QXD_LAUNCHED("k_unpack_to_host");
    return QXD_OK;
}

}  // namespace qxd
