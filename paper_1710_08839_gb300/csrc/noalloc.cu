// qxd_Dw_noalloc: the operator D on lexicographic-layout device spinors
// without any device allocation.
//
// qxd_Dw with the lexicographic layout converts the caller's spinors to the
// library's native layout through two device scratch fields, which it
// allocates with cudaMalloc on its first such call. Some callers cannot let a
// library allocate device memory during a call: frameworks that hand out all
// device memory from their own pool and need the library's footprint fixed
// in advance, serving paths that cannot take the latency of a cudaMalloc
// (which may synchronise the device), and jobs that already hold nearly all
// device memory. For them this entry point keeps the two scratch fields in a
// fixed array in the library's own device memory, so a call allocates
// nothing. The array belongs to this file's module, which holds no kernels:
// with CUDA's lazy module loading (the default) the module, and so the
// array, is loaded on a device by the first call there (its
// cudaGetSymbolAddress), and it stays reserved until the process exits.
// That first call is the set-up step: make it while memory is available and
// before any stream capture; later calls only launch kernels.
#include <mutex>

#include "qxd_internal.cuh"

namespace {

// Largest lattice (simulated sites) the fixed scratch serves.
constexpr long long kNoAllocMaxSites = 65536;
// One native spinor field, FP64 (the larger precision): 24 doubles per site.
constexpr size_t kNoAllocFieldBytes = (size_t)kNoAllocMaxSites * 24 * sizeof(double);

}  // namespace

// Scratch of qxd_Dw_noalloc: input field, then output field (2 x 12 MiB).
// Shared by every call on a device (the contract is in include/qxd.h).
static __device__ __align__(256) unsigned char qxd_noalloc_scratch[2 * kNoAllocFieldBytes];

namespace qxd {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (host code only
// sees a stand-in for the array under its name). Looked up once per device.
int noalloc_scratch(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(QXD_ERR_ARG, "qxd_Dw_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, qxd_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "qxd_Dw_noalloc: cudaGetSymbolAddress(scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = (unsigned char*)g_noalloc_addr[dev];
    return QXD_OK;
}

int dw_noalloc(qxd_lattice* lat, void* out, const void* in, int prec, cudaStream_t st) {
    unsigned char* base = nullptr;
    int rc = noalloc_scratch(lat->device, &base);
    if (rc) return rc;
    unsigned char* nat_in = base;
    unsigned char* nat_out = base + kNoAllocFieldBytes;
    // pack writes every entry of nat_in and the operator every entry of
    // nat_out, so nothing left by an earlier call is read
    if ((rc = launch_pack(lat, nat_in, in, prec, st))) return rc;
    if ((rc = launch_dirac(lat, nat_out, nat_in, prec, st))) return rc;
    return launch_unpack(lat, out, nat_out, prec, st);
}

}  // namespace
}  // namespace qxd

using namespace qxd;

extern "C" int qxd_Dw_noalloc(qxd_lattice* lat, void* out, const void* in, int flags, void* stream) {
    if (!lat || !out || !in) return fail(QXD_ERR_ARG, "qxd_Dw_noalloc: NULL argument");
    if (flags & ~0x1)
        return fail(QXD_ERR_ARG, "qxd_Dw_noalloc: only QXD_FP64 or QXD_FP32 (device buffers, lexicographic layout)");
    if (out == in) return fail(QXD_ERR_ARG, "qxd_Dw_noalloc: in and out must not overlap");
    if (!qxd::clover_ready(lat)) return fail(QXD_ERR_STATE, "qxd_Dw_noalloc: needs qxd_sw_build first");
    if ((long long)lat->g.V > kNoAllocMaxSites)
        return fail(QXD_ERR_ARG, "qxd_Dw_noalloc: lattice has " + std::to_string(lat->g.V) +
                                     " sites, the fixed scratch serves at most " +
                                     std::to_string(kNoAllocMaxSites) + " (use qxd_Dw)");
    const int prec = flags & 0x1;
    cudaStream_t st = stream ? (cudaStream_t)stream : lat->stream;
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e, "qxd_Dw_noalloc: cudaGetDevice");
    if (cur != lat->device && (e = cudaSetDevice(lat->device)) != cudaSuccess)
        return cuda_fail(e, "qxd_Dw_noalloc: cudaSetDevice");
    int rc = dw_noalloc(lat, out, in, prec, st);
    if (cur != lat->device) cudaSetDevice(cur);
    return rc;
}
