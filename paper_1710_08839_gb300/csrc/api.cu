// C ABI of the qxd library: lattice object, argument checks, state machine,
// host<->device marshalling. Every compute step runs in the kernels of the
// other translation units.
#include <cstdio>
#include <cstring>
#include <string>

#include "qxd_internal.cuh"

namespace qxd {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? QXD_ERR_OOM : QXD_ERR_CUDA;
}

static int pick_sweep_rows(int N1, int N2, int N3) {
    // largest divisor R of N2 with N1 * R * N3 <= 64K sites: the x0 neighbours
    // of a site are that many sites apart in the sweep, and their data must
    // still be in L2 (measured on the 96x96x48x48 lattice: 24K-site windows
    // and whole x2 extents are slower, 55K-74K best)
    int best = 1;
    for (int R = 1; R <= N2; ++R)
        if (N2 % R == 0 && (long long)N1 * R * N3 <= 65536) best = R;
    return best;
}

template <typename T>
static int dalloc(T** p, size_t n, const char* what) {
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, what);
    }
    return QXD_OK;
}

static void free_all(qxd_lattice* L) {
    release_hostio(L);
    void* own[] = {L->Zq64, L->C64, L->C32, L->Cinv64, L->Cinv32, L->d_status, L->scratch_in, L->scratch_out,
                   L->scratch_lex, L->sap_r, L->sap_multi};
    for (void* p : own)
        if (p) cudaFree(p);
    if (L->parent) return;  // the gauge field belongs to the parent
    void* gauge[] = {L->U64, L->U32, L->A64, L->Z64, L->A32, L->ftens};
    for (void* p : gauge)
        if (p) cudaFree(p);
}

int ensure_scratch(qxd_lattice* L) {
    if (L->scratch_in) return QXD_OK;
    size_t nat = (size_t)L->g.V * SPINOR_D2 * sizeof(double2);
    int rc;
    if ((rc = dalloc((char**)&L->scratch_in, nat, "cudaMalloc(scratch)"))) return rc;
    if ((rc = dalloc((char**)&L->scratch_out, nat, "cudaMalloc(scratch)"))) return rc;
    if ((rc = dalloc((char**)&L->scratch_lex, nat, "cudaMalloc(scratch)"))) return rc;
    return QXD_OK;
}

}  // namespace qxd

using namespace qxd;

extern "C" {

const char* qxd_last_error(void) { return g_last_error.c_str(); }

int qxd_lattice_create(qxd_lattice** out, int T, int L1, int L2, int L3, unsigned cstar_mask,
                       void* stream) {
    if (!out) return fail(QXD_ERR_ARG, "qxd_lattice_create: out is NULL");
    *out = nullptr;
    if (cstar_mask & ~0xEu) return fail(QXD_ERR_ARG, "qxd_lattice_create: cstar_mask uses bits other than 1..3");
    if (cstar_mask && !(cstar_mask & 2u))
        return fail(QXD_ERR_ARG, "qxd_lattice_create: C* in direction 2 or 3 needs C* in direction 1");
    int L[4] = {T, L1, L2, L3};
    for (int mu = 0; mu < 4; ++mu)
        if (L[mu] < 2 || (L[mu] & 1))
            return fail(QXD_ERR_ARG, "qxd_lattice_create: every extent must be even and >= 2 "
                                     "(even-odd parity on the shifted torus)");
    long long N1 = (cstar_mask & 2u) ? 2LL * L1 : L1;
    long long V = (long long)T * N1 * L2 * L3;
    if (V >= (1LL << 30)) return fail(QXD_ERR_ARG, "qxd_lattice_create: volume must be below 2^30 sites");

    qxd_lattice* lat = new (std::nothrow) qxd_lattice();
    if (!lat) return fail(QXD_ERR_OOM, "qxd_lattice_create: host allocation failed");
    lat->T = T;
    lat->L1 = L1;
    lat->L2 = L2;
    lat->L3 = L3;
    lat->cstar_mask = cstar_mask;
    lat->stream = (cudaStream_t)stream;
    Geom& g = lat->g;
    g.N0 = T;
    g.N1 = (int)N1;
    g.N2 = L2;
    g.N3 = L3;
    g.L1 = L1;
    g.cs2 = (cstar_mask & 4u) ? 1 : 0;
    g.cs3 = (cstar_mask & 8u) ? 1 : 0;
    g.V = (int)V;
    g.Vh = (int)(V / 2);
    g.R = pick_sweep_rows(g.N1, g.N2, g.N3);
    cudaError_t e = cudaGetDevice(&lat->device);
    if (e != cudaSuccess) {
        delete lat;
        return cuda_fail(e, "cudaGetDevice");
    }
    size_t v = (size_t)V;
    int rc = 0;
    if ((rc = dalloc(&lat->U64, 4 * 9 * v, "cudaMalloc(U64)")) ||
        (rc = dalloc(&lat->U32, 4 * 3 * v, "cudaMalloc(U32)")) ||
        (rc = dalloc(&lat->A64, 4 * v, "cudaMalloc(A64)")) ||
        (rc = dalloc(&lat->Z64, 4 * v, "cudaMalloc(Z64)")) ||
        (rc = dalloc(&lat->A32, v, "cudaMalloc(A32)")) ||
        (rc = dalloc(&lat->ftens, FTENS_REALS * v, "cudaMalloc(ftens)")) ||
        (rc = dalloc(&lat->Zq64, 4 * v, "cudaMalloc(Zq64)")) ||
        (rc = dalloc(&lat->C64, CLOVER_REALS * v, "cudaMalloc(C64)")) ||
        (rc = dalloc(&lat->C32, CLOVER_F4 * v, "cudaMalloc(C32)")) ||
        (rc = dalloc(&lat->Cinv64, CLOVER_REALS * v, "cudaMalloc(Cinv64)")) ||
        (rc = dalloc(&lat->Cinv32, CLOVER_F4 * v, "cudaMalloc(Cinv32)")) ||
        (rc = dalloc(&lat->d_status, 64, "cudaMalloc(status)"))) {
        free_all(lat);
        delete lat;
        return rc;
    }
    *out = lat;
    return QXD_OK;
}

int qxd_lattice_destroy(qxd_lattice* lat) {
    if (!lat) return QXD_OK;
    if (lat->nviews > 0)
        return fail(QXD_ERR_STATE, "qxd_lattice_destroy: " + std::to_string(lat->nviews) +
                                       " views still share this lattice's gauge field");
    cudaStreamSynchronize(lat->stream);
    if (lat->parent) --lat->parent->nviews;
    release_solver(lat);
    release_mscg(lat);
    release_dfl(lat);
    free_all(lat);
    delete lat;
    return QXD_OK;
}

int qxd_lattice_dims(const qxd_lattice* lat, int* N4, long long* volume) {
    if (!lat) return fail(QXD_ERR_ARG, "qxd_lattice_dims: lat is NULL");
    if (N4) {
        N4[0] = lat->g.N0;
        N4[1] = lat->g.N1;
        N4[2] = lat->g.N2;
        N4[3] = lat->g.N3;
    }
    if (volume) *volume = lat->g.V;
    return QXD_OK;
}

int qxd_lattice_view(qxd_lattice** out, qxd_lattice* parent, void* stream) {
    if (!out || !parent) return fail(QXD_ERR_ARG, "qxd_lattice_view: NULL argument");
    *out = nullptr;
    qxd_lattice* root = gauge_owner(parent);
    qxd_lattice* v = new (std::nothrow) qxd_lattice();
    if (!v) return fail(QXD_ERR_OOM, "qxd_lattice_view: host allocation failed");
    v->g = root->g;
    v->T = root->T;
    v->L1 = root->L1;
    v->L2 = root->L2;
    v->L3 = root->L3;
    v->cstar_mask = root->cstar_mask;
    v->stream = stream ? (cudaStream_t)stream : root->stream;
    v->device = root->device;
    v->U64 = root->U64;
    v->U32 = root->U32;
    v->A64 = root->A64;
    v->Z64 = root->Z64;
    v->A32 = root->A32;
    v->ftens = root->ftens;
    v->parent = root;
    size_t n = (size_t)root->g.V;
    int rc = 0;
    if ((rc = dalloc(&v->Zq64, 4 * n, "cudaMalloc(Zq64)")) ||
        (rc = dalloc(&v->C64, CLOVER_REALS * n, "cudaMalloc(C64)")) ||
        (rc = dalloc(&v->C32, CLOVER_F4 * n, "cudaMalloc(C32)")) ||
        (rc = dalloc(&v->Cinv64, CLOVER_REALS * n, "cudaMalloc(Cinv64)")) ||
        (rc = dalloc(&v->Cinv32, CLOVER_F4 * n, "cudaMalloc(Cinv32)")) ||
        (rc = dalloc(&v->d_status, 64, "cudaMalloc(status)"))) {
        free_all(v);
        delete v;
        return rc;
    }
    ++root->nviews;
    *out = v;
    return QXD_OK;
}

int qxd_set_gauge(qxd_lattice* lat, const double* su3, const double* u1_angle, int flags) {
    if (!lat || !su3 || !u1_angle) return fail(QXD_ERR_ARG, "qxd_set_gauge: NULL argument");
    if (lat->parent) return fail(QXD_ERR_STATE, "qxd_set_gauge: a view shares its parent's gauge field");
    int kind = flags & 0x3;
    if (kind == 3 || (flags & ~0x13)) return fail(QXD_ERR_ARG, "qxd_set_gauge: bad flags");
    const bool host = flags & QXD_GAUGE_HOST;
    const int extended = kind != QXD_GAUGE_PHYSICAL_HALF;
    size_t nsites = extended ? (size_t)lat->g.V
                             : (size_t)lat->T * lat->L1 * lat->L2 * lat->L3;
    lat->has_gauge = false;
    lat->has_clover = false;
    const double* d_su3 = su3;
    const double* d_ang = u1_angle;
    double* tmp = nullptr;
    if (host) {
        size_t n = nsites * 4 * 18 + nsites * 4;
        int rc = dalloc(&tmp, n, "cudaMalloc(gauge staging)");
        if (rc) return rc;
        cudaError_t e1 = cudaMemcpyAsync(tmp, su3, nsites * 4 * 18 * sizeof(double),
                                         cudaMemcpyHostToDevice, lat->stream);
        cudaError_t e2 = cudaMemcpyAsync(tmp + nsites * 4 * 18, u1_angle, nsites * 4 * sizeof(double),
                                         cudaMemcpyHostToDevice, lat->stream);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            cudaFree(tmp);
            return cuda_fail(e1 != cudaSuccess ? e1 : e2, "cudaMemcpyAsync(gauge)");
        }
        d_su3 = tmp;
        d_ang = tmp + nsites * 4 * 18;
    }
    int rc = launch_gauge_ingest(lat, d_su3, d_ang, kind, lat->d_status);
    if (rc == QXD_OK) rc = launch_field_tensor(lat);
    int st[4] = {0, 0, 0, 0};
    if (rc == QXD_OK) {
        cudaError_t e = cudaMemcpyAsync(st, lat->d_status, sizeof(st), cudaMemcpyDeviceToHost, lat->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "qxd_set_gauge: status readback");
    }
    if (tmp) cudaFree(tmp);
    if (rc) return rc;
    if (st[0]) return fail(QXD_ERR_ARG, "qxd_set_gauge: " + std::to_string(st[0]) +
                                            " links are not SU(3) to 1e-10 or not finite");
    if (st[1]) return fail(QXD_ERR_NOT_ADMISSIBLE, "qxd_set_gauge: " + std::to_string(st[1]) +
                                                       " mirror links violate the orbifold constraint");
    lat->has_gauge = true;
    ++lat->gauge_version;
    return QXD_OK;
}

int qxd_set_params(qxd_lattice* lat, double m0, double csw, double cswqed, int qhat) {
    if (!lat) return fail(QXD_ERR_ARG, "qxd_set_params: lat is NULL");
    if (!(m0 == m0) || !(csw == csw) || !(cswqed == cswqed))
        return fail(QXD_ERR_ARG, "qxd_set_params: NaN parameter");
    lat->m0 = m0;
    lat->csw = csw;
    lat->cswqed = cswqed;
    lat->qhat = qhat;
    lat->has_params = true;
    lat->has_clover = false;
    return QXD_OK;
}

int qxd_sw_build(qxd_lattice* lat) {
    if (!lat) return fail(QXD_ERR_ARG, "qxd_sw_build: lat is NULL");
    if (!gauge_owner(lat)->has_gauge || !lat->has_params)
        return fail(QXD_ERR_STATE, "qxd_sw_build: needs qxd_set_gauge and qxd_set_params first");
    lat->has_clover = false;
    int rc = launch_clover_build(lat, lat->d_status);
    if (rc) return rc;
    int st[4];
    cudaError_t e = cudaMemcpyAsync(st, lat->d_status, sizeof(st), cudaMemcpyDeviceToHost, lat->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "qxd_sw_build: status readback");
    if (st[0]) return fail(QXD_ERR_SW_SINGULAR, "qxd_sw_build: " + std::to_string(st[0]) +
                                                    " clover blocks are singular or not finite");
    lat->has_clover = true;
    lat->built_gauge_version = gauge_owner(lat)->gauge_version;
    ++lat->op_version;
    return QXD_OK;
}

size_t qxd_spinor_bytes(const qxd_lattice* lat, int prec) {
    if (!lat) return 0;
    return (size_t)lat->g.V * 24 * (prec == QXD_FP32 ? sizeof(float) : sizeof(double));
}

int qxd_spinor_pack(qxd_lattice* lat, void* native_out, const void* lex_in, int prec, void* stream) {
    if (!lat || !native_out || !lex_in) return fail(QXD_ERR_ARG, "qxd_spinor_pack: NULL argument");
    if (prec != QXD_FP32 && prec != QXD_FP64) return fail(QXD_ERR_ARG, "qxd_spinor_pack: bad precision");
    cudaStream_t st = stream ? (cudaStream_t)stream : lat->stream;
    return launch_pack(lat, native_out, lex_in, prec, st);
}

int qxd_spinor_unpack(qxd_lattice* lat, void* lex_out, const void* native_in, int prec, void* stream) {
    if (!lat || !lex_out || !native_in) return fail(QXD_ERR_ARG, "qxd_spinor_unpack: NULL argument");
    if (prec != QXD_FP32 && prec != QXD_FP64) return fail(QXD_ERR_ARG, "qxd_spinor_unpack: bad precision");
    cudaStream_t st = stream ? (cudaStream_t)stream : lat->stream;
    return launch_unpack(lat, lex_out, native_in, prec, st);
}

int qxd_Dw(qxd_lattice* lat, void* out, const void* in, int flags, void* stream) {
    if (!lat || !out || !in) return fail(QXD_ERR_ARG, "qxd_Dw: NULL argument");
    if (flags & ~(0x1 | 0x10 | 0x100)) return fail(QXD_ERR_ARG, "qxd_Dw: bad flags");
    if (!qxd::clover_ready(lat)) return fail(QXD_ERR_STATE, "qxd_Dw: needs qxd_sw_build first");
    const int prec = flags & 0x1;
    const bool host = flags & QXD_HOST;
    const bool native = flags & QXD_LAYOUT_NATIVE;
    if (host && native) return fail(QXD_ERR_ARG, "qxd_Dw: host buffers must use the lexicographic layout");
    cudaStream_t st = stream ? (cudaStream_t)stream : lat->stream;
    if (out == in) return fail(QXD_ERR_ARG, "qxd_Dw: in and out must not overlap");
    if (native) return launch_dirac(lat, out, in, prec, st);
    int rc = ensure_scratch(lat);
    if (rc) return rc;
    size_t bytes = qxd_spinor_bytes(lat, prec);
    const void* lex_in = in;
    if (host) {
        // page-locked buffers are read and written by the kernels directly,
        // pipelined over slabs of x0 planes when both are page-locked;
        // pageable ones go through a device staging copy
        void* in_dev = nullptr;
        void* out_dev = nullptr;
        const bool in_pl = host_device_view(in, &in_dev), out_pl = host_device_view(out, &out_dev);
        if (in_pl && out_pl && pick_slabs(lat->g.N0) >= 3) {
            if ((rc = dw_host_pipelined(lat, out_dev, in_dev, prec, st))) return rc;
            QXD_CUDA(cudaStreamSynchronize(st));
            return QXD_OK;
        }
        if (in_pl) {
            if ((rc = launch_pack_from_host(lat, lat->scratch_in, in_dev, prec, st))) return rc;
        } else {
            QXD_CUDA(cudaMemcpyAsync(lat->scratch_lex, in, bytes, cudaMemcpyHostToDevice, st));
            if ((rc = launch_pack(lat, lat->scratch_in, lat->scratch_lex, prec, st))) return rc;
        }
        if ((rc = launch_dirac(lat, lat->scratch_out, lat->scratch_in, prec, st))) return rc;
        if (out_pl) {
            if ((rc = launch_unpack_to_host(lat, out_dev, lat->scratch_out, prec, st))) return rc;
        } else {
            if ((rc = launch_unpack(lat, lat->scratch_lex, lat->scratch_out, prec, st))) return rc;
            QXD_CUDA(cudaMemcpyAsync(out, lat->scratch_lex, bytes, cudaMemcpyDeviceToHost, st));
        }
        QXD_CUDA(cudaStreamSynchronize(st));
        return QXD_OK;
    }
    if ((rc = launch_pack(lat, lat->scratch_in, lex_in, prec, st))) return rc;
    if ((rc = launch_dirac(lat, lat->scratch_out, lat->scratch_in, prec, st))) return rc;
    return launch_unpack(lat, out, lat->scratch_out, prec, st);
}

}  // extern "C"
