// Batched application of D: many right-hand sides on several operators
// (lattices or views, possibly of different sizes) in one launch.
//
// The work is a table of groups; a group is one operator with up to NR
// right-hand sides. A group covers ceil(V * NR / 256) thread blocks and a
// thread handles one (site, right-hand side) pair, with the NR right-hand
// sides of a site in adjacent lanes: their link, angle and clover loads hit
// the same addresses, so they are fetched once (L1) and the DRAM traffic per
// right-hand side drops from 688 B/site to (496 + 192 NR)/NR B/site in FP32.
// A thread block finds its group by binary search over the groups' first
// block indices. NR is chosen per lattice size by a small autotuner that
// times the candidates once and remembers the fastest.
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <cstdio>

#include "batch.cuh"
#include "dirac_common.cuh"
#include "tune.cuh"

namespace qxd {

namespace {

template <typename R>
struct DwGroup {
    Geom g;
    Fields<R> f;  // psi/out unused; U, A, C of the group's operator
    R q;
    int nr;                                     // right-hand sides in this group (<= NR)
    const typename Fields<R>::vec* in[BATCH_MAXR];
    typename Fields<R>::vec* out[BATCH_MAXR];
    int cta_begin;
};

template <typename R, int NR>
__global__ void __launch_bounds__(DW_THREADS, DwMinBlocks<R>::value)
    k_dirac_batch(const DwGroup<R>* __restrict__ groups, int ngroups) {
    // group of this thread block
    int lo = 0, hi = ngroups - 1;
    const int b = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (groups[mid].cta_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    const DwGroup<R>& G = groups[lo];
    const Geom g = G.g;
    const int t = (b - G.cta_begin) * DW_THREADS + threadIdx.x;
    const int tau = t / NR;
    const int r = t - tau * NR;
    if (tau >= g.V || r >= G.nr) return;
    Fields<R> f = G.f;
    const R q = G.q;
    int x0, x1, x2, x3;
    sweep_coords(g, tau, x0, x1, x2, x3);
    const int p = (x0 + x1 + x2 + x3) & 1;
    const int s = native_index(g, lex_index(g, x0, x1, x2, x3), p);
    const int po = 1 - p;
    const typename Fields<R>::vec* psi = G.in[r];
    cplx<R> acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = mk<R>(0, 0);
    // one code path for every charge (qhat = 0 gives the phase 1 exactly)
    dirac_dir<R, true, 0>(g, f, psi, g.V, 0, q, x0, x1, x2, x3, s, po, acc);
    dirac_dir<R, true, 1>(g, f, psi, g.V, 0, q, x0, x1, x2, x3, s, po, acc);
    dirac_dir<R, true, 2>(g, f, psi, g.V, 0, q, x0, x1, x2, x3, s, po, acc);
    dirac_dir<R, true, 3>(g, f, psi, g.V, 0, q, x0, x1, x2, x3, s, po, acc);
    cplx<R> v[12], w[12];
    load_spinor(psi, g.V, s, v);
    clover_mul<true>(f.C, g.V, s, v, w);
#pragma unroll
    for (int i = 0; i < 12; ++i) w[i] = w[i] - R(0.5) * acc[i];
    store_spinor(G.out[r], g.V, s, w);
}

template <typename R>
Fields<R> op_fields(qxd_lattice* lat);
template <>
Fields<float> op_fields<float>(qxd_lattice* lat) {
    return Fields<float>{nullptr, nullptr, lat->U32, lat->A32, lat->C32};
}
template <>
Fields<double> op_fields<double>(qxd_lattice* lat) {
    return Fields<double>{nullptr, nullptr, lat->U64, lat->Zq64, lat->C64};
}

// device buffer for group tables, grown on demand, one per (device, stream)
struct TableBuf {
    void* d = nullptr;
    size_t cap = 0;
};
std::mutex g_tab_mu;
std::map<std::pair<int, cudaStream_t>, TableBuf> g_tabs;

int table_upload(const void* host, size_t bytes, cudaStream_t st, void** dev) {
    int d = 0;
    cudaGetDevice(&d);
    std::lock_guard<std::mutex> lock(g_tab_mu);
    TableBuf& tb = g_tabs[{d, st}];
    if (tb.cap < bytes) {
        if (tb.d) {
            cudaStreamSynchronize(st);
            cudaFree(tb.d);
        }
        size_t cap = std::max<size_t>(bytes, 64 * 1024);
        cudaError_t e = cudaMalloc(&tb.d, cap);
        if (e != cudaSuccess) {
            tb.d = nullptr;
            tb.cap = 0;
            return cuda_fail(e, "cudaMalloc(batch table)");
        }
        tb.cap = cap;
    }
    // the copy is ordered on the stream before the kernel that reads it; the
    // host buffer must stay valid until it completes (pageable: the call
    // returns after the data is staged)
    cudaError_t e = cudaMemcpyAsync(tb.d, host, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(batch table)");
    *dev = tb.d;
    return QXD_OK;
}

template <typename R, int NR>
int launch_batch_nr(const std::vector<BatchItem>& items, cudaStream_t st) {
    // group consecutive items of the same operator, NR per group
    std::vector<DwGroup<R>> groups;
    int ctas = 0;
    size_t i = 0;
    while (i < items.size()) {
        qxd_lattice* lat = items[i].lat;
        DwGroup<R> G{};
        G.g = lat->g;
        G.f = op_fields<R>(lat);
        G.q = (R)lat->qhat;
        G.nr = 0;
        while (i < items.size() && items[i].lat == lat && G.nr < NR) {
            G.in[G.nr] = (const typename Fields<R>::vec*)items[i].in;
            G.out[G.nr] = (typename Fields<R>::vec*)items[i].out;
            ++G.nr;
            ++i;
        }
        G.cta_begin = ctas;
        ctas += (int)(((long long)G.g.V * NR + DW_THREADS - 1) / DW_THREADS);
        groups.push_back(G);
    }
    void* dtab = nullptr;
    int rc = table_upload(groups.data(), groups.size() * sizeof(DwGroup<R>), st, &dtab);
    if (rc) return rc;
    k_dirac_batch<R, NR><<<ctas, DW_THREADS, 0, st>>>((const DwGroup<R>*)dtab, (int)groups.size());
    QXD_LAUNCHED("k_dirac_batch");
    return QXD_OK;
}

template <typename R>
int launch_batch(const std::vector<BatchItem>& items, int nr, cudaStream_t st) {
    switch (nr) {
        case 1: return launch_batch_nr<R, 1>(items, st);
        case 2: return launch_batch_nr<R, 2>(items, st);
        case 4: return launch_batch_nr<R, 4>(items, st);
        default: return launch_batch_nr<R, 8>(items, st);
    }
}

// autotuner: fastest right-hand sides per site for (precision, volume bucket)
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tuned;

}  // namespace

int dw_batch(const std::vector<BatchItem>& items, int prec, int nr, cudaStream_t st) {
    if (items.empty()) return QXD_OK;
    if (nr <= 0) {
        // largest lattice of the batch decides
        int vmax = 0;
        for (const auto& it : items) vmax = std::max(vmax, it.lat->g.V);
        int bucket = 0;
        while ((1 << bucket) < vmax) ++bucket;
        const auto key = std::make_pair(prec, bucket);
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) nr = it->second;
        }
        if (nr <= 0) {
            // time each candidate on this batch (outputs are rewritten every time)
            const int cand[4] = {1, 2, 4, 8};
            float best = 1e30f;
            int best_nr = 1;
            cudaEvent_t e0, e1;
            QXD_CUDA(cudaEventCreate(&e0));
            QXD_CUDA(cudaEventCreate(&e1));
            for (int c : cand) {
                int rc = prec == QXD_FP32 ? launch_batch<float>(items, c, st) : launch_batch<double>(items, c, st);
                if (rc) return rc;
                cudaEventRecord(e0, st);
                for (int rep = 0; rep < 3; ++rep) {
                    rc = prec == QXD_FP32 ? launch_batch<float>(items, c, st) : launch_batch<double>(items, c, st);
                    if (rc) return rc;
                }
                cudaEventRecord(e1, st);
                QXD_CUDA(cudaEventSynchronize(e1));
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    best_nr = c;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            nr = best_nr;
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tuned[key] = nr;
        }
    }
    return prec == QXD_FP32 ? launch_batch<float>(items, nr, st) : launch_batch<double>(items, nr, st);
}

void dw_batch_report(std::string& out) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    char line[160];
    for (const auto& kv : g_tuned) {
        std::snprintf(line, sizeof line, "Dw_batch %s volume<=2^%d: rhs_per_site=%d (tuned)\n",
                      kv.first.first == QXD_FP32 ? "fp32" : "fp64", kv.first.second, kv.second);
        out += line;
    }
}

int dw_batch_tuned_nr(int prec, int volume) {
    int bucket = 0;
    while ((1 << bucket) < volume) ++bucket;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(std::make_pair(prec, bucket));
    return it == g_tuned.end() ? 0 : it->second;
}

}  // namespace qxd

using namespace qxd;

extern "C" int qxd_Dw_batch(int n, qxd_lattice* const* lats, void* const* out, const void* const* in, int flags,
                            int rhs_per_site, void* stream) {
    if (n < 0 || (n > 0 && (!lats || !out || !in))) return fail(QXD_ERR_ARG, "qxd_Dw_batch: NULL argument");
    if (flags & ~0x1) return fail(QXD_ERR_ARG, "qxd_Dw_batch: flags: QXD_FP64 or QXD_FP32 (native device buffers)");
    if (rhs_per_site != 0 && rhs_per_site != 1 && rhs_per_site != 2 && rhs_per_site != 4 && rhs_per_site != 8)
        return fail(QXD_ERR_ARG, "qxd_Dw_batch: rhs_per_site must be 0 (autotune), 1, 2, 4 or 8");
    std::vector<BatchItem> items;
    items.reserve(n);
    int dev = -1;
    for (int i = 0; i < n; ++i) {
        if (!lats[i] || !out[i] || !in[i]) return fail(QXD_ERR_ARG, "qxd_Dw_batch: NULL entry");
        if (!clover_ready(lats[i])) return fail(QXD_ERR_STATE, "qxd_Dw_batch: an operator needs qxd_sw_build");
        if (out[i] == in[i]) return fail(QXD_ERR_ARG, "qxd_Dw_batch: in and out must not overlap");
        if (dev < 0) dev = lats[i]->device;
        if (lats[i]->device != dev) return fail(QXD_ERR_ARG, "qxd_Dw_batch: all operators must be on one device");
        items.push_back(BatchItem{lats[i], in[i], out[i]});
    }
    // keep the right-hand sides of one operator together
    std::stable_sort(items.begin(), items.end(),
                     [](const BatchItem& a, const BatchItem& b) { return a.lat < b.lat; });
    cudaStream_t st = stream ? (cudaStream_t)stream : (n ? lats[0]->stream : nullptr);
    return dw_batch(items, flags & 0x1, rhs_per_site, st);
}
