// Process-wide table of the launch shapes chosen for the D kernels, and the
// C ABI to switch the autotuner, query, pin and list the choices. The paper
// has no counterpart: the shapes are properties of this GPU code.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>

#include "dirac_common.cuh"
#include "tune.cuh"

namespace qxd {
namespace {

struct Entry {
    DwShape sh;
    std::string how;  // "tuned", "default" or "set"
};

std::mutex g_mu;
std::map<DwKey, Entry> g_table;
std::atomic<int> g_autotune{1};

}  // namespace

DwKey dw_key(const qxd_lattice* lat, int prec) {
    const Geom& g = lat->g;
    return DwKey(prec, lat->qhat != 0 ? 1 : 0, g.N0, g.N1, g.N2, g.N3, lat->cstar_mask);
}

DwShape dw_default_shape(const qxd_lattice* lat, int prec) {
    return DwShape{prec == QXD_FP32 ? 1 : 0, DW_THREADS, lat->g.R, 0.f};
}

bool dw_shape_get(const DwKey& key, DwShape* out) {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_table.find(key);
    if (it == g_table.end()) return false;
    *out = it->second.sh;
    return true;
}

void dw_shape_put(const DwKey& key, const DwShape& sh, const char* how) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_table[key] = Entry{sh, how};
}

bool autotune_enabled() { return g_autotune.load() != 0; }

}  // namespace qxd

using namespace qxd;

extern "C" {

int qxd_set_autotune(int enable) { return g_autotune.exchange(enable ? 1 : 0); }

int qxd_dw_shape(const qxd_lattice* lat, int prec, int* pipelined, int* threads, int* rows, float* ms) {
    if (!lat) return fail(QXD_ERR_ARG, "qxd_dw_shape: NULL lattice");
    if (prec != QXD_FP64 && prec != QXD_FP32) return fail(QXD_ERR_ARG, "qxd_dw_shape: prec must be QXD_FP64 or QXD_FP32");
    DwShape sh;
    if (!dw_shape_get(dw_key(lat, prec), &sh))
        return fail(QXD_ERR_STATE, "qxd_dw_shape: no shape chosen yet for this lattice shape and precision");
    if (pipelined) *pipelined = sh.pipelined;
    if (threads) *threads = sh.threads;
    if (rows) *rows = sh.rows;
    if (ms) *ms = sh.ms;
    return QXD_OK;
}

int qxd_dw_set_shape(const qxd_lattice* lat, int prec, int pipelined, int threads, int rows) {
    if (!lat) return fail(QXD_ERR_ARG, "qxd_dw_set_shape: NULL lattice");
    if (prec != QXD_FP64 && prec != QXD_FP32) return fail(QXD_ERR_ARG, "qxd_dw_set_shape: prec must be QXD_FP64 or QXD_FP32");
    if ((pipelined != 0 && pipelined != 1) || (pipelined && prec != QXD_FP32))
        return fail(QXD_ERR_ARG, "qxd_dw_set_shape: the pipelined hop order exists in FP32 only");
    if (threads != 64 && threads != 128) return fail(QXD_ERR_ARG, "qxd_dw_set_shape: threads must be 64 or 128");
    if (rows < 1 || lat->g.N2 % rows) return fail(QXD_ERR_ARG, "qxd_dw_set_shape: rows must divide the x2 extent");
    dw_shape_put(dw_key(lat, prec), DwShape{pipelined, threads, rows, 0.f}, "set");
    return QXD_OK;
}

int qxd_tune_report(char* buf, size_t len, size_t* needed) {
    std::string out;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        char line[256];
        for (const auto& kv : g_table) {
            const DwKey& k = kv.first;
            const DwShape& sh = kv.second.sh;
            std::snprintf(line, sizeof line,
                          "Dw %s qhat%s %dx%dx%dx%d cstar=%u: %s threads=%d rows=%d window=%lld sites ms=%.4f (%s)\n",
                          std::get<0>(k) == QXD_FP32 ? "fp32" : "fp64", std::get<1>(k) ? "!=0" : "=0", std::get<2>(k),
                          std::get<3>(k), std::get<4>(k), std::get<5>(k), std::get<6>(k),
                          sh.pipelined ? "pipelined" : "plain", sh.threads, sh.rows,
                          (long long)std::get<3>(k) * sh.rows * std::get<5>(k), sh.ms, kv.second.how.c_str());
            out += line;
        }
    }
    dw_batch_report(out);
    if (needed) *needed = out.size() + 1;
    if (buf && len) {
        const size_t n = std::min(len - 1, out.size());
        std::memcpy(buf, out.data(), n);
        buf[n] = '\0';
    }
    return QXD_OK;
}

}  // extern "C"
