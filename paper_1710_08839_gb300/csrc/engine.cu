// Batched solve engine: many independent solves D_i x_i = b_i advanced in
// lockstep, one flexible-GCR step per engine step for every active job.
//
// Per step, all active jobs share each kernel launch: one launch per SAP
// half-cycle (k_sap_block_batch over every job's blocks), one batched D
// (k_dirac_batch), and one launch per vector operation (k_blas_batch, with
// grid.y = job). Each job's arithmetic uses exactly the kernels, grids and
// reduction orders it would use alone, so its result does not depend on the
// other jobs in the batch. Between steps the engine retires finished jobs and
// admits queued ones while their device memory fits the budget (continuous
// batching). The algorithm per job is the flexible GCR of solver.cu (full
// system, FP32 inner vectors and preconditioner, FP64 reliable updates).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "batch.cuh"
#include "blas.cuh"
#include "solver.cuh"

namespace qxd {

namespace {

using Clock = std::chrono::steady_clock;

constexpr long long kBigSites = 1 << 20;  // lattices routed to the single-lattice kernels

// caching device allocator: freed blocks go to per-size free lists. The
// device memory it holds (blocks in use plus cached ones) is kept within
// cap: before a new cudaMalloc would take it above cap, cached blocks of
// other sizes are released first, then any cached block.
struct DevicePool {
    std::map<size_t, std::vector<void*>> free_;
    size_t in_use = 0, held = 0;
    size_t cap = (size_t)-1;
    int alloc(size_t bytes, void** p) {
        auto it = free_.find(bytes);
        if (it != free_.end() && !it->second.empty()) {
            *p = it->second.back();
            it->second.pop_back();
            in_use += bytes;
            return QXD_OK;
        }
        if (held + bytes > cap) reclaim(bytes);
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            trim();
            e = cudaMalloc(p, bytes);
        }
        if (e != cudaSuccess) {
            *p = nullptr;
            return cuda_fail(e, "engine: cudaMalloc");
        }
        in_use += bytes;
        held += bytes;
        return QXD_OK;
    }
    void release(void* p, size_t bytes) {
        if (!p) return;
        free_[bytes].push_back(p);
        in_use -= bytes;
    }
    // release cached blocks until a new block of `bytes` fits under cap:
    // blocks of other sizes first (a block of this size would have been reused)
    void reclaim(size_t bytes) {
        for (int pass = 0; pass < 2 && held + bytes > cap; ++pass)
            for (auto& kv : free_) {
                if (pass == 0 && kv.first == bytes) continue;
                while (!kv.second.empty() && held + bytes > cap) {
                    cudaFree(kv.second.back());
                    kv.second.pop_back();
                    held -= kv.first;
                }
            }
    }
    void trim() {
        for (auto& kv : free_)
            for (void* p : kv.second) {
                cudaFree(p);
                held -= kv.first;
            }
        free_.clear();
    }
    ~DevicePool() { trim(); }
};

enum JobState { JOB_PENDING, JOB_ACTIVE, JOB_DONE };

struct Job {
    long long id;
    qxd_lattice* op;
    qxd_solver_params P;
    void* x_user;
    const void* b_user;
    JobState state = JOB_PENDING;
    // device vectors
    size_t f64_bytes = 0, f32_bytes = 0;
    void *b64 = nullptr, *x64 = nullptr, *r64 = nullptr, *t64 = nullptr, *rin = nullptr;
    void* sapw = nullptr;  // work fields of the Schwarz solve (delta, rho of the even sites)
    size_t sapw_bytes = 0;
    void* phi[BLAS_KMAX] = {};
    void* chi[BLAS_KMAX] = {};
    // solver state
    double bn = 0, rn = 0, rin_n = 0, target = 0;
    int k = 0;
    bool restart = true;
    bool cycle_end = false;
    cd Rm[BLAS_KMAX][BLAS_KMAX];
    cd c[BLAS_KMAX], a[BLAS_KMAX];
    qxd_solve_info info{};
    Clock::time_point t0;
    size_t charge = 0;  // job_bytes charged against the budget while admitted
};

// FP32 work fields of a batched Schwarz solve: the last block corrections
// of every site and the block residuals of the even sites
size_t sap_work_bytes(const qxd_lattice* op) { return ((size_t)op->g.V + op->g.Vh) * 24 * sizeof(float); }

// device bytes a request holds at most: four FP64 fields, the FP32 residual,
// nkv Krylov pairs (allocated on demand, but charged at admission so that
// the active requests stay within the budget whatever their Krylov depth)
// and the Schwarz work fields (charged for every request)
size_t job_bytes(const qxd_lattice* op, int nkv) {
    const size_t V = (size_t)op->g.V;
    return V * 24 * sizeof(double) * 4 + V * 24 * sizeof(float) * (1 + 2 * (size_t)nkv) + sap_work_bytes(op);
}

}  // namespace

struct Engine {
    cudaStream_t st;
    size_t budget;
    int max_active;
    long long next_id = 1;
    DevicePool pool;
    std::deque<Job*> pending;
    std::vector<Job*> active;
    std::map<long long, std::unique_ptr<Job>> jobs;
    BatchReducer red;
    SapJob* d_sap = nullptr;
    int d_sap_cap = 0;
    SapGraphCache sap_graphs;  // graphs of the batched SAP launch sets
    long long steps = 0;
    size_t charged = 0;  // sum of the charges of the admitted requests

    ~Engine() {
        sap_graphs.release();
        if (d_sap) cudaFree(d_sap);
        red.release();
        for (auto& kv : jobs) free_job(kv.second.get());
    }

    void free_job(Job* j) {
        charged -= j->charge;
        j->charge = 0;
        pool.release(j->b64, j->f64_bytes);
        pool.release(j->x64, j->f64_bytes);
        pool.release(j->r64, j->f64_bytes);
        pool.release(j->t64, j->f64_bytes);
        pool.release(j->rin, j->f32_bytes);
        pool.release(j->sapw, j->sapw_bytes);
        j->sapw = nullptr;
        for (int i = 0; i < BLAS_KMAX; ++i) {
            pool.release(j->phi[i], j->f32_bytes);
            pool.release(j->chi[i], j->f32_bytes);
        }
        j->b64 = j->x64 = j->r64 = j->t64 = j->rin = nullptr;
        for (int i = 0; i < BLAS_KMAX; ++i) j->phi[i] = j->chi[i] = nullptr;
    }

    int alloc_job(Job* j) {
        const size_t V = (size_t)j->op->g.V;
        j->f64_bytes = V * 24 * sizeof(double);
        j->f32_bytes = V * 24 * sizeof(float);
        int rc;
        void** f64[] = {&j->b64, &j->x64, &j->r64, &j->t64};
        for (void** p : f64)
            if ((rc = pool.alloc(j->f64_bytes, p))) return rc;
        if ((rc = pool.alloc(j->f32_bytes, &j->rin))) return rc;
        if (j->P.precond == QXD_PRECOND_SAP) {
            j->sapw_bytes = sap_work_bytes(j->op);
            if ((rc = pool.alloc(j->sapw_bytes, &j->sapw))) return rc;
        }
        // Krylov vectors are allocated when first used (SAP-preconditioned
        // GCR rarely needs all nkv of them)
        return QXD_OK;
    }

    void finish(Job* j, int status) {
        j->info.status = status;
        j->info.time_ms = std::chrono::duration<double, std::milli>(Clock::now() - j->t0).count();
        j->state = JOB_DONE;
    }

    // copy the solution out and release the job's vectors
    int complete(Job* j, int status) {
        int rc = QXD_OK;
        const size_t bytes = j->f64_bytes;
        if (j->P.flags & QXD_LAYOUT_NATIVE) {
            if (cudaMemcpyAsync(j->x_user, j->x64, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) rc = QXD_ERR_CUDA;
        } else {
            rc = launch_unpack(j->op, j->x_user, j->x64, QXD_FP64, st);
        }
        if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = QXD_ERR_CUDA;
        free_job(j);
        finish(j, rc ? rc : status);
        return rc;
    }

    int admit() {
        std::vector<Job*> fresh;
        while (!pending.empty() && (int)active.size() + (int)fresh.size() < max_active) {
            Job* j = pending.front();
            const size_t need = job_bytes(j->op, j->P.nkv);
            if (charged + need > budget && !(active.empty() && fresh.empty())) break;
            pending.pop_front();
            j->charge = need;
            charged += need;
            int rc = alloc_job(j);
            if (rc) {
                free_job(j);
                finish(j, rc);
                continue;
            }
            j->t0 = Clock::now();
            // b -> native FP64, x = 0, r = b
            if (j->P.flags & QXD_LAYOUT_NATIVE) {
                QXD_CUDA(cudaMemcpyAsync(j->b64, j->b_user, j->f64_bytes, cudaMemcpyDeviceToDevice, st));
            } else if ((rc = launch_pack(j->op, j->b64, j->b_user, QXD_FP64, st))) {
                return rc;
            }
            QXD_CUDA(cudaMemsetAsync(j->x64, 0, j->f64_bytes, st));
            QXD_CUDA(cudaMemcpyAsync(j->r64, j->b64, j->f64_bytes, cudaMemcpyDeviceToDevice, st));
            j->state = JOB_ACTIVE;
            fresh.push_back(j);
        }
        if (fresh.empty()) return QXD_OK;
        int rc = red.ensure((int)fresh.size());
        if (rc) return rc;
        for (size_t i = 0; i < fresh.size(); ++i) {
            BJob& b = red.h_jobs[i];
            b = BJob{};
            b.n = (size_t)fresh[i]->op->g.V * 12;
            b.y = fresh[i]->b64;
        }
        if ((rc = blas_batch(red, B_NORM2_F64, (int)fresh.size(), 1, st))) return rc;
        for (size_t i = 0; i < fresh.size(); ++i) {
            Job* j = fresh[i];
            j->bn = std::sqrt(red.h_res[i * 2 * BLAS_KMAX]);
            j->rn = j->bn;
            j->target = j->P.tol * j->bn;
            j->restart = true;
            if (!std::isfinite(j->bn)) {
                free_job(j);
                finish(j, QXD_ERR_NUMERIC);
            } else if (j->bn == 0.0) {
                j->info.true_relres = 0.0;
                if ((rc = complete(j, QXD_OK))) return rc;
            } else {
                active.push_back(j);
            }
        }
        return QXD_OK;
    }

    // jobs on lattices this large fill the GPU alone: their Schwarz method
    // and D run through the single-lattice kernels (no job-table lookup);
    // the choice depends only on the job's own lattice, so a job's result
    // still does not depend on the batch
    static bool big(const Job* j) { return (long long)j->op->g.V >= kBigSites; }

    int step(int* ndone) {
        int rc, failed = 0;
        if ((rc = admit())) return rc;
        int n = (int)active.size();
        if (n == 0) return QXD_OK;
        ++steps;
        if ((rc = red.ensure(n))) return rc;
        // restart: rin = (float) r64, k = 0
        {
            int m = 0;
            for (Job* j : active)
                if (j->restart) {
                    BJob& b = red.h_jobs[m++];
                    b = BJob{};
                    b.n = (size_t)j->op->g.V;
                    b.y = j->r64;
                    b.out = j->rin;
                    j->k = 0;
                    j->rin_n = j->rn;
                    j->restart = false;
                }
            if ((rc = blas_batch(red, B_D2F_NATIVE, m, 0, st))) return rc;
        }
        // Krylov pair k of every job (allocated on first use). A job whose
        // pair cannot be allocated fails alone; the others go on.
        {
            std::vector<Job*> ok;
            for (Job* j : active) {
                if (!j->phi[j->k]) {
                    int e = pool.alloc(j->f32_bytes, &j->phi[j->k]);
                    if (!e) e = pool.alloc(j->f32_bytes, &j->chi[j->k]);
                    if (e) {
                        free_job(j);
                        finish(j, e);
                        continue;
                    }
                }
                ok.push_back(j);
            }
            if (ok.size() != active.size()) {
                failed = (int)(active.size() - ok.size());
                if (ndone) *ndone = failed;
                active.swap(ok);
                n = (int)active.size();
                if (n == 0) return QXD_OK;
            }
        }
        // phi_k = P(rin); large lattices of one operator (and ncy, nmr) solved
        // together, each thread block staging its links once for all of them
        std::vector<SapJob> sj;
        std::map<std::tuple<qxd_lattice*, int, int>, std::vector<Job*>> same_op;
        for (Job* j : active) {
            if (j->P.precond == QXD_PRECOND_SAP && big(j)) {
                same_op[{j->op, j->P.sap_ncy, j->P.sap_nmr}].push_back(j);
            } else if (j->P.precond == QXD_PRECOND_SAP) {
                SapJob J{};
                J.g = j->op->g;
                J.sg = sap_geom(j->op->g);
                J.f = Fields<float>{(const float4*)j->phi[j->k], nullptr, j->op->U32, j->op->A32, j->op->C32};
                J.Cinv = j->op->Cinv32;
                J.eta = (const float4*)j->rin;
                J.delta = (float4*)j->sapw;
                J.rho = J.delta + (size_t)SPINOR_F4 * j->op->g.V;
                J.q = (float)j->op->qhat;
                sj.push_back(J);
            } else {
                QXD_CUDA(cudaMemcpyAsync(j->phi[j->k], j->rin, j->f32_bytes, cudaMemcpyDeviceToDevice, st));
            }
        }
        for (auto& kv : same_op) {
            std::vector<void*> outs;
            std::vector<const void*> ins;
            std::vector<float4*> works;
            for (Job* j : kv.second) {
                outs.push_back(j->phi[j->k]);
                ins.push_back(j->rin);
                works.push_back((float4*)j->sapw);
            }
            if ((rc = sap_apply_multi(std::get<0>(kv.first), (int)outs.size(), outs.data(), ins.data(), works.data(),
                                      std::get<1>(kv.first), std::get<2>(kv.first), st)))
                return rc;
        }
        if (!sj.empty()) {
            if ((int)sj.size() > d_sap_cap) {
                if (d_sap) {
                    cudaStreamSynchronize(st);
                    sap_graphs.clear();  // they hold the old table address
                    cudaFree(d_sap);
                }
                d_sap_cap = (int)sj.size() * 2;
                QXD_CUDA(cudaMalloc(&d_sap, sizeof(SapJob) * d_sap_cap));
            }
            // all SAP jobs of a step share ncy and nmr of their own params:
            // group by (ncy, nmr)
            std::map<std::pair<int, int>, std::vector<SapJob>> groups;
            size_t idx = 0;
            for (Job* j : active)
                if (j->P.precond == QXD_PRECOND_SAP && !big(j))
                    groups[{j->P.sap_ncy, j->P.sap_nmr}].push_back(sj[idx++]);
            // the table copies are ordered on the stream, so d_sap can be
            // rewritten for the next group
            for (auto& kv : groups)
                if ((rc = sap_apply_batch(kv.second, d_sap, kv.first.first, kv.first.second, st, &sap_graphs)))
                    return rc;
        }
        // chi_k = D phi_k (FP32)
        {
            std::vector<BatchItem> items;
            for (Job* j : active) {
                if (big(j)) {
                    if ((rc = launch_dirac(j->op, j->chi[j->k], j->phi[j->k], QXD_FP32, st))) return rc;
                } else {
                    items.push_back(BatchItem{j->op, j->phi[j->k], j->chi[j->k]});
                }
            }
            std::stable_sort(items.begin(), items.end(),
                             [](const BatchItem& a, const BatchItem& b) { return a.lat < b.lat; });
            if (!items.empty() && (rc = dw_batch(items, QXD_FP32, 0, st))) return rc;
            for (Job* j : active) ++j->info.inner_calls;
        }
        // Gram-Schmidt: a_j = <chi_j, chi_k>
        {
            int m = 0;
            std::vector<Job*> with;
            for (Job* j : active)
                if (j->k > 0) {
                    BJob& b = red.h_jobs[m++];
                    b = BJob{};
                    b.n = (size_t)j->op->g.V * 12;
                    b.k = j->k;
                    for (int i = 0; i < j->k; ++i) b.xs[i] = j->chi[i];
                    b.y = j->chi[j->k];
                    with.push_back(j);
                }
            if (m && (rc = blas_batch(red, B_MDOT_F32, m, 2 * BLAS_KMAX, st))) return rc;
            for (int i = 0; i < m; ++i)
                for (int l = 0; l < with[i]->k; ++l)
                    with[i]->a[l] = cd(red.h_res[i * 2 * BLAS_KMAX + 2 * l], red.h_res[i * 2 * BLAS_KMAX + 2 * l + 1]);
        }
        // chi_k -= sum a_j chi_j, |chi_k|
        for (int i = 0; i < n; ++i) {
            Job* j = active[i];
            BJob& b = red.h_jobs[i];
            b = BJob{};
            b.n = (size_t)j->op->g.V * 12;
            b.k = j->k;
            for (int l = 0; l < j->k; ++l) {
                b.xs[l] = j->chi[l];
                b.cre[l] = j->a[l].real();
                b.cim[l] = j->a[l].imag();
            }
            b.out = j->chi[j->k];
        }
        if ((rc = blas_batch(red, B_MAXPY_NORM_F32, n, 1, st))) return rc;
        std::vector<double> nrm(n);
        for (int i = 0; i < n; ++i) {
            Job* j = active[i];
            nrm[i] = std::sqrt(red.h_res[i * 2 * BLAS_KMAX]);
            if (!std::isfinite(nrm[i]) || nrm[i] == 0.0) {
                j->state = JOB_DONE;  // marked; handled below
            }
            BJob& b = red.h_jobs[i];
            b = BJob{};
            b.n = (size_t)j->op->g.V * 12;
            b.s = nrm[i] > 0 && std::isfinite(nrm[i]) ? 1.0 / nrm[i] : 0.0;
            b.out = j->chi[j->k];
        }
        if ((rc = blas_batch(red, B_SCALE_F32, n, 0, st))) return rc;
        // c_k = <chi_k, rin>
        for (int i = 0; i < n; ++i) {
            Job* j = active[i];
            BJob& b = red.h_jobs[i];
            b = BJob{};
            b.n = (size_t)j->op->g.V * 12;
            b.k = 1;
            b.xs[0] = j->chi[j->k];
            b.y = j->rin;
        }
        if ((rc = blas_batch(red, B_MDOT_F32, n, 2, st))) return rc;
        for (int i = 0; i < n; ++i) {
            Job* j = active[i];
            j->c[j->k] = cd(red.h_res[i * 2 * BLAS_KMAX], red.h_res[i * 2 * BLAS_KMAX + 1]);
            for (int l = 0; l < j->k; ++l) j->Rm[l][j->k] = j->a[l];
            j->Rm[j->k][j->k] = cd(nrm[i], 0.0);
            BJob& b = red.h_jobs[i];
            b = BJob{};
            b.n = (size_t)j->op->g.V * 12;
            b.k = 1;
            b.xs[0] = j->chi[j->k];
            b.cre[0] = j->c[j->k].real();
            b.cim[0] = j->c[j->k].imag();
            b.out = j->rin;
        }
        if ((rc = blas_batch(red, B_MAXPY_NORM_F32, n, 1, st))) return rc;
        std::vector<Job*> ending;
        for (int i = 0; i < n; ++i) {
            Job* j = active[i];
            if (j->state == JOB_DONE) {  // breakdown or non-finite direction
                ending.push_back(j);
                continue;
            }
            j->rin_n = std::sqrt(red.h_res[i * 2 * BLAS_KMAX]);
            ++j->k;
            ++j->info.iterations;
            const qxd_solver_params& P = j->P;
            j->cycle_end = j->k >= P.nkv || j->rin_n <= 0.5 * j->target ||
                           (P.delta > 0 && j->rin_n < P.delta * j->rn) || j->info.iterations >= P.max_iter ||
                           !std::isfinite(j->rin_n);
            if (j->cycle_end) ending.push_back(j);
        }
        // a failure there still leaves every ending job finished or restarting
        rc = ending.empty() ? QXD_OK : end_cycles(ending);
        // retire
        std::vector<Job*> still;
        int done = 0;
        for (Job* j : active)
            if (j->state == JOB_DONE) ++done;
            else still.push_back(j);
        active.swap(still);
        if (ndone) *ndone = done + failed;
        return rc;
    }

    // x += sum beta phi, r = b - D x (FP64) for the jobs whose cycle ended
    int end_cycles(std::vector<Job*>& ending) {
        int rc;
        std::vector<Job*> upd;
        for (Job* j : ending) {
            if (j->state == JOB_DONE) {  // failed direction
                if (j->k == 0) {
                    free_job(j);
                    finish(j, QXD_ERR_NUMERIC);
                    continue;
                }
                j->state = JOB_ACTIVE;
            }
            upd.push_back(j);
        }
        if (upd.empty()) return QXD_OK;
        rc = update_cycles(upd);
        if (rc) {
            // no job may stay active with a finished cycle (k could be nkv):
            // the jobs the update did not finish or restart fail with rc
            for (Job* j : upd)
                if (j->state != JOB_DONE && !j->restart) {
                    free_job(j);
                    finish(j, rc);
                }
        }
        return rc;
    }

    // the FP64 update of end_cycles; every job of upd is processed by the
    // final loop even when one completion fails (the first error is returned)
    int update_cycles(std::vector<Job*>& upd) {
        int rc;
        if ((rc = red.ensure((int)upd.size()))) return rc;
        for (size_t i = 0; i < upd.size(); ++i) {
            Job* j = upd[i];
            cd beta[BLAS_KMAX];
            for (int l = j->k - 1; l >= 0; --l) {
                cd s = j->c[l];
                for (int m = l + 1; m < j->k; ++m) s -= j->Rm[l][m] * beta[m];
                beta[l] = s / j->Rm[l][l];
            }
            BJob& b = red.h_jobs[i];
            b = BJob{};
            b.n = (size_t)j->op->g.V;
            b.k = j->k;
            for (int l = 0; l < j->k; ++l) {
                b.xs[l] = j->phi[l];
                b.cre[l] = beta[l].real();
                b.cim[l] = beta[l].imag();
            }
            b.out = j->x64;
        }
        if ((rc = blas_batch(red, B_UPDATE_X_NATIVE32, (int)upd.size(), 0, st))) return rc;
        std::vector<BatchItem> items;
        for (Job* j : upd) {
            if (big(j)) {
                if ((rc = launch_dirac(j->op, j->t64, j->x64, QXD_FP64, st))) return rc;
            } else {
                items.push_back(BatchItem{j->op, j->x64, j->t64});
            }
        }
        std::stable_sort(items.begin(), items.end(), [](const BatchItem& a, const BatchItem& b) { return a.lat < b.lat; });
        if (!items.empty() && (rc = dw_batch(items, QXD_FP64, 0, st))) return rc;
        for (size_t i = 0; i < upd.size(); ++i) {
            Job* j = upd[i];
            BJob& b = red.h_jobs[i];
            b = BJob{};
            b.n = (size_t)j->op->g.V * 12;
            b.b = j->b64;
            b.y = j->t64;
            b.out = j->r64;
        }
        if ((rc = blas_batch(red, B_SUB_NORM_F64, (int)upd.size(), 1, st))) return rc;
        int first = QXD_OK;
        for (size_t i = 0; i < upd.size(); ++i) {
            Job* j = upd[i];
            j->rn = std::sqrt(red.h_res[i * 2 * BLAS_KMAX]);
            ++j->info.restarts;
            ++j->info.dw64_calls;
            j->info.true_relres = j->rn / j->bn;
            if (!std::isfinite(j->rn)) {
                free_job(j);
                finish(j, QXD_ERR_NUMERIC);
            } else if (j->rn <= j->target) {
                if ((rc = complete(j, QXD_OK)) && !first) first = rc;
            } else if (j->info.iterations >= j->P.max_iter) {
                if ((rc = complete(j, QXD_ERR_NOT_CONVERGED)) && !first) first = rc;
            } else {
                j->restart = true;
            }
        }
        return first;
    }
};

}  // namespace qxd

struct qxd_engine : public qxd::Engine {};

namespace qxd {
// checks of a request the engine accepts (also used by the server)
int engine_check_request(qxd_lattice* op, void* x, const void* b, const qxd_solver_params* p, const char* who) {
    const std::string w(who);
    if (!op || !x || !b || !p) return fail(QXD_ERR_ARG, w + ": NULL argument");
    const qxd_solver_params& P = *p;
    if (!(P.tol > 0) || P.max_iter < 1 || P.nkv < 1 || P.nkv > BLAS_KMAX)
        return fail(QXD_ERR_ARG, w + ": tol > 0, max_iter >= 1 and 1 <= nkv <= 16 required");
    if (P.system != QXD_SOLVE_FULL || P.inner_prec != QXD_FP32 ||
        (P.precond != QXD_PRECOND_SAP && P.precond != QXD_PRECOND_NONE) || (P.flags & ~0x100))
        return fail(QXD_ERR_ARG, w + ": the engine runs full-system FGCR with FP32 inner vectors on device buffers");
    if (P.precond == QXD_PRECOND_SAP && (P.sap_ncy < 1 || P.sap_nmr < 1))
        return fail(QXD_ERR_ARG, w + ": sap_ncy and sap_nmr must be >= 1");
    if (!clover_ready(op)) return fail(QXD_ERR_STATE, w + ": the operator needs qxd_sw_build");
    if (P.precond == QXD_PRECOND_SAP) return sap_check(op);
    return QXD_OK;
}
}  // namespace qxd

using namespace qxd;

extern "C" {

int qxd_engine_create(qxd_engine** out, size_t hbm_budget_bytes, int max_active, void* stream) {
    if (!out || max_active < 1) return fail(QXD_ERR_ARG, "qxd_engine_create: NULL out or max_active < 1");
    qxd_engine* e = new (std::nothrow) qxd_engine();
    if (!e) return fail(QXD_ERR_OOM, "qxd_engine_create: host allocation failed");
    e->st = (cudaStream_t)stream;
    e->budget = hbm_budget_bytes;
    e->pool.cap = hbm_budget_bytes;
    e->max_active = max_active;
    *out = e;
    return QXD_OK;
}

int qxd_engine_destroy(qxd_engine* e) {
    if (!e) return QXD_OK;
    cudaStreamSynchronize(e->st);
    delete e;
    return QXD_OK;
}

int qxd_engine_submit(qxd_engine* e, qxd_lattice* op, void* x, const void* b, const qxd_solver_params* p,
                      long long* id) {
    if (!e || !id) return fail(QXD_ERR_ARG, "qxd_engine_submit: NULL argument");
    int rc = engine_check_request(op, x, b, p, "qxd_engine_submit");
    if (rc) return rc;
    const qxd_solver_params& P = *p;
    std::unique_ptr<Job> j(new (std::nothrow) Job());
    if (!j) return fail(QXD_ERR_OOM, "qxd_engine_submit: host allocation failed");
    j->id = e->next_id++;
    j->op = op;
    j->P = P;
    j->x_user = x;
    j->b_user = b;
    j->info.status = QXD_ERR_STATE;  // pending
    *id = j->id;
    e->pending.push_back(j.get());
    e->jobs[j->id] = std::move(j);
    return QXD_OK;
}

int qxd_engine_step(qxd_engine* e, int* n_active, int* n_pending, int* n_done) {
    if (!e) return fail(QXD_ERR_ARG, "qxd_engine_step: NULL engine");
    int done = 0;
    int rc = e->step(&done);
    if (n_active) *n_active = (int)e->active.size();
    if (n_pending) *n_pending = (int)e->pending.size();
    if (n_done) *n_done = done;
    return rc;
}

int qxd_engine_poll(qxd_engine* e, long long id, qxd_solve_info* info, int* done) {
    if (!e) return fail(QXD_ERR_ARG, "qxd_engine_poll: NULL engine");
    auto it = e->jobs.find(id);
    if (it == e->jobs.end()) return fail(QXD_ERR_ARG, "qxd_engine_poll: unknown request id");
    Job* j = it->second.get();
    if (info) *info = j->info;
    if (done) *done = j->state == JOB_DONE;
    return QXD_OK;
}

int qxd_engine_forget(qxd_engine* e, long long id) {
    if (!e) return fail(QXD_ERR_ARG, "qxd_engine_forget: NULL engine");
    auto it = e->jobs.find(id);
    if (it == e->jobs.end()) return fail(QXD_ERR_ARG, "qxd_engine_forget: unknown request id");
    if (it->second->state != JOB_DONE) return fail(QXD_ERR_STATE, "qxd_engine_forget: request not finished");
    e->jobs.erase(it);
    return QXD_OK;
}

int qxd_engine_run(qxd_engine* e) {
    if (!e) return fail(QXD_ERR_ARG, "qxd_engine_run: NULL engine");
    while (!e->active.empty() || !e->pending.empty()) {
        int rc = e->step(nullptr);
        if (rc) return rc;
    }
    return QXD_OK;
}

int qxd_engine_stats(const qxd_engine* e, size_t* bytes_in_use, size_t* bytes_held, long long* steps) {
    if (!e) return fail(QXD_ERR_ARG, "qxd_engine_stats: NULL engine");
    if (bytes_in_use) *bytes_in_use = e->pool.in_use;
    if (bytes_held) *bytes_held = e->pool.held;
    if (steps) *steps = e->steps;
    return QXD_OK;
}

int qxd_engine_graph_stats(const qxd_engine* e, long long* captures, long long* replays) {
    if (!e) return fail(QXD_ERR_ARG, "qxd_engine_graph_stats: NULL engine");
    if (captures) *captures = e->sap_graphs.captures;
    if (replays) *replays = e->sap_graphs.replays;
    return QXD_OK;
}

}  // extern "C"
