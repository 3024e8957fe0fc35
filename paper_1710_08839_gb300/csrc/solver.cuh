// Solver workspace and the Schwarz (SAP) preconditioner interface.
#pragma once

#include <vector>

#include "blas.cuh"
#include "dirac_common.cuh"
#include "qxd_internal.cuh"

namespace qxd {

// block decomposition of the SAP preconditioner: 4^4 blocks, coloured by the
// parity of the block coordinates
struct SapGeom {
    int nb0, nb1, nb2, nb3;
    int nblk;   // all blocks
    int nhalf;  // blocks of one colour
};

struct SapWork {
    SapGeom sg{};
};

// one job of a batched SAP application (FP32): out = SAP(eta) on the job's
// operator; f.psi is the output field
struct SapJob {
    Geom g;
    SapGeom sg;
    Fields<float> f;
    const float4* Cinv;
    const float4* eta;
    float4* delta;  // work fields: last block corrections (V sites) and
    float4* rho;    // block residuals of the even sites (Vh), 6 float4 each
    float q;
    int cta_begin;
};
SapGeom sap_geom(const Geom& g);

// CUDA graphs of the batched Schwarz launch set. For a given job table, job
// count, CTA count, ncy and nmr the 2 ncy launches of one application have
// fixed arguments (the table contents are copied in before each replay), so
// the set is captured once on a private stream and replayed with one graph
// launch. At most kMax graphs are kept, the least recently used is dropped.
struct SapGraphCache {
    static constexpr int kMax = 16;
    struct Entry {
        const void* table;
        int njobs, ctas, ncy, nmr;
        cudaGraphExec_t exec;
        unsigned long long last;
    };
    std::vector<Entry> entries;
    cudaStream_t cap = nullptr;
    unsigned long long tick = 0;
    long long captures = 0, replays = 0;
    void clear();    // destroys the graphs (those in flight finish first)
    void release();  // clear() and the capture stream
};

// every job's SAP in one launch per half-cycle; d_jobs: device table with
// room for jobs.size() entries; graphs: replay the launch set from this
// cache (nullptr: plain launches)
int sap_apply_batch(std::vector<SapJob>& jobs, SapJob* d_jobs, int ncy, int nmr, cudaStream_t st,
                    SapGraphCache* graphs = nullptr);

struct SolverWork {
    int V = 0, nkv = 0, prec = -1;
    void *b64 = nullptr, *x64 = nullptr, *r64 = nullptr, *t64 = nullptr;  // full-lattice FP64
    void *xs = nullptr, *rs = nullptr, *ts = nullptr, *bs = nullptr;      // system vectors FP64
    void* tmp64 = nullptr;                                                // odd-parity FP64 temp
    void* tmp_in = nullptr;                                               // inner-precision temp
    void* rin = nullptr;                                                  // inner residual
    void* phi[BLAS_KMAX] = {};
    void* chi[BLAS_KMAX] = {};
    Reducer red;
    SapWork sap;
    double last_true_rn = 0.0;  // |b - A x| of the last reliable update
    int ensure(int V, int nkv, int prec);
    void release();
};

// checks that the lattice admits the 4^4 SAP block colouring
int sap_check(qxd_lattice* lat);
// out = SAP(in): ncy cycles of the multiplicative Schwarz method over the
// black and white blocks, nmr minimal-residual steps per block solve
template <typename R>
int sap_apply(qxd_lattice* lat, SapWork& w, void* out, const void* in, int ncy, int nmr, cudaStream_t st);
// outs[i] = SAP(ins[i]) in FP32 (native layout) for nrhs right-hand sides of
// the operator lat, solved together (each thread block stages its block's
// links once for all of them); works[i]: the work fields of right-hand side
// i, (V + Vh) * 6 float4 (delta of every site, then rho of the even sites).
// Each result is the same as with the right-hand side alone.
int sap_apply_multi(qxd_lattice* lat, int nrhs, void* const* outs, const void* const* ins, float4* const* works,
                    int ncy, int nmr, cudaStream_t st);

int run_solve(qxd_lattice* lat, const qxd_solver_params& P, qxd_solve_info& info, cudaStream_t st);

// the checks qxd_engine_submit applies to a request (who: name in the message)
int engine_check_request(qxd_lattice* op, void* x, const void* b, const qxd_solver_params* p, const char* who);

}  // namespace qxd
