// Local deflation work space (deflation subspace, little operator, little solver).
#pragma once

#include "blas.cuh"
#include "qxd_internal.cuh"
#include "solver.cuh"

namespace qxd {

constexpr int DFL_NKV = 16;  // Krylov vectors of the little GCR before a restart

struct DflGeom {
    int nb[4];  // blocks per direction (4^4 blocks)
    int nblk;
};

// device state of the little solver (one GCR step reads the coefficients
// the previous kernels left here; the host reads it once per restart cycle)
struct LittleState {
    double a[2 * BLAS_KMAX];  // Gram-Schmidt coefficients <q_j, q_k>
    double qq;                // |q_k|^2 after orthogonalisation
    double al[2];             // <q_k, r> after normalisation
    double rn2, target2;      // |r|^2, tol^2 |c|^2
    int it, max_iter;         // steps taken, step limit
    int done, status;         // status 1: breakdown or non-finite residual
    unsigned count;           // blocks arrived at the current reduction
};

struct DflWork {
    int ns = 0;
    DflGeom d{};
    float4* basis = nullptr;   // [ns] native FP32 fields phi_k = sum_b phi_{b,k}
    float2* A = nullptr;       // little operator [nblk][9][ns][ns]
    float4* chi = nullptr;     // prolongation (FP32 field)
    float4* tfield = nullptr;  // FP32 work field
    float4* H = nullptr;       // [4] face hops (FP32 fields)
    double2 *lx = nullptr, *lc = nullptr;  // little solution and source [nblk * ns] (FP64)
    float2* lr = nullptr;                  // little residual (FP32)
    float2* lt = nullptr;                  // even-odd work vector (FP32)
    float2* Ainv = nullptr;                // [nblk][ns][ns]: inverse self-coupling of the odd blocks
    bool eo = false;                       // little solve on the even blocks (Schur complement)
    float2* lp[DFL_NKV] = {};              // little Krylov vectors (FP32)
    float2* lq[DFL_NKV] = {};
    int* d_bad = nullptr;
    LittleState* lstate = nullptr;    // device
    LittleState* h_lstate = nullptr;  // pinned host copy
    cudaStream_t cap = nullptr;       // capture stream of the cycle graph
    cudaGraphExec_t cycle = nullptr;  // one restart cycle (DFL_NKV steps) of the little GCR
    Reducer red;
    SapWork sap;
    unsigned op_version = 0;   // operator the little operator was built for
    bool ready = false;
    int ensure(const Geom& g, int ns);
    void release();
};

void release_dfl(qxd_lattice* lat);
// out = M_dfl in (FP32 native full-lattice fields); little_iters accumulates
// the little-solver steps
int dfl_precondition(qxd_lattice* lat, void* out, const void* in, int ncy, int nmr, double tol, int max_iter,
                     int* little_iters, cudaStream_t st);
// deflation subspace built and matching the current operator
inline bool dfl_ready(const qxd_lattice* lat) { return lat->dfl && lat->dfl->ready && lat->dfl->op_version == lat->op_version && clover_ready(lat); }

}  // namespace qxd
