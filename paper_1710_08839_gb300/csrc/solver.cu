// Flexible GCR solver for D x = b (full lattice) or D_hat x_e = b_hat_e
// (even-odd form, Sec. 2.4), with optional SAP preconditioning.
//
// The paper names the SAP-preconditioned GCR solver (Sec. 1-2) without
// specifying it; this is the textbook flexible GCR: at step k the direction
// phi_k = P(r) comes from the preconditioner P, chi_k = A phi_k is made
// orthonormal against chi_0..chi_{k-1} (classical Gram-Schmidt with FP64
// accumulated inner products), and r -= <chi_k, r> chi_k. At a restart the
// upper-triangular Gram-Schmidt system R beta = c is solved, x += sum beta_k
// phi_k in FP64, and the true residual b - A x is recomputed in FP64
// (reliable update). A restart happens after nkv steps, or earlier when the
// inner residual drops below delta times the last true residual.
#include <chrono>
#include <cmath>
#include <vector>

#include "blas.cuh"
#include "dfl.cuh"
#include "eo.cuh"
#include "solver.cuh"

namespace qxd {

namespace {

template <typename R>
struct V2T;
template <>
struct V2T<float> {
    using type = float2;
};
template <>
struct V2T<double> {
    using type = double2;
};

__global__ void k_copy_parity(Geom g, int p, SpRef<double> in, SpRefOut<double> out) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    const int s = p * g.Vh + h;
#pragma unroll
    for (int k = 0; k < 12; ++k) out.p[(size_t)k * out.stride + s - out.off] = in.p[(size_t)k * in.stride + s - in.off];
}

int copy_parity(qxd_lattice* lat, int p, SpRef<double> in, SpRefOut<double> out, cudaStream_t st) {
    k_copy_parity<<<(lat->g.Vh + 255) / 256, 256, 0, st>>>(lat->g, p, in, out);
    QXD_LAUNCHED("k_copy_parity");
    return QXD_OK;
}

int alloc(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMalloc(solver work)");
    }
    return QXD_OK;
}

}  // namespace

void SolverWork::release() {
    void* ps[] = {b64, x64, r64, t64, xs, rs, ts, bs, tmp64, tmp_in, rin};
    for (void* p : ps)
        if (p) cudaFree(p);
    for (int k = 0; k < BLAS_KMAX; ++k) {
        if (phi[k]) cudaFree(phi[k]);
        if (chi[k]) cudaFree(chi[k]);
        phi[k] = chi[k] = nullptr;
    }
    b64 = x64 = r64 = t64 = xs = rs = ts = bs = tmp64 = tmp_in = rin = nullptr;
    red.release();
    nkv = 0;
    prec = -1;
    V = 0;
}

int SolverWork::ensure(int V_, int nkv_, int prec_) {
    // inner vectors are sized for FP64, so switching the inner precision
    // reuses them; a new lattice size or more Krylov vectors reallocate
    (void)prec_;
    if (V == V_ && nkv >= nkv_) return QXD_OK;
    release();
    const size_t b64n = (size_t)V_ * 12 * sizeof(double2);
    const size_t binn = b64n;
    int rc;
    void** full[] = {&b64, &x64, &r64, &t64, &xs, &rs, &ts, &bs, &tmp64};
    for (void** p : full)
        if ((rc = alloc(p, b64n))) return rc;
    if ((rc = alloc(&tmp_in, binn)) || (rc = alloc(&rin, binn))) return rc;
    for (int k = 0; k < nkv_; ++k)
        if ((rc = alloc(&phi[k], binn)) || (rc = alloc(&chi[k], binn))) return rc;
    if ((rc = red.init())) return rc;
    V = V_;
    nkv = nkv_;
    prec = QXD_FP64;
    return QXD_OK;
}

namespace {

// the FP64 operator of the system: D (full) or D_hat (even sites)
int apply_a64(qxd_lattice* lat, SolverWork& w, bool eo, double2* out, const double2* in, cudaStream_t st) {
    if (!eo) return launch_dirac(lat, out, in, QXD_FP64, st);
    const int Vh = lat->g.Vh;
    return apply_dhat<double>(lat, half_out<double>(out, Vh, 0), half_ref<double>(in, Vh, 0),
                              half_out<double>(w.tmp64, Vh, 1), st);
}

template <typename R>
int apply_ain(qxd_lattice* lat, SolverWork& w, bool eo, void* out, const void* in, cudaStream_t st) {
    const int prec = sizeof(R) == 4 ? QXD_FP32 : QXD_FP64;
    if (!eo) return launch_dirac(lat, out, in, prec, st);
    const int Vh = lat->g.Vh;
    return apply_dhat<R>(lat, half_out<R>(out, Vh, 0), half_ref<R>(in, Vh, 0), half_out<R>(w.tmp_in, Vh, 1), st);
}

template <typename R>
int precondition(qxd_lattice* lat, SolverWork& w, const qxd_solver_params& P, void* out, const void* in,
                 size_t bytes, cudaStream_t st, qxd_solve_info& info) {
    if (P.precond == QXD_PRECOND_SAP) return sap_apply<R>(lat, w.sap, out, in, P.sap_ncy, P.sap_nmr, st);
    if constexpr (sizeof(R) == 4) {
        if (P.precond == QXD_PRECOND_DFL_SAP)
            return dfl_precondition(lat, out, in, P.sap_ncy, P.sap_nmr, P.dfl_tol, P.dfl_max_iter,
                                    &info.little_iters, st);
    }
    QXD_CUDA(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st));
    return QXD_OK;
}

template <typename R>
int fgcr(qxd_lattice* lat, SolverWork& w, const qxd_solver_params& P, double bn, qxd_solve_info& info,
         cudaStream_t st) {
    using V2 = typename V2T<R>::type;
    const bool eo = P.system == QXD_SOLVE_EO;
    const size_t n = (size_t)(eo ? lat->g.Vh : lat->g.V) * 12;  // complex numbers per vector
    const size_t bytes_in = n * sizeof(V2);
    double2* xs = (double2*)w.xs;
    double2* rs = (double2*)w.rs;
    double2* ts = (double2*)w.ts;
    const double2* bs = (const double2*)w.bs;
    V2* rin = (V2*)w.rin;
    const double target = P.tol * bn;
    int rc;

    QXD_CUDA(cudaMemsetAsync(xs, 0, n * sizeof(double2), st));
    QXD_CUDA(cudaMemcpyAsync(rs, bs, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    double rn2;
    if ((rc = blas_norm2<double2>(w.red, n, rs, &rn2, st))) return rc;
    double rn = std::sqrt(rn2);
    std::vector<cd> Rm(BLAS_KMAX * BLAS_KMAX), c(BLAS_KMAX), a(BLAS_KMAX);
    while (true) {
        if (!std::isfinite(rn)) return fail(QXD_ERR_NUMERIC, "qxd_solve: non-finite residual");
        if (rn <= target) break;
        if (info.iterations >= P.max_iter) break;
        // inner residual in the inner precision
        if (sizeof(R) == 4) {
            if ((rc = blas_d2f_native(n / 12, rs, (float2*)rin, st))) return rc;
        } else {
            QXD_CUDA(cudaMemcpyAsync(rin, rs, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        }
        double rin_n = rn;
        int k = 0;
        while (k < P.nkv && info.iterations < P.max_iter) {
            V2* phk = (V2*)w.phi[k];
            V2* chk = (V2*)w.chi[k];
            if ((rc = precondition<R>(lat, w, P, phk, rin, bytes_in, st, info))) return rc;
            if ((rc = apply_ain<R>(lat, w, eo, chk, phk, st))) return rc;
            ++info.inner_calls;
            // classical Gram-Schmidt against chi_0..chi_{k-1}
            VecList<V2> prev{};
            for (int j = 0; j < k; ++j) prev.p[j] = (const V2*)w.chi[j];
            double nrm2;
            CoefList cl{};
            if (k > 0) {
                if ((rc = blas_mdot<V2>(w.red, n, k, prev, chk, a.data(), st))) return rc;
                for (int j = 0; j < k; ++j) {
                    cl.re[j] = a[j].real();
                    cl.im[j] = a[j].imag();
                }
            }
            if ((rc = blas_maxpy_norm<V2>(w.red, n, k, cl, prev, chk, &nrm2, st))) return rc;
            const double nrm = std::sqrt(nrm2);
            if (!std::isfinite(nrm)) return fail(QXD_ERR_NUMERIC, "qxd_solve: non-finite Krylov vector");
            if (nrm == 0.0) break;  // breakdown: the direction adds nothing
            if ((rc = blas_scale<V2>(n, 1.0 / nrm, chk, st))) return rc;
            for (int j = 0; j < k; ++j) Rm[j * BLAS_KMAX + k] = a[j];
            Rm[k * BLAS_KMAX + k] = cd(nrm, 0.0);
            // c_k = <chi_k, r>, r -= c_k chi_k
            VecList<V2> one{};
            one.p[0] = chk;
            cd ck;
            if ((rc = blas_mdot<V2>(w.red, n, 1, one, rin, &ck, st))) return rc;
            c[k] = ck;
            CoefList c1{};
            c1.re[0] = ck.real();
            c1.im[0] = ck.imag();
            double r2;
            if ((rc = blas_maxpy_norm<V2>(w.red, n, 1, c1, one, rin, &r2, st))) return rc;
            rin_n = std::sqrt(r2);
            ++k;
            ++info.iterations;
            if (!std::isfinite(rin_n)) return fail(QXD_ERR_NUMERIC, "qxd_solve: non-finite inner residual");
            if (rin_n <= 0.5 * target) break;
            if (P.delta > 0 && rin_n < P.delta * rn) break;
        }
        if (k == 0) return fail(QXD_ERR_NUMERIC, "qxd_solve: Krylov breakdown at a restart");
        // R beta = c (upper triangular), x += sum beta_j phi_j
        std::vector<cd> beta(k);
        for (int j = k - 1; j >= 0; --j) {
            cd s = c[j];
            for (int l = j + 1; l < k; ++l) s -= Rm[j * BLAS_KMAX + l] * beta[l];
            beta[j] = s / Rm[j * BLAS_KMAX + j];
        }
        CoefList bl{};
        VecList<V2> phis{};
        for (int j = 0; j < k; ++j) {
            bl.re[j] = beta[j].real();
            bl.im[j] = beta[j].imag();
            phis.p[j] = (const V2*)w.phi[j];
        }
        if (sizeof(R) == 4)
            rc = blas_update_x_native32(n / 12, k, bl, (const VecList<float2>&)phis, xs, st);
        else
            rc = blas_update_x<V2>(n, k, bl, phis, xs, st);
        if (rc) return rc;
        // reliable update: true residual in FP64
        if ((rc = apply_a64(lat, w, eo, ts, xs, st))) return rc;
        ++info.dw64_calls;
        if ((rc = blas_sub_norm(w.red, n, bs, ts, rs, &rn2, st))) return rc;
        rn = std::sqrt(rn2);
        ++info.restarts;
        w.last_true_rn = rn;
    }
    return QXD_OK;
}

}  // namespace

void release_solver(qxd_lattice* lat) {
    if (!lat->solver) return;
    lat->solver->release();
    delete lat->solver;
    lat->solver = nullptr;
}

int run_solve(qxd_lattice* lat, const qxd_solver_params& P, qxd_solve_info& info, cudaStream_t st) {
    SolverWork& w = *lat->solver;
    const bool eo = P.system == QXD_SOLVE_EO;
    const Geom& g = lat->g;
    const size_t nfull = (size_t)g.V * 12;
    int rc;
    double bn2;
    if ((rc = blas_norm2<double2>(w.red, nfull, (const double2*)w.b64, &bn2, st))) return rc;
    const double bn = std::sqrt(bn2);
    if (bn == 0.0) {
        QXD_CUDA(cudaMemsetAsync(w.x64, 0, nfull * sizeof(double2), st));
        info.true_relres = 0.0;
        return QXD_OK;
    }
    if (!std::isfinite(bn)) return fail(QXD_ERR_NUMERIC, "qxd_solve: non-finite source");
    // system right-hand side
    if (eo) {
        // b_hat_e = b_e - H_eo M_oo^-1 b_o
        const int Vh = g.Vh;
        if ((rc = launch_clover_half<double>(lat, 1, full_ref<double>(w.b64, g.V), half_out<double>(w.tmp64, Vh, 1),
                                             true, st)))
            return rc;
        if ((rc = launch_eo<double>(lat, EO_AUX_MHOP, 0, half_ref<double>(w.tmp64, Vh, 1),
                                    full_ref<double>(w.b64, g.V), half_out<double>(w.bs, Vh, 0), false, st)))
            return rc;
    } else {
        QXD_CUDA(cudaMemcpyAsync(w.bs, w.b64, nfull * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    }
    if (P.inner_prec == QXD_FP32) rc = fgcr<float>(lat, w, P, bn, info, st);
    else rc = fgcr<double>(lat, w, P, bn, info, st);
    if (rc) return rc;
    // solution on the full lattice
    if (eo) {
        const int Vh = g.Vh;
        if ((rc = copy_parity(lat, 0, half_ref<double>(w.xs, Vh, 0), full_out<double>(w.x64, g.V), st))) return rc;
        if ((rc = launch_eo<double>(lat, EO_INV_AUX_MHOP, 1, half_ref<double>(w.xs, Vh, 0),
                                    full_ref<double>(w.b64, g.V), full_out<double>(w.x64, g.V), true, st)))
            return rc;
    } else {
        QXD_CUDA(cudaMemcpyAsync(w.x64, w.xs, nfull * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    }
    // true residual of the full system; for the full system the solver's
    // last step computed exactly b - D x in FP64 already
    if (eo || info.restarts == 0) {
        if ((rc = launch_dirac(lat, w.t64, w.x64, QXD_FP64, st))) return rc;
        ++info.dw64_calls;
        double r2;
        if ((rc = blas_sub_norm(w.red, nfull, (const double2*)w.b64, (const double2*)w.t64, (double2*)w.r64, &r2,
                                st)))
            return rc;
        info.true_relres = std::sqrt(r2) / bn;
    } else {
        info.true_relres = w.last_true_rn / bn;
    }
    if (!std::isfinite(info.true_relres)) return fail(QXD_ERR_NUMERIC, "qxd_solve: non-finite final residual");
    if (info.true_relres > P.tol)
        return fail(QXD_ERR_NOT_CONVERGED, "qxd_solve: true relative residual " + std::to_string(info.true_relres) +
                                               " above tol after " + std::to_string(info.iterations) + " steps");
    return QXD_OK;
}

}  // namespace qxd

using namespace qxd;

extern "C" {

void qxd_solver_defaults(qxd_solver_params* p) {
    if (!p) return;
    p->tol = 1e-10;
    p->max_iter = 2000;
    p->nkv = 16;
    p->precond = QXD_PRECOND_NONE;
    p->system = QXD_SOLVE_FULL;
    p->inner_prec = QXD_FP64;
    p->sap_ncy = 5;
    p->sap_nmr = 5;
    p->delta = 1e-4;
    p->flags = QXD_DEVICE | QXD_LAYOUT_LEX;
    p->dfl_tol = 1e-2;
    p->dfl_max_iter = 64;
}

int qxd_solve(qxd_lattice* lat, void* x, const void* b, const qxd_solver_params* params, qxd_solve_info* info_out,
              void* stream) {
    auto t0 = std::chrono::steady_clock::now();
    qxd_solve_info info{};
    info.status = QXD_ERR_ARG;
    if (info_out) *info_out = info;
    if (!lat || !x || !b || !params) return fail(QXD_ERR_ARG, "qxd_solve: NULL argument");
    const qxd_solver_params& P = *params;
    if (!(P.tol > 0) || P.max_iter < 1 || P.nkv < 1 || P.nkv > BLAS_KMAX)
        return fail(QXD_ERR_ARG, "qxd_solve: tol > 0, max_iter >= 1 and 1 <= nkv <= 16 required");
    if ((P.precond != QXD_PRECOND_NONE && P.precond != QXD_PRECOND_SAP && P.precond != QXD_PRECOND_DFL_SAP) ||
        (P.system != QXD_SOLVE_FULL && P.system != QXD_SOLVE_EO) ||
        (P.inner_prec != QXD_FP32 && P.inner_prec != QXD_FP64) || (P.flags & ~(0x10 | 0x100)))
        return fail(QXD_ERR_ARG, "qxd_solve: bad precond/system/inner_prec/flags");
    if (P.precond != QXD_PRECOND_NONE && P.system != QXD_SOLVE_FULL)
        return fail(QXD_ERR_ARG, "qxd_solve: SAP preconditions the full system only");
    if (P.precond == QXD_PRECOND_DFL_SAP &&
        (P.inner_prec != QXD_FP32 || !(P.dfl_tol > 0) || P.dfl_max_iter < 1))
        return fail(QXD_ERR_ARG, "qxd_solve: deflation needs inner_prec FP32, dfl_tol > 0, dfl_max_iter >= 1");
    if (P.precond != QXD_PRECOND_NONE && (P.sap_ncy < 1 || P.sap_nmr < 1))
        return fail(QXD_ERR_ARG, "qxd_solve: sap_ncy and sap_nmr must be >= 1");
    if ((P.flags & QXD_HOST) && (P.flags & QXD_LAYOUT_NATIVE))
        return fail(QXD_ERR_ARG, "qxd_solve: host buffers must use the lexicographic layout");
    if (!qxd::clover_ready(lat)) return fail(QXD_ERR_STATE, "qxd_solve: needs qxd_sw_build first");
    cudaStream_t st = stream ? (cudaStream_t)stream : lat->stream;
    int rc;
    if (P.precond != QXD_PRECOND_NONE && (rc = sap_check(lat))) return rc;
    if (P.precond == QXD_PRECOND_DFL_SAP && !dfl_ready(lat))
        return fail(QXD_ERR_STATE, "qxd_solve: no deflation subspace for the current operator "
                                   "(qxd_dfl_subspace, or qxd_dfl_refresh after qxd_sw_build)");
    if (!lat->solver) lat->solver = new SolverWork();
    SolverWork& w = *lat->solver;
    if ((rc = w.ensure(lat->g.V, P.nkv, P.inner_prec))) return rc;
    if ((rc = ensure_scratch(lat))) return rc;
    const size_t bytes = (size_t)lat->g.V * 12 * sizeof(double2);
    // b -> native FP64
    if (P.flags & QXD_LAYOUT_NATIVE) {
        QXD_CUDA(cudaMemcpyAsync(w.b64, b, bytes, cudaMemcpyDeviceToDevice, st));
    } else {
        const void* src = b;
        if (P.flags & QXD_HOST) {
            QXD_CUDA(cudaMemcpyAsync(lat->scratch_lex, b, bytes, cudaMemcpyHostToDevice, st));
            src = lat->scratch_lex;
        }
        if ((rc = launch_pack(lat, w.b64, src, QXD_FP64, st))) return rc;
    }
    rc = run_solve(lat, P, info, st);
    info.status = rc;
    if (rc == QXD_OK || rc == QXD_ERR_NOT_CONVERGED) {
        int rc2 = QXD_OK;
        if (P.flags & QXD_LAYOUT_NATIVE) {
            if (cudaMemcpyAsync(x, w.x64, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) rc2 = QXD_ERR_CUDA;
        } else if (P.flags & QXD_HOST) {
            rc2 = launch_unpack(lat, lat->scratch_lex, w.x64, QXD_FP64, st);
            if (!rc2 && cudaMemcpyAsync(x, lat->scratch_lex, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
                rc2 = QXD_ERR_CUDA;
        } else {
            rc2 = launch_unpack(lat, x, w.x64, QXD_FP64, st);
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) rc2 = QXD_ERR_CUDA;
        if (rc2) {
            rc = rc2;
            info.status = rc;
        }
    }
    info.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info_out) *info_out = info;
    return rc;
}

}  // extern "C"
