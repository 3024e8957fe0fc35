// Pseudofermion action of the RHMC (Sec. 2.4):
//   S_pf = -1/2 ln|Det D_oo| + sum_k phi_k^dag P_k phi_k,
//   P_k  = prod_j (A + nu_j^2) / (A + mu_j^2),  A = D_hat^dag D_hat.
//
// * qxd_sw_logdet: ln|det| of the 12x12 site blocks M(x) of D summed over the
//   sites of one parity (D_oo is diagonal in the lattice index, so
//   ln|Det D_oo| is exact). One thread per (site, chirality block).
// * qxd_mscg: multi-shift CG for (A + sigma_j) x_j = b. A = Q^2 with
//   Q = gamma5 D_hat Hermitian (D_hat^dag = gamma5 D_hat gamma5), so one CG
//   step costs two applications of Q, i.e. four even-odd hopping kernels.
//   The shifted systems share the base system's Krylov space: their
//   residuals are r_j = zeta_j r, and with the base coefficients alpha_n,
//   beta_n the shifted ones follow from
//     zeta_{n+1} = zeta_n zeta_{n-1} alpha_{n-1} /
//                  [alpha_{n-1} zeta_{n-1} (1 + alpha_n s) + alpha_n beta_{n-1} (zeta_{n-1} - zeta_n)],
//     alpha_n^s = alpha_n zeta_{n+1} / zeta_n,  beta_n^s = beta_n (zeta_{n+1} / zeta_n)^2,
//   s = sigma_j - sigma_base (the three-term recurrence of the CG residuals
//   written for A + s and matched term by term). The base is the smallest
//   shift, the slowest to converge.
// * qxd_rational_apply: P phi = phi + sum_j rho_j (A + mu_j^2)^-1 phi
//   (partial fractions of P), one multi-shift CG for all poles.
//
// Vectors are even-site FP64 arrays in the native layout (12 components x
// V/2 sites, component-major), so the vector kernels see flat arrays of
// 12 V/2 complex numbers. Reductions use the fixed grid and order of the
// solver's vector kernels.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "blas.cuh"
#include "eo.cuh"
#include "rhmc.cuh"

namespace qxd {

namespace {

using C64 = cplx<double>;

// ---------------------------------------------------------------------------
// ln|det| of the clover blocks
// ---------------------------------------------------------------------------

// ln|det A| of a Hermitian 6x6 block given packed (real diagonal d, strictly
// lower part l row major), by Gaussian elimination with partial pivoting;
// -inf when a pivot column is exactly zero
__device__ double ln_abs_det6(const double d[6], const C64 l[15]) {
    C64 A[6][6];
    int k = 0;
    for (int i = 0; i < 6; ++i) {
        A[i][i] = mk(d[i], 0.0);
        for (int j = 0; j < i; ++j, ++k) {
            A[i][j] = l[k];
            A[j][i] = mk(l[k].re, -l[k].im);
        }
    }
    double acc = 0.0;
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        double best = A[c][c].re * A[c][c].re + A[c][c].im * A[c][c].im;
        for (int i = c + 1; i < 6; ++i) {
            const double m = A[i][c].re * A[i][c].re + A[i][c].im * A[i][c].im;
            if (m > best) {
                best = m;
                piv = i;
            }
        }
        if (!(best > 0.0)) return -INFINITY;
        if (piv != c)
            for (int j = c; j < 6; ++j) {
                C64 t = A[c][j];
                A[c][j] = A[piv][j];
                A[piv][j] = t;
            }
        acc += 0.5 * log(best);
        const double inv = 1.0 / best;
        // 1 / pivot = conj(pivot) / |pivot|^2
        const C64 ip = mk(A[c][c].re * inv, -A[c][c].im * inv);
        for (int i = c + 1; i < 6; ++i) {
            const C64 f = A[i][c] * ip;
            for (int j = c + 1; j < 6; ++j) A[i][j] = A[i][j] - f * A[c][j];
        }
    }
    return acc;
}

// sum over the selected sites and both chirality blocks; fixed grid
__global__ void __launch_bounds__(RED_THREADS) k_sw_logdet(int V, int first, int count,
                                                          const double* __restrict__ C,
                                                          double* __restrict__ partials) {
    double acc[2] = {0.0, 0.0};  // sum, number of non-finite blocks
    const size_t n = (size_t)count * 2;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int s = first + (int)(i >> 1);
        const int blk = (int)(i & 1);
        double d[6];
        C64 l[15];
#pragma unroll
        for (int r = 0; r < 6; ++r) d[r] = C[(size_t)(36 * blk + r) * V + s];
#pragma unroll
        for (int q = 0; q < 15; ++q)
            l[q] = mk(C[(size_t)(36 * blk + 6 + 2 * q) * V + s], C[(size_t)(36 * blk + 7 + 2 * q) * V + s]);
        const double v = ln_abs_det6(d, l);
        if (isfinite(v)) acc[0] += v;
        else acc[1] += 1.0;
    }
    block_reduce_store<2>(acc, 2, partials);
}

// ---------------------------------------------------------------------------
// vector kernels of the multi-shift CG (flat arrays of n complex numbers)
// ---------------------------------------------------------------------------

// r -= alpha (w + sigma0 p); returns |r|^2
__global__ void __launch_bounds__(RED_THREADS) k_ms_residual(size_t n, double alpha, double sigma0,
                                                            const double2* __restrict__ w,
                                                            const double2* __restrict__ p, double2* __restrict__ r,
                                                            double* __restrict__ partials) {
    double acc[1] = {0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 a = w[i], b = p[i];
        double2 v = r[i];
        v.x -= alpha * (a.x + sigma0 * b.x);
        v.y -= alpha * (a.y + sigma0 * b.y);
        r[i] = v;
        acc[0] += v.x * v.x + v.y * v.y;
    }
    block_reduce_store<1>(acc, 1, partials);
}

struct ShiftUpdate {
    int k;                   // shifts updated
    int base;                // entry whose |p|^2 is returned (-1: none)
    double a[BLAS_KMAX];     // x_j += a_j p_j
    double z[BLAS_KMAX];     // p_j = z_j r + b_j p_j
    double b[BLAS_KMAX];
    double2* x[BLAS_KMAX];
    double2* p[BLAS_KMAX];
};

// for every listed shift: x_j += a_j p_j, then p_j = z_j r + b_j p_j;
// returns |p_base|^2 (the new base direction)
__global__ void __launch_bounds__(RED_THREADS) k_ms_xp(size_t n, ShiftUpdate u, const double2* __restrict__ r,
                                                      double* __restrict__ partials) {
    double acc[1] = {0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 rv = r[i];
#pragma unroll
        for (int j = 0; j < BLAS_KMAX; ++j) {
            if (j >= u.k) break;
            double2 pv = u.p[j][i];
            double2 xv = u.x[j][i];
            xv.x += u.a[j] * pv.x;
            xv.y += u.a[j] * pv.y;
            u.x[j][i] = xv;
            pv.x = u.z[j] * rv.x + u.b[j] * pv.x;
            pv.y = u.z[j] * rv.y + u.b[j] * pv.y;
            u.p[j][i] = pv;
            if (j == u.base) acc[0] += pv.x * pv.x + pv.y * pv.y;
        }
    }
    block_reduce_store<1>(acc, 1, partials);
}

// |b - w - sigma x|^2 (true residual of one shift; nothing written)
__global__ void __launch_bounds__(RED_THREADS) k_ms_true_res(size_t n, double sigma, const double2* __restrict__ b,
                                                            const double2* __restrict__ w,
                                                            const double2* __restrict__ x,
                                                            double* __restrict__ partials) {
    double acc[1] = {0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 bv = b[i], wv = w[i], xv = x[i];
        const double re = bv.x - wv.x - sigma * xv.x;
        const double im = bv.y - wv.y - sigma * xv.y;
        acc[0] += re * re + im * im;
    }
    block_reduce_store<1>(acc, 1, partials);
}

// FP32 native half-lattice layout: component k of site s at float2 index
// ((k / 2) * S + s) * 2 + k % 2 (two components per float4)
__device__ __forceinline__ size_t f32_half_index(size_t S, size_t i) {
    const size_t k = i / S, s = i - k * S;
    return ((k >> 1) * S + s) * 2 + (k & 1);
}

// r -= alpha (w32 + sigma0 p), w32 in the FP32 native layout; returns |r|^2
__global__ void __launch_bounds__(RED_THREADS) k_ms_residual32(size_t n, size_t S, double alpha, double sigma0,
                                                              const float2* __restrict__ w,
                                                              const double2* __restrict__ p,
                                                              double2* __restrict__ r,
                                                              double* __restrict__ partials) {
    double acc[1] = {0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 a = w[f32_half_index(S, i)];
        const double2 b = p[i];
        double2 v = r[i];
        v.x -= alpha * ((double)a.x + sigma0 * b.x);
        v.y -= alpha * ((double)a.y + sigma0 * b.y);
        r[i] = v;
        acc[0] += v.x * v.x + v.y * v.y;
    }
    block_reduce_store<1>(acc, 1, partials);
}

// r = b - w - sigma x (FP64), returns |r|^2
__global__ void __launch_bounds__(RED_THREADS) k_ms_true_res_store(size_t n, double sigma,
                                                                  const double2* __restrict__ b,
                                                                  const double2* __restrict__ w,
                                                                  const double2* __restrict__ x,
                                                                  double2* __restrict__ r,
                                                                  double* __restrict__ partials) {
    double acc[1] = {0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 bv = b[i], wv = w[i], xv = x[i];
        const double re = bv.x - wv.x - sigma * xv.x;
        const double im = bv.y - wv.y - sigma * xv.y;
        r[i] = make_double2(re, im);
        acc[0] += re * re + im * im;
    }
    block_reduce_store<1>(acc, 1, partials);
}

// x += a p (FP64)
__global__ void k_ms_axpy(size_t n, double a, const double2* __restrict__ p, double2* __restrict__ x) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double2 v = x[i];
        const double2 q = p[i];
        v.x += a * q.x;
        v.y += a * q.y;
        x[i] = v;
    }
}

struct Combine {
    int k;
    double rho[BLAS_KMAX];
    const double2* x[BLAS_KMAX];
};

// out = phi + sum_j rho_j x_j; returns Re <phi, out>
__global__ void __launch_bounds__(RED_THREADS) k_rat_combine(size_t n, Combine c, const double2* __restrict__ phi,
                                                            double2* __restrict__ out,
                                                            double* __restrict__ partials) {
    double acc[1] = {0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 f = phi[i];
        double2 v = f;
#pragma unroll
        for (int j = 0; j < BLAS_KMAX; ++j) {
            if (j >= c.k) break;
            const double2 xv = c.x[j][i];
            v.x += c.rho[j] * xv.x;
            v.y += c.rho[j] * xv.y;
        }
        out[i] = v;
        acc[0] += f.x * v.x + f.y * v.y;
    }
    block_reduce_store<1>(acc, 1, partials);
}

// even sites of a full native FP64 field <-> an even-site array; the odd
// sites of the full field are set to zero
__global__ void k_even_from_full(int V, int Vh, const double2* __restrict__ full, double2* __restrict__ half) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)12 * Vh) return;
    const size_t k = i / Vh, s = i % Vh;
    half[i] = full[k * V + s];
}
__global__ void k_full_from_even(int V, int Vh, const double2* __restrict__ half, double2* __restrict__ full) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)12 * V) return;
    const size_t k = i / V, s = i % V;
    full[i] = s < (size_t)Vh ? half[k * Vh + s] : make_double2(0.0, 0.0);
}

int dev_alloc(double2** p, size_t bytes) {
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMalloc(multi-shift CG work)");
    }
    return QXD_OK;
}

}  // namespace

void MscgWork::release() {
    double2** ps[] = {&b, &r, &t, &w, &tmp_o, &full, &out, &e, &src2};
    float4** fs[] = {&p32, &t32, &w32, &tmp32};
    for (float4** p : fs)
        if (*p) {
            cudaFree(*p);
            *p = nullptr;
        }
    for (double2** p : ps)
        if (*p) {
            cudaFree(*p);
            *p = nullptr;
        }
    for (int j = 0; j < BLAS_KMAX; ++j) {
        if (x[j]) cudaFree(x[j]);
        if (p[j]) cudaFree(p[j]);
        x[j] = p[j] = nullptr;
    }
    red.release();
    Vh = 0;
    nshift = 0;
}

int MscgWork::ensure(int V_, int Vh_, int nshift_) {
    if (Vh == Vh_ && nshift >= nshift_) return QXD_OK;
    const size_t hb = (size_t)12 * Vh_ * sizeof(double2);
    int rc;
    if (Vh != Vh_) {
        release();
        double2** ps[] = {&b, &r, &t, &w, &tmp_o, &out, &e, &src2};
        for (double2** p : ps)
            if ((rc = dev_alloc(p, hb))) return rc;
        float4** fs[] = {&p32, &t32, &w32, &tmp32};
        for (float4** p : fs)
            if ((rc = dev_alloc((double2**)p, hb / 2))) return rc;
        if ((rc = dev_alloc(&full, (size_t)12 * V_ * sizeof(double2)))) return rc;
        if ((rc = red.init())) return rc;
        Vh = Vh_;
    }
    for (int j = nshift; j < nshift_; ++j)
        if ((rc = dev_alloc(&x[j], hb)) || (rc = dev_alloc(&p[j], hb))) return rc;
    nshift = nshift_;
    return QXD_OK;
}

void release_mscg(qxd_lattice* lat) {
    if (!lat->mscg) return;
    lat->mscg->release();
    delete lat->mscg;
    lat->mscg = nullptr;
}

namespace {

// out = Q in = gamma5 D_hat in (even-site arrays)
int apply_q(qxd_lattice* lat, MscgWork& W, double2* out, const double2* in, cudaStream_t st) {
    const int Vh = lat->g.Vh;
    return apply_g5dhat<double>(lat, half_out<double>(out, Vh, 0), half_ref<double>(in, Vh, 0),
                                half_out<double>(W.tmp_o, Vh, 1), st);
}

// W.w = A in = Q (Q in), W.t = Q in
int apply_normal(qxd_lattice* lat, MscgWork& W, const double2* in, cudaStream_t st) {
    int rc = apply_q(lat, W, W.t, in, st);
    if (rc) return rc;
    return apply_q(lat, W, W.w, W.t, st);
}

template <typename K, typename... Args>
int reduce_launch(MscgWork& W, K kernel, int nc, double* out, cudaStream_t st, Args... args) {
    kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(args..., W.red.partials);
    QXD_LAUNCHED("multi-shift CG vector kernel");
    int rc = reduce_finish(W.red, nc, st);
    if (rc) return rc;
    for (int c = 0; c < nc; ++c) out[c] = W.red.h_res[c];
    return QXD_OK;
}

}  // namespace

// Multi-shift CG on the even-site arrays: W.b holds b; x_j land in W.x[j].
int mscg_core(qxd_lattice* lat, MscgWork& W, int ns, const double* sigma, double tol, int max_iter,
              qxd_mscg_info& info, double* relres, cudaStream_t st) {
    const size_t n = (size_t)12 * lat->g.Vh;
    const size_t hb = n * sizeof(double2);
    int base = 0;
    for (int j = 1; j < ns; ++j)
        if (sigma[j] < sigma[base]) base = j;
    const double s0 = sigma[base];
    int rc;
    double bb;
    if ((rc = blas_norm2<double2>(W.red, n, W.b, &bb, st))) return rc;
    for (int j = 0; j < ns; ++j) QXD_CUDA(cudaMemsetAsync(W.x[j], 0, hb, st));
    if (relres)
        for (int j = 0; j < ns; ++j) relres[j] = 0.0;
    info.true_relres = 0.0;
    if (bb == 0.0) return QXD_OK;
    if (!std::isfinite(bb)) return fail(QXD_ERR_NUMERIC, "qxd_mscg: non-finite source");
    const double bn = std::sqrt(bb);
    QXD_CUDA(cudaMemcpyAsync(W.r, W.b, hb, cudaMemcpyDeviceToDevice, st));
    for (int j = 0; j < ns; ++j) QXD_CUDA(cudaMemcpyAsync(W.p[j], W.b, hb, cudaMemcpyDeviceToDevice, st));

    std::vector<double> zeta(ns, 1.0), zeta_prev(ns, 1.0), zeta_new(ns, 1.0);
    std::vector<char> active(ns, 1);
    double rr = bb, pp = bb, alpha_prev = 1.0, beta_prev = 0.0;
    int it = 0;
    bool converged = false;
    while (it < max_iter) {
        // w = A p_base, t = Q p_base; <p, A p> = |Q p|^2
        if ((rc = apply_normal(lat, W, W.p[base], st))) return rc;
        info.dhat_calls += 2;
        double tt;
        if ((rc = blas_norm2<double2>(W.red, n, W.t, &tt, st))) return rc;
        const double alpha = rr / (tt + s0 * pp);
        if (!std::isfinite(alpha) || !(alpha > 0.0))
            return fail(QXD_ERR_NUMERIC, "qxd_mscg: breakdown (non-finite or non-positive step)");
        double rr_new;
        if ((rc = reduce_launch(W, k_ms_residual, 1, &rr_new, st, n, alpha, s0, (const double2*)W.w,
                                (const double2*)W.p[base], W.r)))
            return rc;
        const double beta = rr_new / rr;
        ShiftUpdate u{};
        u.base = -1;
        for (int j = 0; j < ns; ++j) {
            if (!active[j]) continue;
            double a, z, b;
            if (j == base) {
                a = alpha;
                z = 1.0;
                b = beta;
                zeta_new[j] = 1.0;
                u.base = u.k;
            } else {
                const double ds = sigma[j] - s0;
                const double den = alpha_prev * zeta_prev[j] * (1.0 + alpha * ds) +
                                   alpha * beta_prev * (zeta_prev[j] - zeta[j]);
                zeta_new[j] = zeta[j] * zeta_prev[j] * alpha_prev / den;
                const double q = zeta_new[j] / zeta[j];
                a = alpha * q;
                z = zeta_new[j];
                b = beta * q * q;
            }
            u.a[u.k] = a;
            u.z[u.k] = z;
            u.b[u.k] = b;
            u.x[u.k] = W.x[j];
            u.p[u.k] = W.p[j];
            ++u.k;
        }
        double pp_new = 0.0;
        if ((rc = reduce_launch(W, k_ms_xp, 1, &pp_new, st, n, u, (const double2*)W.r))) return rc;
        ++it;
        for (int j = 0; j < ns; ++j) {
            if (!active[j]) continue;
            zeta_prev[j] = zeta[j];
            zeta[j] = zeta_new[j];
            if (std::fabs(zeta[j]) * std::sqrt(rr_new) <= tol * bn) active[j] = 0;
        }
        alpha_prev = alpha;
        beta_prev = beta;
        rr = rr_new;
        pp = pp_new;
        if (!active[base]) {
            converged = true;
            break;
        }
    }
    info.iterations = it;
    // true residuals |b - (A + sigma_j) x_j| in FP64
    double worst = 0.0;
    for (int j = 0; j < ns; ++j) {
        if ((rc = apply_normal(lat, W, W.x[j], st))) return rc;
        info.dhat_calls += 2;
        double r2;
        if ((rc = reduce_launch(W, k_ms_true_res, 1, &r2, st, n, sigma[j], (const double2*)W.b,
                                (const double2*)W.w, (const double2*)W.x[j])))
            return rc;
        const double rel = std::sqrt(r2) / bn;
        if (relres) relres[j] = rel;
        if (!std::isfinite(rel)) return fail(QXD_ERR_NUMERIC, "qxd_mscg: non-finite true residual");
        worst = std::max(worst, rel);
    }
    info.true_relres = worst;
    if (!converged || worst > tol)
        return fail(QXD_ERR_NOT_CONVERGED, "qxd_mscg: largest true relative residual " + std::to_string(worst) +
                                               " (tol " + std::to_string(tol) + ") after " + std::to_string(it) +
                                               " steps");
    return QXD_OK;
}

namespace {

// Q32 in = gamma5 D_hat in with the FP32 operator (even-site FP32 arrays)
int apply_q32(qxd_lattice* lat, MscgWork& W, float4* out, const float4* in, cudaStream_t st) {
    const int Vh = lat->g.Vh;
    return apply_g5dhat<float>(lat, half_out<float>(out, Vh, 0), half_ref<float>(in, Vh, 0),
                               half_out<float>(W.tmp32, Vh, 1), st);
}

// Multi-shift CG with the FP32 operator: the Krylov vectors, x_j and all
// scalars are FP64; the base residual is replaced by the true FP64 residual
// src - (A + s0) x_base whenever it has fallen by delta since the last
// replacement, and before the run ends. Solves (A + sigma_j) x_j = src into
// x[j] until every shift's iterated residual is below target (absolute).
// *true_rr: |src - (A + s0) x_base|^2 from the last reliable update when the
// run ended converged (that update is the last step), else -1.
int run_mixed(qxd_lattice* lat, MscgWork& W, const double2* src, double ss, int ns, const double* sigma,
              double2* const* x, double target, double delta, int max_iter, int* iters, double* true_rr,
              qxd_mscg_info& info, cudaStream_t st) {
    const size_t Vh = (size_t)lat->g.Vh;
    const size_t n = 12 * Vh;
    const size_t hb = n * sizeof(double2);
    int base = 0;
    for (int j = 1; j < ns; ++j)
        if (sigma[j] < sigma[base]) base = j;
    const double s0 = sigma[base];
    int rc;
    for (int j = 0; j < ns; ++j) QXD_CUDA(cudaMemsetAsync(x[j], 0, hb, st));
    *iters = 0;
    *true_rr = -1.0;
    if (ss == 0.0) {
        *true_rr = 0.0;
        return QXD_OK;
    }
    QXD_CUDA(cudaMemcpyAsync(W.r, src, hb, cudaMemcpyDeviceToDevice, st));
    for (int j = 0; j < ns; ++j) QXD_CUDA(cudaMemcpyAsync(W.p[j], src, hb, cudaMemcpyDeviceToDevice, st));
    std::vector<double> zeta(ns, 1.0), zeta_prev(ns, 1.0), zeta_new(ns, 1.0);
    std::vector<char> active(ns, 1);
    double rr = ss, pp = ss, alpha_prev = 1.0, beta_prev = 0.0, rr_max = ss;
    int it = 0;
    const unsigned ew = (unsigned)std::min<size_t>((n + 255) / 256, 4 * 152 * 4);
    while (it < max_iter) {
        if ((rc = blas_d2f_native(Vh, W.p[base], (float2*)W.p32, st))) return rc;
        if ((rc = apply_q32(lat, W, W.t32, W.p32, st)) || (rc = apply_q32(lat, W, W.w32, W.t32, st))) return rc;
        info.dhat_calls += 2;
        double tt;
        if ((rc = blas_norm2<float2>(W.red, n, (const float2*)W.t32, &tt, st))) return rc;
        const double alpha = rr / (tt + s0 * pp);
        if (!std::isfinite(alpha) || !(alpha > 0.0))
            return fail(QXD_ERR_NUMERIC, "qxd_mscg: breakdown (non-finite or non-positive step)");
        double rr_new;
        if ((rc = reduce_launch(W, k_ms_residual32, 1, &rr_new, st, n, Vh, alpha, s0, (const float2*)W.w32,
                                (const double2*)W.p[base], W.r)))
            return rc;
        // reliable update of the base residual
        const bool base_done = std::sqrt(rr_new) <= target;
        const bool reliable = rr_new < delta * delta * rr_max || base_done;
        if (reliable) {
            k_ms_axpy<<<ew, 256, 0, st>>>(n, alpha, W.p[base], x[base]);
            QXD_LAUNCHED("k_ms_axpy");
            if ((rc = apply_normal(lat, W, x[base], st))) return rc;
            info.dhat_calls += 2;
            if ((rc = reduce_launch(W, k_ms_true_res_store, 1, &rr_new, st, n, s0, src, (const double2*)W.w,
                                    (const double2*)x[base], W.r)))
                return rc;
            rr_max = rr_new;
        }
        const double beta = rr_new / rr;
        ShiftUpdate u{};
        u.base = -1;
        for (int j = 0; j < ns; ++j) {
            if (!active[j]) continue;
            double a, z, b;
            if (j == base) {
                a = reliable ? 0.0 : alpha;  // already added on a reliable update
                z = 1.0;
                b = beta;
                zeta_new[j] = 1.0;
                u.base = u.k;
            } else {
                const double ds = sigma[j] - s0;
                const double den = alpha_prev * zeta_prev[j] * (1.0 + alpha * ds) +
                                   alpha * beta_prev * (zeta_prev[j] - zeta[j]);
                zeta_new[j] = zeta[j] * zeta_prev[j] * alpha_prev / den;
                const double q = zeta_new[j] / zeta[j];
                a = alpha * q;
                z = zeta_new[j];
                b = beta * q * q;
            }
            u.a[u.k] = a;
            u.z[u.k] = z;
            u.b[u.k] = b;
            u.x[u.k] = x[j];
            u.p[u.k] = W.p[j];
            ++u.k;
        }
        double pp_new = 0.0;
        if ((rc = reduce_launch(W, k_ms_xp, 1, &pp_new, st, n, u, (const double2*)W.r))) return rc;
        ++it;
        for (int j = 0; j < ns; ++j) {
            if (!active[j]) continue;
            zeta_prev[j] = zeta[j];
            zeta[j] = zeta_new[j];
            if (j != base && std::fabs(zeta[j]) * std::sqrt(rr_new) <= target) active[j] = 0;
        }
        alpha_prev = alpha;
        beta_prev = beta;
        rr = rr_new;
        pp = pp_new;
        if (reliable && std::sqrt(rr) <= target) {  // the true base residual (just replaced)
            *true_rr = rr;
            break;
        }
    }
    *iters = it;
    return QXD_OK;
}

// FP32-operator multi-shift CG, then every shift checked in FP64 and
// refined by FP32-operator CG on its own residual until it meets tol
int mscg_mixed(qxd_lattice* lat, MscgWork& W, int ns, const double* sigma, double tol, double delta,
               int max_iter, qxd_mscg_info& info, double* relres, cudaStream_t st) {
    const size_t n = (size_t)12 * lat->g.Vh;
    const unsigned ew = (unsigned)std::min<size_t>((n + 255) / 256, 4 * 152 * 4);
    int rc;
    double bb;
    if ((rc = blas_norm2<double2>(W.red, n, W.b, &bb, st))) return rc;
    if (relres)
        for (int j = 0; j < ns; ++j) relres[j] = 0.0;
    info.true_relres = 0.0;
    if (bb == 0.0) {
        for (int j = 0; j < ns; ++j) QXD_CUDA(cudaMemsetAsync(W.x[j], 0, n * sizeof(double2), st));
        return QXD_OK;
    }
    if (!std::isfinite(bb)) return fail(QXD_ERR_NUMERIC, "qxd_mscg: non-finite source");
    const double bn = std::sqrt(bb);
    int it = 0;
    double rr_fin;
    if ((rc = run_mixed(lat, W, W.b, bb, ns, sigma, W.x, tol * bn, delta, max_iter, &it, &rr_fin, info, st)))
        return rc;
    int total = it;
    double worst = 0.0;
    bool ok = true;
    for (int j = 0; j < ns; ++j) {
        double rel = 0.0;
        double r2 = -1.0;  // true |b - (A + sigma_j) x_j|^2 when known
        for (int pass = 0;; ++pass) {
            if (r2 < 0.0) {
                if ((rc = apply_normal(lat, W, W.x[j], st))) return rc;
                info.dhat_calls += 2;
                if ((rc = reduce_launch(W, k_ms_true_res_store, 1, &r2, st, n, sigma[j], (const double2*)W.b,
                                        (const double2*)W.w, (const double2*)W.x[j], W.src2)))
                    return rc;
            }
            rel = std::sqrt(r2) / bn;
            if (!std::isfinite(rel)) return fail(QXD_ERR_NUMERIC, "qxd_mscg: non-finite true residual");
            if (rel <= tol || pass == 4 || total >= max_iter) break;
            // x_j += e, (A + sigma_j) e = r_j to half the target; the refinement
            // ends with the true residual of its system, which is the new
            // residual r_j - (A + sigma_j) e of x_j
            double2* xe[1] = {W.e};
            int it2 = 0;
            double rr_e;
            if ((rc = run_mixed(lat, W, W.src2, r2, 1, &sigma[j], xe, 0.5 * tol * bn, delta, max_iter - total,
                                &it2, &rr_e, info, st)))
                return rc;
            total += it2;
            k_ms_axpy<<<ew, 256, 0, st>>>(n, 1.0, W.e, W.x[j]);
            QXD_LAUNCHED("k_ms_axpy");
            r2 = rr_e;  // -1 (recompute) unless the refinement converged
        }
        if (relres) relres[j] = rel;
        worst = std::max(worst, rel);
        if (rel > tol) ok = false;
    }
    info.iterations = total;
    info.true_relres = worst;
    if (!ok)
        return fail(QXD_ERR_NOT_CONVERGED, "qxd_mscg: largest true relative residual " + std::to_string(worst) +
                                               " (tol " + std::to_string(tol) + ") after " + std::to_string(total) +
                                               " steps");
    return QXD_OK;
}

int solve_shifts(qxd_lattice* lat, MscgWork& W, int ns, const double* sigma, const qxd_mscg_params& P,
                 qxd_mscg_info& info, double* relres, cudaStream_t st) {
    if (P.prec == QXD_FP32) return mscg_mixed(lat, W, ns, sigma, P.tol, P.delta, P.max_iter, info, relres, st);
    return mscg_core(lat, W, ns, sigma, P.tol, P.max_iter, info, relres, st);
}

int check_params(const qxd_mscg_params* P, const char* name) {
    if (!P) return fail(QXD_ERR_ARG, std::string(name) + ": NULL params");
    if (!(P->tol > 0) || P->max_iter < 1) return fail(QXD_ERR_ARG, std::string(name) + ": tol > 0, max_iter >= 1");
    if (P->prec != QXD_FP64 && P->prec != QXD_FP32)
        return fail(QXD_ERR_ARG, std::string(name) + ": prec must be QXD_FP64 or QXD_FP32");
    if (P->prec == QXD_FP32 && !(P->delta > 0.0 && P->delta < 1.0))
        return fail(QXD_ERR_ARG, std::string(name) + ": 0 < delta < 1 required with QXD_FP32");
    if (P->flags & ~(QXD_HOST | QXD_LAYOUT_NATIVE))
        return fail(QXD_ERR_ARG, std::string(name) + ": flags: QXD_HOST, QXD_LAYOUT_NATIVE only (FP64 fields)");
    if ((P->flags & QXD_HOST) && (P->flags & QXD_LAYOUT_NATIVE))
        return fail(QXD_ERR_ARG, std::string(name) + ": host buffers must use the lexicographic layout");
    return QXD_OK;
}

int prepare(qxd_lattice* lat, int nshift, const char* name) {
    if (!qxd::clover_ready(lat)) return fail(QXD_ERR_STATE, std::string(name) + ": needs qxd_sw_build first");
    int rc;
    if ((rc = ensure_scratch(lat))) return rc;
    if (!lat->mscg) lat->mscg = new MscgWork();
    return lat->mscg->ensure(lat->g.V, lat->g.Vh, nshift);
}

// caller's full-lattice field -> W.b (even sites, native FP64)
int load_source(qxd_lattice* lat, MscgWork& W, const void* b, int flags, cudaStream_t st) {
    const Geom& g = lat->g;
    const size_t fb = (size_t)12 * g.V * sizeof(double2);
    const double2* nat = (const double2*)b;
    int rc;
    if (!(flags & QXD_LAYOUT_NATIVE)) {
        const void* src = b;
        if (flags & QXD_HOST) {
            QXD_CUDA(cudaMemcpyAsync(lat->scratch_lex, b, fb, cudaMemcpyHostToDevice, st));
            src = lat->scratch_lex;
        }
        if ((rc = launch_pack(lat, W.full, src, QXD_FP64, st))) return rc;
        nat = W.full;
    }
    const size_t n = (size_t)12 * g.Vh;
    k_even_from_full<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g.V, g.Vh, nat, W.b);
    QXD_LAUNCHED("k_even_from_full");
    return QXD_OK;
}

// even-site array -> caller's full-lattice field (odd sites zero)
int store_field(qxd_lattice* lat, MscgWork& W, void* x, const double2* half, int flags, cudaStream_t st) {
    const Geom& g = lat->g;
    const size_t fb = (size_t)12 * g.V * sizeof(double2);
    const size_t n = (size_t)12 * g.V;
    double2* nat = (flags & QXD_LAYOUT_NATIVE) ? (double2*)x : W.full;
    k_full_from_even<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g.V, g.Vh, half, nat);
    QXD_LAUNCHED("k_full_from_even");
    if (flags & QXD_LAYOUT_NATIVE) return QXD_OK;
    int rc;
    if (flags & QXD_HOST) {
        if ((rc = launch_unpack(lat, lat->scratch_lex, W.full, QXD_FP64, st))) return rc;
        QXD_CUDA(cudaMemcpyAsync(x, lat->scratch_lex, fb, cudaMemcpyDeviceToHost, st));
        return QXD_OK;
    }
    return launch_unpack(lat, x, W.full, QXD_FP64, st);
}

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

}  // namespace qxd

using namespace qxd;

extern "C" {

int qxd_sw_logdet(qxd_lattice* lat, int sites, double* out) {
    if (!lat || !out) return fail(QXD_ERR_ARG, "qxd_sw_logdet: NULL argument");
    if (sites != QXD_SITES_EVEN && sites != QXD_SITES_ODD && sites != QXD_SITES_ALL)
        return fail(QXD_ERR_ARG, "qxd_sw_logdet: sites must be QXD_SITES_EVEN, _ODD or _ALL");
    if (!qxd::clover_ready(lat)) return fail(QXD_ERR_STATE, "qxd_sw_logdet: needs qxd_sw_build first");
    const Geom& g = lat->g;
    const int first = sites == QXD_SITES_ODD ? g.Vh : 0;
    const int count = sites == QXD_SITES_ALL ? g.V : g.Vh;
    if (!lat->mscg) lat->mscg = new MscgWork();
    int rc;
    if ((rc = lat->mscg->red.init())) return rc;
    cudaStream_t st = lat->stream;
    k_sw_logdet<<<RED_BLOCKS, RED_THREADS, 0, st>>>(g.V, first, count, lat->C64, lat->mscg->red.partials);
    QXD_LAUNCHED("k_sw_logdet");
    if ((rc = reduce_finish(lat->mscg->red, 2, st))) return rc;
    const double v = lat->mscg->red.h_res[0], bad = lat->mscg->red.h_res[1];
    if (bad > 0.0 || !std::isfinite(v))
        return fail(QXD_ERR_SW_SINGULAR, "qxd_sw_logdet: " + std::to_string((long long)bad) +
                                             " singular or non-finite site blocks");
    *out = v;
    return QXD_OK;
}

void qxd_mscg_defaults(qxd_mscg_params* p) {
    if (!p) return;
    p->tol = 1e-10;
    p->max_iter = 10000;
    p->flags = QXD_DEVICE | QXD_LAYOUT_LEX;
    p->prec = QXD_FP64;
    p->delta = 0.01;
}

int qxd_mscg(qxd_lattice* lat, int nshift, const double* sigma, void* const* x, const void* b,
             const qxd_mscg_params* params, qxd_mscg_info* info_out, double* relres, void* stream) {
    const auto t0 = std::chrono::steady_clock::now();
    qxd_mscg_info info{};
    info.status = QXD_ERR_ARG;
    if (info_out) *info_out = info;
    if (!lat || !sigma || !x || !b) return fail(QXD_ERR_ARG, "qxd_mscg: NULL argument");
    if (nshift < 1 || nshift > BLAS_KMAX) return fail(QXD_ERR_ARG, "qxd_mscg: 1 <= nshift <= 16");
    for (int j = 0; j < nshift; ++j) {
        if (!x[j]) return fail(QXD_ERR_ARG, "qxd_mscg: NULL solution buffer");
        if (!(sigma[j] >= 0.0) || !std::isfinite(sigma[j]))
            return fail(QXD_ERR_ARG, "qxd_mscg: shifts must be finite and >= 0");
    }
    int rc;
    if ((rc = check_params(params, "qxd_mscg"))) return rc;
    if ((rc = prepare(lat, nshift, "qxd_mscg"))) return rc;
    cudaStream_t st = stream ? (cudaStream_t)stream : lat->stream;
    MscgWork& W = *lat->mscg;
    if ((rc = load_source(lat, W, b, params->flags, st))) return rc;
    rc = solve_shifts(lat, W, nshift, sigma, *params, info, relres, st);
    if (rc == QXD_OK || rc == QXD_ERR_NOT_CONVERGED) {
        int rc2 = QXD_OK;
        for (int j = 0; j < nshift && !rc2; ++j) rc2 = store_field(lat, W, x[j], W.x[j], params->flags, st);
        if (!rc2 && cudaStreamSynchronize(st) != cudaSuccess) rc2 = fail(QXD_ERR_CUDA, "qxd_mscg: stream sync");
        if (rc2) rc = rc2;
    }
    info.status = rc;
    info.time_ms = ms_since(t0);
    if (info_out) *info_out = info;
    return rc;
}

int qxd_rational_apply(qxd_lattice* lat, int n, const double* nu, const double* mu, void* out, const void* phi,
                       const qxd_mscg_params* params, qxd_mscg_info* info_out, void* stream) {
    const auto t0 = std::chrono::steady_clock::now();
    qxd_mscg_info info{};
    info.status = QXD_ERR_ARG;
    if (info_out) *info_out = info;
    if (!lat || !nu || !mu || !out || !phi) return fail(QXD_ERR_ARG, "qxd_rational_apply: NULL argument");
    if (n < 1 || n > BLAS_KMAX) return fail(QXD_ERR_ARG, "qxd_rational_apply: 1 <= n <= 16");
    std::vector<double> s(n), rho(n);
    for (int j = 0; j < n; ++j) {
        if (!std::isfinite(nu[j]) || !std::isfinite(mu[j]))
            return fail(QXD_ERR_ARG, "qxd_rational_apply: non-finite nu or mu");
        s[j] = mu[j] * mu[j];
    }
    // residues of prod_l (lambda + nu_l^2) / (lambda + mu_l^2) at lambda = -mu_j^2
    for (int j = 0; j < n; ++j) {
        double num = 1.0, den = 1.0;
        for (int l = 0; l < n; ++l) {
            num *= nu[l] * nu[l] - s[j];
            if (l != j) den *= s[l] - s[j];
        }
        if (den == 0.0) return fail(QXD_ERR_ARG, "qxd_rational_apply: the poles mu_j must be distinct");
        rho[j] = num / den;
    }
    int rc;
    if ((rc = check_params(params, "qxd_rational_apply"))) return rc;
    if ((rc = prepare(lat, n, "qxd_rational_apply"))) return rc;
    cudaStream_t st = stream ? (cudaStream_t)stream : lat->stream;
    MscgWork& W = *lat->mscg;
    if ((rc = load_source(lat, W, phi, params->flags, st))) return rc;
    rc = solve_shifts(lat, W, n, s.data(), *params, info, nullptr, st);
    if (rc == QXD_OK || rc == QXD_ERR_NOT_CONVERGED) {
        Combine c{};
        c.k = n;
        for (int j = 0; j < n; ++j) {
            c.rho[j] = rho[j];
            c.x[j] = W.x[j];
        }
        double act = 0.0;
        int rc2 = reduce_launch(W, k_rat_combine, 1, &act, st, (size_t)12 * lat->g.Vh, c, (const double2*)W.b,
                                W.out);
        if (!rc2) rc2 = store_field(lat, W, out, W.out, params->flags, st);
        if (!rc2 && cudaStreamSynchronize(st) != cudaSuccess)
            rc2 = fail(QXD_ERR_CUDA, "qxd_rational_apply: stream sync");
        if (rc2) rc = rc2;
        info.action = act;
    }
    info.status = rc;
    info.time_ms = ms_since(t0);
    if (info_out) *info_out = info;
    return rc;
}

}  // extern "C"
