// Work space of the multi-shift CG (pseudofermion action of the RHMC).
#pragma once

#include "blas.cuh"
#include "qxd_internal.cuh"

namespace qxd {

struct MscgWork {
    int Vh = 0;       // even sites the vectors are sized for
    int nshift = 0;   // shifts with x and p allocated
    // even-site FP64 arrays (12 V/2 complex numbers each)
    double2 *b = nullptr, *r = nullptr, *t = nullptr, *w = nullptr, *out = nullptr;
    double2* tmp_o = nullptr;  // odd-site temporary of D_hat
    double2 *e = nullptr, *src2 = nullptr;  // refinement: correction and residual
    float4 *p32 = nullptr, *t32 = nullptr, *w32 = nullptr, *tmp32 = nullptr;  // FP32 operator (even/odd sites)
    double2* full = nullptr;   // full-lattice native FP64 staging field
    double2* x[BLAS_KMAX] = {};
    double2* p[BLAS_KMAX] = {};
    Reducer red;
    int ensure(int V, int Vh, int nshift);
    void release();
};

// x_j = (D_hat^dag D_hat + sigma_j)^-1 W.b into W.x[j] (even-site arrays)
int mscg_core(qxd_lattice* lat, MscgWork& W, int ns, const double* sigma, double tol, int max_iter,
              qxd_mscg_info& info, double* relres, cudaStream_t st);

}  // namespace qxd
