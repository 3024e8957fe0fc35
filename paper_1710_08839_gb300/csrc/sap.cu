// Schwarz alternating procedure (SAP) preconditioner on 4^4 blocks.
//
// The paper names the SAP-preconditioned GCR solver (Sec. 1-2) without
// giving it; this is the standard multiplicative Schwarz method. The lattice
// is cut into 4^4 blocks, coloured by the parity of their block coordinates
// so that blocks of one colour never touch. One cycle visits the blocks of
// colour 0, then of colour 1; for each block B (all blocks of a colour in
// parallel, one thread block each):
//   r_B   = eta_B - (D psi)_B                 (D over the whole lattice)
//   solve D_B delta = r_B approximately, D_B = D restricted to B with
//         the hops leaving B dropped, by nmr minimal-residual steps on the
//         even-odd form D_hat_B = M_ee - H_eo M_oo^-1 H_oe of the block
//   psi_B += delta
// Starting from psi = 0, ncy cycles give psi = SAP(eta).
// The block spinors live in shared memory; links and clover blocks are read
// from the global fields.
#include <vector>

#include "dirac_common.cuh"
#include "solver.cuh"

namespace qxd {

namespace {

constexpr int SAP_BS = 4;          // block extent in every direction
constexpr int SAP_SITES = 256;     // sites per block
constexpr int SAP_HALF = 128;      // sites of one parity per block
constexpr int SAP_THREADS = 128;   // one thread per (even, odd) site pair

// shared-memory half-spinor field of one block: R[24][128], conflict-free
template <typename R>
struct SmemField {
    R* a;
    __device__ __forceinline__ void load(int slot, cplx<R> v[12]) const {
#pragma unroll
        for (int i = 0; i < 12; ++i) v[i] = mk(a[(2 * i) * SAP_HALF + slot], a[(2 * i + 1) * SAP_HALF + slot]);
    }
    __device__ __forceinline__ void store(int slot, const cplx<R> v[12]) const {
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            a[(2 * i) * SAP_HALF + slot] = v[i].re;
            a[(2 * i + 1) * SAP_HALF + slot] = v[i].im;
        }
    }
};

// Links of the block: FP32 keeps them in shared memory (two rows + angle,
// 53 KB per block), loaded once per block visit; FP64 reads the global field.
template <typename R>
struct BlockLinks;

template <>
struct BlockLinks<float> {
    static constexpr bool kStaged = true;
    float4* U;   // [4][3][256] by local site index
    float2* Z;   // [4][256] z^qhat = exp(i qhat A), computed once per block visit
    __device__ __forceinline__ void link(const Fields<float>&, const Geom&, int mu, int lidx, int,
                                         cplx<float> u[3][3]) const {
        const float4 a = U[(mu * 3 + 0) * SAP_SITES + lidx];
        const float4 b = U[(mu * 3 + 1) * SAP_SITES + lidx];
        const float4 c = U[(mu * 3 + 2) * SAP_SITES + lidx];
        u[0][0] = mk(a.x, a.y);
        u[0][1] = mk(a.z, a.w);
        u[0][2] = mk(b.x, b.y);
        u[1][0] = mk(b.z, b.w);
        u[1][1] = mk(c.x, c.y);
        u[1][2] = mk(c.z, c.w);
        u[2][0] = conj(u[0][1] * u[1][2] - u[0][2] * u[1][1]);
        u[2][1] = conj(u[0][2] * u[1][0] - u[0][0] * u[1][2]);
        u[2][2] = conj(u[0][0] * u[1][1] - u[0][1] * u[1][0]);
    }
    __device__ __forceinline__ cplx<float> phase(const Fields<float>&, const Geom&, int mu, int lidx, int,
                                                 float) const {
        const float2 z = Z[mu * SAP_SITES + lidx];
        return mk(z.x, z.y);
    }
};

template <>
struct BlockLinks<double> {
    static constexpr bool kStaged = false;
    __device__ __forceinline__ void link(const Fields<double>& f, const Geom& g, int mu, int, int s,
                                         cplx<double> u[3][3]) const {
        load_link(f.U, g.V, mu, s, u);
    }
    __device__ __forceinline__ cplx<double> phase(const Fields<double>& f, const Geom& g, int mu, int, int s,
                                                  double q) const {
        return link_phase(f.A, g.V, mu, s, q);
    }
};

struct Site {
    int l[4];   // coordinates inside the block
    int x[4];   // global coordinates
    int s;      // native index
    int lidx;   // local lexicographic index (0..255)
};

__device__ __forceinline__ Site make_site(const Geom& g, const int org[4], int lidx) {
    Site t;
    t.lidx = lidx;
    t.l[3] = lidx & 3;
    t.l[2] = (lidx >> 2) & 3;
    t.l[1] = (lidx >> 4) & 3;
    t.l[0] = (lidx >> 6) & 3;
#pragma unroll
    for (int m = 0; m < 4; ++m) t.x[m] = org[m] + t.l[m];
    const int p = (t.x[0] + t.x[1] + t.x[2] + t.x[3]) & 1;
    t.s = native_index(g, lex_index(g, t.x[0], t.x[1], t.x[2], t.x[3]), p);
    return t;
}

// native index of the in-block site one step back in direction MU
template <int MU>
__device__ __forceinline__ int back_native(const Geom& g, const Site& t) {
    int y[4] = {t.x[0], t.x[1], t.x[2], t.x[3]};
    y[MU] -= 1;
    return native_index(g, lex_index(g, y[0], y[1], y[2], y[3]), (y[0] + y[1] + y[2] + y[3]) & 1);
}

// hops of direction MU that stay inside the block (Dirichlet block boundary);
// the neighbour spinor comes from shared memory (field of the other parity)
template <typename R, bool QNZ, int MU>
__device__ __forceinline__ void block_dir(const Geom& g, const Fields<R>& f, const BlockLinks<R>& bl,
                                          const SmemField<R>& src, R q, const Site& t, cplx<R> acc[12]) {
    constexpr int stride = MU == 0 ? 64 : MU == 1 ? 16 : MU == 2 ? 4 : 1;
    cplx<R> v[12], h0[3], h1[3], g0[3], g1[3], u[3][3];
    if (t.l[MU] < SAP_BS - 1) {
        src.load((t.lidx + stride) >> 1, v);
        project<R, MU, +1>(v, h0, h1);
        bl.link(f, g, MU, t.lidx, t.s, u);
        su3_mul(u, h0, g0);
        su3_mul(u, h1, g1);
        if (QNZ) {
            cplx<R> ph = bl.phase(f, g, MU, t.lidx, t.s, q);
            times3(ph, g0);
            times3(ph, g1);
        }
        accumulate<R, MU, +1>(acc, g0, g1);
    }
    if (t.l[MU] > 0) {
        src.load((t.lidx - stride) >> 1, v);
        project<R, MU, -1>(v, h0, h1);
        const int sb = BlockLinks<R>::kStaged ? 0 : back_native<MU>(g, t);
        bl.link(f, g, MU, t.lidx - stride, sb, u);
        su3_dag_mul(u, h0, g0);
        su3_dag_mul(u, h1, g1);
        if (QNZ) {
            cplx<R> ph = conj(bl.phase(f, g, MU, t.lidx - stride, sb, q));
            times3(ph, g0);
            times3(ph, g1);
        }
        accumulate<R, MU, -1>(acc, g0, g1);
    }
}

template <typename R, bool QNZ>
__device__ __forceinline__ void block_hops(const Geom& g, const Fields<R>& f, const BlockLinks<R>& bl,
                                        const SmemField<R> src, R q, const Site& t, cplx<R> acc[12]) {
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = mk<R>(0, 0);
    block_dir<R, QNZ, 0>(g, f, bl, src, q, t, acc);
    block_dir<R, QNZ, 1>(g, f, bl, src, q, t, acc);
    block_dir<R, QNZ, 2>(g, f, bl, src, q, t, acc);
    block_dir<R, QNZ, 3>(g, f, bl, src, q, t, acc);
}

// r = eta - (D psi)(x), D over the whole lattice, at one site
template <typename R, bool QNZ>
__device__ __noinline__ void residual_at(const Geom& g, const Fields<R>& f, const typename Fields<R>::vec* eta,
                                         R q, const Site& t, bool psi_zero, cplx<R> r[12]) {
    load_spinor(eta, g.V, t.s, r);
    if (psi_zero) return;
    const int po = 1 - ((t.x[0] + t.x[1] + t.x[2] + t.x[3]) & 1);
    cplx<R> acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = mk<R>(0, 0);
    dirac_dir<R, QNZ, 0>(g, f, f.psi, g.V, 0, q, t.x[0], t.x[1], t.x[2], t.x[3], t.s, po, acc);
    dirac_dir<R, QNZ, 1>(g, f, f.psi, g.V, 0, q, t.x[0], t.x[1], t.x[2], t.x[3], t.s, po, acc);
    dirac_dir<R, QNZ, 2>(g, f, f.psi, g.V, 0, q, t.x[0], t.x[1], t.x[2], t.x[3], t.s, po, acc);
    dirac_dir<R, QNZ, 3>(g, f, f.psi, g.V, 0, q, t.x[0], t.x[1], t.x[2], t.x[3], t.s, po, acc);
    cplx<R> v[12], w[12];
    load_spinor(f.psi, g.V, t.s, v);
    clover_mul(f.C, g.V, t.s, v, w);
#pragma unroll
    for (int i = 0; i < 12; ++i) r[i] = r[i] - (w[i] - R(0.5) * acc[i]);
}

// sum over the 128 threads of the block, result in every thread
template <typename R>
__device__ __forceinline__ void block_sum3(R a, R b, R c, R* red, R out[3]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[3 * warp] = a;
        red[3 * warp + 1] = b;
        red[3 * warp + 2] = c;
    }
    __syncthreads();
    out[0] = out[1] = out[2] = R(0);
#pragma unroll
    for (int w = 0; w < SAP_THREADS / 32; ++w) {
        out[0] += red[3 * w];
        out[1] += red[3 * w + 1];
        out[2] += red[3 * w + 2];
    }
    __syncthreads();
}

template <typename R>
constexpr size_t sap_link_bytes() {
    return BlockLinks<R>::kStaged ? (12 * SAP_SITES * sizeof(float4) + 4 * SAP_SITES * sizeof(float2)) : 0;
}

// Each thread owns one even and one odd site of the block: the local pair
// (2t, 2t + 1). Phases in order (each block-hop phase is one call of
// block_hops from a single call site, which keeps the code small):
//   residual on both sites; t_o = M_oo^-1 r_o
//   step 0:            rho = r_e - H_eo t_o                       (even)
//   step 2k+1, 2k+2:   t_o = M_oo^-1 H_oe rho (odd); w = M_ee rho - H_eo t_o,
//                      omega = <w,rho>/<w,w>, delta_e += omega rho,
//                      rho -= omega w (even)             for k < nmr
//   last step:         delta_o = M_oo^-1 (r_o - H_oe delta_e)     (odd)
template <typename R, bool QNZ>
__device__ __forceinline__ void sap_block_body(const Geom& g, const SapGeom& sg, int bidx, int colour, int psi_zero,
                                               const Fields<R>& f, const typename Fields<R>::cvec* __restrict__ Cinv,
                                               const typename Fields<R>::vec* __restrict__ eta, int nmr, R q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BlockLinks<R> bl;
    unsigned char* sp = smem_raw;
    if constexpr (BlockLinks<R>::kStaged) {
        bl.U = reinterpret_cast<float4*>(sp);
        bl.Z = reinterpret_cast<float2*>(sp + 12 * SAP_SITES * sizeof(float4));
        sp += sap_link_bytes<R>();
    }
    R* sm = reinterpret_cast<R*>(sp);
    const SmemField<R> s_ro{sm};                    // r on the odd sites
    const SmemField<R> s_rho{sm + 24 * SAP_HALF};   // MR residual (even)
    const SmemField<R> s_t{sm + 48 * SAP_HALF};     // odd temporary / delta_e at the end
    R* red = sm + 72 * SAP_HALF;                    // 3 * warps reduction slots

    // block of this colour handled by this thread block
    int org[4];
    {
        const int bi2 = 2 * bidx;
        const int b3e = bi2 % sg.nb3;
        int rest = bi2 / sg.nb3;
        const int b2 = rest % sg.nb2;
        rest /= sg.nb2;
        const int b1 = rest % sg.nb1;
        const int b0 = rest / sg.nb1;
        const int b3 = b3e + ((b0 + b1 + b2 + b3e + colour) & 1);
        org[0] = SAP_BS * b0;
        org[1] = SAP_BS * b1;
        org[2] = SAP_BS * b2;
        org[3] = SAP_BS * b3;
    }
    const int t = threadIdx.x;
    const int base = 2 * t;
    const int par0 = ((base >> 6) + ((base >> 4) & 3) + ((base >> 2) & 3) + (base & 3)) & 1;
    const Site se = make_site(g, org, base + par0);
    const Site so = make_site(g, org, base + 1 - par0);

    if constexpr (BlockLinks<R>::kStaged) {
        // links and angles of the block's sites, all four directions
#pragma unroll 1
        for (int k = 0; k < 2; ++k) {
            const Site& st_ = k ? so : se;
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    bl.U[(mu * 3 + j) * SAP_SITES + st_.lidx] = f.U[((size_t)mu * 3 + j) * g.V + st_.s];
            }
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
                const cplx<float> z = QNZ ? link_phase(f.A, g.V, mu, st_.s, q) : mk(1.f, 0.f);
                bl.Z[mu * SAP_SITES + st_.lidx] = make_float2(z.re, z.im);
            }
        }
    }

    // residual r = eta - D psi on both sites (one call site)
    cplx<R> re[12], v[12], w[12], acc[12];
#pragma unroll 1
    for (int k = 0; k < 2; ++k) {
        residual_at<R, QNZ>(g, f, eta, q, k ? so : se, psi_zero, k ? v : re);
    }
    s_ro.store(t, v);
    clover_mul(Cinv, g.V, so.s, v, w);  // t_o = M_oo^-1 r_o
    s_t.store(t, w);
    __syncthreads();

    cplx<R> rho[12], de[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) de[i] = mk<R>(0, 0);
    const int nsteps = 2 * nmr + 2;
#pragma unroll 1
    for (int step = 0; step < nsteps; ++step) {
        const bool odd = (step & 1) != 0;   // steps 1, 3, ..., 2 nmr + 1 work on the odd sites
        const bool last = step == nsteps - 1;
        // odd steps read rho (or delta_e on the last step), even steps read t_o
        block_hops<R, QNZ>(g, f, bl, odd ? (last ? s_t : s_rho) : s_t, q, odd ? so : se, acc);
        if (step == 0) {
#pragma unroll
            for (int i = 0; i < 12; ++i) rho[i] = re[i] + R(0.5) * acc[i];
            s_rho.store(t, rho);
        } else if (last) {
            s_ro.load(t, v);
#pragma unroll
            for (int i = 0; i < 12; ++i) v[i] = v[i] + R(0.5) * acc[i];
            clover_mul(Cinv, g.V, so.s, v, w);  // delta_o
        } else if (odd) {
#pragma unroll
            for (int i = 0; i < 12; ++i) v[i] = R(-0.5) * acc[i];
            clover_mul(Cinv, g.V, so.s, v, w);
            s_t.store(t, w);
        } else {
            clover_mul(f.C, g.V, se.s, rho, w);
#pragma unroll
            for (int i = 0; i < 12; ++i) w[i] = w[i] + R(0.5) * acc[i];
            R a_re = 0, a_im = 0, b = 0;
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                a_re += w[i].re * rho[i].re + w[i].im * rho[i].im;
                a_im += w[i].re * rho[i].im - w[i].im * rho[i].re;
                b += w[i].re * w[i].re + w[i].im * w[i].im;
            }
            R sums[3];
            block_sum3(a_re, a_im, b, red, sums);
            if (sums[2] > R(0)) {  // else rho = 0 on the whole block: nothing to add
                const cplx<R> om = mk(sums[0] / sums[2], sums[1] / sums[2]);
#pragma unroll
                for (int i = 0; i < 12; ++i) {
                    de[i] = de[i] + om * rho[i];
                    rho[i] = rho[i] - om * w[i];
                }
            }
            if (step == nsteps - 2) s_t.store(t, de);  // delta_e for the last step
            else s_rho.store(t, rho);
        }
        __syncthreads();
    }
    // psi_B += delta (w holds delta_o)
    typename Fields<R>::vec* psi = const_cast<typename Fields<R>::vec*>(f.psi);
    if (psi_zero) {
        store_spinor(psi, g.V, se.s, de);
        store_spinor(psi, g.V, so.s, w);
    } else {
        load_spinor(f.psi, g.V, se.s, v);
#pragma unroll
        for (int i = 0; i < 12; ++i) v[i] = v[i] + de[i];
        store_spinor(psi, g.V, se.s, v);
        load_spinor(f.psi, g.V, so.s, v);
#pragma unroll
        for (int i = 0; i < 12; ++i) v[i] = v[i] + w[i];
        store_spinor(psi, g.V, so.s, v);
    }
}

template <typename R, bool QNZ>
__global__ void __launch_bounds__(SAP_THREADS, 2) k_sap_block(Geom g, SapGeom sg, int colour, int psi_zero,
                                                              Fields<R> f, const typename Fields<R>::cvec* __restrict__ Cinv,
                                                              const typename Fields<R>::vec* __restrict__ eta, int nmr,
                                                              R q) {
    sap_block_body<R, QNZ>(g, sg, blockIdx.x, colour, psi_zero, f, Cinv, eta, nmr, q);
}

// batched form: thread block b works on block (b - cta_begin) of the job
// whose range holds b (one launch serves every job of a batch)
__global__ void __launch_bounds__(SAP_THREADS, 2) k_sap_block_batch(const SapJob* __restrict__ jobs, int njobs,
                                                                    int colour, int psi_zero, int nmr) {
    int lo = 0, hi = njobs - 1;
    const int b = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].cta_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    const SapJob& J = jobs[lo];
    sap_block_body<float, true>(J.g, J.sg, b - J.cta_begin, colour, psi_zero, J.f, J.Cinv, J.eta, nmr, J.q);
}

template <typename R>
size_t sap_smem_bytes() {
    return sap_link_bytes<R>() + (72 * SAP_HALF + 3 * (SAP_THREADS / 32)) * sizeof(R);
}

template <typename R, bool QNZ>
int launch_sap_block(qxd_lattice* lat, const SapGeom& sg, int colour, int psi_zero, Fields<R> f,
                     const typename Fields<R>::cvec* Cinv, const typename Fields<R>::vec* eta, int nmr,
                     cudaStream_t st) {
    const size_t smem = sap_smem_bytes<R>();
    QXD_CUDA(cudaFuncSetAttribute(k_sap_block<R, QNZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_sap_block<R, QNZ><<<sg.nhalf, SAP_THREADS, smem, st>>>(lat->g, sg, colour, psi_zero, f, Cinv, eta, nmr,
                                                              (R)lat->qhat);
    QXD_LAUNCHED("k_sap_block");
    return QXD_OK;
}

template <typename R>
Fields<R> sap_fields(qxd_lattice* lat, void* psi);
template <>
Fields<float> sap_fields<float>(qxd_lattice* lat, void* psi) {
    return Fields<float>{(const float4*)psi, nullptr, lat->U32, lat->A32, lat->C32};
}
template <>
Fields<double> sap_fields<double>(qxd_lattice* lat, void* psi) {
    return Fields<double>{(const double2*)psi, nullptr, lat->U64, lat->Zq64, lat->C64};
}
const float4* sap_cinv(qxd_lattice* lat, float) { return lat->Cinv32; }
const double* sap_cinv(qxd_lattice* lat, double) { return lat->Cinv64; }

}  // namespace

int sap_check(qxd_lattice* lat) {
    const Geom& g = lat->g;
    const int N[4] = {g.N0, g.N1, g.N2, g.N3};
    for (int m = 0; m < 4; ++m)
        if (N[m] % SAP_BS || (N[m] / SAP_BS) % 2)
            return fail(QXD_ERR_ARG, "SAP: every simulated extent must be a multiple of 8 "
                                     "(4^4 blocks, even number of blocks per direction)");
    if (g.cs2 || g.cs3) {
        if (g.L1 % SAP_BS)
            return fail(QXD_ERR_ARG, "SAP: with C* boundaries L1 must be a multiple of 4");
        const int sh = g.L1 / SAP_BS;
        if ((g.cs2 && (N[2] / SAP_BS + sh) % 2) || (g.cs3 && (N[3] / SAP_BS + sh) % 2))
            return fail(QXD_ERR_ARG, "SAP: the block colouring is not consistent across the shifted "
                                     "C* boundary (L_k/4 + L1/4 must be even)");
    }
    return QXD_OK;
}

template <typename R>
int sap_apply(qxd_lattice* lat, SapWork& w, void* out, const void* in, int ncy, int nmr, cudaStream_t st) {
    const Geom& g = lat->g;
    SapGeom& sg = w.sg;
    sg.nb0 = g.N0 / SAP_BS;
    sg.nb1 = g.N1 / SAP_BS;
    sg.nb2 = g.N2 / SAP_BS;
    sg.nb3 = g.N3 / SAP_BS;
    sg.nblk = sg.nb0 * sg.nb1 * sg.nb2 * sg.nb3;
    sg.nhalf = sg.nblk / 2;
    Fields<R> f = sap_fields<R>(lat, out);
    const typename Fields<R>::cvec* Cinv = sap_cinv(lat, R(0));
    const typename Fields<R>::vec* eta = (const typename Fields<R>::vec*)in;
    const bool qnz = lat->qhat != 0;
    // psi starts at zero: the first half-cycle writes the blocks of colour 0
    // without reading psi, and the blocks of colour 1 must read zeros there
    QXD_CUDA(cudaMemsetAsync(out, 0, (size_t)g.V * 24 * sizeof(R), st));
    int rc;
    for (int cy = 0; cy < ncy; ++cy)
        for (int colour = 0; colour < 2; ++colour) {
            const int psi_zero = (cy == 0 && colour == 0) ? 1 : 0;
            rc = qnz ? launch_sap_block<R, true>(lat, sg, colour, psi_zero, f, Cinv, eta, nmr, st)
                     : launch_sap_block<R, false>(lat, sg, colour, psi_zero, f, Cinv, eta, nmr, st);
            if (rc) return rc;
        }
    return QXD_OK;
}

template int sap_apply<float>(qxd_lattice*, SapWork&, void*, const void*, int, int, cudaStream_t);

SapGeom sap_geom(const Geom& g) {
    SapGeom sg;
    sg.nb0 = g.N0 / SAP_BS;
    sg.nb1 = g.N1 / SAP_BS;
    sg.nb2 = g.N2 / SAP_BS;
    sg.nb3 = g.N3 / SAP_BS;
    sg.nblk = sg.nb0 * sg.nb1 * sg.nb2 * sg.nb3;
    sg.nhalf = sg.nblk / 2;
    return sg;
}

int sap_apply_batch(std::vector<SapJob>& jobs, SapJob* d_jobs, int ncy, int nmr, cudaStream_t st) {
    if (jobs.empty()) return QXD_OK;
    int ctas = 0;
    for (auto& J : jobs) {
        J.cta_begin = ctas;
        ctas += J.sg.nhalf;
        QXD_CUDA(cudaMemsetAsync((void*)J.f.psi, 0, (size_t)J.g.V * 24 * sizeof(float), st));
    }
    QXD_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(SapJob), cudaMemcpyHostToDevice, st));
    const size_t smem = sap_smem_bytes<float>();
    QXD_CUDA(cudaFuncSetAttribute(k_sap_block_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int cy = 0; cy < ncy; ++cy)
        for (int colour = 0; colour < 2; ++colour) {
            const int psi_zero = (cy == 0 && colour == 0) ? 1 : 0;
            k_sap_block_batch<<<ctas, SAP_THREADS, smem, st>>>(d_jobs, (int)jobs.size(), colour, psi_zero, nmr);
            QXD_LAUNCHED("k_sap_block_batch");
        }
    return QXD_OK;
}
template int sap_apply<double>(qxd_lattice*, SapWork&, void*, const void*, int, int, cudaStream_t);

}  // namespace qxd

using namespace qxd;

extern "C" int qxd_sap(qxd_lattice* lat, void* out, const void* in, int ncy, int nmr, int flags, void* stream) {
    if (!lat || !out || !in) return fail(QXD_ERR_ARG, "qxd_sap: NULL argument");
    if (flags & ~(0x1 | 0x100)) return fail(QXD_ERR_ARG, "qxd_sap: bad flags (device buffers only)");
    if (ncy < 1 || nmr < 1) return fail(QXD_ERR_ARG, "qxd_sap: ncy and nmr must be >= 1");
    if (out == in) return fail(QXD_ERR_ARG, "qxd_sap: in and out must not overlap");
    if (!qxd::clover_ready(lat)) return fail(QXD_ERR_STATE, "qxd_sap: needs qxd_sw_build first");
    int rc = sap_check(lat);
    if (rc) return rc;
    const int prec = flags & 0x1;
    cudaStream_t st = stream ? (cudaStream_t)stream : lat->stream;
    SapWork w;
    if (flags & QXD_LAYOUT_NATIVE)
        return prec == QXD_FP32 ? sap_apply<float>(lat, w, out, in, ncy, nmr, st)
                                : sap_apply<double>(lat, w, out, in, ncy, nmr, st);
    if ((rc = ensure_scratch(lat))) return rc;
    if ((rc = launch_pack(lat, lat->scratch_in, in, prec, st))) return rc;
    rc = prec == QXD_FP32 ? sap_apply<float>(lat, w, lat->scratch_out, lat->scratch_in, ncy, nmr, st)
                          : sap_apply<double>(lat, w, lat->scratch_out, lat->scratch_in, ncy, nmr, st);
    if (rc) return rc;
    return launch_unpack(lat, out, lat->scratch_out, prec, st);
}
