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
// FP32, single lattice (k_sap_split): two threads per site pair, the block's
// interior compound links W' = -1/2 z^qhat U (all three rows) and two block
// fields in shared memory, the clover blocks read through L1. The residual
// of a block is not recomputed from eta - D psi: the even-odd block solve
// leaves the block residual r_B - D_B delta equal to the MR residual rho on
// the even sites and to zero on the odd sites (delta_o = M_oo^-1 (r_o - H_oe
// delta_e) solves the odd rows exactly), and between two visits of a block
// psi changes only on the blocks of the other colour, by their last
// corrections delta. So a visit starts from
//   r_B = rho_B (even sites), 0 (odd sites)  -  D_cross delta,
// where D_cross keeps the hops of D that cross the faces of B (all other
// terms of D delta vanish on B), and r_B = eta_B on the first visit. The
// kernel keeps rho on the even sites and delta of every site in two work
// fields. FP32, batched (k_sap_block_batch): the same block solve over the
// blocks of several lattices in one launch, each job with its own work
// fields. FP64 (k_sap_block): one thread per site pair, the block fields in
// shared memory, links and clover blocks from the global fields.
#include <algorithm>
#include <vector>

#include "dirac_common.cuh"
#include "solver.cuh"

namespace qxd {

namespace {

constexpr int SAP_BS = 4;          // block extent in every direction
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

// Links of the block for the one-thread-per-pair form (FP64): read from the
// global field.
template <typename R>
struct BlockLinks;

template <>
struct BlockLinks<double> {
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
        const int sb = back_native<MU>(g, t);
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
__device__ __forceinline__ void residual_body(const Geom& g, const Fields<R>& f, const typename Fields<R>::vec* eta,
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

// out-of-line form for the one-thread-per-pair kernel, which calls it twice
template <typename R, bool QNZ>
__device__ __noinline__ void residual_at(const Geom& g, const Fields<R>& f, const typename Fields<R>::vec* eta,
                                         R q, const Site& t, bool psi_zero, cplx<R> r[12]) {
    residual_body<R, QNZ>(g, f, eta, q, t, psi_zero, r);
}

// sum over the NT threads of the block, result in every thread. TAIL_SYNC
// guards red against the next call; a caller that passes a barrier before it
// reuses red may drop it.
template <typename R, int NT = SAP_THREADS, bool TAIL_SYNC = true>
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
    for (int w = 0; w < NT / 32; ++w) {
        out[0] += red[3 * w];
        out[1] += red[3 * w + 1];
        out[2] += red[3 * w + 2];
    }
    if (TAIL_SYNC) __syncthreads();
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
    R* sm = reinterpret_cast<R*>(smem_raw);
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

// ---------------------------------------------------------------------------
// FP32 block solve with two threads per site pair (spin split)
//
// Thread 2t + sg owns the spin-sg half of every block spinor of local pair t:
// components 3 sg + c (upper chirality) and 6 + 3 sg + c (lower chirality,
// spin 2 + sg), c = 0..2. In the chiral basis (1 -+ g_mu) psi is fixed by a
// half spinor (h_0, h_1): the upper spins are U h and the lower ones a fixed
// 2x2 spin matrix times U h. Thread sg forms h_sg from two spin components of
// the neighbour, multiplies it by the link, and adds U h_sg to its own upper
// spin and to one lower spin: its own (mu = 0, 3) or its partner's
// (mu = 1, 2). The partner's share is exchanged once per hop set with a warp
// shuffle. The clover term acts within a chirality, so each thread computes
// its three rows of both 6x6 blocks after one shuffle of the partner's half.
// The block's compound links W' = -1/2 z^qhat U are staged once per launch
// with all three rows, so a hop is a projection, one 3x3 complex product and
// the accumulation: no third-row rebuild, no U(1) phase, no factor -1/2.
// ---------------------------------------------------------------------------
constexpr int SPLIT_THREADS = 256;
constexpr unsigned FULL_MASK = 0xffffffffu;

// Shared-memory block fields of the split kernel: float2 [12][128], entry
// (3 spin + colour, pair slot) a complex number, with the slots of spins 1
// and 3 rotated by 8. The two threads of a pair read the same slot in spins
// of opposite parity; the rotation puts the eight pairs of a half warp on
// disjoint halves of the 32 banks.
__device__ __forceinline__ int spin_slot(int spin, int slot) { return (slot + 8 * (spin & 1)) & (SAP_HALF - 1); }
__device__ __forceinline__ void ld_spin(const float2* a, int spin, int slot, cplx<float> v[3]) {
    const float2* p = a + 3 * spin * SAP_HALF + spin_slot(spin, slot);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 x = p[c * SAP_HALF];
        v[c] = mk(x.x, x.y);
    }
}
__device__ __forceinline__ void st_spin(float2* a, int spin, int slot, const cplx<float> v[3]) {
    float2* p = a + 3 * spin * SAP_HALF + spin_slot(spin, slot);
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c * SAP_HALF] = make_float2(v[c].re, v[c].im);
}
// own half: v[0..2] spin sg, v[3..5] spin 2 + sg
__device__ __forceinline__ void ld_half(const float2* a, int sg, int slot, cplx<float> v[6]) {
    ld_spin(a, sg, slot, v);
    ld_spin(a, 2 + sg, slot, v + 3);
}
__device__ __forceinline__ void st_half(float2* a, int sg, int slot, const cplx<float> v[6]) {
    st_spin(a, sg, slot, v);
    st_spin(a, 2 + sg, slot, v + 3);
}
__device__ __forceinline__ void ld_full(const float2* a, int slot, cplx<float> v[12]) {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) ld_spin(a, sp, slot, v + 3 * sp);
}
__device__ __forceinline__ void st_full(float2* a, int slot, const cplx<float> v[12]) {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) st_spin(a, sp, slot, v + 3 * sp);
}

// Block links of the split kernel in shared memory. The block operator uses
// only the links that stay inside the block, those of sites with l[mu] < 3,
// 192 per direction. Entry of the site of parity p and local index lidx in
// direction mu (stride S = 64, 16, 4, 1 in lidx):
//   mu = 0, 1, 2: p * 96 + compact pair slot, with the pair slot lidx >> 1
//                 written as hi * 2S + l * S/2 + lo (l = l[mu]) and compacted to
//                 hi * 3S/2 + l * S/2 + lo, so that consecutive pairs read
//                 consecutive entries;
//   mu = 3:       3 (lidx >> 2) + (lidx & 3).
constexpr int SPLIT_LINKS = 192;  // interior links per direction

template <int MU>
__device__ __forceinline__ int link_entry(int p, int lidx) {
    if constexpr (MU == 3) {
        return 3 * (lidx >> 2) + (lidx & 3);
    } else {
        constexpr int H = MU == 0 ? 32 : MU == 1 ? 8 : 2;  // S / 2
        const int slot = lidx >> 1;
        return p * (SPLIT_LINKS / 2) + (slot / (4 * H)) * (3 * H) + ((slot / H) & 3) * H + (slot & (H - 1));
    }
}

// Compound block links of the split kernel, W'(x,mu) = -1/2 z(x,mu)^qhat
// U(x,mu), all three rows, staged once per launch so that the hops need
// neither the third-row reconstruction nor the U(1) phase nor the factor
// -1/2. Entry e of direction mu: float4 W4[mu][k][e], k = 0..3, holds the
// complex entries (00, 01), (02, 10), (11, 12), (20, 21); float2 W2[mu][e]
// holds (22).
struct SplitLinks {
    const float4* W4;  // [4][4][192]
    const float2* W2;  // [4][192]
    __device__ __forceinline__ void link(int mu, int e, cplx<float> u[3][3]) const {
        const float4 a = W4[(mu * 4 + 0) * SPLIT_LINKS + e];
        const float4 b = W4[(mu * 4 + 1) * SPLIT_LINKS + e];
        const float4 c = W4[(mu * 4 + 2) * SPLIT_LINKS + e];
        const float4 d = W4[(mu * 4 + 3) * SPLIT_LINKS + e];
        const float2 z = W2[mu * SPLIT_LINKS + e];
        u[0][0] = mk(a.x, a.y);
        u[0][1] = mk(a.z, a.w);
        u[0][2] = mk(b.x, b.y);
        u[1][0] = mk(b.z, b.w);
        u[1][1] = mk(c.x, c.y);
        u[1][2] = mk(c.z, c.w);
        u[2][0] = mk(d.x, d.y);
        u[2][1] = mk(d.z, d.w);
        u[2][2] = mk(z.x, z.y);
    }
};

constexpr size_t split_link_bytes() { return 16 * SPLIT_LINKS * sizeof(float4) + 4 * SPLIT_LINKS * sizeof(float2); }

// Hops of direction MU inside the block for thread sg (sgn = +1 for sg = 0,
// -1 for sg = 1). With a the neighbour's spin sg and b the lower spin named
// below, h_sg = a + DIR c_MU b with c_0 = 1, c_1 = i, c_2 = sgn, c_3 = sgn i;
// g = U h_sg (U^+ backwards) goes to au (upper spin sg) and, times
// DIR, 1 / -i / sgn / -sgn i for MU = 0..3, to al (lower spin 2 + sg, MU =
// 0, 3) or ax (lower spin 3 - sg, the partner's, MU = 1, 2).
template <bool QNZ, int MU>
__device__ __forceinline__ void split_dir(const SplitLinks& bl, const float2* src, const Site& t, int p, int sg,
                                          float sgn, cplx<float> au[3], cplx<float> al[3], cplx<float> ax[3]) {
    constexpr int stride = MU == 0 ? 64 : MU == 1 ? 16 : MU == 2 ? 4 : 1;
    const int lspin = (MU == 0 || MU == 3) ? 2 + sg : 3 - sg;
    cplx<float> a[3], b[3], h[3], gv[3], u[3][3];
    if (t.l[MU] < SAP_BS - 1) {
        const int slot = (t.lidx + stride) >> 1;
        ld_spin(src, sg, slot, a);
        ld_spin(src, lspin, slot, b);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (MU == 0) h[c] = a[c] + b[c];
            else if (MU == 1) h[c] = a[c] + times_i(b[c]);
            else if (MU == 2) h[c] = a[c] + sgn * b[c];
            else h[c] = a[c] + sgn * times_i(b[c]);
        }
        const int e = link_entry<MU>(p, t.lidx);
        bl.link(MU, e, u);
        su3_mul(u, h, gv);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            au[c] = au[c] + gv[c];
            if (MU == 0) al[c] = al[c] + gv[c];
            else if (MU == 1) ax[c] = ax[c] + times_mi(gv[c]);
            else if (MU == 2) ax[c] = ax[c] + sgn * gv[c];
            else al[c] = al[c] - sgn * times_i(gv[c]);
        }
    }
    if (t.l[MU] > 0) {
        const int slot = (t.lidx - stride) >> 1;
        ld_spin(src, sg, slot, a);
        ld_spin(src, lspin, slot, b);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (MU == 0) h[c] = a[c] - b[c];
            else if (MU == 1) h[c] = a[c] - times_i(b[c]);
            else if (MU == 2) h[c] = a[c] - sgn * b[c];
            else h[c] = a[c] - sgn * times_i(b[c]);
        }
        const int e = link_entry<MU>(1 - p, t.lidx - stride);  // link of the neighbour (other parity)
        bl.link(MU, e, u);
        su3_dag_mul(u, h, gv);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            au[c] = au[c] + gv[c];
            if (MU == 0) al[c] = al[c] - gv[c];
            else if (MU == 1) ax[c] = ax[c] + times_i(gv[c]);
            else if (MU == 2) ax[c] = ax[c] - sgn * gv[c];
            else al[c] = al[c] + sgn * times_i(gv[c]);
        }
    }
}

// raw block-hop sum at site t, own half (acc[0..2] spin sg, acc[3..5] spin 2 + sg);
// every thread of the warp must call it (one shuffle at the end)
// (site t of parity p)
template <bool QNZ>
__device__ __forceinline__ void split_hops(const SplitLinks& bl, const float2* src, const Site& t, int p, int sg,
                                           float sgn, cplx<float> acc[6]) {
    cplx<float> au[3], al[3], ax[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) au[c] = al[c] = ax[c] = mk(0.f, 0.f);
    split_dir<QNZ, 0>(bl, src, t, p, sg, sgn, au, al, ax);
    split_dir<QNZ, 1>(bl, src, t, p, sg, sgn, au, al, ax);
    split_dir<QNZ, 2>(bl, src, t, p, sg, sgn, au, al, ax);
    split_dir<QNZ, 3>(bl, src, t, p, sg, sgn, au, al, ax);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float xr = __shfl_xor_sync(FULL_MASK, ax[c].re, 1);
        const float xi = __shfl_xor_sync(FULL_MASK, ax[c].im, 1);
        acc[c] = au[c];
        acc[3 + c] = al[c] + mk(xr, xi);
    }
}

// Own rows (3 sg + a, a = 0..2) of both packed Hermitian 6x6 blocks of C at
// site s times v; v and y are own halves, the partner's half is shuffled in.
// In block order the rows of thread sg see a Hermitian 3x3 diagonal block
// (entries d[3 sg + a] and L(3 sg + a, 3 sg + b)) and the off-diagonal
// 3x3 block B[a][b] = L(3 + a, b) for sg = 1, B^+ for sg = 0. Every thread
// of the warp must call it.
__device__ __forceinline__ void clover_half(const float4* __restrict__ C, int V, int s, int sg, float sgn,
                                            const cplx<float> v[6], cplx<float> y[6]) {
    cplx<float> p[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) p[k] = mk(__shfl_xor_sync(FULL_MASK, v[k].re, 1), __shfl_xor_sync(FULL_MASK, v[k].im, 1));
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        const float4* Cb = C + (size_t)(9 * blk) * V + s;
        const float4 q0 = Cb[0], q1 = Cb[(size_t)V], q3 = Cb[(size_t)3 * V], q4 = Cb[(size_t)4 * V];
        const float4 q5 = Cb[(size_t)5 * V], q6 = Cb[(size_t)6 * V], q7 = Cb[(size_t)7 * V];
        const float4 X = Cb[(size_t)(sg ? 8 : 2) * V];
        // packed floats: d_i at i, L_k at (6 + 2k, 7 + 2k); float4 n holds 4n..4n+3
        const float d0 = sg ? q0.w : q0.x, d1 = sg ? q1.x : q0.y, d2 = sg ? q1.y : q0.z;
        const cplx<float> l10 = sg ? mk(q6.x, q6.y) : mk(q1.z, q1.w);  // L(4,3) : L(1,0)
        const cplx<float> l20 = mk(X.x, X.y);                          // L(5,3) : L(2,0)
        const cplx<float> l21 = mk(X.z, X.w);                          // L(5,4) : L(2,1)
        const cplx<float> B[3][3] = {{mk(q3.x, q3.y), mk(q3.z, q3.w), mk(q4.x, q4.y)},
                                     {mk(q4.z, q4.w), mk(q5.x, q5.y), mk(q5.z, q5.w)},
                                     {mk(q6.z, q6.w), mk(q7.x, q7.y), mk(q7.z, q7.w)}};
        const cplx<float>* w = v + 3 * blk;
        const cplx<float>* pp = p + 3 * blk;
        cplx<float> z[3];
        z[0] = d0 * w[0] + cmul(l10, w[1]) + cmul(l20, w[2]);
        z[1] = l10 * w[0] + d1 * w[1] + cmul(l21, w[2]);
        z[2] = l20 * w[0] + l21 * w[1] + d2 * w[2];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                // E[a][b] = sg ? B[a][b] : conj(B[b][a])
                const cplx<float> e = mk(sg ? B[a][b].re : B[b][a].re, sg ? B[a][b].im : -B[b][a].im);
                z[a] = z[a] + e * pp[b];
            }
#pragma unroll
        for (int a = 0; a < 3; ++a) y[3 * blk + a] = z[a];
    }
    (void)sgn;
}

// Hop of D from x to its neighbour x + DIR mu across the face of x's block,
// applied to the field d (raw: without the factor -1/2), added to acc
template <bool QNZ, int MU, int DIR>
__device__ __forceinline__ void crossing_hop(const Geom& g, const Fields<float>& f, const float4* __restrict__ d,
                                             float q, const Site& t, int po, cplx<float> acc[12]) {
    cplx<float> v[12], h0[3], h1[3], g0[3], g1[3], u[3][3];
    const int sn = native_index(g, neighbour_lex<MU, DIR>(g, t.x[0], t.x[1], t.x[2], t.x[3]), po);
    load_spinor(d, g.V, sn, v);
    project<float, MU, DIR>(v, h0, h1);
    const int sl = DIR > 0 ? t.s : sn;  // the link of x forwards, of the neighbour backwards
    load_link(f.U, g.V, MU, sl, u);
    if (DIR > 0) {
        su3_mul(u, h0, g0);
        su3_mul(u, h1, g1);
    } else {
        su3_dag_mul(u, h0, g0);
        su3_dag_mul(u, h1, g1);
    }
    if (QNZ) {
        const cplx<float> ph0 = link_phase(f.A, g.V, MU, sl, q);
        const cplx<float> ph = DIR > 0 ? ph0 : conj(ph0);
        times3(ph, g0);
        times3(ph, g1);
    }
    accumulate<float, MU, DIR>(acc, g0, g1);
}

// acc += raw sum of the hops of D at site t that leave its block (t on the
// upper face in mu: forward hop; on the lower face: backward hop)
template <bool QNZ, int MU>
__device__ __forceinline__ void crossing_dir(const Geom& g, const Fields<float>& f, const float4* __restrict__ d,
                                             float q, const Site& t, int po, cplx<float> acc[12]) {
    if (t.l[MU] == SAP_BS - 1) crossing_hop<QNZ, MU, +1>(g, f, d, q, t, po, acc);
    if (t.l[MU] == 0) crossing_hop<QNZ, MU, -1>(g, f, d, q, t, po, acc);
}

// How k_sap_split forms the residual of its blocks and what it keeps
enum SplitFlags : int {
    SF_FIRST = 1,  // first visit of this colour: r = eta, psi = delta (psi is not read)
    SF_CROSS = 2,  // subtract D_cross of the other colour's last corrections
    SF_KEEP_RHO = 4,    // keep rho of the even sites for the next visit of this colour
    SF_KEEP_DELTA = 8,  // keep delta for the next visit of the other colour
};

// One right-hand side of the FP32 block solve: source eta, output psi and the
// work fields, delta of every site (6 float4 per site, stride V) and rho of
// the even sites (stride Vh)
struct SplitWork {
    const float4* eta;
    float4* psi;
    float4* delta;
    float4* rho;
};

// right-hand sides of one operator solved in one launch: each thread block
// stages its block's links once and solves the block for each of them
constexpr int SPLIT_MAXR = 12;
struct SplitRhsList {
    SplitWork r[SPLIT_MAXR];
    int n;
};

// Same phases as sap_block_body, with the site-pair work split over the
// two threads of a pair, for the right-hand sides rhs[0 .. nrhs) in turn
// (the arithmetic of each is the same whatever the others); the residual
// comes from eta on the first visit of a colour, else from the kept rho and
// the crossing hops of the kept delta.
template <bool QNZ>
__device__ __forceinline__ void sap_split_body(const Geom& g, const SapGeom& sgm, int bidx, int colour,
                                               const Fields<float>& f, const float4* __restrict__ Cinv,
                                               const SplitWork* rhs, int nrhs, int flags, int nmr, float q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* sW4 = reinterpret_cast<float4*>(smem_raw);
    float2* sW2 = reinterpret_cast<float2*>(smem_raw + 16 * SPLIT_LINKS * sizeof(float4));
    const SplitLinks bl{sW4, sW2};
    float2* sm = reinterpret_cast<float2*>(smem_raw + split_link_bytes());
    float2* s_rho = sm;                 // r on the even sites, the MR residual, delta_o at the end
    float2* s_t = sm + 12 * SAP_HALF;   // r on the odd sites, the odd temporary, delta_e at the end
    float* red = reinterpret_cast<float*>(sm + 24 * SAP_HALF);  // 3 * warps reduction slots

    // blocks (b0, b1, b2, b3e) and (.., b3e + 1), b3e even: one of each colour
    int org[4];
    {
        const int bi2 = 2 * bidx;
        const int b3e = bi2 % sgm.nb3;
        int rest = bi2 / sgm.nb3;
        const int b2 = rest % sgm.nb2;
        rest /= sgm.nb2;
        const int b1 = rest % sgm.nb1;
        const int b0 = rest / sgm.nb1;
        const int b3 = b3e + ((b0 + b1 + b2 + b3e + colour) & 1);
        org[0] = SAP_BS * b0;
        org[1] = SAP_BS * b1;
        org[2] = SAP_BS * b2;
        org[3] = SAP_BS * b3;
    }
    const int t = threadIdx.x >> 1;
    const int sg = threadIdx.x & 1;
    const float sgn = sg ? -1.f : 1.f;
    const int base = 2 * t;
    const int par0 = ((base >> 6) + ((base >> 4) & 3) + ((base >> 2) & 3) + (base & 3)) & 1;
    const Site se = make_site(g, org, base + par0);
    const Site so = make_site(g, org, base + 1 - par0);
    const Site& me = sg ? so : se;  // the site this thread stages, and whose residual it computes

    // compound links W' = -1/2 z^qhat U of this thread's site that stay
    // inside the block (se has parity 0, so parity sg)
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        if (me.l[mu] == SAP_BS - 1) continue;
        const int e = mu == 0   ? link_entry<0>(sg, me.lidx)
                      : mu == 1 ? link_entry<1>(sg, me.lidx)
                      : mu == 2 ? link_entry<2>(sg, me.lidx)
                                : link_entry<3>(sg, me.lidx);
        cplx<float> u[3][3];
        load_link(f.U, g.V, mu, me.s, u);
        cplx<float> z = QNZ ? link_phase(f.A, g.V, mu, me.s, q) : mk(1.f, 0.f);
        z = -0.5f * z;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) u[a][b] = z * u[a][b];
        sW4[(mu * 4 + 0) * SPLIT_LINKS + e] = make_float4(u[0][0].re, u[0][0].im, u[0][1].re, u[0][1].im);
        sW4[(mu * 4 + 1) * SPLIT_LINKS + e] = make_float4(u[0][2].re, u[0][2].im, u[1][0].re, u[1][0].im);
        sW4[(mu * 4 + 2) * SPLIT_LINKS + e] = make_float4(u[1][1].re, u[1][1].im, u[1][2].re, u[1][2].im);
        sW4[(mu * 4 + 3) * SPLIT_LINKS + e] = make_float4(u[2][0].re, u[2][0].im, u[2][1].re, u[2][1].im);
        sW2[mu * SPLIT_LINKS + e] = make_float2(u[2][2].re, u[2][2].im);
    }

#pragma unroll 1
    for (int ir = 0; ir < nrhs; ++ir) {
        const SplitWork& wk = rhs[ir];
        {
            cplx<float> r[12];
            if (flags & SF_FIRST) {
                load_spinor(wk.eta, g.V, me.s, r);
            } else if (sg == 0) {  // even site: the kept rho
                load_spinor(wk.rho, g.Vh, me.s, r);
            } else {  // odd site: the block solve left no residual
#pragma unroll
                for (int i = 0; i < 12; ++i) r[i] = mk(0.f, 0.f);
            }
            if (flags & SF_CROSS) {  // r -= D_cross delta = r + 1/2 (crossing hops of delta)
                cplx<float> acc[12];
#pragma unroll
                for (int i = 0; i < 12; ++i) acc[i] = mk(0.f, 0.f);
                const int po = 1 - sg;  // parity of the neighbours
                crossing_dir<QNZ, 0>(g, f, wk.delta, q, me, po, acc);
                crossing_dir<QNZ, 1>(g, f, wk.delta, q, me, po, acc);
                crossing_dir<QNZ, 2>(g, f, wk.delta, q, me, po, acc);
                crossing_dir<QNZ, 3>(g, f, wk.delta, q, me, po, acc);
#pragma unroll
                for (int i = 0; i < 12; ++i) r[i] = r[i] + 0.5f * acc[i];
            }
            st_full(sg ? s_t : s_rho, t, r);
        }
        __syncthreads();

        // r_o (this thread's half) stays in registers until the last step; the
        // pair overwrites its own halves of s_t with t_o = M_oo^-1 r_o
        cplx<float> ro[6], v[6], w[6], acc[6], rho[6];
        ld_half(s_t, sg, t, ro);
        clover_half(Cinv, g.V, so.s, sg, sgn, ro, w);
        st_half(s_t, sg, t, w);
        __syncthreads();

        // rho stays in shared memory between steps (fewer live registers)
        cplx<float> de[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) de[i] = mk(0.f, 0.f);
        const int nsteps = 2 * nmr + 2;
#pragma unroll 1
        for (int step = 0; step < nsteps; ++step) {
            const bool odd = (step & 1) != 0;
            const bool last = step == nsteps - 1;
            split_hops<QNZ>(bl, odd ? (last ? s_t : s_rho) : s_t, odd ? so : se, odd ? 1 : 0, sg, sgn, acc);
            // acc = H psi on the sites of this step's parity (the links carry the -1/2)
            if (step == 0) {
                ld_half(s_rho, sg, t, rho);  // r_e
#pragma unroll
                for (int i = 0; i < 6; ++i) rho[i] = rho[i] - acc[i];
                st_half(s_rho, sg, t, rho);
            } else if (last) {
#pragma unroll
                for (int i = 0; i < 6; ++i) v[i] = ro[i] - acc[i];
                clover_half(Cinv, g.V, so.s, sg, sgn, v, w);  // delta_o (s_rho is no longer read)
                st_half(s_rho, sg, t, w);
            } else if (odd) {
                clover_half(Cinv, g.V, so.s, sg, sgn, acc, w);
                st_half(s_t, sg, t, w);
            } else {
                ld_half(s_rho, sg, t, rho);
                clover_half(f.C, g.V, se.s, sg, sgn, rho, w);
#pragma unroll
                for (int i = 0; i < 6; ++i) w[i] = w[i] - acc[i];
                float a_re = 0.f, a_im = 0.f, b = 0.f;
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    a_re += w[i].re * rho[i].re + w[i].im * rho[i].im;
                    a_im += w[i].re * rho[i].im - w[i].im * rho[i].re;
                    b += w[i].re * w[i].re + w[i].im * w[i].im;
                }
                float sums[3];
                // red is next written two steps later, after the barriers that end each step
                block_sum3<float, SPLIT_THREADS, false>(a_re, a_im, b, red, sums);
                if (sums[2] > 0.f) {  // else rho = 0 on the whole block: nothing to add
                    const cplx<float> om = mk(sums[0] / sums[2], sums[1] / sums[2]);
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        de[i] = de[i] + om * rho[i];
                        rho[i] = rho[i] - om * w[i];
                    }
                }
                if (step == nsteps - 2) {
                    st_half(s_t, sg, t, de);  // delta_e for the last step
                    if (flags & SF_KEEP_RHO) {
                        // this thread's half of rho at the even site: components 3 sg + c and 6 + 3 sg + c
                        float2* kr = reinterpret_cast<float2*>(wk.rho);
#pragma unroll
                        for (int h = 0; h < 2; ++h)
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                const int i = 6 * h + 3 * sg + c;
                                kr[2 * ((size_t)(i >> 1) * g.Vh + se.s) + (i & 1)] = make_float2(rho[3 * h + c].re, rho[3 * h + c].im);
                            }
                    }
                } else {
                    st_half(s_rho, sg, t, rho);
                }
            }
            __syncthreads();
        }
        // psi_B += delta on this thread's site: delta_e in s_t, delta_o in s_rho
        cplx<float> d[12];
        ld_full(sg ? s_rho : s_t, t, d);
        if (flags & SF_KEEP_DELTA) store_spinor(wk.delta, g.V, me.s, d);
        if (!(flags & SF_FIRST)) {
            cplx<float> o[12];
            load_spinor(wk.psi, g.V, me.s, o);
#pragma unroll
            for (int i = 0; i < 12; ++i) d[i] = d[i] + o[i];
        }
        store_spinor(wk.psi, g.V, me.s, d);
        if (ir + 1 < nrhs) __syncthreads();  // the next right-hand side reuses the block fields
    }
}

// MULTI: several right-hand sides per launch (else exactly one, and the
// loop over them compiles away)
template <bool QNZ, bool MULTI>
__global__ void __launch_bounds__(SPLIT_THREADS, 2) k_sap_split(const __grid_constant__ Geom g,
                                                                const __grid_constant__ SapGeom sgm, int colour,
                                                                const __grid_constant__ Fields<float> f,
                                                                const float4* __restrict__ Cinv,
                                                                const __grid_constant__ SplitRhsList rl, int flags,
                                                                int nmr, float q) {
    sap_split_body<QNZ>(g, sgm, blockIdx.x, colour, f, Cinv, rl.r, MULTI ? rl.n : 1, flags, nmr, q);
}

// batched form: thread block b works on block (b - cta_begin) of the job
// whose range holds b (one launch serves every job of a batch)
__global__ void __launch_bounds__(SPLIT_THREADS, 2) k_sap_block_batch(const SapJob* __restrict__ jobs, int njobs,
                                                                      int colour, int flags, int nmr) {
    int lo = 0, hi = njobs - 1;
    const int b = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].cta_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    const SapJob& J = jobs[lo];
    const SplitWork wk{J.eta, const_cast<float4*>(J.f.psi), J.delta, J.rho};
    sap_split_body<true>(J.g, J.sg, b - J.cta_begin, colour, J.f, J.Cinv, &wk, 1, flags, nmr, J.q);
}

template <typename R>
size_t sap_smem_bytes() {
    if (sizeof(R) == 4)  // split kernel: interior compound links, two block fields, reduction slots of 8 warps
        return split_link_bytes() + 24 * SAP_HALF * sizeof(float2) + 3 * (SPLIT_THREADS / 32) * sizeof(float);
    return (72 * SAP_HALF + 3 * (SAP_THREADS / 32)) * sizeof(R);
}

// Dynamic shared memory of the split kernel, and an L1/shared carveout just
// large enough for two blocks per SM: the rest of the SM's L1 caches the
// clover blocks that every MR step re-reads.
template <typename K>
int split_attrs(K kernel, size_t smem) {
    int dev = 0, per_sm = 0;
    QXD_CUDA(cudaGetDevice(&dev));
    QXD_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    QXD_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (per_sm > 0) {
        const long need = 2L * ((long)smem + 1024);
        const int pct = (int)std::min(100L, (100 * need + per_sm - 1) / per_sm);
        QXD_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    }
    return QXD_OK;
}

// flags of visit `cy` of colour `colour` out of ncy cycles
int split_flags(int cy, int colour, int ncy) {
    int fl = 0;
    if (cy == 0) fl |= SF_FIRST;
    if (cy > 0 || colour == 1) fl |= SF_CROSS;  // the other colour has a correction
    if (cy + 1 < ncy) fl |= SF_KEEP_RHO;
    if (cy + 1 < ncy || colour == 0) fl |= SF_KEEP_DELTA;
    return fl;
}

// FP64 visit `cy` of colour `colour` out of ncy cycles
template <bool QNZ>
int launch_sap_block64(qxd_lattice* lat, const SapGeom& sg, int cy, int colour, Fields<double> f,
                       const double* Cinv, const double2* eta, int nmr, cudaStream_t st) {
    const size_t smem = sap_smem_bytes<double>();
    const int psi_zero = (cy == 0 && colour == 0) ? 1 : 0;
    QXD_CUDA(cudaFuncSetAttribute(k_sap_block<double, QNZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_sap_block<double, QNZ><<<sg.nhalf, SAP_THREADS, smem, st>>>(lat->g, sg, colour, psi_zero, f, Cinv, eta, nmr,
                                                                   (double)lat->qhat);
    QXD_LAUNCHED("k_sap_block");
    return QXD_OK;
}

// FP32: the ncy cycles for the right-hand sides of rl (one operator)
template <bool QNZ, bool MULTI>
int split_cycles(qxd_lattice* lat, const SapGeom& sg, const SplitRhsList& rl, int ncy, int nmr, cudaStream_t st) {
    const size_t smem = sap_smem_bytes<float>();
    int rc = split_attrs(k_sap_split<QNZ, MULTI>, smem);
    if (rc) return rc;
    const Fields<float> f{nullptr, nullptr, lat->U32, lat->A32, lat->C32};
    for (int cy = 0; cy < ncy; ++cy)
        for (int colour = 0; colour < 2; ++colour) {
            k_sap_split<QNZ, MULTI><<<sg.nhalf, SPLIT_THREADS, smem, st>>>(lat->g, sg, colour, f, lat->Cinv32, rl,
                                                                           split_flags(cy, colour, ncy), nmr,
                                                                           (float)lat->qhat);
            QXD_LAUNCHED("k_sap_split");
        }
    return QXD_OK;
}

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

int sap_apply_multi(qxd_lattice* lat, int nrhs, void* const* outs, const void* const* ins, float4* const* works,
                    int ncy, int nmr, cudaStream_t st) {
    const SapGeom sg = sap_geom(lat->g);
    const size_t V = (size_t)lat->g.V;
    for (int i0 = 0; i0 < nrhs; i0 += SPLIT_MAXR) {
        SplitRhsList rl{};
        rl.n = std::min(SPLIT_MAXR, nrhs - i0);
        for (int i = 0; i < rl.n; ++i)
            rl.r[i] = SplitWork{(const float4*)ins[i0 + i], (float4*)outs[i0 + i], works[i0 + i],
                                works[i0 + i] + (size_t)SPINOR_F4 * V};
        int rc;
        if (rl.n > 1)
            rc = lat->qhat != 0 ? split_cycles<true, true>(lat, sg, rl, ncy, nmr, st)
                                : split_cycles<false, true>(lat, sg, rl, ncy, nmr, st);
        else
            rc = lat->qhat != 0 ? split_cycles<true, false>(lat, sg, rl, ncy, nmr, st)
                                : split_cycles<false, false>(lat, sg, rl, ncy, nmr, st);
        if (rc) return rc;
    }
    return QXD_OK;
}

template <typename R>
int sap_apply(qxd_lattice* lat, SapWork& w, void* out, const void* in, int ncy, int nmr, cudaStream_t st) {
    const Geom& g = lat->g;
    w.sg = sap_geom(g);
    if constexpr (sizeof(R) == 4) {
        // the first visit of each colour writes psi = delta; work fields: delta
        // (V sites) and rho (Vh even sites), kept with the lattice
        if (!lat->sap_r) {
            const cudaError_t e = cudaMalloc(&lat->sap_r, ((size_t)g.V + g.Vh) * SPINOR_F4 * sizeof(float4));
            if (e != cudaSuccess) {
                lat->sap_r = nullptr;
                return cuda_fail(e, "SAP: cudaMalloc(work fields)");
            }
        }
        float4* work = lat->sap_r;
        return sap_apply_multi(lat, 1, &out, &in, &work, ncy, nmr, st);
    } else {
        // psi starts at zero; the first half-cycle writes the blocks of colour 0
        // without reading psi, and the blocks of colour 1 must read zeros there
        QXD_CUDA(cudaMemsetAsync(out, 0, (size_t)g.V * 24 * sizeof(R), st));
        const Fields<double> f{(const double2*)out, nullptr, lat->U64, lat->Zq64, lat->C64};
        for (int cy = 0; cy < ncy; ++cy)
            for (int colour = 0; colour < 2; ++colour) {
                const int rc = lat->qhat != 0
                                   ? launch_sap_block64<true>(lat, w.sg, cy, colour, f, lat->Cinv64,
                                                              (const double2*)in, nmr, st)
                                   : launch_sap_block64<false>(lat, w.sg, cy, colour, f, lat->Cinv64,
                                                               (const double2*)in, nmr, st);
                if (rc) return rc;
            }
        return QXD_OK;
    }
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

void SapGraphCache::clear() {
    for (auto& e : entries) cudaGraphExecDestroy(e.exec);
    entries.clear();
}

void SapGraphCache::release() {
    clear();
    if (cap) cudaStreamDestroy(cap);
    cap = nullptr;
}

namespace {

void launch_batch_set(const SapJob* d_jobs, int njobs, int ctas, int ncy, int nmr, size_t smem, cudaStream_t st) {
    for (int cy = 0; cy < ncy; ++cy)
        for (int colour = 0; colour < 2; ++colour)
            k_sap_block_batch<<<ctas, SPLIT_THREADS, smem, st>>>(d_jobs, njobs, colour, split_flags(cy, colour, ncy),
                                                                 nmr);
}

// the executable graph of this launch set, captured on first use
int batch_graph(SapGraphCache& gc, const SapJob* d_jobs, int njobs, int ctas, int ncy, int nmr, size_t smem,
                cudaGraphExec_t* out) {
    ++gc.tick;
    for (auto& e : gc.entries)
        if (e.table == d_jobs && e.njobs == njobs && e.ctas == ctas && e.ncy == ncy && e.nmr == nmr) {
            e.last = gc.tick;
            ++gc.replays;
            *out = e.exec;
            return QXD_OK;
        }
    if (!gc.cap) QXD_CUDA(cudaStreamCreateWithFlags(&gc.cap, cudaStreamNonBlocking));
    QXD_CUDA(cudaStreamBeginCapture(gc.cap, cudaStreamCaptureModeThreadLocal));
    launch_batch_set(d_jobs, njobs, ctas, ncy, nmr, smem, gc.cap);
    const cudaError_t le = cudaGetLastError();
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(gc.cap, &graph);  // always ends the capture
    if (le != cudaSuccess || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(le != cudaSuccess ? le : ce, "k_sap_block_batch graph capture");
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate (SAP launch set)");
    if ((int)gc.entries.size() >= SapGraphCache::kMax) {
        auto lru = std::min_element(gc.entries.begin(), gc.entries.end(),
                                    [](const SapGraphCache::Entry& a, const SapGraphCache::Entry& b) { return a.last < b.last; });
        cudaGraphExecDestroy(lru->exec);
        gc.entries.erase(lru);
    }
    gc.entries.push_back(SapGraphCache::Entry{d_jobs, njobs, ctas, ncy, nmr, exec, gc.tick});
    ++gc.captures;
    *out = exec;
    return QXD_OK;
}

}  // namespace

int sap_apply_batch(std::vector<SapJob>& jobs, SapJob* d_jobs, int ncy, int nmr, cudaStream_t st,
                    SapGraphCache* graphs) {
    if (jobs.empty()) return QXD_OK;
    int ctas = 0;
    for (auto& J : jobs) {  // the first visit of each colour writes psi without reading it
        J.cta_begin = ctas;
        ctas += J.sg.nhalf;
    }
    QXD_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(SapJob), cudaMemcpyHostToDevice, st));
    const size_t smem = sap_smem_bytes<float>();
    int rc = split_attrs(k_sap_block_batch, smem);
    if (rc) return rc;
    const int njobs = (int)jobs.size();
    if (graphs) {
        cudaGraphExec_t exec = nullptr;
        if ((rc = batch_graph(*graphs, d_jobs, njobs, ctas, ncy, nmr, smem, &exec))) return rc;
        QXD_CUDA(cudaGraphLaunch(exec, st));
        return QXD_OK;
    }
    launch_batch_set(d_jobs, njobs, ctas, ncy, nmr, smem, st);
    QXD_LAUNCHED("k_sap_block_batch");
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

extern "C" int qxd_sap_multi(qxd_lattice* lat, int nrhs, void* const* out, const void* const* in, int ncy, int nmr,
                             void* stream) {
    if (!lat || !out || !in || nrhs < 1) return fail(QXD_ERR_ARG, "qxd_sap_multi: NULL argument or nrhs < 1");
    if (ncy < 1 || nmr < 1) return fail(QXD_ERR_ARG, "qxd_sap_multi: ncy and nmr must be >= 1");
    for (int i = 0; i < nrhs; ++i) {
        if (!out[i] || !in[i]) return fail(QXD_ERR_ARG, "qxd_sap_multi: NULL field");
        for (int j = 0; j < nrhs; ++j)
            if (out[i] == in[j] || (j != i && out[i] == out[j]))
                return fail(QXD_ERR_ARG, "qxd_sap_multi: outputs must differ from each other and from the inputs");
    }
    if (!qxd::clover_ready(lat)) return fail(QXD_ERR_STATE, "qxd_sap_multi: needs qxd_sw_build first");
    int rc = sap_check(lat);
    if (rc) return rc;
    const size_t per = ((size_t)lat->g.V + lat->g.Vh) * SPINOR_F4;  // float4 of one right-hand side's work fields
    if (lat->sap_multi_n < nrhs) {
        if (lat->sap_multi) cudaFree(lat->sap_multi);
        lat->sap_multi = nullptr;
        lat->sap_multi_n = 0;
        const cudaError_t e = cudaMalloc(&lat->sap_multi, per * nrhs * sizeof(float4));
        if (e != cudaSuccess) {
            lat->sap_multi = nullptr;
            return cuda_fail(e, "qxd_sap_multi: cudaMalloc(work fields)");
        }
        lat->sap_multi_n = nrhs;
    }
    std::vector<float4*> works(nrhs);
    for (int i = 0; i < nrhs; ++i) works[i] = lat->sap_multi + per * i;
    cudaStream_t st = stream ? (cudaStream_t)stream : lat->stream;
    return sap_apply_multi(lat, nrhs, out, in, works.data(), ncy, nmr, st);
}
