"""Pseudofermion action on the GPU (ln|Det D_oo|, multi-shift CG, rational
factors P_k of Sec. 2.4) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle as O
import pins_rhmc as PR
from qxd_cases import Case, rel_norm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qxd():
    import __graft_entry__ as ge
    ge.build()
    from paper_1710_08839_gb300 import qxd as q
    return q


CASES = {
    "cstar_q2": dict(T=4, L1=4, L2=4, L3=4, mask=0b1110, qhat=2, m0=0.1),
    "cstar_qm1_ragged": dict(T=6, L1=2, L2=6, L3=4, mask=0b1110, qhat=-1, m0=0.2),
    "periodic_q0": dict(T=4, L1=4, L2=4, L3=6, mask=0, qhat=0, m0=0.15),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_sw_logdet_matches_oracle(qxd, name):
    c = Case(**CASES[name])
    eo = O.EvenOdd(c.oracle())
    lat = c.lattice()
    ref_o = O.ln_abs_det_blocks(eo.Doo_blocks)
    ref_e = O.ln_abs_det_blocks(eo.Dee_blocks)
    got_o = lat.sw_logdet(qxd.QXD_SITES_ODD)
    got_e = lat.sw_logdet(qxd.QXD_SITES_EVEN)
    got_a = lat.sw_logdet(qxd.QXD_SITES_ALL)
    assert abs(got_o - ref_o) <= 1e-12 * abs(ref_o)
    assert abs(got_e - ref_e) <= 1e-12 * abs(ref_e)
    assert abs(got_a - (ref_o + ref_e)) <= 1e-12 * abs(ref_o + ref_e)
    # deterministic: the same bits on every call
    assert lat.sw_logdet(qxd.QXD_SITES_ODD) == got_o


@pytest.mark.parametrize("name", sorted(CASES))
def test_mscg_matches_oracle_shifted_solves(qxd, name):
    c = Case(**CASES[name])
    eo = O.EvenOdd(c.oracle())
    lat = c.lattice()
    sig = [0.3, 0.04, 2.5, 1.0]        # base (smallest) not first
    b = c.psi.to(torch.complex128).cuda().contiguous()
    xs = [torch.full_like(b, float("nan")) for _ in sig]
    rc, info, rel = lat.mscg(xs, b, sig, tol=1e-12)
    assert rc == qxd.QXD_OK, info
    assert info["true_relres"] <= 1e-12 and max(rel) == info["true_relres"]
    be = c.psi.numpy()[eo.even]
    odd = eo.odd
    for s, x in zip(sig, xs):
        xh = x.cpu().numpy()
        assert np.all(xh[odd] == 0)
        ref, _, res = O.shifted_solve(eo, be, s, tol=1e-13)
        assert res < 1e-12
        assert rel_norm(xh[eo.even], ref) < 1e-8, s


@pytest.mark.parametrize("k", [1, 2])
def test_rational_apply_matches_oracle_product_form(qxd, k):
    c = Case(**CASES["cstar_q2"])
    eo = O.EvenOdd(c.oracle())
    lat = c.lattice()
    nu, mu = PR.factor_P(k)
    phi = c.psi.to(torch.complex128).cuda().contiguous()
    out = torch.empty_like(phi)
    rc, info = lat.rational_apply(out, phi, nu, mu, tol=1e-12)
    assert rc == qxd.QXD_OK, info
    pe = c.psi.numpy()[eo.even]
    ref = O.rational_apply(eo, pe, nu, mu)
    oh = out.cpu().numpy()
    assert np.all(oh[eo.odd] == 0)
    assert rel_norm(oh[eo.even], ref) < 1e-9
    s_ref = O.vdot(pe, ref).real
    assert abs(info["action"] - s_ref) <= 1e-10 * abs(s_ref)


def test_mscg_layouts_and_host_buffers_agree(qxd):
    c = Case(**CASES["cstar_qm1_ragged"])
    lat = c.lattice()
    sig = [0.05, 0.5]
    b = c.psi.to(torch.complex128).cuda().contiguous()
    x_lex = [torch.empty_like(b) for _ in sig]
    assert lat.mscg(x_lex, b, sig)[0] == qxd.QXD_OK
    # host buffers
    bh = c.psi.to(torch.complex128).contiguous()
    x_host = [torch.empty_like(bh) for _ in sig]
    assert lat.mscg(x_host, bh, sig)[0] == qxd.QXD_OK
    # native layout
    nbytes = lat.spinor_bytes(qxd.QXD_FP64)
    bn = torch.empty(nbytes // 16, dtype=torch.complex128, device="cuda")
    lat.pack(bn, b, qxd.QXD_FP64)
    x_nat = [torch.empty_like(bn) for _ in sig]
    assert lat.mscg(x_nat, bn, sig, native=True)[0] == qxd.QXD_OK
    for j in range(len(sig)):
        back = torch.empty_like(b)
        lat.unpack(back, x_nat[j], qxd.QXD_FP64)
        torch.cuda.synchronize()
        assert torch.equal(x_lex[j].cpu(), x_host[j])
        assert torch.equal(x_lex[j], back)


def test_mscg_edge_cases_and_errors(qxd):
    c = Case(**CASES["cstar_q2"])
    lat = c.lattice()
    b = c.psi.to(torch.complex128).cuda().contiguous()
    x = [torch.empty_like(b)]
    # zero source: zero solution, nothing to iterate
    z = torch.zeros_like(b)
    rc, info, rel = lat.mscg(x, z, [0.1])
    assert rc == qxd.QXD_OK and info["iterations"] == 0 and torch.count_nonzero(x[0]) == 0
    # not converged within max_iter: solution and info still written
    rc, info, rel = lat.mscg(x, b, [0.01], max_iter=3)
    assert rc == qxd.QXD_ERR_NOT_CONVERGED and info["iterations"] == 3 and rel[0] > 1e-10
    assert torch.isfinite(x[0]).all()
    # one shift equals plain CG on the base system, whatever else is listed
    x1 = [torch.empty_like(b)]
    x2 = [torch.empty_like(b), torch.empty_like(b)]
    lat.mscg(x1, b, [0.2])
    lat.mscg(x2, b, [0.2, 3.0])
    assert torch.equal(x1[0], x2[0])
    for bad in ([], [-1.0], [float("nan")], [0.1] * 17):
        with pytest.raises(qxd.QxdError) as e:
            lat.mscg([torch.empty_like(b) for _ in bad], b, bad)
        assert e.value.code == qxd.QXD_ERR_ARG
    with pytest.raises(qxd.QxdError) as e:
        lat.rational_apply(torch.empty_like(b), b, [0.5, 0.6], [0.3, 0.3])
    assert e.value.code == qxd.QXD_ERR_ARG
    # FP32 fields are not accepted
    p = qxd.qxd_mscg_defaults()
    p.flags = qxd.QXD_FP32
    with pytest.raises(qxd.QxdError) as e:
        qxd.qxd_mscg(lat.handle, [0.1], [x[0].data_ptr()], b.data_ptr(), p)
    assert e.value.code == qxd.QXD_ERR_ARG
    # before sw_build
    l2 = qxd.Lattice(c.T, c.L1, c.L2, c.L3, c.mask)
    l2.set_gauge(c.su3.cuda(), c.ang.cuda())
    l2.set_params(c.m0, c.csw, c.cswqed, c.qhat)
    for call in (lambda: l2.sw_logdet(), lambda: l2.mscg(x, b, [0.1])):
        with pytest.raises(qxd.QxdError) as e:
            call()
        assert e.value.code == qxd.QXD_ERR_STATE


def _g5(f):
    g = f.clone()
    g[..., 2:, :] *= -1
    return g


@pytest.mark.slow
def test_rational_apply_full_size_properties(qxd):
    """64x64x32x32 doubled lattice (the 64 x 32^3 lattice of the paper, C*
    in three directions), Table 2's P_1: every shift's residual checked
    through the public FP64 D_hat entry point, and the action against
    <phi, P phi> formed from the output."""
    c = Case(T=64, L1=32, L2=32, L3=32, mask=0b1110, qhat=2, m0=0.05, device="cuda")
    lat = c.lattice()
    nu, mu = PR.factor_P(1)
    phi = c.psi.to(torch.complex128).cuda().contiguous()
    out = torch.empty_like(phi)
    rc, info = lat.rational_apply(out, phi, nu, mu, tol=1e-10)
    assert rc == qxd.QXD_OK and info["true_relres"] <= 1e-10, info
    V = c.V
    even = torch.zeros(V, dtype=torch.bool, device="cuda")
    sh = (c.T, c.N1, c.L2, c.L3)
    co = torch.stack(torch.meshgrid(*[torch.arange(n, device="cuda") for n in sh], indexing="ij"), -1).reshape(V, 4)
    even = co.sum(-1) % 2 == 0
    pe = phi.reshape(V, 4, 3).clone()
    pe[~even] = 0
    act = torch.vdot(pe.flatten(), out.reshape(V, 4, 3).flatten()).real.item()
    assert abs(act - info["action"]) <= 1e-11 * abs(act)
    # one shift by multi-shift CG, residual through qxd_Dhat (FP64, lexicographic)
    s = float(mu[-1]) ** 2
    x = [torch.empty_like(phi)]
    rc, info2, rel = lat.mscg(x, phi, [s], tol=1e-10)
    assert rc == qxd.QXD_OK
    t = torch.empty_like(phi)
    w = torch.empty_like(phi)
    lat.Dhat(t, x[0])
    lat.Dhat(w, _g5(t.reshape(V, 4, 3)).reshape(phi.shape).contiguous())
    res = _g5(w.reshape(V, 4, 3)) + s * x[0].reshape(V, 4, 3) - pe
    res[~even] = 0
    assert (res.norm() / pe.norm()).item() <= 1e-9


@pytest.mark.parametrize("name", ["cstar_q2", "periodic_q0"])
def test_mixed_precision_mscg_matches_oracle(qxd, name):
    """FP32 operator with FP64 reliable updates and per-shift refinement:
    the same solutions (to the cond * tol bound) and true residuals <= tol."""
    c = Case(**CASES[name])
    eo = O.EvenOdd(c.oracle())
    lat = c.lattice()
    sig = [0.3, 0.04, 2.5, 1.0]
    b = c.psi.to(torch.complex128).cuda().contiguous()
    xs = [torch.empty_like(b) for _ in sig]
    rc, info, rel = lat.mscg(xs, b, sig, tol=1e-12, prec=qxd.QXD_FP32)
    assert rc == qxd.QXD_OK, info
    assert max(rel) <= 1e-12
    be = c.psi.numpy()[eo.even]
    for s, x in zip(sig, xs):
        xh = x.cpu().numpy()
        assert np.all(xh[eo.odd] == 0)
        ref, _, _ = O.shifted_solve(eo, be, s, tol=1e-13)
        assert rel_norm(xh[eo.even], ref) < 1e-8, s


def test_mixed_precision_rational_apply(qxd):
    c = Case(**CASES["cstar_qm1_ragged"])
    eo = O.EvenOdd(c.oracle())
    lat = c.lattice()
    nu, mu = PR.factor_P(1)
    phi = c.psi.to(torch.complex128).cuda().contiguous()
    out = torch.empty_like(phi)
    rc, info = lat.rational_apply(out, phi, nu, mu, tol=1e-12, prec=qxd.QXD_FP32)
    assert rc == qxd.QXD_OK and info["true_relres"] <= 1e-12, info
    pe = c.psi.numpy()[eo.even]
    ref = O.rational_apply(eo, pe, nu, mu)
    assert rel_norm(out.cpu().numpy()[eo.even], ref) < 1e-9
    # a bad delta is an argument error
    with pytest.raises(qxd.QxdError) as e:
        lat.rational_apply(out, phi, nu, mu, prec=qxd.QXD_FP32, delta=1.5)
    assert e.value.code == qxd.QXD_ERR_ARG


@pytest.mark.slow
def test_mixed_precision_rational_apply_full_size(qxd):
    """64x64x32x32 doubled lattice, Table 2's P_1: the FP32-operator path
    gives the FP64 result (to the tolerance) with true residuals <= tol."""
    c = Case(T=64, L1=32, L2=32, L3=32, mask=0b1110, qhat=-1, m0=0.05, device="cuda")
    lat = c.lattice()
    nu, mu = PR.factor_P(1)
    phi = c.psi.to(torch.complex128).cuda().contiguous()
    o64, o32 = torch.empty_like(phi), torch.empty_like(phi)
    rc, i64 = lat.rational_apply(o64, phi, nu, mu, tol=1e-10)
    assert rc == qxd.QXD_OK
    rc, i32 = lat.rational_apply(o32, phi, nu, mu, tol=1e-10, prec=qxd.QXD_FP32)
    assert rc == qxd.QXD_OK and i32["true_relres"] <= 1e-10
    assert float((o32 - o64).norm() / o64.norm()) < 1e-9
    assert abs(i32["action"] - i64["action"]) <= 1e-10 * abs(i64["action"])
