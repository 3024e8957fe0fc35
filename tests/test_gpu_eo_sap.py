"""GPU parity of the even-odd operator (Sec. 2.4) and of the SAP
preconditioner against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from qxd_cases import Case, rel_max, rel_norm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


EO_CASES = {
    "cfg0_q-1": dict(T=8, L1=4, L2=4, L3=4, eps=0.4, sigma=0.5, m0=0.2, qhat=-1),
    "ragged_q2": dict(T=6, L1=6, L2=4, L3=2, qhat=2, csw=1.9, cswqed=0.7),
    "periodic_q0": dict(T=4, L1=4, L2=6, L3=4, mask=0, qhat=0),
}


def to_dev(x, dt):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()


@pytest.mark.parametrize("name", list(EO_CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_even_odd_operators(name, prec):
    c = Case(**EO_CASES[name])
    op = c.oracle()
    eo = O.EvenOdd(op)
    lat = c.lattice()
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    check = (lambda a, b: rel_max(a, b) < 1e-13) if prec == "fp64" else (lambda a, b: rel_norm(a, b) < 1e-5)
    psi = c.psi.numpy()
    x = to_dev(psi, dt)
    # D_hat on the even sites, zeros on the odd sites
    y = torch.empty_like(x)
    lat.Dhat(y, x)
    yh = y.cpu().numpy().astype(np.complex128)
    assert check(yh[eo.even], eo.D_hat(psi[eo.even]))
    assert np.count_nonzero(yh[eo.odd]) == 0
    # b_hat_e = b_e - D_eo D_oo^-1 b_o
    lat.eo_prepare(y, x)
    assert check(y.cpu().numpy()[eo.even], eo.prepare_source(psi))
    # x_o = D_oo^-1 (b_o - D_oe x_e)
    rng = np.random.default_rng(5)
    xe = rng.normal(size=(c.V, 4, 3)) + 1j * rng.normal(size=(c.V, 4, 3))
    xd = to_dev(xe, dt)
    xe_in = xd.cpu().numpy().astype(np.complex128)
    lat.eo_reconstruct(xd, x)
    full = eo.reconstruct(xe[eo.even], psi)
    got = xd.cpu().numpy().astype(np.complex128)
    assert check(got[eo.odd], full[eo.odd])
    assert np.array_equal(got[eo.even], xe_in[eo.even])
    lat.close()


SAP_CASES = {
    # smallest C* lattice the 4^4 block colouring admits: 8 x 16 x 8 x 8
    "cstar_8x16x8x8_q2": dict(T=8, L1=8, L2=8, L3=8, qhat=2, m0=0.3),
    # qhat = 0: the kernels' template without the U(1) phases
    "cstar_8x16x8x8_q0": dict(T=8, L1=8, L2=8, L3=8, qhat=0, m0=0.1),
    "periodic_8x8x8x8_q-1": dict(T=8, L1=8, L2=8, L3=8, mask=0, qhat=-1, m0=0.1),
}


@pytest.mark.parametrize("ncy,nmr", [(2, 3), (5, 5)])
@pytest.mark.parametrize("name", list(SAP_CASES))
def test_sap_matches_oracle(name, ncy, nmr):
    """qxd_sap against the oracle's Schwarz method, FP64 to 1e-12 relative
    max and FP32 to 1e-5 relative norm; (5, 5) is the solver workload's
    setting (5 cycles, 5 minimal-residual steps)."""
    c = Case(**SAP_CASES[name])
    op = c.oracle()
    ref = O.sap(op, c.psi.numpy(), ncy, nmr)
    lat = c.lattice()
    for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 1e-5)):
        x = c.psi.to(dt).cuda()
        y = torch.empty_like(x)
        lat.sap(y, x, ncy=ncy, nmr=nmr)
        torch.cuda.synchronize()
        got = y.cpu().numpy().astype(np.complex128)
        err = rel_max(got, ref) if dt == torch.complex128 else rel_norm(got, ref)
        assert err < tol, (dt, err)
    lat.close()


def test_sap_rejects_incompatible_lattice():
    from paper_1710_08839_gb300 import qxd
    c = Case(T=8, L1=4, L2=4, L3=4)   # 8 x 8 x 4 x 4: extents not multiples of 8
    lat = c.lattice()
    x = c.psi.cuda()
    with pytest.raises(qxd.QxdError) as e:
        lat.sap(torch.empty_like(x), x)
    assert e.value.code == qxd.QXD_ERR_ARG
    lat.close()


@pytest.mark.parametrize("name", ["cstar_8x16x8x8_q2", "cstar_8x16x8x8_q0"])
def test_sap_multi_equals_sap_per_rhs(name):
    """qxd_sap_multi (several right-hand sides per launch, links staged once
    per block for all of them) gives each right-hand side the bits of
    qxd_sap alone; the first is also checked against the oracle."""
    from paper_1710_08839_gb300 import qxd
    c = Case(**SAP_CASES[name])
    lat = c.lattice()
    rng = np.random.default_rng(17)
    srcs = [c.psi] + [torch.from_numpy(rng.normal(size=(c.V, 4, 3)) + 1j * rng.normal(size=(c.V, 4, 3)))
                      for _ in range(3)]
    nb = lat.spinor_bytes(qxd.QXD_FP32)
    ins, singles = [], []
    for s_ in srcs:
        xn = torch.empty(nb, dtype=torch.uint8, device="cuda")
        lat.pack(xn, s_.to(torch.complex64).cuda(), qxd.QXD_FP32)
        ins.append(xn)
        yn = torch.empty_like(xn)
        lat.sap(yn, xn, 5, 5, native=True, prec=qxd.QXD_FP32)
        singles.append(yn)
    outs = [torch.empty_like(x) for x in ins]
    lat.sap_multi(outs, ins, 5, 5)
    torch.cuda.synchronize()
    for o, s_ in zip(outs, singles):
        assert torch.equal(o, s_)
    y = torch.empty(c.V, 4, 3, dtype=torch.complex64, device="cuda")
    lat.unpack(y, outs[0], qxd.QXD_FP32)
    ref = O.sap(c.oracle(), c.psi.numpy(), 5, 5)
    assert rel_norm(y.cpu().numpy().astype(np.complex128), ref) < 1e-5
    lat.close()
