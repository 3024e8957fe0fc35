"""Gauge observables and the Wilson flow on the GPU against the FP64 oracle,
through the C ABI."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import qxd_flow as F
from qxd_cases import Case, rel_max, rel_norm

pytestmark = pytest.mark.gpu

Q_EL = 1.0 / 6.0


@pytest.fixture(scope="module")
def qxd():
    import __graft_entry__ as ge
    ge.build()
    from paper_1710_08839_gb300 import qxd as q
    return q


CASES = {
    "cstar": dict(T=4, L1=4, L2=4, L3=4, mask=0b1110, qhat=2, m0=0.1, eps=0.5, sigma=0.6),
    "cstar_ragged": dict(T=6, L1=2, L2=6, L3=4, mask=0b1110, qhat=-1, m0=0.2, eps=0.6, sigma=0.5),
    "cstar12": dict(T=4, L1=4, L2=4, L3=6, mask=0b0110, qhat=1, m0=0.2, eps=0.4, sigma=0.4),
    "periodic": dict(T=4, L1=4, L2=6, L3=4, mask=0, qhat=0, m0=0.15, eps=0.5, sigma=0.7),
}


def _oracle_lattice(c):
    return O.Lattice(c.T, c.L1, c.L2, c.L3, c.mask)


def _oracle_gauge(c):
    return O.GaugeField.from_physical(_oracle_lattice(c), c.su3.numpy(), c.ang.numpy())


@pytest.mark.parametrize("name", sorted(CASES))
def test_observables_match_oracle(qxd, name):
    c = Case(**CASES[name])
    lat = c.lattice()
    got = lat.gauge_observables(Q_EL)
    ref = F.observables(_oracle_lattice(c), _oracle_gauge(c), Q_EL)
    assert abs(got[0] - ref[0]) <= 1e-12 * ref[0]
    assert abs(got[1] - ref[1]) <= 1e-12 * ref[1]
    # Q_top is a sum of terms of either sign: compare against the size of E V
    assert abs(got[2] - ref[2]) <= 1e-12 * ref[0] * c.V
    # a view sees the same field
    v = lat.view()
    assert v.gauge_observables(Q_EL) == got


@pytest.mark.parametrize("name", sorted(CASES))
def test_flow_matches_oracle_through_D(qxd, name):
    """Flow three steps; D (FP64 and FP32) built on the flowed field agrees
    with the oracle's operator on its own flowed field, and so do the
    observables at t = 3 eps."""
    c = Case(**CASES[name])
    lat = c.lattice()
    eps, n = 0.03, 3
    lat.wflow(eps, n)
    olat = _oracle_lattice(c)
    gf = F.wilson_flow(olat, _oracle_gauge(c), eps, n)
    got = lat.gauge_observables(Q_EL)
    ref = F.observables(olat, gf, Q_EL)
    assert abs(got[0] - ref[0]) <= 1e-11 * ref[0]
    assert abs(got[1] - ref[1]) <= 1e-11 * ref[1]
    assert abs(got[2] - ref[2]) <= 1e-11 * ref[0] * c.V
    # the clover term is stale until rebuilt
    psi = c.psi.to(torch.complex128).cuda().contiguous()
    out = torch.empty_like(psi)
    with pytest.raises(qxd.QxdError) as e:
        lat.Dw(out, psi)
    assert e.value.code == qxd.QXD_ERR_STATE
    lat.sw_build()
    op = O.Dirac(olat, gf, c.m0, c.csw, c.cswqed, c.qhat)
    ref_d = op.apply(c.psi.numpy())
    lat.Dw(out, psi)
    torch.cuda.synchronize()
    assert rel_max(out.cpu().numpy(), ref_d) < 1e-12
    psi32 = c.psi.to(torch.complex64).cuda().contiguous()
    out32 = torch.empty_like(psi32)
    lat.Dw(out32, psi32)
    torch.cuda.synchronize()
    assert rel_norm(out32.cpu().numpy(), ref_d) < 1e-5


def test_flow_errors_and_views(qxd):
    c = Case(**CASES["cstar"])
    lat = c.lattice()
    v = lat.view()
    v.set_params(0.3, 1.0, 1.0, 2)
    v.sw_build()
    with pytest.raises(qxd.QxdError) as e:
        v.wflow(0.01, 1)
    assert e.value.code == qxd.QXD_ERR_STATE
    for eps, n in ((0.01, -1), (float("nan"), 1)):
        with pytest.raises(qxd.QxdError) as e:
            lat.wflow(eps, n)
        assert e.value.code == qxd.QXD_ERR_ARG
    with pytest.raises(qxd.QxdError) as e:
        lat.gauge_observables(0.0)
    assert e.value.code == qxd.QXD_ERR_ARG
    # zero steps change nothing: the clover terms stay valid
    before = lat.gauge_observables(Q_EL)
    lat.wflow(0.01, 0)
    psi = c.psi.to(torch.complex128).cuda().contiguous()
    out = torch.empty_like(psi)
    lat.Dw(out, psi)
    v.Dw(out, psi)
    assert lat.gauge_observables(Q_EL) == before
    # a flow of the parent makes the view's clover term stale too
    lat.wflow(0.01, 1)
    with pytest.raises(qxd.QxdError) as e:
        v.Dw(out, psi)
    assert e.value.code == qxd.QXD_ERR_STATE
    assert v.gauge_observables(Q_EL) == lat.gauge_observables(Q_EL)
    # flowing forward then backward returns to the start (RK3 error only)
    lat.wflow(-0.01, 1)
    after = lat.gauge_observables(Q_EL)
    assert abs(after[0] - before[0]) < 1e-6 * before[0]


@pytest.mark.slow
def test_flow_full_size_properties(qxd):
    """Doubled 64x64x32x32 C* lattice (the paper's 64 x 32^3): along the flow
    both action densities fall monotonically, Q_top stays finite and the
    operator on the flowed field is still built (admissible, invertible
    clover)."""
    c = Case(T=64, L1=32, L2=32, L3=32, mask=0b1110, qhat=2, m0=0.05, device="cuda")
    lat = c.lattice()
    obs = [lat.gauge_observables(Q_EL)]
    for _ in range(4):
        lat.wflow(0.02, 5)
        obs.append(lat.gauge_observables(Q_EL))
    e = np.array(obs)
    assert np.all(np.diff(e[:, 0]) < 0) and np.all(np.diff(e[:, 1]) < 0)
    assert np.all(np.isfinite(e))
    lat.sw_build()
