"""Local deflation on the GPU against the FP64 oracle, through the C ABI:
block-orthonormal basis and little operator for the same input fields, and
deflated solves checked with the oracle's D."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import qxd_dfl as DF
import synth
from qxd_cases import Case, rel_max, rel_norm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qxd():
    import __graft_entry__ as ge
    ge.build()
    from paper_1710_08839_gb300 import qxd as q
    return q


# 4^4 blocks need extents that are multiples of 8 and, with C* boundaries,
# N_k/4 + L1/4 even (the Schwarz colouring)
CASES = {
    "cstar": dict(T=8, L1=8, L2=8, L3=8, mask=0b1110, qhat=2, m0=0.1, eps=0.4, sigma=0.4),
    "periodic": dict(T=8, L1=8, L2=8, L3=8, mask=0, qhat=-1, m0=0.05, eps=0.4, sigma=0.4),
}
NS = 4


def _fields(c, ns=NS):
    return [synth.spinor_field(c.T, c.N1, c.L2, c.L3, synth.SEED_SOURCE + 100 + k).reshape(c.V, 4, 3)
            for k in range(ns)]


def _block_neighbour(lat, b, mu, dirn, bs=4):
    bid = DF.block_index(lat, bs)
    site = np.nonzero(bid == b)[0][0]
    for _ in range(bs):
        site = lat.shift(site, mu, dirn)
    return int(bid[site])


@pytest.mark.parametrize("name", sorted(CASES))
def test_basis_and_little_operator_match_oracle(qxd, name):
    c = Case(**CASES[name])
    psi = _fields(c)
    lat = c.lattice()
    lat.dfl_set_basis([p.to(torch.complex128).cuda().contiguous() for p in psi])
    A = lat.dfl_little()
    olat = O.Lattice(c.T, c.L1, c.L2, c.L3, c.mask)
    phi = DF.block_orthonormalize(olat, np.stack([p.numpy() for p in psi]), 4)
    for k in range(NS):
        got = torch.empty(c.V, 4, 3, dtype=torch.complex128, device="cuda")
        lat.dfl_basis(k, got)
        assert rel_max(got.cpu().numpy(), phi[k]) < 2e-5
    Ao = DF.little_operator(c.oracle(), phi, 4)
    nblk = A.shape[0]
    Ao = Ao.reshape(nblk, NS, nblk, NS)
    # the nine couplings of block b, summed per neighbouring block (with two
    # blocks in a direction, b + mu and b - mu are the same block)
    got = np.zeros_like(Ao)
    for b in range(nblk):
        got[b, :, b, :] += A[b, 0]
        for mu in range(4):
            got[b, :, _block_neighbour(olat, b, mu, +1), :] += A[b, 1 + 2 * mu]
            got[b, :, _block_neighbour(olat, b, mu, -1), :] += A[b, 2 + 2 * mu]
    assert rel_max(got, Ao) < 2e-5


@pytest.mark.parametrize("ns", [8, 16, 32, 6])
@pytest.mark.parametrize("name", sorted(CASES))
def test_deflated_solve(qxd, name, ns):
    """Deflated SAP-GCR to 1e-10 through the oracle's D, with subspaces of
    8, 16 and 32 fields (the warp-per-block little operator) and 6 (the
    one-thread-per-row form)."""
    c = Case(**CASES[name])
    lat = c.lattice()
    lat.dfl_subspace(ns, niter=4, ncy=4, seed=7)
    b = c.psi.to(torch.complex128).cuda().contiguous()
    x = torch.zeros_like(b)
    rc, info = lat.solve(x, b, tol=1e-10, precond=qxd.QXD_PRECOND_DFL_SAP, inner_prec=qxd.QXD_FP32)
    assert rc == qxd.QXD_OK, info
    assert info["little_iters"] > 0 and info["true_relres"] <= 1e-10
    r = c.psi.numpy() - c.oracle().apply(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(c.psi.numpy()) < 1e-10
    # the same solution as the undeflated SAP solver
    x2 = torch.zeros_like(b)
    lat.solve(x2, b, tol=1e-10, precond=qxd.QXD_PRECOND_SAP, inner_prec=qxd.QXD_FP32)
    assert rel_norm(x.cpu().numpy(), x2.cpu().numpy()) < 1e-8


def test_deflation_state_and_errors(qxd):
    c = Case(**CASES["cstar"])
    lat = c.lattice()
    b = c.psi.to(torch.complex128).cuda().contiguous()
    x = torch.zeros_like(b)
    kw = dict(precond=qxd.QXD_PRECOND_DFL_SAP, inner_prec=qxd.QXD_FP32)
    with pytest.raises(qxd.QxdError) as e:
        lat.solve(x, b, **kw)
    assert e.value.code == qxd.QXD_ERR_STATE
    with pytest.raises(qxd.QxdError) as e:
        lat.dfl_refresh()
    assert e.value.code == qxd.QXD_ERR_STATE
    for ns in (0, 65):
        with pytest.raises(qxd.QxdError) as e:
            lat.dfl_subspace(ns)
        assert e.value.code == qxd.QXD_ERR_ARG
    lat.dfl_subspace(6, niter=2)
    with pytest.raises(qxd.QxdError) as e:
        lat.solve(x, b, precond=qxd.QXD_PRECOND_DFL_SAP, inner_prec=qxd.QXD_FP64)
    assert e.value.code == qxd.QXD_ERR_ARG
    assert lat.solve(x, b, **kw)[0] == qxd.QXD_OK
    # a new operator makes the little operator stale until refreshed
    lat.set_params(0.3, 1.0, 1.0, 0)
    lat.sw_build()
    with pytest.raises(qxd.QxdError) as e:
        lat.solve(x, b, **kw)
    assert e.value.code == qxd.QXD_ERR_STATE
    lat.dfl_refresh()
    rc, info = lat.solve(x, b, **kw)
    assert rc == qxd.QXD_OK and info["true_relres"] <= 1e-10
    # a lattice whose blocks cannot be coloured is rejected
    c2 = Case(T=8, L1=4, L2=8, L3=8, mask=0b1110, qhat=1)
    l2 = c2.lattice()
    with pytest.raises(qxd.QxdError) as e:
        l2.dfl_subspace(4)
    assert e.value.code == qxd.QXD_ERR_ARG


@pytest.mark.slow
def test_deflated_solve_full_size_near_critical(qxd):
    """64x64x32x32 doubled lattice near its critical mass (m0 = -0.62, where
    the SAP solver needs about 40 steps): the deflated solver reaches the same
    solution with fewer outer steps."""
    c = Case(T=64, L1=32, L2=32, L3=32, mask=0b1110, qhat=2, m0=-0.62, device="cuda")
    lat = c.lattice()
    b = c.psi.to(torch.complex128).cuda().contiguous()
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    rc, i1 = lat.solve(x1, b, tol=1e-10, precond=qxd.QXD_PRECOND_SAP, inner_prec=qxd.QXD_FP32)
    assert rc == qxd.QXD_OK
    lat.dfl_subspace(16, niter=5, ncy=4, seed=3)
    rc, i2 = lat.solve(x2, b, tol=1e-10, precond=qxd.QXD_PRECOND_DFL_SAP, inner_prec=qxd.QXD_FP32)
    assert rc == qxd.QXD_OK and i2["true_relres"] <= 1e-10
    assert i2["iterations"] < i1["iterations"]
    assert float((x2 - x1).norm() / x1.norm()) < 1e-8
