"""GPU solves of D x = b: plain FP64 GCR (full and even-odd systems) and the
mixed-precision SAP-preconditioned flexible GCR, checked against the oracle
(dense LU on tiny lattices, the oracle's GCR, the oracle's D for the true
residual)."""
import numpy as np
import pytest
import torch

import oracle as O
from qxd_cases import Case, rel_norm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def solve(lat, b, **kw):
    x = torch.zeros_like(b)
    rc, info = lat.solve(x, b, **kw)
    torch.cuda.synchronize()
    return rc, info, x.cpu().numpy()


def true_relres(op, x, b):
    return np.linalg.norm(b - op.apply(x)) / np.linalg.norm(b)


@pytest.mark.parametrize("system", [0, 1])
def test_tiny_solve_matches_dense_lu(system):
    """4 x 4 x 2 x 2 doubled lattice (128 sites): GCR vs dense LU."""
    from paper_1710_08839_gb300 import qxd
    c = Case(T=4, L1=2, L2=2, L3=2, eps=0.5, sigma=0.6, m0=0.2, qhat=-1)
    op = c.oracle()
    b = c.psi.numpy()
    x_lu = np.linalg.solve(O.dense_matrix(op), b.ravel()).reshape(b.shape)
    lat = c.lattice()
    rc, info, x = solve(lat, c.psi.cuda(), tol=1e-12, system=system)
    lat.close()
    assert rc == qxd.QXD_OK and info["true_relres"] <= 1e-12
    assert rel_norm(x, x_lu) < 1e-9
    assert true_relres(op, x, b) < 1e-11


@pytest.mark.parametrize("system", [0, 1])
def test_cfg0_solve_matches_oracle(system):
    """The small workload (T=8, L=4 doubled, q=-1, m0=0.2): FP64 GCR to 1e-12."""
    from paper_1710_08839_gb300 import qxd
    c = Case(T=8, L1=4, L2=4, L3=4, eps=0.4, sigma=0.5, m0=0.2, qhat=-1)
    op = c.oracle()
    b = c.psi.numpy()
    x_ref, it, res = O.gcr(op.apply, b, tol=1e-13)
    assert res < 1e-12
    lat = c.lattice()
    rc, info, x = solve(lat, c.psi.cuda(), tol=1e-12, system=system)
    lat.close()
    assert rc == qxd.QXD_OK, info
    assert true_relres(op, x, b) < 1e-11
    assert rel_norm(x, x_ref) < 1e-9


@pytest.mark.parametrize("inner", ["fp32", "fp64"])
def test_sap_gcr_solve(inner):
    """SAP-preconditioned flexible GCR (4^4 blocks, ncy=5, nmr=5) to 1e-10 on
    an 8 x 16 x 8 x 8 C* lattice; checked with the oracle's D and against the
    plain FP64 even-odd GCR solution."""
    from paper_1710_08839_gb300 import qxd
    c = Case(T=8, L1=8, L2=8, L3=8, qhat=2, m0=0.05)
    op = c.oracle()
    b = c.psi.numpy()
    lat = c.lattice()
    prec = qxd.QXD_FP32 if inner == "fp32" else qxd.QXD_FP64
    rc, info, x = solve(lat, c.psi.cuda(), tol=1e-10, precond=qxd.QXD_PRECOND_SAP, inner_prec=prec)
    rc2, info2, x2 = solve(lat, c.psi.cuda(), tol=1e-12, system=qxd.QXD_SOLVE_EO)
    lat.close()
    assert rc == qxd.QXD_OK, info
    assert info["true_relres"] <= 1e-10
    assert true_relres(op, x, b) < 2e-10
    assert rc2 == qxd.QXD_OK
    assert rel_norm(x, x2) < 1e-8
    assert info["iterations"] < info2["iterations"]


def test_solver_host_buffers_and_zero_source():
    from paper_1710_08839_gb300 import qxd
    c = Case(T=4, L1=2, L2=2, L3=2, m0=0.3, qhat=2)
    lat = c.lattice()
    rc, info, xd = solve(lat, c.psi.cuda(), tol=1e-11)
    xh = torch.zeros_like(c.psi)
    rc2, info2 = lat.solve(xh, c.psi.contiguous(), tol=1e-11)
    assert rc == rc2 == qxd.QXD_OK
    assert np.array_equal(xd, xh.numpy())
    z = torch.zeros_like(c.psi).cuda()
    rc3, info3, x3 = solve(lat, z)
    assert rc3 == qxd.QXD_OK and np.count_nonzero(x3) == 0
    lat.close()


def test_not_converged_is_reported_with_info():
    from paper_1710_08839_gb300 import qxd
    c = Case(T=8, L1=4, L2=4, L3=4, m0=0.05, qhat=-1)
    lat = c.lattice()
    rc, info, x = solve(lat, c.psi.cuda(), tol=1e-12, max_iter=3)
    lat.close()
    assert rc == qxd.QXD_ERR_NOT_CONVERGED
    assert info["iterations"] == 3 and info["true_relres"] > 1e-12
    assert np.count_nonzero(x) > 0


def test_solver_argument_errors():
    from paper_1710_08839_gb300 import qxd
    c = Case(T=4, L1=2, L2=2, L3=2)
    lat = c.lattice()
    b = c.psi.cuda()
    for kw in ({"nkv": 0}, {"nkv": 17}, {"tol": 0.0}, {"precond": 1, "system": 1}, {"precond": 1}):
        with pytest.raises(qxd.QxdError) as e:
            lat.solve(torch.zeros_like(b), b, **kw)
        assert e.value.code == qxd.QXD_ERR_ARG
    lat.close()
