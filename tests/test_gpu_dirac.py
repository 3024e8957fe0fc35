"""GPU parity: D through the C ABI (FP64 and FP32) against the FP64 oracle.

Tolerances: FP64 relative max error 1e-13, FP32 relative norm error 1e-5
(relative max error = max|a-b| / max|b| over all reals)."""
import numpy as np
import pytest
import torch

import oracle as O
import pins as P
from qxd_cases import Case, rel_max, rel_norm

pytestmark = pytest.mark.gpu

TOL64 = 1e-13
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def gpu_apply(lat, psi, prec):
    from paper_1710_08839_gb300 import qxd
    x = psi.to(torch.complex64 if prec == qxd.QXD_FP32 else torch.complex128).cuda().contiguous()
    y = torch.empty_like(x)
    lat.Dw(y, x)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128)


CASES = {
    # the small workload: T=8, L=4, C* in x,y,z, eps 0.4, sigma 0.5, q=-1, m0 0.2
    "cfg0_q-1": dict(T=8, L1=4, L2=4, L3=4, eps=0.4, sigma=0.5, m0=0.2, qhat=-1),
    "cfg0_q0": dict(T=8, L1=4, L2=4, L3=4, eps=0.4, sigma=0.5, m0=0.2, qhat=0),
    "cfg0_q2": dict(T=8, L1=4, L2=4, L3=4, eps=0.4, sigma=0.5, m0=0.2, qhat=2),
    "tiny_64": dict(T=2, L1=2, L2=2, L3=2, eps=0.5, sigma=0.6, qhat=2),
    "tiny_128": dict(T=4, L1=2, L2=2, L3=2, eps=0.5, sigma=0.6, qhat=-1),
    "ragged_576": dict(T=6, L1=6, L2=4, L3=2, qhat=2, csw=1.9, cswqed=0.7),
    "cstar_xy": dict(T=4, L1=4, L2=6, L3=4, mask=0b0110, qhat=-1),
    "cstar_x": dict(T=4, L1=4, L2=4, L3=6, mask=0b0010, qhat=2),
    "periodic": dict(T=4, L1=4, L2=6, L3=4, mask=0, qhat=-1),
    "rough": dict(T=4, L1=4, L2=4, L3=4, eps=1.5, sigma=2.0, qhat=3, csw=2.0, cswqed=1.5),
}


@pytest.mark.parametrize("name", list(CASES))
def test_dirac_parity(name):
    from paper_1710_08839_gb300 import qxd
    c = Case(**CASES[name])
    ref = c.oracle().apply(c.psi.numpy())
    lat = c.lattice()
    y64 = gpu_apply(lat, c.psi, qxd.QXD_FP64)
    y32 = gpu_apply(lat, c.psi, qxd.QXD_FP32)
    lat.close()
    assert rel_max(y64, ref) < TOL64
    assert rel_norm(y32, ref) < TOL32


def test_multi_chunk_sweep_sampled():
    """A lattice whose sweep has several x2 chunks (N1*N2*N3 > 64K sites, so
    the x2 extent is cut into chunks): FP64 and FP32 against the oracle on 3000
    sampled sites plus every site of the rows next to the chunk boundary."""
    from paper_1710_08839_gb300 import qxd
    c = Case(T=4, L1=8, L2=128, L3=64, qhat=2)
    lat = c.lattice()
    y64 = gpu_apply(lat, c.psi, qxd.QXD_FP64)
    y32 = gpu_apply(lat, c.psi, qxd.QXD_FP32)
    lat.close()
    rng = np.random.default_rng(0)
    olat = O.Lattice(c.T, c.L1, c.L2, c.L3, c.mask)
    x2 = olat.coords(olat.all_sites())[:, 2]
    rows = np.nonzero(np.isin(x2, (0, 63, 64, 127)))[0]
    idx = np.union1d(rng.choice(c.V, size=3000, replace=False), rows[::7])
    ref = c.oracle().apply_at(c.psi.numpy(), idx)
    assert rel_max(y64[idx], ref) < TOL64
    assert rel_norm(y32[idx], ref) < TOL32


def test_host_pointer_path_matches_device_path():
    from paper_1710_08839_gb300 import qxd
    c = Case(T=8, L1=4, L2=4, L3=4, qhat=-1)
    lat = c.lattice()
    for prec, dt in ((qxd.QXD_FP64, torch.complex128), (qxd.QXD_FP32, torch.complex64)):
        x = c.psi.to(dt).contiguous()
        yh = torch.empty_like(x)
        lat.Dw(yh, x)                      # host buffers
        yd = torch.empty_like(x.cuda())
        lat.Dw(yd, x.cuda())               # device buffers
        torch.cuda.synchronize()
        assert torch.equal(yh, yd.cpu())
        # page-locked buffers: read and written by the kernels directly, also
        # when only one of the two is page-locked
        xp = x.pin_memory()
        for yp in (torch.empty_like(x).pin_memory(), torch.empty_like(x)):
            yp.zero_()
            lat.Dw(yp, xp)
            assert torch.equal(yp, yd.cpu())
        yp = torch.empty_like(x).pin_memory()
        lat.Dw(yp, x)
        assert torch.equal(yp, yd.cpu())
    lat.close()


@pytest.mark.parametrize("T", [2, 6, 10, 14])
def test_pipelined_host_path_matches_device_path(T):
    """Page-locked input and output: qxd_Dw pipelines reading, applying and
    writing over slabs of x0 planes (3, 5 and 7 slabs for T = 6, 10, 14; T = 2
    cannot be cut and takes the unpipelined path). Same bits as the device
    path, and the oracle's D."""
    from paper_1710_08839_gb300 import qxd
    c = Case(T=T, L1=4, L2=4, L3=2, qhat=2)
    lat = c.lattice()
    ref = c.oracle().apply(c.psi.numpy())
    for prec, dt in ((qxd.QXD_FP64, torch.complex128), (qxd.QXD_FP32, torch.complex64)):
        x = c.psi.to(dt).contiguous()
        yd = torch.empty_like(x.cuda())
        lat.Dw(yd, x.cuda())
        xp, yp = x.pin_memory(), torch.full_like(x, float("nan")).pin_memory()
        for _ in range(2):
            lat.Dw(yp, xp)
            torch.cuda.synchronize()
            assert torch.equal(yp, yd.cpu())
        got = yp.numpy().astype(np.complex128)
        assert (rel_max(got, ref) < TOL64) if prec == qxd.QXD_FP64 else (rel_norm(got, ref) < TOL32)
    lat.close()


def test_native_layout_roundtrip_and_apply():
    from paper_1710_08839_gb300 import qxd
    c = Case(T=4, L1=4, L2=4, L3=4, qhat=2)
    lat = c.lattice()
    for prec, dt in ((qxd.QXD_FP64, torch.complex128), (qxd.QXD_FP32, torch.complex64)):
        x = c.psi.to(dt).cuda().contiguous()
        nb = lat.spinor_bytes(prec)
        xn = torch.empty(nb, dtype=torch.uint8, device="cuda")
        yn = torch.empty_like(xn)
        lat.pack(xn, x, prec)
        back = torch.empty_like(x)
        lat.unpack(back, xn, prec)
        assert torch.equal(back, x)
        lat.Dw(yn, xn, prec=prec, native=True)
        y = torch.empty_like(x)
        lat.unpack(y, yn, prec)
        ylex = torch.empty_like(x)
        lat.Dw(ylex, x)
        torch.cuda.synchronize()
        assert torch.equal(y, ylex)
    lat.close()


def test_zero_source_gives_zero():
    c = Case(T=4, L1=2, L2=2, L3=2)
    lat = c.lattice()
    x = torch.zeros(c.V, 4, 3, dtype=torch.complex128, device="cuda")
    y = torch.full_like(x, 7.0)
    lat.Dw(y, x)
    assert torch.count_nonzero(y) == 0
    lat.close()


# --- pins re-run through the GPU path ------------------------------------


def test_gpu_free_field_plane_waves():
    """U = 1, A = 0 on the C* lattice: D on plane waves of the shifted torus."""
    from paper_1710_08839_gb300 import qxd
    T, L1, L2, L3 = 4, 4, 6, 2
    lo = O.Lattice(T, L1, L2, L3, 0b1110)
    lat = qxd.Lattice(T, L1, L2, L3, 0b1110)
    su3 = torch.eye(3, dtype=torch.complex128).expand(T, L1, L2, L3, 4, 3, 3).contiguous()
    lat.set_gauge(su3.cuda(), torch.zeros(T, L1, L2, L3, 4, dtype=torch.float64, device="cuda"))
    m0 = 0.3
    lat.set_params(m0, 1.3, 0.7, 2)
    lat.sw_build()
    rng = np.random.default_rng(1)
    for _ in range(4):
        p = P.allowed_momentum(lo, rng.integers(-5, 6, size=4))
        u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        pw = P.plane_wave(lo, p, u)
        y = gpu_apply(lat, torch.from_numpy(pw), qxd.QXD_FP64)
        expect = P.plane_wave(lo, p, P.free_symbol(p, m0) @ u)
        assert np.abs(y - expect).max() < 1e-12
    lat.close()


def test_gpu_gamma5_hermiticity_and_mirror_identity():
    """<chi, g5 D phi> = <g5 D chi, phi>; T D[U*,z*] T^-1 = D[U,z] (Eq. (26))."""
    from paper_1710_08839_gb300 import qxd
    c = Case(T=4, L1=4, L2=4, L3=4, qhat=2, eps=0.6, sigma=0.8)
    lat = c.lattice()
    rng = np.random.default_rng(2)
    chi = torch.from_numpy(P.random_spinor(rng, (c.V,)))
    phi = torch.from_numpy(P.random_spinor(rng, (c.V,)))
    G5 = np.diag([1, 1, -1, -1]).astype(complex)
    Dphi = gpu_apply(lat, phi, qxd.QXD_FP64)
    Dchi = gpu_apply(lat, chi, qxd.QXD_FP64)
    a = np.vdot(chi.numpy(), O.spin_mul(G5, Dphi))
    b = np.vdot(O.spin_mul(G5, Dchi), phi.numpy())
    assert abs(a - b) / abs(a) < 1e-12
    # conjugated field on a second lattice
    latc = Case.__new__(Case)
    latc.__dict__.update(c.__dict__)
    latc.su3 = c.su3.conj().resolve_conj()
    latc.ang = -c.ang
    lc = latc.lattice()
    lo = O.Lattice(c.T, c.L1, c.L2, c.L3, c.mask)
    tr = lo.translate(lo.all_sites())
    lhs = gpu_apply(lc, phi[tr], qxd.QXD_FP64)[tr]
    assert rel_max(lhs, Dphi) < 1e-13
    lat.close()
    lc.close()


# --- errors ------------------------------------------------------------------


def test_state_and_argument_errors():
    from paper_1710_08839_gb300 import qxd
    lat = qxd.Lattice(4, 2, 2, 2, 0b1110)
    x = torch.zeros(lat.V, 4, 3, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(qxd.QxdError) as e:
        lat.Dw(y, x)
    assert e.value.code == qxd.QXD_ERR_STATE
    with pytest.raises(qxd.QxdError) as e:
        lat.sw_build()
    assert e.value.code == qxd.QXD_ERR_STATE
    # non-SU(3) links are rejected
    su3 = 2 * torch.eye(3, dtype=torch.complex128).expand(4, 2, 2, 2, 4, 3, 3).contiguous()
    with pytest.raises(qxd.QxdError) as e:
        lat.set_gauge(su3.cuda(), torch.zeros(4, 2, 2, 2, 4, dtype=torch.float64, device="cuda"))
    assert e.value.code == qxd.QXD_ERR_ARG
    # in == out
    c = Case(T=4, L1=2, L2=2, L3=2)
    l2 = c.lattice()
    with pytest.raises(qxd.QxdError) as e:
        l2.Dw(x, x)
    assert e.value.code == qxd.QXD_ERR_ARG
    l2.close()
    lat.close()


def test_extended_checked_admissibility():
    from paper_1710_08839_gb300 import qxd
    c = Case(T=4, L1=2, L2=2, L3=2, qhat=1)
    lo = O.Lattice(c.T, c.L1, c.L2, c.L3, c.mask)
    U, A = O.GaugeField.from_physical(lo, c.su3.numpy(), c.ang.numpy()).extended_arrays()
    lat = qxd.Lattice(c.T, c.L1, c.L2, c.L3, c.mask)
    lat.set_gauge(torch.from_numpy(U).cuda(), torch.from_numpy(A).cuda(), qxd.QXD_GAUGE_EXTENDED_CHECKED)
    # break one mirror link
    U2 = U.copy()
    mirror = lo.index(np.array([0, c.L1, 0, 0]))
    U2[mirror, 1] = U2[mirror, 1] @ np.diag(np.exp(1j * np.array([0.1, -0.1, 0.0])))
    with pytest.raises(qxd.QxdError) as e:
        lat.set_gauge(torch.from_numpy(U2).cuda(), torch.from_numpy(A).cuda(),
                      qxd.QXD_GAUGE_EXTENDED_CHECKED)
    assert e.value.code == qxd.QXD_ERR_NOT_ADMISSIBLE
    # unchecked accepts it, and D matches the oracle on that non-admissible field
    lat.set_gauge(torch.from_numpy(U2).cuda(), torch.from_numpy(A).cuda(),
                  qxd.QXD_GAUGE_EXTENDED_UNCHECKED)
    lat.set_params(c.m0, c.csw, c.cswqed, c.qhat)
    lat.sw_build()
    y = gpu_apply(lat, c.psi, qxd.QXD_FP64)
    op = O.Dirac(lo, O.GaugeField.from_extended(lo, U2, A), c.m0, c.csw, c.cswqed, c.qhat)
    assert rel_max(y, op.apply(c.psi.numpy())) < TOL64
    lat.close()


def test_singular_clover_is_reported():
    from paper_1710_08839_gb300 import qxd
    lat = qxd.Lattice(4, 2, 2, 2, 0b1110)
    su3 = torch.eye(3, dtype=torch.complex128).expand(4, 2, 2, 2, 4, 3, 3).contiguous()
    lat.set_gauge(su3.cuda(), torch.zeros(4, 2, 2, 2, 4, dtype=torch.float64, device="cuda"))
    lat.set_params(-4.0, 1.0, 1.0, 1)   # M(x) = 0 on unit links
    with pytest.raises(qxd.QxdError) as e:
        lat.sw_build()
    assert e.value.code == qxd.QXD_ERR_SW_SINGULAR
    lat.close()
