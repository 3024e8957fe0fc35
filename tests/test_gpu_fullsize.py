"""Parity at the full benchmark size (doubled 96x96x48x48 C* lattice, 21.2M
sites) in the launch configuration bench.py times: FP64 and FP32 D against
the oracle on sampled sites."""
import numpy as np
import pytest
import torch

from qxd_cases import rel_max, rel_norm

pytestmark = pytest.mark.gpu


def test_full_size_sampled_parity():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import bench
    import oracle as O
    from paper_1710_08839_gb300 import qxd
    w = bench.WORKLOAD
    su3, ang, psi, V = bench.make_inputs("cuda")
    lat = qxd.Lattice(w["T"], w["L1"], w["L2"], w["L3"], w["mask"])
    lat.set_gauge(su3, ang)
    lat.set_params(w["m0"], w["csw"], w["cswqed"], w["qhat"])
    lat.sw_build()
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(V, size=2000, replace=False))
    # include the corners of the shifted boundaries
    lo = O.Lattice(w["T"], w["L1"], w["L2"], w["L3"], w["mask"])
    corners = lo.index(np.array([[0, 0, 0, 0], [w["T"] - 1, 2 * w["L1"] - 1, w["L2"] - 1, w["L3"] - 1],
                                 [5, w["L1"] - 1, 0, w["L3"] - 1], [7, w["L1"], w["L2"] - 1, 0]]))
    idx = np.unique(np.concatenate([idx, corners]))
    out = {}
    for prec, dt in ((qxd.QXD_FP64, torch.complex128), (qxd.QXD_FP32, torch.complex64)):
        x = psi.to(dt).cuda()
        y = torch.empty_like(x)
        lat.Dw(y, x)
        torch.cuda.synchronize()
        out[prec] = y[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
        del x, y
    lat.close()
    op = O.Dirac(lo, O.GaugeField.from_physical(lo, su3.cpu().numpy(), ang.cpu().numpy()),
                 w["m0"], w["csw"], w["cswqed"], w["qhat"])
    ref = op.apply_at(psi.numpy(), idx)
    assert rel_max(out[qxd.QXD_FP64], ref) < 1e-13
    assert rel_norm(out[qxd.QXD_FP32], ref) < 1e-5


def test_solver_workload_sampled_oracle_residual():
    """The solver workload at full size (doubled 64x64x32x32 C* lattice,
    4.2M sites, m0 = 0.05, qhat = -1): one mixed-precision SAP-FGCR solve to
    1e-10, then the residual b - D x recomputed by the oracle on 2000 sampled
    sites plus the corners of the shifted boundaries. Site by site it must
    match the GPU's FP64 residual to 1e-12 of max|b| (two FP64 evaluations of
    D x, which is of the size of b), and its sampled norm must stay at the
    solver's tolerance."""
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import bench
    import oracle as O
    from paper_1710_08839_gb300 import qxd
    w = dict(bench.SOLVE_WORKLOAD)
    m0, q = 0.05, -1
    su3, ang, psi, V = bench.make_inputs("cuda", w)
    lat = qxd.Lattice(w["T"], w["L1"], w["L2"], w["L3"], w["mask"])
    lat.set_gauge(su3, ang)
    lat.set_params(m0, w["csw"], w["cswqed"], q)
    lat.sw_build()
    b = psi.cuda()
    x = torch.zeros_like(b)
    rc, info = lat.solve(x, b, tol=w["tol"], precond=qxd.QXD_PRECOND_SAP, inner_prec=qxd.QXD_FP32)
    assert rc == qxd.QXD_OK and info["true_relres"] <= w["tol"], info
    r_gpu = torch.empty_like(x)
    lat.Dw(r_gpu, x)
    r_gpu = b - r_gpu
    lo = O.Lattice(w["T"], w["L1"], w["L2"], w["L3"], w["mask"])
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(V, size=2000, replace=False))
    N1 = 2 * w["L1"]
    corners = lo.index(np.array([[0, 0, 0, 0], [w["T"] - 1, N1 - 1, w["L2"] - 1, w["L3"] - 1],
                                 [3, w["L1"] - 1, 0, w["L3"] - 1], [9, w["L1"], w["L2"] - 1, 0],
                                 [1, 0, w["L2"] - 1, w["L3"] - 1], [2, N1 - 1, 0, 0]]))
    idx = np.unique(np.concatenate([idx, corners]))
    ti = torch.from_numpy(idx).cuda()
    r_gpu_s = r_gpu[ti].cpu().numpy()
    x_h = x.cpu().numpy()
    b_s = psi.numpy()[idx]
    lat.close()
    del x, b, r_gpu
    op = O.Dirac(lo, O.GaugeField.from_physical(lo, su3.cpu().numpy(), ang.cpu().numpy()),
                 m0, w["csw"], w["cswqed"], q)
    del su3, ang
    r_orc = b_s - op.apply_at(x_h, idx)
    assert np.abs(r_gpu_s - r_orc).max() / np.abs(b_s).max() < 1e-12
    # sampled estimate of the true relative residual (the full value is <= 1e-10)
    assert np.linalg.norm(r_orc) / np.linalg.norm(b_s) < 3e-10
