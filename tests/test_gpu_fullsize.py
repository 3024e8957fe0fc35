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
