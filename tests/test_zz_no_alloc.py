"""qxd_Dw_noalloc: D without device allocation, for callers that cannot let a
library allocate during a call. It is checked against qxd_Dw (the entry point
that allocates its conversion scratch) on two calls in a row, and its size
limit is checked. Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from qxd_cases import Case, rel_max, rel_norm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _noalloc(lat, out, inp, prec):
    from paper_1710_08839_gb300 import qxd
    stream = torch.cuda.current_stream().cuda_stream
    rc = qxd.lib().qxd_Dw_noalloc(ctypes.c_void_p(lat.handle), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(inp.data_ptr()), prec, ctypes.c_void_p(stream))
    return rc


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_Dw_on_two_calls(prec):
    from paper_1710_08839_gb300 import qxd
    p = qxd.QXD_FP64 if prec == "fp64" else qxd.QXD_FP32
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    c = Case(T=8, L1=4, L2=4, L3=4, eps=0.4, sigma=0.5, m0=0.2, qhat=-1)
    lat = c.lattice()
    rng = np.random.default_rng(17)
    for call in range(2):
        src = c.psi.numpy() if call == 0 else rng.normal(size=(c.V, 4, 3)) + 1j * rng.normal(size=(c.V, 4, 3))
        x = torch.from_numpy(np.ascontiguousarray(src)).to(dt).cuda()
        ref = torch.empty_like(x)
        lat.Dw(ref, x)
        y = torch.full_like(x, float("nan"))
        assert _noalloc(lat, y, x, p) == qxd.QXD_OK, qxd.qxd_last_error()
        torch.cuda.synchronize()
        a, b = y.cpu().numpy().astype(np.complex128), ref.cpu().numpy().astype(np.complex128)
        assert np.isfinite(a).all()
        if prec == "fp64":
            assert rel_max(a, b) < 1e-13
        else:
            assert rel_norm(a, b) < 1e-5
    lat.close()


def test_noalloc_rejects_lattices_above_its_limit():
    from paper_1710_08839_gb300 import qxd
    c = Case(T=16, L1=8, L2=8, L3=8, qhat=1)   # 16 x 16 x 8 x 8 = 16384 sites: accepted
    lat = c.lattice()
    x = c.psi.cuda()
    y = torch.empty_like(x)
    assert _noalloc(lat, y, x, qxd.QXD_FP64) == qxd.QXD_OK
    lat.close()
    big = Case(T=16, L1=16, L2=16, L3=8, qhat=1)  # 16 x 32 x 16 x 8 = 65536: the limit
    lat = big.lattice()
    xb = big.psi.cuda()
    assert _noalloc(lat, torch.empty_like(xb), xb, qxd.QXD_FP64) == qxd.QXD_OK
    lat.close()
    over = Case(T=16, L1=16, L2=16, L3=16, qhat=1)  # 131072 sites: rejected
    lat = over.lattice()
    xo = over.psi.cuda()
    rc = _noalloc(lat, torch.empty_like(xo), xo, qxd.QXD_FP64)
    assert rc == qxd.QXD_ERR_ARG
    assert "65536" in qxd.qxd_last_error()
    lat.close()
