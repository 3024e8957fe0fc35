"""qxd_Dw_noalloc: D without device allocation, for callers that cannot let a
library allocate during a call (their own memory pools, nearly full
devices, paths that cannot wait for a cudaMalloc). Two calls in a row are
checked to leave the device's free memory unchanged and against qxd_Dw (the
entry point that allocates its conversion scratch); the size limit is
checked too. Collected last on purpose."""
import ctypes
import gc

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
    """On a fresh lattice: one set-up call, then two calls in a row that must
    leave the device's free memory unchanged (nothing allocated, not even the
    conversion scratch qxd_Dw would create), then both results against
    qxd_Dw."""
    from paper_1710_08839_gb300 import qxd
    p = qxd.QXD_FP64 if prec == "fp64" else qxd.QXD_FP32
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    c = Case(T=8, L1=4, L2=4, L3=4, eps=0.4, sigma=0.5, m0=0.2, qhat=-1)
    lat = c.lattice()
    rng = np.random.default_rng(17)
    srcs = [c.psi.numpy(), rng.normal(size=(c.V, 4, 3)) + 1j * rng.normal(size=(c.V, 4, 3))]
    xs = [torch.from_numpy(np.ascontiguousarray(s)).to(dt).cuda() for s in srcs]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    # set-up call: the first call on a device loads the scratch array
    warm = torch.empty_like(xs[0])
    assert _noalloc(lat, warm, xs[0], p) == qxd.QXD_OK, qxd.qxd_last_error()
    torch.cuda.synchronize()
    # no Python garbage collection in the measured window: a lattice left by
    # an earlier test and finalised there would free device memory
    gc.collect()
    gc.disable()
    try:
        free_before = torch.cuda.mem_get_info()[0]
        for x, y in zip(xs, ys):
            assert _noalloc(lat, y, x, p) == qxd.QXD_OK, qxd.qxd_last_error()
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
    finally:
        gc.enable()
    assert free_after == free_before, (free_before, free_after)
    for x, y in zip(xs, ys):
        ref = torch.empty_like(x)
        lat.Dw(ref, x)
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
