"""Launch-shape autotuning of D: every shape the tuner may pick gives the
same result, bit for bit, and the oracle's; the chosen shape is reported and
can be pinned."""
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


# a lattice shape no other test uses, so its first D here does the tuning:
# doubled 12 x 16 x 8 x 8 C* lattice, window candidates rows in {2, 4, 8}
SHAPE = dict(T=12, L1=8, L2=8, L3=8, qhat=2, m0=0.1)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_every_shape_gives_the_same_result(prec):
    from paper_1710_08839_gb300 import qxd
    p = qxd.QXD_FP32 if prec == "fp32" else qxd.QXD_FP64
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    c = Case(**SHAPE)
    lat = c.lattice()
    x = c.psi.to(dt).cuda()
    y = torch.empty_like(x)
    lat.Dw(y, x)                      # first call on this shape: tunes
    torch.cuda.synchronize()
    sh = lat.dw_shape(p)
    assert sh["threads"] in (64, 128) and c.L2 % sh["rows"] == 0 and sh["ms"] > 0
    assert sh["pipelined"] == (sh["pipelined"] and prec == "fp32")
    report = qxd.tune_report()
    assert f"{c.T}x{2 * c.L1}x{c.L2}x{c.L3}" in report and "(tuned)" in report
    ref = c.oracle().apply(c.psi.numpy())
    got = y.cpu().numpy().astype(np.complex128)
    assert (rel_max(got, ref) < 1e-13) if prec == "fp64" else (rel_norm(got, ref) < 1e-5)
    outs = []
    for pl in ((0, 1) if prec == "fp32" else (0,)):
        for th in (64, 128):
            for rows in (1, 2, 4, 8):
                lat.set_dw_shape(p, pl, th, rows)
                z = torch.full_like(x, float("nan"))
                lat.Dw(z, x)
                torch.cuda.synchronize()
                outs.append(((pl, th, rows), z))
    for shape, z in outs:
        assert torch.equal(z, y), shape
    lat.close()


def test_pinned_and_default_shapes_and_errors():
    from paper_1710_08839_gb300 import qxd
    c = Case(T=20, L1=8, L2=8, L3=8, qhat=-1)     # another fresh shape
    lat = c.lattice()
    with pytest.raises(qxd.QxdError) as e:
        lat.dw_shape(qxd.QXD_FP32)                # nothing chosen yet
    assert e.value.code == qxd.QXD_ERR_STATE
    prev = qxd.set_autotune(False)
    try:
        x = c.psi.to(torch.complex64).cuda()
        lat.Dw(torch.empty_like(x), x)
        sh = lat.dw_shape(qxd.QXD_FP32)
        assert sh["pipelined"] and sh["threads"] == 128 and sh["ms"] == 0
        assert "(default)" in qxd.tune_report()
    finally:
        qxd.set_autotune(prev)
    for args in ((qxd.QXD_FP64, 1, 128, 2), (qxd.QXD_FP32, 2, 128, 2), (qxd.QXD_FP32, 1, 96, 2),
                 (qxd.QXD_FP32, 1, 128, 3), (qxd.QXD_FP32, 1, 128, 0)):
        with pytest.raises(qxd.QxdError) as e:
            lat.set_dw_shape(*args)
        assert e.value.code == qxd.QXD_ERR_ARG
    lat.close()
