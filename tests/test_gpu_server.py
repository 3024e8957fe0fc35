"""The serving runtime: engine lanes by lattice size, each with its own
stream and worker thread. Requests submitted from several host threads and
at different times finish with the same result, bit for bit, as each request
solved alone, and pass the oracle's D."""
import threading
import time

import numpy as np
import pytest
import torch

import oracle as O
from qxd_cases import Case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _requests():
    small = Case(T=8, L1=8, L2=8, L3=8, qhat=2)               # 8192 sites: lane 0
    large = Case(T=16, L1=8, L2=8, L3=8, qhat=-1, seed=5)     # 16384 sites: lane 1
    parents, reqs = [], []
    rng = np.random.default_rng(21)
    for c in (small, large):
        par = c.lattice()
        parents.append(par)
        for m0, q in ((0.05, -1), (0.1, 2)):
            v = par.view()
            v.set_params(m0, 1.0, 1.0, q)
            v.sw_build()
            b = torch.from_numpy(rng.normal(size=(c.V, 4, 3)) + 1j * rng.normal(size=(c.V, 4, 3))).cuda()
            reqs.append((c, v, b, m0, q))
    return parents, reqs


def _wait(srv, ids, timeout=300.0):
    t0 = time.time()
    while True:
        states = [srv.poll(i) for i in ids]
        if all(d for d, _ in states):
            return [info for _, info in states]
        assert time.time() - t0 < timeout, "server requests did not finish"
        time.sleep(0.002)


def test_server_lanes_match_requests_alone():
    from paper_1710_08839_gb300 import qxd
    parents, reqs = _requests()
    srv = qxd.Server(lane_sites=[10000], lane_budgets=[8 << 30, 8 << 30], max_active=16)
    xs = [torch.zeros_like(b) for _, _, b, _, _ in reqs]
    ids = [None] * len(reqs)

    def submit(idx):
        for i in idx:
            _, v, b, _, _ = reqs[i]
            ids[i] = srv.submit(v, xs[i], b, tol=1e-10)

    # two host threads submit at once; then two more requests arrive later
    th = [threading.Thread(target=submit, args=([0],)), threading.Thread(target=submit, args=([2],))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    time.sleep(0.01)
    submit([1, 3])
    infos = _wait(srv, ids)
    for info in infos:
        assert info["status"] == qxd.QXD_OK and info["true_relres"] <= 1e-10, info
    assert srv.stats(0)["completed"] == 2 and srv.stats(1)["completed"] == 2
    assert srv.stats(0)["submitted"] == 2 and srv.stats(1)["submitted"] == 2
    for i in ids:
        srv.forget(i)
    with pytest.raises(qxd.QxdError) as e:
        srv.poll(ids[0])
    assert e.value.code == qxd.QXD_ERR_ARG
    srv.close()
    for (c, v, b, m0, q), x in zip(reqs, xs):
        eng = qxd.Engine(hbm_budget_bytes=8 << 30, max_active=4)
        x1 = torch.zeros_like(b)
        rid = eng.submit(v, x1, b, tol=1e-10)
        eng.run()
        assert eng.poll(rid)[0]
        eng.close()
        torch.cuda.synchronize()
        assert torch.equal(x1, x)
        lo = O.Lattice(c.T, c.L1, c.L2, c.L3, c.mask)
        op = O.Dirac(lo, O.GaugeField.from_physical(lo, c.su3.numpy(), c.ang.numpy()), m0, 1.0, 1.0, q)
        bb = b.cpu().numpy()
        assert np.linalg.norm(bb - op.apply(x.cpu().numpy())) / np.linalg.norm(bb) < 2e-10
    for _, v, _, _, _ in reqs:
        v.close()
    for p in parents:
        p.close()


def test_server_argument_errors():
    from paper_1710_08839_gb300 import qxd
    with pytest.raises(qxd.QxdError) as e:
        qxd.Server(lane_sites=[100, 50], lane_budgets=[1 << 30] * 3)
    assert e.value.code == qxd.QXD_ERR_ARG
    c = Case(T=8, L1=8, L2=8, L3=8, qhat=2)
    lat = c.lattice()
    b = c.psi.cuda()
    srv = qxd.Server(lane_sites=[], lane_budgets=[1 << 30])
    for kw in ({"tol": 0.0}, {"nkv": 17}, {"system": qxd.QXD_SOLVE_EO}):
        with pytest.raises(qxd.QxdError) as e:
            srv.submit(lat, torch.zeros_like(b), b, **kw)
        assert e.value.code == qxd.QXD_ERR_ARG
    # a request not converged within max_iter is reported as such
    x = torch.zeros_like(b)
    rid = srv.submit(lat, x, b, tol=1e-14, max_iter=2)
    info = _wait(srv, [rid])[0]
    assert info["status"] == qxd.QXD_ERR_NOT_CONVERGED and info["iterations"] == 2
    srv.close()
    lat.close()
