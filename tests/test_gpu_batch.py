"""Views (several quarks on one resident gauge field), the batched
multi-right-hand-side D over operators of different lattice sizes, and the
batched solve engine (continuous batching), on the GPU."""
import numpy as np
import pytest
import torch

import oracle as O
from qxd_cases import Case, rel_max, rel_norm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def native(lat, x, prec):
    n = torch.empty(lat.spinor_bytes(prec), dtype=torch.uint8, device="cuda")
    lat.pack(n, x, prec)
    return n


def test_views_share_the_gauge_field():
    from paper_1710_08839_gb300 import qxd
    c = Case(T=8, L1=4, L2=4, L3=4, qhat=2)
    parent = c.lattice()
    params = [(0.05, 1.0, 1.0, -1), (0.2, 1.3, 0.7, 2), (0.1, 1.0, 1.0, 0)]
    views = []
    for m0, csw, cq, q in params:
        v = parent.view()
        v.set_params(m0, csw, cq, q)
        v.sw_build()
        views.append(v)
    x = c.psi.cuda()
    for (m0, csw, cq, q), v in zip(params, views):
        y = torch.empty_like(x)
        v.Dw(y, x)
        c2 = Case(T=8, L1=4, L2=4, L3=4, m0=m0, csw=csw, cswqed=cq, qhat=q)
        ref = c2.oracle(c.su3, c.ang).apply(c.psi.numpy())
        assert rel_max(y.cpu().numpy(), ref) < 1e-13
    with pytest.raises(qxd.QxdError) as e:
        views[0].set_gauge(c.su3.cuda(), c.ang.cuda())
    assert e.value.code == qxd.QXD_ERR_STATE
    with pytest.raises(qxd.QxdError) as e:
        parent.close()
    assert e.value.code == qxd.QXD_ERR_STATE
    # a new gauge field on the parent makes the views stale until sw_build
    parent.set_gauge(c.su3.cuda(), c.ang.cuda())
    with pytest.raises(qxd.QxdError) as e:
        views[0].Dw(torch.empty_like(x), x)
    assert e.value.code == qxd.QXD_ERR_STATE
    views[0].sw_build()
    views[0].Dw(torch.empty_like(x), x)
    for v in views:
        v.close()
    parent.close()


# operators of the batched-D test: two lattice sizes, two quarks on each,
# three Gaussian right-hand sides per operator
BATCH_LATTICES = (dict(T=8, L1=4, L2=4, L3=4, qhat=2), dict(T=8, L1=8, L2=8, L3=8, qhat=-1, seed=3))
BATCH_QUARKS = ((0.05, -1), (0.1, 2))


@pytest.fixture(scope="module")
def batch_refs():
    """Sources and the oracle's D applied to them, once for all parametrisations."""
    rng = np.random.default_rng(9)
    out = []
    for kw in BATCH_LATTICES:
        c = Case(**kw)
        lo = O.Lattice(c.T, c.L1, c.L2, c.L3, c.mask)
        g = O.GaugeField.from_physical(lo, c.su3.numpy(), c.ang.numpy())
        for m0, q in BATCH_QUARKS:
            op = O.Dirac(lo, g, m0, 1.0, 1.0, q)
            for r in range(3):
                src = rng.normal(size=(c.V, 4, 3)) + 1j * rng.normal(size=(c.V, 4, 3))
                out.append((kw, m0, q, src, op.apply(src)))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nr", [0, 1, 2, 4, 8])
def test_batched_dw_matches_oracle(prec, nr, batch_refs):
    """qxd_Dw_batch over 12 right-hand sides of 4 operators on 2 lattice
    sizes, rhs_per_site nr (0: autotuned), against the oracle's D per
    operator (FP64 1e-13 relative max, FP32 1e-5 relative norm) and against
    qxd_Dw on the same input."""
    from paper_1710_08839_gb300 import qxd
    p = qxd.QXD_FP64 if prec == "fp64" else qxd.QXD_FP32
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    lats, views = {}, {}
    for kw in BATCH_LATTICES:
        c = Case(**kw)
        par = c.lattice()
        lats[id(kw)] = par
        for m0, q in BATCH_QUARKS:
            v = par.view()
            v.set_params(m0, 1.0, 1.0, q)
            v.sw_build()
            views[(id(kw), m0, q)] = v
    handles, ins, outs, checks = [], [], [], []
    for kw, m0, q, src, ref in batch_refs:
        v = views[(id(kw), m0, q)]
        x = torch.from_numpy(src).to(dt).cuda()
        xn = native(v, x, p)
        yn = torch.empty_like(xn)
        y = torch.empty_like(x)
        v.Dw(y, x)
        handles.append(v.handle)
        ins.append(xn)
        outs.append(yn)
        checks.append((v, y, ref))
    qxd.qxd_Dw_batch(handles, [o.data_ptr() for o in outs], [i.data_ptr() for i in ins], p, nr,
                     torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for (v, y, ref), yn in zip(checks, outs):
        got = torch.empty_like(y)
        v.unpack(got, yn, p)
        a, b = got.cpu().numpy().astype(np.complex128), y.cpu().numpy().astype(np.complex128)
        if prec == "fp64":
            assert rel_max(a, ref) < 1e-13
            assert rel_max(a, b) < 1e-13
        else:
            assert rel_norm(a, ref) < 1e-5
            assert rel_norm(a, b) < 1e-6
    for v in views.values():
        v.close()
    for l in lats.values():
        l.close()


ENGINE_QUARKS = ((0.05, -1), (0.1, 2))


def _engine_setup():
    # two lattices that admit the 4^4 SAP blocks, two quarks on each
    a = Case(T=8, L1=8, L2=8, L3=8, qhat=2)
    b = Case(T=16, L1=8, L2=8, L3=8, qhat=-1, seed=5)
    pa, pb = a.lattice(), b.lattice()
    reqs = []
    rng = np.random.default_rng(13)
    for c, par in ((a, pa), (b, pb)):
        for m0, q in ENGINE_QUARKS:
            v = par.view()
            v.set_params(m0, 1.0, 1.0, q)
            v.sw_build()
            bsrc = torch.from_numpy(rng.normal(size=(c.V, 4, 3)) + 1j * rng.normal(size=(c.V, 4, 3))).cuda()
            reqs.append((c, v, bsrc, m0, q))
    return (pa, pb), reqs


def _oracle_relres(c, m0, q, x, b):
    """||b - D x|| / ||b|| with the oracle's D of request (c, m0, q)."""
    lo = O.Lattice(c.T, c.L1, c.L2, c.L3, c.mask)
    op = O.Dirac(lo, O.GaugeField.from_physical(lo, c.su3.numpy(), c.ang.numpy()), m0, 1.0, 1.0, q)
    bb = b.cpu().numpy()
    return float(np.linalg.norm(bb - op.apply(x.cpu().numpy())) / np.linalg.norm(bb))


def _alone(v, b, **kw):
    """The request solved alone, in a fresh engine."""
    from paper_1710_08839_gb300 import qxd
    e1 = qxd.Engine(hbm_budget_bytes=64 << 30, max_active=16)
    x1 = torch.zeros_like(b)
    rid = e1.submit(v, x1, b, tol=1e-10, **kw)
    e1.run()
    done, info = e1.poll(rid)
    assert done and info["status"] == qxd.QXD_OK, info
    e1.close()
    torch.cuda.synchronize()
    return x1


def test_engine_results_same_alone_and_in_mix():
    from paper_1710_08839_gb300 import qxd
    parents, reqs = _engine_setup()
    # all requests together
    eng = qxd.Engine(hbm_budget_bytes=64 << 30, max_active=16)
    xs_mix = [torch.zeros_like(b) for _, _, b, _, _ in reqs]
    ids = [eng.submit(v, x, b, tol=1e-10) for (_, v, b, _, _), x in zip(reqs, xs_mix)]
    eng.run()
    for rid in ids:
        done, info = eng.poll(rid)
        assert done and info["status"] == qxd.QXD_OK, info
        assert info["true_relres"] <= 1e-10
    # the batched SAP launch set is captured once per job mix and replayed
    gs = eng.graph_stats()
    assert gs["captures"] >= 1 and gs["replays"] >= 1, gs
    assert gs["captures"] + gs["replays"] <= eng.stats()["steps"], gs
    eng.close()
    for (c, v, b, m0, q), xm in zip(reqs, xs_mix):
        # each alone, in a fresh engine: bit-identical
        assert torch.equal(_alone(v, b), xm)
        # every request's true residual with the oracle's D
        assert _oracle_relres(c, m0, q, xm, b) < 2e-10
    for _, v, _, _, _ in reqs:
        v.close()
    for p in parents:
        p.close()


def test_engine_staggered_arrivals():
    """Continuous batching: two requests start, the engine steps, two more
    arrive while the first two are on the GPU and join the running batch.
    Every result equals the same request solved alone, bit for bit, and
    passes the oracle's D."""
    from paper_1710_08839_gb300 import qxd
    parents, reqs = _engine_setup()
    eng = qxd.Engine(hbm_budget_bytes=64 << 30, max_active=16)
    xs = [torch.zeros_like(b) for _, _, b, _, _ in reqs]
    first, later = (0, 2), (1, 3)     # one request of each lattice in each wave
    ids = {}
    for i in first:
        _, v, b, _, _ = reqs[i]
        ids[i] = eng.submit(v, xs[i], b, tol=1e-10)
    for _ in range(2):
        active, pending, done = eng.step()
        assert active == 2 and pending == 0 and done == 0
    for i in first:
        assert not eng.poll(ids[i])[0]
    for i in later:
        _, v, b, _, _ = reqs[i]
        ids[i] = eng.submit(v, xs[i], b, tol=1e-10)
    active, pending, done = eng.step()
    assert active + done == 4 and pending == 0     # admitted beside the running two
    eng.run()
    for i in range(4):
        done, info = eng.poll(ids[i])
        assert done and info["status"] == qxd.QXD_OK, info
    eng.close()
    for (c, v, b, m0, q), x in zip(reqs, xs):
        assert torch.equal(_alone(v, b), x)
        assert _oracle_relres(c, m0, q, x, b) < 2e-10
    for _, v, _, _, _ in reqs:
        v.close()
    for p in parents:
        p.close()


def test_engine_budget_holds_with_full_krylov_depth():
    """Requests with nkv = 16 under a budget of 2.5 of the larger requests:
    the engine charges each its full Krylov depth, so the four requests (two
    of 8192 sites, two of 16384) are never all active at once, and the bytes
    in use and held by its allocator never exceed the budget."""
    from paper_1710_08839_gb300 import qxd
    parents, reqs = _engine_setup()
    V = max(c.V for c, _, _, _, _ in reqs)
    per_req = 24 * V * (4 * 8 + (1 + 2 * 16) * 4)
    budget = int(2.5 * per_req)
    eng = qxd.Engine(hbm_budget_bytes=budget, max_active=16)
    xs = [torch.zeros_like(b) for _, _, b, _, _ in reqs]
    # a loose inner tolerance and no SAP: many Krylov steps per cycle
    ids = [eng.submit(v, x, b, tol=1e-10, nkv=16, precond=qxd.QXD_PRECOND_NONE, delta=0.0, max_iter=4000)
           for (_, v, b, _, _), x in zip(reqs, xs)]
    max_active = 0
    while True:
        a, p, d = eng.step()
        st = eng.stats()
        assert st["bytes_in_use"] <= budget and st["bytes_held"] <= budget, st
        max_active = max(max_active, a)
        if a == 0 and p == 0:
            break
    charge = {c.V: 24 * c.V * (4 * 8 + (1 + 2 * 16) * 4) for c, _, _, _, _ in reqs}
    assert sum(charge[c.V] for c, _, _, _, _ in reqs) > budget     # not all four fit
    assert 2 <= max_active < 4
    for rid in ids:
        done, info = eng.poll(rid)
        assert done and info["status"] == qxd.QXD_OK, info
        assert info["iterations"] > 16      # the Krylov space was filled at least once
    eng.close()
    for _, v, _, _, _ in reqs:
        v.close()
    for p in parents:
        p.close()


def test_engine_admission_by_budget_and_agreement_with_solve():
    from paper_1710_08839_gb300 import qxd
    parents, reqs = _engine_setup()
    c, v, b, _, _ = reqs[0]
    # budget below one request: requests run one at a time, all complete
    eng = qxd.Engine(hbm_budget_bytes=1 << 20, max_active=16)
    xs = [torch.zeros_like(bb) for _, _, bb, _, _ in reqs]
    ids = [eng.submit(vv, x, bb, tol=1e-10) for (_, vv, bb, _, _), x in zip(reqs, xs)]
    max_active = 0
    while True:
        a, p, d = eng.step()
        max_active = max(max_active, a)
        if a == 0 and p == 0:
            break
    assert max_active == 1
    for rid in ids:
        done, info = eng.poll(rid)
        assert done and info["status"] == qxd.QXD_OK
    st = eng.stats()
    assert st["bytes_in_use"] == 0 and st["steps"] > 0
    eng.close()
    # same problem through qxd_solve (mixed precision, SAP)
    x2 = torch.zeros_like(b)
    rc, info = v.solve(x2, b, tol=1e-10, precond=qxd.QXD_PRECOND_SAP, inner_prec=qxd.QXD_FP32)
    assert rc == qxd.QXD_OK
    assert float((x2 - xs[0]).norm() / x2.norm()) < 1e-8
    for _, vv, _, _, _ in reqs:
        vv.close()
    for p in parents:
        p.close()


def test_engine_not_converged_and_argument_errors():
    from paper_1710_08839_gb300 import qxd
    c = Case(T=8, L1=8, L2=8, L3=8, qhat=2, m0=0.05)
    lat = c.lattice()
    b = c.psi.cuda()
    eng = qxd.Engine(hbm_budget_bytes=8 << 30, max_active=4)
    x = torch.zeros_like(b)
    rid = eng.submit(lat, x, b, tol=1e-14, max_iter=2)
    eng.run()
    done, info = eng.poll(rid)
    assert done and info["status"] == qxd.QXD_ERR_NOT_CONVERGED
    assert info["iterations"] == 2 and 0 < info["true_relres"] < 1
    assert torch.count_nonzero(x) > 0
    for kw in ({"system": qxd.QXD_SOLVE_EO}, {"inner_prec": qxd.QXD_FP64}, {"nkv": 17}, {"tol": 0.0}):
        with pytest.raises(qxd.QxdError) as e:
            eng.submit(lat, torch.zeros_like(b), b, **kw)
        assert e.value.code == qxd.QXD_ERR_ARG
    fresh = lat.view()                     # parameters never set: no clover term
    with pytest.raises(qxd.QxdError) as e:
        eng.submit(fresh, torch.zeros_like(b), b)
    assert e.value.code == qxd.QXD_ERR_STATE
    with pytest.raises(qxd.QxdError):
        eng.forget(123456)
    eng.close()
    fresh.close()
    lat.close()


def test_native_layout_solve_matches_lexicographic():
    from paper_1710_08839_gb300 import qxd
    c = Case(T=8, L1=8, L2=8, L3=8, qhat=-1, m0=0.1)
    lat = c.lattice()
    b = c.psi.cuda()
    x_lex = torch.zeros_like(b)
    rc, _ = lat.solve(x_lex, b, tol=1e-10, precond=qxd.QXD_PRECOND_SAP, inner_prec=qxd.QXD_FP32)
    assert rc == qxd.QXD_OK
    bn = torch.empty(lat.spinor_bytes(qxd.QXD_FP64), dtype=torch.uint8, device="cuda")
    lat.pack(bn, b, qxd.QXD_FP64)
    xn = torch.zeros_like(bn)
    rc, _ = lat.solve(xn, bn, tol=1e-10, precond=qxd.QXD_PRECOND_SAP, inner_prec=qxd.QXD_FP32,
                      flags=qxd.QXD_LAYOUT_NATIVE)
    assert rc == qxd.QXD_OK
    x2 = torch.empty_like(b)
    lat.unpack(x2, xn, qxd.QXD_FP64)
    torch.cuda.synchronize()
    assert torch.equal(x2, x_lex)
    lat.close()


def test_engine_large_lattice_path():
    """Jobs on lattices of 1M sites or more run their Schwarz method and D
    through the single-lattice kernels: mixed with a small job, the large
    job's result is the same as alone, and it agrees with qxd_solve."""
    from paper_1710_08839_gb300 import qxd
    big = Case(T=48, L1=24, L2=24, L3=24, qhat=2, m0=0.1)           # 1,327,104 sites
    small = Case(T=8, L1=8, L2=8, L3=8, qhat=-1)
    lb, ls = big.lattice(), small.lattice()
    bb = big.psi.to(torch.complex128).cuda().contiguous()
    bs = small.psi.to(torch.complex128).cuda().contiguous()
    eng = qxd.Engine(hbm_budget_bytes=64 << 30, max_active=16)
    xb, xs = torch.zeros_like(bb), torch.zeros_like(bs)
    ib, i_s = eng.submit(lb, xb, bb, tol=1e-10), eng.submit(ls, xs, bs, tol=1e-10)
    eng.run()
    for rid in (ib, i_s):
        done, info = eng.poll(rid)
        assert done and info["status"] == qxd.QXD_OK and info["true_relres"] <= 1e-10
    x1 = torch.zeros_like(bb)
    rid = eng.submit(lb, x1, bb, tol=1e-10)
    eng.run()
    assert eng.poll(rid)[0]
    eng.close()
    torch.cuda.synchronize()
    assert torch.equal(x1, xb)
    x2 = torch.zeros_like(bb)
    rc, info = lb.solve(x2, bb, tol=1e-10, precond=qxd.QXD_PRECOND_SAP, inner_prec=qxd.QXD_FP32)
    assert rc == qxd.QXD_OK
    assert float((x2 - xb).norm() / x2.norm()) < 1e-8
    lb.close()
    ls.close()


def test_engine_same_operator_large_lattice():
    """Requests on a lattice of 2^20 sites take the single-lattice Schwarz
    kernels, and the requests of one operator are solved together (each
    thread block stages its block's links once for all of them). Each result
    equals the same request solved alone, bit for bit, and its residual with
    the oracle's D at sampled sites (and the corners of the shifted
    boundaries) stays at the tolerance."""
    from paper_1710_08839_gb300 import qxd
    c = Case(T=32, L1=16, L2=32, L3=32, qhat=2, m0=0.1, seed=9)
    assert c.V == 1 << 20
    lat = c.lattice()
    rng = np.random.default_rng(29)
    bs = [torch.from_numpy(rng.normal(size=(c.V, 4, 3)) + 1j * rng.normal(size=(c.V, 4, 3))).cuda()
          for _ in range(3)]
    eng = qxd.Engine(hbm_budget_bytes=64 << 30, max_active=16)
    xs = [torch.zeros_like(b) for b in bs]
    ids = [eng.submit(lat, x, b, tol=1e-10) for x, b in zip(xs, bs)]
    eng.run()
    for rid in ids:
        done, info = eng.poll(rid)
        assert done and info["status"] == qxd.QXD_OK and info["true_relres"] <= 1e-10, info
    eng.close()
    for x, b in zip(xs, bs):
        assert torch.equal(_alone(lat, b), x)
    lo = O.Lattice(c.T, c.L1, c.L2, c.L3, c.mask)
    op = c.oracle()
    idx = np.sort(rng.choice(c.V, size=400, replace=False))
    corners = lo.index(np.array([[0, 0, 0, 0], [c.T - 1, c.N1 - 1, c.L2 - 1, c.L3 - 1],
                                 [3, c.L1 - 1, 0, c.L3 - 1], [9, c.L1, c.L2 - 1, 0]]))
    idx = np.unique(np.concatenate([idx, corners]))
    for x, b in zip(xs, bs):
        b_h = b.cpu().numpy()
        r = b_h[idx] - op.apply_at(x.cpu().numpy(), idx)
        assert np.linalg.norm(r) / np.linalg.norm(b_h[idx]) < 3e-10
    lat.close()
