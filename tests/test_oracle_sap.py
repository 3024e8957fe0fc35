"""Pins of the oracle's SAP preconditioner (no GPU).

SAP is an approximate inverse, so what the mathematics fixes is:
* with enough minimal-residual steps the block solve is exact, so right after
  the half-cycle of colour c the residual eta - D psi vanishes on the blocks
  of colour c (and not on the other colour);
* the Schwarz iteration converges: the residual of SAP(eta) falls with the
  number of cycles;
* with exact block solves SAP is linear: SAP(a eta) = a SAP(eta).
The block size is a parameter of the oracle; these pins use 2^4 blocks on a
512-site C* lattice so that they run in seconds (the GPU comparisons use the
4^4 blocks of the library).
"""
import inspect

import numpy as np
import pytest

import oracle as O
import pins as P

BS = 2


def setup(m0=0.6, qhat=2, seed=21):
    lat = O.Lattice(4, 4, 4, 4, 0b1110)     # 4 x 8 x 4 x 4, C* in x, y, z
    r = P.rng(seed)
    g = P.random_physical_gauge(r, lat, eps=0.3, sigma=0.3)
    op = O.Dirac(lat, g, m0, 1.0, 1.0, qhat)
    eta = P.random_spinor(r, (lat.V,))
    return lat, op, eta


def colour_of(lat, bs=BS):
    c = lat.coords(lat.all_sites())
    return (c // bs).sum(axis=1) % 2


def last_colour_residual(op, eta, lat, nmr):
    psi = O.sap(op, eta, ncy=1, nmr=nmr, bs=BS)
    r = eta - op.apply(psi)
    col = colour_of(lat)
    n = np.linalg.norm(eta)
    return np.linalg.norm(r[col == 1]) / n, np.linalg.norm(r[col == 0]) / n


def test_exact_block_solves_zero_the_residual_on_the_last_colour():
    lat, op, eta = setup()
    r1, r0 = last_colour_residual(op, eta, lat, nmr=60)
    assert r1 < 1e-10
    assert r0 > 1e-3   # colour 0 was disturbed by the colour-1 updates


def test_schwarz_iteration_converges():
    lat, op, eta = setup()
    res = []
    for ncy in (1, 2, 4):
        psi = O.sap(op, eta, ncy=ncy, nmr=20, bs=BS)
        res.append(np.linalg.norm(eta - op.apply(psi)) / np.linalg.norm(eta))
    assert all(b < 0.7 * a for a, b in zip(res, res[1:])), res
    assert res[-1] < 2e-2


def test_exact_block_solves_are_linear():
    lat, op, eta = setup()
    a = 0.7 - 1.3j
    p1 = O.sap(op, eta, ncy=1, nmr=60, bs=BS)
    p2 = O.sap(op, a * eta, ncy=1, nmr=60, bs=BS)
    assert np.abs(p2 - a * p1).max() / np.abs(p2).max() < 1e-10


def test_inconsistent_colouring_is_rejected():
    lat = O.Lattice(4, 2, 4, 4, 0b1110)      # 4 x 4 x 4 x 4: N_k/2 + L1/2 odd
    r = P.rng(1)
    op = O.Dirac(lat, P.random_physical_gauge(r, lat), 0.5, 1.0, 1.0, 1)
    with pytest.raises(ValueError):
        O.sap(op, P.random_spinor(r, (lat.V,)), 1, 1, bs=2)


def test_planted_wrong_block_inverse_is_caught(monkeypatch):
    """A wrong D_oo^-1 inside the block solves (identity instead of the clover
    inverse) makes the block solves inexact, which the first pin detects."""
    lat, op, eta = setup()
    monkeypatch.setattr(O.EvenOdd, "_diag_blocks",
                        lambda self, sites: np.broadcast_to(np.eye(12, dtype=complex),
                                                            (len(sites), 12, 12)).copy())
    r1, _ = last_colour_residual(op, eta, lat, nmr=60)
    assert r1 > 1e-6


# Plausible mistakes planted in a copy of the oracle's sap (one line each).
# Every one must fail at least one of the pins above: a pin that cannot fail
# pins nothing.
PLANTED = {
    "sign of the odd-site reconstruction": ("yo = Doo_inv_B(restrict(r, odd_b) - D_B_eo(y, odd_b, even_b))",
                                            "yo = Doo_inv_B(restrict(r, odd_b) + D_B_eo(y, odd_b, even_b))"),
    "sign of the even-odd source": ("ce = restrict(r, even_b) - D_B_eo(Doo_inv_B(r), even_b, odd_b)",
                                    "ce = restrict(r, even_b) + D_B_eo(Doo_inv_B(r), even_b, odd_b)"),
    "sign of the Schur complement": ("return D_B_eo(f, even_b, even_b) - D_B_eo(",
                                     "return D_B_eo(f, even_b, even_b) + D_B_eo("),
    "residual not updated after the first colour": ("r = restrict(eta - op.apply(psi), inb)",
                                                    "r = restrict(eta, inb)"),
    "one colour visited twice": ("for col in (0, 1):", "for col in (0, 0):"),
}


def planted_sap(old, new):
    src = inspect.getsource(O.qxd_oracle.sap)
    assert src.count(old) == 1, old
    ns = dict(vars(O.qxd_oracle))
    exec(compile(src.replace(old, new), "<planted sap>", "exec"), ns)
    return ns["sap"]


def pins_hold(sap):
    """The three pins above, for a given implementation of SAP."""
    lat, op, eta = setup()
    col = colour_of(lat)
    n = np.linalg.norm(eta)
    p1 = sap(op, eta, ncy=1, nmr=60, bs=BS)
    r = eta - op.apply(p1)
    if not (np.linalg.norm(r[col == 1]) / n < 1e-10 and np.linalg.norm(r[col == 0]) / n > 1e-3):
        return False
    a = 0.7 - 1.3j
    p2 = sap(op, a * eta, ncy=1, nmr=60, bs=BS)
    if not np.abs(p2 - a * p1).max() / np.abs(p2).max() < 1e-10:
        return False
    res = [np.linalg.norm(eta - op.apply(sap(op, eta, ncy=k, nmr=20, bs=BS))) / n for k in (1, 2, 4)]
    return all(b < 0.7 * a for a, b in zip(res, res[1:])) and res[-1] < 2e-2


@pytest.mark.parametrize("name", list(PLANTED))
def test_planted_sap_mistakes_are_caught(name):
    assert not pins_hold(planted_sap(*PLANTED[name])), name


# The block solve itself (nmr minimal-residual steps). Its defining
# properties: rho = c - A y after every step, and each step's omega minimises
# the block norm of rho - omega w, i.e. the new rho is orthogonal to w = A rho
# on every block (so the block residual never grows). Checked on a random
# non-Hermitian block-diagonal operator with a masked support.

def mr_problem(seed=4):
    rng = np.random.default_rng(seed)
    nb, per = 3, 8                              # 3 blocks of 8 sites
    V = nb * per
    block_id = np.arange(V) // per
    mask = (np.arange(V) % 2) == 0              # the operator lives on half the sites
    idx = [np.flatnonzero((block_id == b) & mask) for b in range(nb)]
    mats = [np.eye(12 * len(i)) + 0.3 * (rng.normal(size=(12 * len(i),) * 2)
                                         + 1j * rng.normal(size=(12 * len(i),) * 2)) / np.sqrt(12 * len(i))
            for i in idx]

    def A(f):
        g = np.zeros_like(f)
        for i, m in zip(idx, mats):
            g[i] = (m @ f[i].reshape(-1)).reshape(len(i), 4, 3)
        return g

    c = np.zeros((V, 4, 3), dtype=complex)
    c[mask] = rng.normal(size=(mask.sum(), 4, 3)) + 1j * rng.normal(size=(mask.sum(), 4, 3))
    return A, c, block_id, nb, mask


def mr_pins_hold(block_mr):
    A, c, block_id, nb, mask = mr_problem()
    prev = None
    for k in range(5):
        y, rho = block_mr(A, c, block_id, nb, k, mask)
        if np.linalg.norm(c - A(y) - rho) > 1e-12 * np.linalg.norm(c):
            return False
        if np.count_nonzero(y[~mask]) or np.count_nonzero(rho[~mask]):
            return False
        if prev is not None:
            w = A(prev)
            for b in range(nb):
                sel = block_id == b
                overlap = abs(np.vdot(w[sel], rho[sel]))
                if overlap > 1e-12 * np.linalg.norm(w[sel]) * np.linalg.norm(prev[sel]):
                    return False
                if np.linalg.norm(rho[sel]) > np.linalg.norm(prev[sel]) * (1 + 1e-14):
                    return False
        prev = rho
    return np.linalg.norm(prev) < 0.9 * np.linalg.norm(c)


def test_block_minimal_residual_steps():
    assert mr_pins_hold(O.block_mr)


PLANTED_MR = {
    "conjugated step length": ('wr = np.einsum("nsc,nsc->n", np.conj(w), rho)',
                               'wr = np.einsum("nsc,nsc->n", w, np.conj(rho))'),
    "one omega for all blocks": ("omega = om[block_id][:, None, None]",
                                 "omega = num.sum() / max(den.sum(), 1e-300)"),
    "solution updated along w": ("y = restrict(y + omega * rho)", "y = restrict(y + omega * w)"),
    "step length without the conjugate of w": ('wr = np.einsum("nsc,nsc->n", np.conj(w), rho)',
                                               'wr = np.einsum("nsc,nsc->n", w, rho)'),
}


@pytest.mark.parametrize("name", list(PLANTED_MR))
def test_planted_mr_mistakes_are_caught(name):
    old, new = PLANTED_MR[name]
    src = inspect.getsource(O.qxd_oracle.block_mr)
    assert src.count(old) == 1, old
    ns = dict(vars(O.qxd_oracle))
    exec(compile(src.replace(old, new), "<planted block_mr>", "exec"), ns)
    assert not mr_pins_hold(ns["block_mr"]), name


def sap_carried(op, eta, ncy, nmr, bs, cross_sign=1.0):
    """The Schwarz sweep of oracle.sap with the residual of a block visit
    carried instead of recomputed: the even-odd block solve leaves the block
    residual r_B - D_B delta_B equal to the MR residual rho on the even sites
    and to zero on the odd ones (the odd rows are solved exactly), and
    between two visits of a colour psi changes only by the other colour's
    last correction, whose D reaches the blocks of this colour only through
    the hops crossing their faces. So a visit starts from eta (first visit)
    or the kept rho, minus D of the other colour's last correction there.
    cross_sign plants a sign mistake in that term."""
    lat = op.lat
    V = lat.V
    c = lat.coords(lat.all_sites())
    B = c // bs
    nb = [lat.N[mu] // bs for mu in range(4)]
    block_id = ((B[:, 0] * nb[1] + B[:, 1]) * nb[2] + B[:, 2]) * nb[3] + B[:, 3]
    colour = B.sum(axis=1) % 2
    parity = c.sum(axis=1) % 2
    eo = O.EvenOdd(op)
    inv_full = np.zeros((V, 12, 12), dtype=np.complex128)
    inv_full[eo.odd] = np.linalg.inv(eo.Doo_blocks)

    def restrict(f, mask):
        g = np.zeros_like(f)
        g[mask] = f[mask]
        return g

    psi = np.zeros_like(eta)
    kept = [None, None]
    last = [np.zeros_like(eta), np.zeros_like(eta)]   # each colour's last correction
    for cy in range(ncy):
        for col in (0, 1):
            inb = colour == col
            even_b, odd_b = inb & (parity == 0), inb & (parity == 1)

            def D_B_eo(f, rows, cols):
                return restrict(restrict(op.apply(restrict(restrict(f, cols), inb)), inb), rows)

            def Doo_inv_B(f):
                return restrict(np.einsum("nij,nj->ni", inv_full, f.reshape(V, 12)).reshape(V, 4, 3), odd_b)

            def D_hat_B(f):
                return D_B_eo(f, even_b, even_b) - D_B_eo(Doo_inv_B(D_B_eo(f, odd_b, even_b)), even_b, odd_b)

            base = restrict(eta, inb) if cy == 0 else kept[col]
            r = base - cross_sign * restrict(op.apply(last[1 - col]), inb)
            ce = restrict(r, even_b) - D_B_eo(Doo_inv_B(r), even_b, odd_b)
            y, rho = O.block_mr(D_hat_B, ce, block_id, int(np.prod(nb)), nmr, even_b)
            yo = Doo_inv_B(restrict(r, odd_b) - D_B_eo(y, odd_b, even_b))
            last[col] = y + yo
            kept[col] = rho
            psi = psi + y + yo
    return psi


def test_carried_residual_equals_recomputed_residual():
    """The identity behind the FP32 Schwarz kernel, which carries the
    residual of a block visit from the previous visits instead of computing
    eta - D psi: with the same sweep the two agree to rounding, and the
    check is sharp (the crossing term with the wrong sign fails it)."""
    _, op, eta = setup()
    ref = O.sap(op, eta, 3, 3, bs=BS)
    got = sap_carried(op, eta, 3, 3, BS)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12
    bad = sap_carried(op, eta, 3, 3, BS, cross_sign=-1.0)
    assert np.abs(bad - ref).max() / np.abs(ref).max() > 1e-3
