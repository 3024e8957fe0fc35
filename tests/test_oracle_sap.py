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
