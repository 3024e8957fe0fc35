"""Pins of the local-deflation oracle (``oracle.qxd_dfl``).

Closed form used below (derived by hand from D, free field U = 1, z = 1,
block size bs, Ns = 12 block-constant basis vectors phi_{b,a} = e_a /
sqrt(bs^4) with e_a the spin-colour unit vectors): for x in block b,
(D chi_b e)(x) = (4 + m0) e - 1/2 sum_mu [(1 - g_mu) chi_b(x+mu) + (1 + g_mu)
chi_b(x-mu)] e, and of the bs^4 sites of b, bs^4 - bs^3 have x+mu in b while
bs^3 have it in b+mu. Hence
  A_{b,b}     = (4 + m0) - 4 (1 - 1/bs) = m0 + 4/bs,
  A_{b,b+-mu} = -(1 - -+ g_mu) / (2 bs),
and on block plane waves c_b = exp(i P.B) u, with P = bs p for an allowed
site momentum p of the shifted torus (so the phases close across the
shifted block boundaries),
  (A c)_b = [m0 + 4/bs - (1/bs) sum_mu cos P_mu + (i/bs) sum_mu g_mu sin P_mu] c_b.
"""
from __future__ import annotations

import numpy as np

import oracle as O
from oracle import qxd_dfl as DF
import pins as P

BS = 2


def pin_block_qr(lat=O.Lattice(4, 2, 4, 2, 0b1110), ns=5, seed=41):
    """phi is block-orthonormal, <phi_{b,l}, psi_k> = R_lk upper triangular
    with R_kk > 0, and psi_k = sum_l R_lk phi_{b,l} on every block."""
    r = P.rng(seed)
    psi = P.random_spinor(r, (ns, lat.V))
    phi = DF.block_orthonormalize(lat, psi, BS)
    err = 0.0
    for k in range(ns):
        c = DF.restrict(lat, phi, psi[k], BS)             # (nblk, ns): R_lk per block
        err = max(err, np.abs(c[:, k + 1:]).max() if k + 1 < ns else 0.0)
        assert np.all(c[:, k].real > 0)
        err = max(err, np.abs(c[:, k].imag).max())
        err = max(err, np.abs(DF.prolong(lat, phi, c, BS) - psi[k]).max())
        for l in range(ns):
            g = DF.restrict(lat, phi, phi[l], BS)           # <phi_{b,k'}, phi_{b,l}>
            err = max(err, np.abs(g - (np.arange(ns) == l)[None, :]).max())
    return err


def free_symbol(P_, m0, bs=BS):
    M = (m0 + 4.0 / bs) * np.eye(4, dtype=complex)
    for mu in range(4):
        M += -np.cos(P_[mu]) / bs * np.eye(4) + 1j * np.sin(P_[mu]) / bs * P.GAMMA_HAND[mu]
    return M


def pin_free_little_operator(lat=O.Lattice(4, 4, 4, 4, 0b1110), m0=0.2, ntrial=4, seed=42):
    """Free field, block-constant basis: block plane waves are eigenvectors of
    A with the coarse Wilson symbol (C* block boundaries included)."""
    r = P.rng(seed)
    op = O.Dirac(lat, P.unit_gauge(lat), m0, 1.3, 0.8, 2)
    e = np.eye(12, dtype=complex).reshape(12, 4, 3)
    psi = np.broadcast_to(e[:, None], (12, lat.V, 4, 3)).copy()
    phi = DF.block_orthonormalize(lat, psi, BS)
    A = DF.little_operator(op, phi, BS)
    nb = [lat.N[mu] // BS for mu in range(4)]
    nblk = int(np.prod(nb))
    B = np.stack(np.meshgrid(*[np.arange(n) for n in nb], indexing="ij"), -1).reshape(nblk, 4)
    err = 0.0
    for _ in range(ntrial):
        n = [int(r.integers(0, 2 * lat.N[k])) for k in range(4)]
        Pm = BS * P.allowed_momentum(lat, n)
        u = P.random_spinor(r, ())                         # (4, 3)
        c = np.exp(1j * (B @ Pm))[:, None, None] * u[None]  # (nblk, 4, 3); index a = 3 spin + colour
        got = (A @ c.reshape(-1)).reshape(nblk, 4, 3)
        ref = np.einsum("st,btc->bsc", free_symbol(Pm, m0), c)
        err = max(err, np.abs(got - ref).max() / np.abs(ref).max())
    return err


def _random_case(lat, seed, ns=4):
    r = P.rng(seed)
    g = P.random_physical_gauge(r, lat, 0.4, 0.4)
    op = O.Dirac(lat, g, 0.2, 1.0, 1.0, -1)
    phi = DF.block_orthonormalize(lat, P.random_spinor(r, (ns, lat.V)), BS)
    return r, op, phi


def pin_prolong_restrict(lat=O.Lattice(4, 2, 4, 2, 0b1110), seed=43):
    """P^dag P = 1 on coefficient vectors, and A c = P^dag D P c."""
    r, op, phi = _random_case(lat, seed)
    nblk = DF.block_index(lat, BS).max() + 1
    c = r.normal(size=(nblk, phi.shape[0])) + 1j * r.normal(size=(nblk, phi.shape[0]))
    e1 = np.abs(DF.restrict(lat, phi, DF.prolong(lat, phi, c, BS), BS) - c).max()
    A = DF.little_operator(op, phi, BS)
    lhs = (A @ c.reshape(-1)).reshape(c.shape)
    rhs = DF.restrict(lat, phi, op.apply(DF.prolong(lat, phi, c, BS)), BS)
    return max(e1, np.abs(lhs - rhs).max() / np.abs(rhs).max())


def pin_preconditioner_exact_on_DS(lat=O.Lattice(4, 4, 4, 4, 0b1110), seed=44):
    """For eta = D P c the deflated preconditioner returns P c exactly (the
    coarse correction solves it and the Schwarz step sees a zero residual)."""
    r, op, phi = _random_case(lat, seed)
    nblk = DF.block_index(lat, BS).max() + 1
    c = r.normal(size=(nblk, phi.shape[0])) + 1j * r.normal(size=(nblk, phi.shape[0]))
    x = DF.prolong(lat, phi, c, BS)
    A = DF.little_operator(op, phi, BS)
    got = DF.deflated_preconditioner(op, phi, A, op.apply(x), 2, 2, BS)
    return np.abs(got - x).max() / np.abs(x).max()


def pin_little_even_odd(lat=O.Lattice(4, 4, 4, 4, 0b1110), seed=45, planted_colouring=False):
    """The structure the GPU's even-odd little solve relies on: neighbouring
    blocks have opposite colours (parity of the block coordinates, also
    across the shifted C* boundary), so A couples no two different blocks of
    one colour; hence A_oo is block diagonal and A y = c is solved by
    y_e = (A_ee - A_eo A_oo^-1 A_oe)^-1 (c_e - A_eo A_oo^-1 c_o),
    y_o = A_oo^-1 (c_o - A_oe y_e). Returns the larger of the same-colour
    coupling (relative to max |A|) and the relative error of that solve
    against the dense solve. planted_colouring colours the blocks by B3 alone
    (a plausible mistake), which leaves same-colour couplings."""
    r, op, phi = _random_case(lat, seed)
    ns = phi.shape[0]
    nblk = DF.block_index(lat, BS).max() + 1
    nb = [lat.N[mu] // BS for mu in range(4)]
    B = np.array(np.unravel_index(np.arange(nblk), nb))
    colour = (B[3] if planted_colouring else B.sum(axis=0)) % 2
    A = DF.little_operator(op, phi, BS)
    A4 = A.reshape(nblk, ns, nblk, ns)
    same = (colour[:, None] == colour[None, :]) & ~np.eye(nblk, dtype=bool)
    off = np.abs(A4.transpose(0, 2, 1, 3)[same]).max() / np.abs(A).max()
    ie = np.nonzero(np.repeat(colour == 0, ns))[0]
    io = np.nonzero(np.repeat(colour == 1, ns))[0]
    c = r.normal(size=nblk * ns) + 1j * r.normal(size=nblk * ns)
    Aee, Aeo, Aoe, Aoo = A[np.ix_(ie, ie)], A[np.ix_(ie, io)], A[np.ix_(io, ie)], A[np.ix_(io, io)]
    schur = Aee - Aeo @ np.linalg.solve(Aoo, Aoe)
    y = np.zeros_like(c)
    y[ie] = np.linalg.solve(schur, c[ie] - Aeo @ np.linalg.solve(Aoo, c[io]))
    y[io] = np.linalg.solve(Aoo, c[io] - Aoe @ y[ie])
    ref = np.linalg.solve(A, c)
    return max(off, np.abs(y - ref).max() / np.abs(ref).max())
