"""Plain FP64 CPU oracle for local deflation of the SAP-preconditioned GCR solver.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and
its Python binding) may import, call or link this module. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and its
``--impl reference`` arm) use it. It shares no code with the GPU path.

The paper names openQ*D's deflation-accelerated solver (Sec. 1, Sec. 3 and
Table 2) without giving it; this is the standard local deflation of Luscher
(2007), written from its definitions:

* blocks: the lattice is cut into bs^4 blocks, numbered lexicographically in
  the block coordinates B = floor(x / bs) (B3 fastest).
* ``block_orthonormalize`` -- given Ns global fields psi_k, the fields
  restricted to each block b are orthonormalised in order:
  psi_k|_b = sum_{l <= k} phi_{b,l} R_{lk} with R upper triangular and
  R_kk > 0 (the unique QR factorisation). The phi_{b,k} span the deflation
  subspace S.
* ``little_operator`` -- A_{(b,k),(b',l)} = <phi_{b,k}, D phi_{b',l}>, dense
  on small lattices (non-zero for b' = b and the 8 neighbouring blocks).
* ``restrict`` / ``prolong`` -- c_{b,k} = <phi_{b,k}, eta> and P c =
  sum c_{b,k} phi_{b,k}.
* ``deflated_preconditioner`` -- the two-level preconditioner
  M eta = P A^-1 P^dag eta + M_SAP(eta - D P A^-1 P^dag eta), i.e. a coarse
  correction on S followed by the Schwarz method on the remainder (with the
  little system solved exactly here).

Pins (tests/test_oracle_dfl.py): orthonormality and the QR relation; the
free field with block-constant basis vectors, where A is the coarse Wilson
operator (1 + m0) c_b - 1/8 sum_mu [(1 - g_mu) c_{b+mu} + (1 + g_mu)
c_{b-mu}] with closed-form plane waves on the block torus (shifted
boundaries included); P^dag P = 1; the preconditioner inverts D exactly on
D S; a deflated GCR solve equals the dense solution.
"""
from __future__ import annotations

import numpy as np

from .qxd_oracle import Dirac, Lattice, sap


def block_index(lat: Lattice, bs: int = 4) -> np.ndarray:
    """Block number of every site (lexicographic site order)."""
    for mu in range(4):
        if lat.N[mu] % bs:
            raise ValueError("every extent must be a multiple of the block size")
    c = lat.coords(lat.all_sites()) // bs
    nb = [lat.N[mu] // bs for mu in range(4)]
    return ((c[:, 0] * nb[1] + c[:, 1]) * nb[2] + c[:, 2]) * nb[3] + c[:, 3]


def block_orthonormalize(lat: Lattice, psi, bs: int = 4) -> np.ndarray:
    """phi[k] (Ns, V, 4, 3): block-wise orthonormalisation of psi[k] in order."""
    psi = np.asarray(psi, dtype=np.complex128)
    ns = psi.shape[0]
    bid = block_index(lat, bs)
    phi = np.zeros_like(psi)
    for b in range(bid.max() + 1):
        sites = np.nonzero(bid == b)[0]
        M = psi[:, sites].reshape(ns, -1).T          # (12 * sites, Ns)
        Q, R = np.linalg.qr(M)
        sgn = np.sign(np.real(np.diag(R)))
        Q = Q * sgn[None, :]                           # R_kk > 0
        phi[:, sites] = Q.T.reshape(ns, len(sites), 4, 3)
    return phi


def restrict(lat: Lattice, phi, eta, bs: int = 4) -> np.ndarray:
    """c[b, k] = <phi_{b,k}, eta> (the sum over the sites of block b)."""
    bid = block_index(lat, bs)
    nblk = bid.max() + 1
    w = np.einsum("kxsc,xsc->kx", np.conj(phi), eta)  # per site
    c = np.zeros((nblk, phi.shape[0]), dtype=np.complex128)
    for k in range(phi.shape[0]):
        c[:, k] = np.bincount(bid, weights=w[k].real, minlength=nblk) + \
            1j * np.bincount(bid, weights=w[k].imag, minlength=nblk)
    return c


def prolong(lat: Lattice, phi, c, bs: int = 4) -> np.ndarray:
    """sum_{b,k} c[b, k] phi_{b,k} (a field (V, 4, 3))."""
    bid = block_index(lat, bs)
    return np.einsum("xk,kxsc->xsc", c[bid], phi)


def little_operator(op: Dirac, phi, bs: int = 4) -> np.ndarray:
    """Dense A[(b,k), (b',l)] = <phi_{b,k}, D phi_{b',l}>, shape (nblk Ns, nblk Ns)."""
    lat = op.lat
    bid = block_index(lat, bs)
    nblk = bid.max() + 1
    ns = phi.shape[0]
    A = np.zeros((nblk, ns, nblk, ns), dtype=np.complex128)
    for bp in range(nblk):
        mask = (bid == bp)[:, None, None]
        cols = np.where(mask[None], phi, 0.0)        # phi_{b',l} for l < Ns
        Dcols = op.apply(cols)                        # (Ns, V, 4, 3)
        for l in range(ns):
            A[:, :, bp, l] = restrict(lat, phi, Dcols[l], bs)
    return A.reshape(nblk * ns, nblk * ns)


def deflated_preconditioner(op: Dirac, phi, A, eta, ncy: int, nmr: int, bs: int = 4):
    """M eta = P A^-1 P^dag eta + M_SAP(eta - D P A^-1 P^dag eta)."""
    lat = op.lat
    nblk, ns = A.shape[0] // phi.shape[0], phi.shape[0]
    c = restrict(lat, phi, eta, bs).reshape(-1)
    y = np.linalg.solve(A, c).reshape(nblk, ns)
    chi = prolong(lat, phi, y, bs)
    return chi + sap(op, eta - op.apply(chi), ncy, nmr, bs)
