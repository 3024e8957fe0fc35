"""Plain FP64 CPU oracle for the pseudofermion action of the RHMC.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and
its Python binding) may import, call or link this module. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and its
``--impl reference`` arm) use it. It shares no code with the GPU path.

What it computes (Sec. 2.4 of the openQ*D proceedings, arXiv:1710.08839):

* ``ln_abs_det_blocks`` / ``ln_abs_det_Doo`` -- ln|Det D_oo|, the exact term
  of the pseudofermion action S_pf. D_oo is diagonal in the lattice index, so
  its determinant is the product of the determinants of its 12x12 site
  blocks (read off from D itself by ``EvenOdd``).
* ``D_hat_dagger`` -- the adjoint of D_hat = D_ee - D_eo D_oo^-1 D_oe. D is
  gamma5-hermitian, and gamma5 commutes with the site-diagonal part M, so
  D_hat^dag = gamma5 D_hat gamma5 on the even sites. (Pinned against the dense
  conjugate transpose, not assumed.)
* ``normal_apply`` -- (D_hat^dag D_hat + sigma) on an even-site field.
* ``cg`` -- plain conjugate gradient (Hestenes and Stiefel) for a Hermitian
  positive definite operator. The paper solves these systems with CG and
  multi-shift CG (Sec. 2.4, App. A); it prints neither.
* ``rational_apply`` -- P phi with
  P = prod_j (D_hat^dag D_hat + nu_j^2) / (D_hat^dag D_hat + mu_j^2),
  the frequency-splitting factor of the rational approximation (Sec. 2.4),
  applied factor by factor: multiply by (A + nu_j^2), then solve with
  (A + mu_j^2). The factors commute, so the order is immaterial.
* ``pf_action_term`` -- phi^dag P phi, one term of S_pf.

Pins (tests/test_oracle_rhmc.py): closed form of D_hat^dag D_hat on the
even-site plane waves of the free field, ln|Det D_oo| of the free field,
Det D = Det D_oo Det D_hat on tiny lattices, the dense conjugate transpose,
dense solves and the dense eigen-decomposition of P, and the rational
approximation of Table 2 (tests/golden/table2_rational.txt).
"""
from __future__ import annotations

import numpy as np

from .qxd_oracle import GAMMA5, EvenOdd, norm, spin_mul, vdot


def ln_abs_det_blocks(blocks) -> float:
    """sum_x ln|det B(x)| over an array of square blocks (n, k, k)."""
    _, logdet = np.linalg.slogdet(np.asarray(blocks))
    return float(np.sum(logdet))


def ln_abs_det_Doo(eo: EvenOdd) -> float:
    """ln|Det D_oo| (Sec. 2.4): D_oo is block-diagonal, one 12x12 block per odd site."""
    return ln_abs_det_blocks(eo.Doo_blocks)


def gamma5_mul(f):
    return spin_mul(GAMMA5, f)


def D_hat_dagger(eo: EvenOdd, fe):
    """D_hat^dag fe = gamma5 D_hat gamma5 fe."""
    return gamma5_mul(eo.D_hat(gamma5_mul(fe)))


def normal_apply(eo: EvenOdd, fe, sigma: float = 0.0):
    """(D_hat^dag D_hat + sigma) fe."""
    return D_hat_dagger(eo, eo.D_hat(fe)) + sigma * fe


# iteration limit of ``cg`` (a module constant so that tests can lower it)
CG_MAX_ITER = 100000


def cg(apply, b, tol: float = 1e-13, max_iter: int | None = None):
    """Conjugate gradient for a Hermitian positive definite operator.

    x0 = 0, r = p = b; per step alpha = |r|^2 / <p, A p>, x += alpha p,
    r -= alpha A p, beta = |r_new|^2 / |r|^2, p = r + beta p; stop when
    |r| <= tol |b|. Returns (x, iterations, true relative residual).
    """
    if max_iter is None:
        max_iter = CG_MAX_ITER
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    bn = norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    r = b.copy()
    p = r.copy()
    rr = vdot(r, r).real
    it = 0
    while it < max_iter and np.sqrt(rr) > tol * bn:
        q = apply(p)
        alpha = rr / vdot(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        rr_new = vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, norm(b - apply(x)) / bn


def shifted_solve(eo: EvenOdd, b, sigma: float, tol: float = 1e-13):
    """x = (D_hat^dag D_hat + sigma)^-1 b by CG; returns (x, iterations, relres)."""
    return cg(lambda v: normal_apply(eo, v, sigma), b, tol=tol)


def rational_apply(eo: EvenOdd, phi, nu, mu, tol: float = 1e-13):
    """P phi, P = prod_j (A + nu_j^2)(A + mu_j^2)^-1, A = D_hat^dag D_hat (Sec. 2.4)."""
    v = np.asarray(phi, dtype=np.complex128)
    for n_j, m_j in zip(nu, mu):
        v = normal_apply(eo, v, n_j * n_j)
        v, _, _ = shifted_solve(eo, v, m_j * m_j, tol=tol)
    return v


def pf_action_term(eo: EvenOdd, phi, nu, mu, tol: float = 1e-13) -> float:
    """phi^dag P phi (real: P is Hermitian positive definite)."""
    return vdot(phi, rational_apply(eo, phi, nu, mu, tol=tol)).real
