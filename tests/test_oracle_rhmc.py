"""The pseudofermion-action oracle against closed forms, dense linear algebra
and the paper's Table 2 (no GPU); and planted mistakes that the pins catch."""
import numpy as np
import pytest

import oracle as O
from oracle import qxd_rhmc as R
import pins_rhmc as PR

FREE = O.Lattice(4, 2, 4, 2, 0b1110)        # C* in x, y, z; 128 sites
FREE_PERIODIC = O.Lattice(4, 4, 2, 4, 0)    # plain torus
TINY = O.Lattice(2, 2, 2, 2, 0b1110)        # 64 sites: dense matrices
TINY2 = O.Lattice(4, 2, 2, 2, 0b0110)       # 128 sites, z periodic
TOL = 1e-10


@pytest.mark.parametrize("lat", [FREE, FREE_PERIODIC], ids=["cstar3", "periodic"])
def test_free_field_closed_forms(lat):
    assert PR.pin_free_normal(lat) < TOL
    assert PR.pin_free_logdet(lat) < 1e-14


@pytest.mark.parametrize("lat", [TINY, TINY2], ids=["64", "128"])
def test_dense_identities(lat):
    assert PR.pin_dagger_dense(lat) < 1e-13
    assert PR.pin_logdet_factorisation(lat) < 1e-12
    assert PR.pin_shifted_cg_dense(lat) < 1e-10


@pytest.mark.parametrize("k", [1, 2])
def test_rational_factor_eigen(k):
    assert PR.pin_rational_eigen(TINY, k=k) < 1e-10


def test_table2_is_the_quarter_root_approximation():
    # the 14 zero/pole pairs approximate (y^2 + mu_hat^2)^(-1/4) over the
    # stated range; the paper's 1e-6 is limited here by its 5-digit rounding
    assert PR.table2_deviation() < 1e-4
    # without the regulator the small-y end is far off: mu_hat is needed
    assert PR.table2_deviation(mu_hat=0.0) > 1e-2
    j, nu, mu, fac = PR.table2()
    assert list(j) == list(range(1, 15)) and list(np.unique(fac)) == list(range(1, 9))
    # zeros and poles interlace (every residue of P is positive)
    assert np.all(nu > mu) and np.all(nu[1:] < mu[:-1])


# ---------------------------------------------------------------------------
# planted mistakes
# ---------------------------------------------------------------------------


CAUGHT = 1e-6


def _all_pins():
    """Largest deviation over the pins, cheapest first; stops at the first pin
    that catches the mistake."""
    worst = 0.0
    for c in (lambda: PR.pin_free_logdet(FREE),
              lambda: PR.pin_dagger_dense(TINY),
              lambda: PR.pin_logdet_factorisation(TINY),
              lambda: PR.pin_free_normal(FREE, ntrial=2),
              lambda: PR.pin_shifted_cg_dense(TINY),
              lambda: PR.pin_rational_eigen(TINY)):
        v = float(c())
        worst = max(worst, v if np.isfinite(v) else np.inf)
        if worst > CAUGHT:
            break
    return worst


def _dagger_without_gamma5(eo, fe):
    return eo.D_hat(fe)


def _rational_shift_not_squared(eo, phi, nu, mu, tol=1e-13):
    v = np.asarray(phi, dtype=np.complex128)
    for n_j, m_j in zip(nu, mu):
        v = R.normal_apply(eo, v, n_j * n_j)
        v, _, _ = R.shifted_solve(eo, v, m_j, tol=tol)
    return v


def _logdet_even_blocks(eo):
    return R.ln_abs_det_blocks(eo.Dee_blocks)


def _logdet_one_chirality(eo):
    # determinant of the upper-left 6x6 (one chirality) only
    return R.ln_abs_det_blocks(eo.Doo_blocks[:, :6, :6])


def _normal_drops_shift(eo, fe, sigma=0.0):
    return R.D_hat_dagger(eo, eo.D_hat(fe))


def _cg_beta_inverted(apply, b, tol=1e-13, max_iter=None):
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = O.vdot(r, r).real
    for _ in range(max_iter or R.CG_MAX_ITER):
        q = apply(p)
        alpha = rr / O.vdot(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        rr_new = O.vdot(r, r).real
        p = r + (rr / rr_new) * p
        rr = rr_new
        if np.sqrt(rr) <= tol * O.norm(b):
            break
    return x, 0, O.norm(b - apply(x)) / O.norm(b)


MUTATIONS = {
    "dagger_without_gamma5": ("D_hat_dagger", _dagger_without_gamma5),
    "rational_shift_not_squared": ("rational_apply", _rational_shift_not_squared),
    "logdet_even_blocks": ("ln_abs_det_Doo", _logdet_even_blocks),
    "logdet_one_chirality": ("ln_abs_det_Doo", _logdet_one_chirality),
    "normal_drops_shift": ("normal_apply", _normal_drops_shift),
    "cg_beta_inverted": ("cg", _cg_beta_inverted),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(R, attr, fn)
    # a planted mistake may keep CG from converging: bound its work
    monkeypatch.setattr(R, "CG_MAX_ITER", 400)
    assert _all_pins() > CAUGHT
