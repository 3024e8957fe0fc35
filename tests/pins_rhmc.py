"""Pins of the pseudofermion-action oracle (``oracle.qxd_rhmc``).

Each ``pin_*`` returns the largest deviation from what the paper or
mathematics fixes; ``test_oracle_rhmc.py`` checks the deviations and plants
mistakes in the oracle to show that each pin can fail.

Closed form used below (derived by hand from Sec. 2.3-2.4, free field U = 1,
z = 1, where the SW term vanishes and M = 4 + m0 at every site): write
D = (4 + m0) + H with H the hopping part. On a plane wave of allowed momentum
p, H acts as h(p) = -c + i gamma.s with c = sum_mu cos p_mu,
s_mu = sin p_mu. The even-site restriction of the wave is the mean of the
waves at p and p + (pi, pi, pi, pi), where h changes sign, so H^2 acts on it
as h(p)^2 = c^2 - s^2 - 2ic gamma.s. Hence
  D_hat = (4 + m0) - H^2 / (4 + m0) = (a + 2ic gamma.s) / (4 + m0),
  a = (4 + m0)^2 - c^2 + s^2,
and, gamma.s being Hermitian with square s^2,
  D_hat^dag D_hat = (a^2 + 4 c^2 s^2) / (4 + m0)^2   (a multiple of 1).
"""
from __future__ import annotations

import os

import numpy as np

import oracle as O
from oracle import qxd_rhmc as R
import pins as P

MU_HAT = 1.0e-3   # twisted-mass regulator of the QCD runs (Sec. 3 states mu_hat = 0.001)
SPECTRUM = (1.98e-3, 7.62)  # range of |gamma5 D_hat| of the QCD2 rational approximation (App. A)


def table2():
    """(j, nu, mu, factor) columns of tests/golden/table2_rational.txt."""
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_rational.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    j = np.array([int(r[0]) for r in rows])
    nu = np.array([float(r[1]) for r in rows])
    mu = np.array([float(r[2]) for r in rows])
    fac = np.array([int(r[3]) for r in rows])
    return j, nu, mu, fac


def factor_P(k):
    """(nu, mu) of the frequency-splitting factor P_k of Table 2."""
    _, nu, mu, fac = table2()
    return nu[fac == k], mu[fac == k]


def free_lambda(p, m0):
    """Eigenvalue of D_hat^dag D_hat on the even-site plane waves of momentum p (free field)."""
    c = np.sum(np.cos(p))
    s2 = np.sum(np.sin(p) ** 2)
    a = (4 + m0) ** 2 - c * c + s2
    return (a * a + 4 * c * c * s2) / (4 + m0) ** 2


def pin_free_normal(lat, m0=0.15, ntrial=4, seed=21):
    """Free field: D_hat^dag D_hat, its shifted CG solve and P act on even-site
    plane waves as the numbers lambda(p), 1/(lambda + sigma), f(lambda)."""
    r = P.rng(seed)
    op = O.Dirac(lat, P.unit_gauge(lat), m0, 1.4, 0.8, 2)
    eo = O.EvenOdd(op)
    nu, mu = factor_P(1)
    err = 0.0
    for _ in range(ntrial):
        n = [int(r.integers(0, 2 * lat.N[k])) for k in range(4)]
        p = P.allowed_momentum(lat, n)
        u = P.random_spinor(r, ())
        phi = P.plane_wave(lat, p, u)[eo.even]
        lam = free_lambda(p, m0)
        scale = np.abs(phi).max()
        err = max(err, np.abs(R.normal_apply(eo, phi) - lam * phi).max() / (lam * scale))
        sig = 0.37
        x, _, _ = R.shifted_solve(eo, phi, sig)
        err = max(err, np.abs(x - phi / (lam + sig)).max() * (lam + sig) / scale)
        f = np.prod((lam + nu ** 2) / (lam + mu ** 2))
        err = max(err, np.abs(R.rational_apply(eo, phi, nu, mu) - f * phi).max() / (f * scale))
    return err


def pin_free_logdet(lat, m0=0.15):
    """Free field: every site block of D_oo is (4 + m0) times the 12x12 identity."""
    op = O.Dirac(lat, P.unit_gauge(lat), m0, 1.4, 0.8, -1)
    eo = O.EvenOdd(op)
    exact = (lat.V // 2) * 12 * np.log(4 + m0)
    return abs(R.ln_abs_det_Doo(eo) - exact) / exact


def _dense_dhat(eo):
    ne = len(eo.even)
    e = np.eye(12 * ne, dtype=complex).reshape(12 * ne, ne, 4, 3)
    return eo.D_hat(e).reshape(12 * ne, 12 * ne).T, e


def _random_eo(lat, seed, m0=0.1, qhat=2):
    r = P.rng(seed)
    g = P.random_physical_gauge(r, lat)
    return r, O.EvenOdd(O.Dirac(lat, g, m0, 1.2, 0.9, qhat))


def pin_dagger_dense(lat, seed=22):
    """D_hat_dagger equals the conjugate transpose of the dense D_hat."""
    _, eo = _random_eo(lat, seed)
    Dh, e = _dense_dhat(eo)
    n = Dh.shape[0]
    Ddag = R.D_hat_dagger(eo, e).reshape(n, n).T
    return np.abs(Ddag - Dh.conj().T).max() / np.abs(Dh).max()


def pin_logdet_factorisation(lat, seed=23):
    """ln|Det D| = ln|Det D_oo| + ln|Det D_hat| (Sec. 2.4) with dense determinants."""
    _, eo = _random_eo(lat, seed, qhat=-1)
    M = O.dense_matrix(eo.op)
    Dh, _ = _dense_dhat(eo)
    _, ld_full = np.linalg.slogdet(M)
    _, ld_hat = np.linalg.slogdet(Dh)
    return abs(ld_full - (R.ln_abs_det_Doo(eo) + ld_hat)) / abs(ld_full)


def pin_shifted_cg_dense(lat, sigma=0.05, seed=24):
    """CG solve of (D_hat^dag D_hat + sigma) x = b against a dense solve."""
    r, eo = _random_eo(lat, seed)
    Dh, _ = _dense_dhat(eo)
    A = Dh.conj().T @ Dh + sigma * np.eye(Dh.shape[0])
    b = P.random_spinor(r, (len(eo.even),))
    x_ref = np.linalg.solve(A, b.ravel()).reshape(b.shape)
    x, _, res = R.shifted_solve(eo, b, sigma)
    return max(np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref), res * 1e-2)


def pin_rational_eigen(lat, k=1, seed=25):
    """P_k phi against the eigen-decomposition of the dense D_hat^dag D_hat,
    and phi^dag P_k phi against the same."""
    r, eo = _random_eo(lat, seed)
    nu, mu = factor_P(k)
    Dh, _ = _dense_dhat(eo)
    lam, V = np.linalg.eigh(Dh.conj().T @ Dh)
    f = np.prod((lam[:, None] + nu ** 2) / (lam[:, None] + mu ** 2), axis=1)
    phi = P.random_spinor(r, (len(eo.even),))
    ref = (V @ (f * (V.conj().T @ phi.ravel()))).reshape(phi.shape)
    got = R.rational_apply(eo, phi, nu, mu)
    e1 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    s_ref = float(np.vdot(phi.ravel(), ref.ravel()).real)
    e2 = abs(R.pf_action_term(eo, phi, nu, mu) - s_ref) / s_ref
    return max(e1, e2)


def table2_deviation(mu_hat=MU_HAT, lo=SPECTRUM[0], hi=SPECTRUM[1], npts=20001):
    """max_y |A R(y^2) (y^2 + mu_hat^2)^(1/4) - 1| over y in [lo, hi], with the
    Table 2 zeros and poles and the best constant A (App. A: R approximates
    (D_hat^dag D_hat + mu_hat^2)^(-1/4) over the spectrum of |gamma5 D_hat|)."""
    _, nu, mu, _ = table2()
    y = np.geomspace(lo, hi, npts)
    f = np.prod((y[:, None] ** 2 + nu ** 2) / (y[:, None] ** 2 + mu ** 2), axis=1)
    g = f * (y ** 2 + mu_hat ** 2) ** 0.25
    return (g.max() - g.min()) / (g.max() + g.min())
