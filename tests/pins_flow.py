"""Pins of the gauge-observable and Wilson-flow oracle (``oracle.qxd_flow``).

Closed forms used below (derived by hand from the definitions): a constant
abelian field strength on the periodic torus, with plaquette angle
phi^c_munu in plane (mu, nu) for colour c, is realised by the diagonal links
  A^c_nu(x) += phi x_mu,   A^c_mu(x) += -phi N_mu x_nu  where x_mu = N_mu - 1,
phi = 2 pi n / (N_mu N_nu) with integer flux n (sum_c n^c = 0 keeps the links
in SU(3)). Every plaquette of the plane then carries exp(i phi^c), the four
clover leaves agree, and F_munu = i diag(sin phi^c_munu). Hence
  E_SU(3) = sum_{mu<nu} sum_c sin^2 phi^c_munu,
  Q_top   = V/(4 pi^2) sum_c [-s01 s23 + s02 s13 - s03 s12]^c,  s = sin phi,
  E_U(1)  = sum_{mu<nu} sin^2 phi_munu / q_el^2  (the same for a U(1) field),
and the Wilson flow leaves the field unchanged (the six plaquettes through a
link cancel pairwise in W - W^dag).
"""
from __future__ import annotations

import numpy as np

import oracle as O
from oracle import qxd_flow as F
import pins as P

PLANES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def flux_angles(lat, nflux):
    """Angles (V, 4) of a constant abelian field with nflux[(mu, nu)] quanta;
    returns the angles and the plaquette angles phi[(mu, nu)]."""
    c = lat.coords(lat.all_sites())
    N = lat.N
    A = np.zeros((lat.V, 4))
    phi = {}
    for (mu, nu), n in nflux.items():
        ph = 2 * np.pi * n / (N[mu] * N[nu])
        phi[mu, nu] = ph
        A[:, nu] += ph * c[:, mu]
        A[:, mu] += np.where(c[:, mu] == N[mu] - 1, -ph * N[mu] * c[:, nu], 0.0)
    return A, phi


def diag_su3_field(lat, flux_c):
    """SU(3) links diag(exp(i A^c)) for per-colour fluxes flux_c[c] (c = 0, 1;
    colour 2 carries minus their sum)."""
    A0, phi0 = flux_angles(lat, flux_c[0])
    A1, phi1 = flux_angles(lat, flux_c[1])
    A2 = -(A0 + A1)
    U = np.zeros((lat.V, 4, 3, 3), dtype=complex)
    for c, Ac in enumerate((A0, A1, A2)):
        U[:, :, c, c] = np.exp(1j * Ac)
    phis = []
    for pl in PLANES:
        a, b = phi0.get(pl, 0.0), phi1.get(pl, 0.0)
        phis.append((a, b, -(a + b)))
    return U, dict(zip(PLANES, phis))


def closed_forms(lat, phis):
    s = {pl: np.sin(np.array(v)) for pl, v in phis.items()}
    e = sum(np.sum(v ** 2) for v in s.values())
    q = lat.V / (4 * np.pi ** 2) * np.sum(-s[0, 1] * s[2, 3] + s[0, 2] * s[1, 3] - s[0, 3] * s[1, 2])
    return e, q


TORUS = O.Lattice(4, 4, 6, 4, 0)
FLUX_C = [{(0, 1): 1, (2, 3): 2, (0, 2): -1}, {(0, 1): -2, (2, 3): 1, (1, 3): 1, (0, 3): 1, (1, 2): -1}]
FLUX_U1 = {(0, 1): 1, (0, 3): -1, (1, 2): 2}
Q_EL = 1.0 / 6.0


def pin_constant_flux(lat=TORUS):
    """E_SU(3), Q_top, E_U(1) against the closed forms."""
    U, phis = diag_su3_field(lat, FLUX_C)
    A, phi_u1 = flux_angles(lat, FLUX_U1)
    g = O.GaugeField.from_extended(lat, U, A)
    e, eu1, q = F.observables(lat, g, Q_EL)
    e_ref, q_ref = closed_forms(lat, phis)
    eu1_ref = sum(np.sin(v) ** 2 for v in phi_u1.values()) / Q_EL ** 2
    assert abs(q_ref) > 0.1 and e_ref > 0.1  # the case is not degenerate
    return max(abs(e - e_ref) / e_ref, abs(q - q_ref) / abs(q_ref), abs(eu1 - eu1_ref) / eu1_ref)


def pin_constant_flux_is_stationary(lat=TORUS, eps=0.05, nsteps=2):
    U, _ = diag_su3_field(lat, FLUX_C)
    A, _ = flux_angles(lat, FLUX_U1)
    g = O.GaugeField.from_extended(lat, U, np.remainder(A + np.pi, 2 * np.pi) - np.pi)
    h = F.wilson_flow(lat, g, eps, nsteps)
    U0, A0 = g.extended_arrays()
    U1, A1 = h.extended_arrays()
    dA = np.remainder(A1 - A0 + np.pi, 2 * np.pi) - np.pi
    return max(np.abs(U1 - U0).max(), np.abs(dA).max())


def pin_unit_field(lat=O.Lattice(4, 2, 4, 2, 0b1110)):
    g = P.unit_gauge(lat)
    e, eu1, q = F.observables(lat, g, Q_EL)
    h = F.wilson_flow(lat, g, 0.1, 1)
    U, A = h.extended_arrays()
    return max(abs(e), abs(eu1), abs(q), np.abs(U - np.eye(3)).max(), np.abs(A).max())


def _gauge_transform(lat, U, A, r):
    Lam = P.random_su3(r, lat.V)
    al = r.uniform(-np.pi, np.pi, lat.V)
    x = lat.all_sites()
    U2 = np.empty_like(U)
    A2 = np.empty_like(A)
    for mu in range(4):
        xp = lat.shift(x, mu, +1)
        U2[:, mu] = Lam @ U[:, mu] @ O.dagger(Lam[xp])
        A2[:, mu] = A[:, mu] + al - al[xp]
    return U2, np.remainder(A2 + np.pi, 2 * np.pi) - np.pi, Lam, al


def random_field(lat, r, eps=0.6, sigma=0.8):
    """Admissible random field (C* lattices) or plain random field (periodic)."""
    return P.random_physical_gauge(r, lat, eps, sigma) if lat.cstar[1] else \
        O.GaugeField.from_extended(lat, P.random_su3(r, lat.V * 4).reshape(lat.V, 4, 3, 3),
                                   r.uniform(-np.pi, np.pi, (lat.V, 4)))


def pin_gauge_invariance_and_covariance(lat=TORUS, seed=31, eps=0.04, nsteps=2):
    """Observables are gauge invariant; the flow is gauge covariant."""
    r = P.rng(seed)
    g = random_field(lat, r)
    U, A = g.extended_arrays()
    U2, A2, Lam, al = _gauge_transform(lat, U, A, r)
    g2 = O.GaugeField.from_extended(lat, U2, A2)
    o1 = np.array(F.observables(lat, g, Q_EL))
    o2 = np.array(F.observables(lat, g2, Q_EL))
    e1 = np.abs(o1 - o2).max() / np.abs(o1).max()
    h1 = F.wilson_flow(lat, g, eps, nsteps).extended_arrays()
    h2 = F.wilson_flow(lat, g2, eps, nsteps).extended_arrays()
    x = lat.all_sites()
    err = 0.0
    for mu in range(4):
        xp = lat.shift(x, mu, +1)
        err = max(err, np.abs(Lam @ h1[0][:, mu] @ O.dagger(Lam[xp]) - h2[0][:, mu]).max())
        dA = np.remainder(h1[1][:, mu] + al - al[xp] - h2[1][:, mu] + np.pi, 2 * np.pi) - np.pi
        err = max(err, np.abs(dA).max())
    return max(e1, err)


def pin_reflection(lat=TORUS, seed=32):
    """x0 -> -x0: E is unchanged and Q_top changes sign."""
    r = P.rng(seed)
    g = random_field(lat, r)
    U, A = g.extended_arrays()
    c = lat.coords(lat.all_sites())
    pc = c.copy()
    pc[:, 0] = (-c[:, 0]) % lat.N[0]
    px = lat.index(pc)
    U2 = np.empty_like(U)
    A2 = np.empty_like(A)
    back = lat.shift(px, 0, -1)
    U2[:, 0] = O.dagger(U[back, 0])
    A2[:, 0] = -A[back, 0]
    for k in (1, 2, 3):
        U2[:, k] = U[px, k]
        A2[:, k] = A[px, k]
    e1, u1, q1 = F.observables(lat, g, Q_EL)
    e2, u2, q2 = F.observables(lat, O.GaugeField.from_extended(lat, U2, A2), Q_EL)
    assert abs(q1) > 1e-3
    return max(abs(e1 - e2) / e1, abs(u1 - u2) / u1, abs(q1 + q2) / abs(q1))


def pin_action_derivative(lat=O.Lattice(4, 2, 4, 2, 0b1110), seed=33, h=1e-3):
    """d/dt of g0^2 S_w at t = 0 equals 2 sum tr Z^2; for U(1), d/dt of
    sum (1 - cos theta_p) equals -sum Z_U(1)^2 (central differences)."""
    r = P.rng(seed)
    g = random_field(lat, r)
    U, A = g.extended_arrays()
    Up, Ap = F.wilson_flow_step(lat, U, A, h)
    Um, Am = F.wilson_flow_step(lat, U, A, -h)
    dS = (F.wilson_action(lat, Up) - F.wilson_action(lat, Um)) / (2 * h)
    Z = F.force_su3(lat, U)
    ref = 2.0 * np.einsum("nmij,nmji->", Z, Z).real

    def s_u1(A_):
        x = lat.all_sites()
        return sum(np.sum(1 - np.cos(F.plaquette_angle(lat, A_, x, mu, nu))) for mu, nu in PLANES)

    dS1 = (s_u1(Ap) - s_u1(Am)) / (2 * h)
    ref1 = -np.sum(F.force_u1(lat, A) ** 2)
    return max(abs(dS - ref) / abs(ref), abs(dS1 - ref1) / abs(ref1))


def pin_runge_kutta_order(lat=O.Lattice(4, 2, 4, 2, 0b1110), seed=34, t=0.1):
    """Global error of the scheme falls by 2^3 per halving of the step."""
    r = P.rng(seed)
    g = random_field(lat, r)
    U, A = g.extended_arrays()
    runs = []
    for n in (4, 8, 16):
        Un, An = U, A
        for _ in range(n):
            Un, An = F.wilson_flow_step(lat, Un, An, t / n)
        runs.append((Un, An))
    d1 = np.abs(runs[0][0] - runs[1][0]).max()
    d2 = np.abs(runs[1][0] - runs[2][0]).max()
    a1 = np.abs(runs[0][1] - runs[1][1]).max()
    a2 = np.abs(runs[1][1] - runs[2][1]).max()
    # the ratios of third-order schemes are near 8; report the distance
    return max(abs(np.log2(d1 / d2) - 3.0), abs(np.log2(a1 / a2) - 3.0))


def pin_action_decreases(lat=O.Lattice(4, 2, 4, 2, 0b1110), seed=35, eps=0.05, nsteps=6):
    r = P.rng(seed)
    g = random_field(lat, r)
    U, A = g.extended_arrays()
    s = [F.wilson_action(lat, U)]
    for _ in range(nsteps):
        U, A = F.wilson_flow_step(lat, U, A, eps)
        s.append(F.wilson_action(lat, U))
    return float(max(0.0, np.max(np.diff(s))))


def pin_mirror_densities(lat=O.Lattice(4, 2, 4, 2, 0b1110), seed=36):
    """C* (Sec. 2.1): the mirror half carries the conjugate field, so every
    density at T x equals the one at x; E is then the mean over the physical
    half and Q_top the sum over it."""
    r = P.rng(seed)
    g = random_field(lat, r)
    d = F.densities(lat, g, Q_EL)
    x = lat.all_sites()
    phys = lat.is_physical(x)
    err = max(np.abs(v - v[lat.translate(x)]).max() / np.abs(v).max() for v in d)
    e, eu1, q = F.observables(lat, g, Q_EL)
    err = max(err, abs(e - d[0][phys].mean()) / e, abs(eu1 - d[1][phys].mean()) / eu1,
              abs(q - d[2][phys].sum()) / max(abs(q), 1e-300))
    return err
