"""Plain FP64 CPU oracle for the gauge observables and the Wilson flow.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and
its Python binding) may import, call or link this module. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and its
``--impl reference`` arm) use it. It shares no code with the GPU path.

What it computes (App. A of the openQ*D proceedings, arXiv:1710.08839, and
the Wilson flow of Luscher (2010), which Sec. 3 names for these
observables):

* ``observables`` -- the SU(3) and U(1) action densities and the SU(3)
  topological charge built from the clover field tensors:
    E_SU(3) = -1/(2 V) sum_x sum_{mu,nu} tr{F_munu(x) F_munu(x)},
    E_U(1)  = -1/(2 V) sum_x sum_{mu,nu} A_munu(x)^2,
    Q_top   = 1/(32 pi^2) sum_x sum_{mu nu rho sigma} eps_{mu nu rho sigma}
              tr{F_munu(x) F_rhosigma(x)},
  with F the SU(3) clover tensor of the Dirac operator (F = (Q_munu -
  Q_numu)/8) and A_munu = i/(4 q_el) Im{four U(1) plaquettes} (Sec. 2.3).
  Readings: the paper prints E without the minus sign; both tensors are
  anti-Hermitian (Sec. 2.3), so the printed form is <= 0 and the minus sign
  makes E the (non-negative) action density. The sums run over the physical
  lattice of volume V = L^3 T; on the doubled lattice of C* boundaries the
  mirror half carries the complex-conjugate field, whose densities are the
  same, so the code sums over the whole simulated lattice and divides by its
  volume (E), or halves the sum (Q).
* ``wilson_flow`` -- Luscher's flow dV/dt = Z(V) V with
  Z(x,mu) = -g0^2 d_{x,mu} S_w = -1/2 (W - W^dag) + 1/6 tr(W - W^dag),
  W = U(x,mu) sum_{nu != mu} (staple of the plaquettes through the link),
  S_w = 1/g0^2 sum over oriented plaquettes Re tr(1 - U_p), integrated with
  his third-order Runge-Kutta scheme:
    W1 = exp(Z0/4) W0, W2 = exp(8/9 Z1 - 17/36 Z0) W1,
    V(t + eps) = exp(3/4 Z2 - 8/9 Z1 + 17/36 Z0) W2,  Z_i = eps Z(W_i).
  The U(1) field flows by the same scheme with the compact plaquette action
  (abelian, so the exponentials add to the angle):
    dA(x,mu)/dt = -sum_{nu != mu} [sin theta_munu(x) - sin theta_munu(x - nu)],
  theta_munu the plaquette angle. The angles are kept in [-pi, pi)
  (Sec. 2.1).

Pins (tests/test_oracle_flow.py): zero for the unit field, closed forms for
constant abelian field strength embedded in SU(3) (E, E_U(1), Q_top, and a
stationary flow), gauge invariance, the sign change of Q_top under a
reflection, dS_w/dt = 2 sum tr Z^2 at t = 0, the monotone decrease of S_w,
and the third-order convergence of the Runge-Kutta scheme.
"""
from __future__ import annotations

import itertools

import numpy as np

from .qxd_oracle import Dirac, GaugeField, Lattice, dagger


def _levi_civita():
    eps = {}
    for p in itertools.permutations(range(4)):
        inv = sum(1 for i in range(4) for j in range(i + 1, 4) if p[i] > p[j])
        eps[p] = -1 if inv % 2 else 1
    return eps


LEVI_CIVITA = _levi_civita()


def _plain_op(lat: Lattice, g: GaugeField) -> Dirac:
    # the clover tensors only: mass, c_sw and charge do not enter them
    return Dirac(lat, g, 0.0, 0.0, 0.0, 0)


def densities(lat: Lattice, g: GaugeField, q_el: float):
    """Per-site densities (V,) each:
    e_SU(3)(x) = -1/2 sum_{mu,nu} tr{F_munu F_munu},
    e_U(1)(x)  = -1/2 sum_{mu,nu} A_munu^2,
    q(x) = 1/(32 pi^2) sum eps_{mu nu rho sigma} tr{F_munu F_rhosigma}."""
    op = _plain_op(lat, g)
    idx = lat.all_sites()
    F = {}
    Au1 = {}
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            F[mu, nu] = op.F_hat(idx, mu, nu)
            xm = lat.shift(idx, mu, -1)
            xn = lat.shift(idx, nu, -1)
            xmn = lat.shift(xm, nu, -1)
            tot = (op.z_plaquette(idx, mu, nu) + op.z_plaquette(xm, mu, nu)
                   + op.z_plaquette(xn, mu, nu) + op.z_plaquette(xmn, mu, nu))
            Au1[mu, nu] = 1j / (4.0 * q_el) * np.imag(tot)
    e_su3 = np.zeros(lat.V)
    e_u1 = np.zeros(lat.V)
    for (mu, nu), f in F.items():
        e_su3 -= 0.5 * np.einsum("nij,nji->n", f, f).real
        e_u1 -= 0.5 * (Au1[mu, nu] * Au1[mu, nu]).real
    q = np.zeros(lat.V)
    for (mu, nu, rho, sig), s in LEVI_CIVITA.items():
        q += s * np.einsum("nij,nji->n", F[mu, nu], F[rho, sig]).real
    q /= 32.0 * np.pi ** 2
    return e_su3, e_u1, q


def observables(lat: Lattice, g: GaugeField, q_el: float):
    """(E_SU(3), E_U(1), Q_top) of the gauge field g (App. A): E is the mean
    density, Q the sum of q(x) over the physical lattice."""
    e_su3, e_u1, q = densities(lat, g, q_el)
    Q = np.sum(q)
    if lat.cstar[1]:
        Q *= 0.5  # the physical lattice is half of the simulated one
    return float(np.mean(e_su3)), float(np.mean(e_u1)), float(Q)


# ---------------------------------------------------------------------------
# Wilson flow
# ---------------------------------------------------------------------------


def omega(lat: Lattice, U: np.ndarray, mu: int) -> np.ndarray:
    """W(x,mu) = U(x,mu) times the sum of the six staples, for all x."""
    x = lat.all_sites()
    xp = lat.shift(x, mu, +1)
    st = np.zeros((lat.V, 3, 3), dtype=np.complex128)
    for nu in range(4):
        if nu == mu:
            continue
        xn = lat.shift(x, nu, +1)
        xmn = lat.shift(x, nu, -1)
        xpmn = lat.shift(xp, nu, -1)
        # U(x+mu,nu) U(x+nu,mu)^dag U(x,nu)^dag
        st += U[xp, nu] @ dagger(U[xn, mu]) @ dagger(U[x, nu])
        # U(x+mu-nu,nu)^dag U(x-nu,mu)^dag U(x-nu,nu)
        st += dagger(U[xpmn, nu]) @ dagger(U[xmn, mu]) @ U[xmn, nu]
    return U[x, mu] @ st


def force_su3(lat: Lattice, U: np.ndarray) -> np.ndarray:
    """Z(x,mu) = -1/2 (W - W^dag) + 1/6 tr(W - W^dag), shape (V, 4, 3, 3)."""
    Z = np.empty((lat.V, 4, 3, 3), dtype=np.complex128)
    for mu in range(4):
        W = omega(lat, U, mu)
        D = W - dagger(W)
        tr = np.trace(D, axis1=-2, axis2=-1)
        Z[:, mu] = -0.5 * D + (tr / 6.0)[:, None, None] * np.eye(3)
    return Z


def plaquette_angle(lat: Lattice, A: np.ndarray, idx, mu: int, nu: int):
    xm = lat.shift(idx, mu, +1)
    xn = lat.shift(idx, nu, +1)
    return A[idx, mu] + A[xm, nu] - A[xn, mu] - A[idx, nu]


def force_u1(lat: Lattice, A: np.ndarray) -> np.ndarray:
    """-d/dA(x,mu) of sum over plaquettes of (1 - cos theta_p), shape (V, 4)."""
    x = lat.all_sites()
    Z = np.zeros((lat.V, 4))
    for mu in range(4):
        for nu in range(4):
            if nu == mu:
                continue
            Z[:, mu] -= np.sin(plaquette_angle(lat, A, x, mu, nu))
            Z[:, mu] += np.sin(plaquette_angle(lat, A, lat.shift(x, nu, -1), mu, nu))
    return Z


def expm_antihermitian(X: np.ndarray) -> np.ndarray:
    """exp(X) for anti-Hermitian X (..., 3, 3) through the eigenvectors of iX."""
    w, v = np.linalg.eigh(-1j * X)  # X = i H, H Hermitian
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), np.conj(v))


def _wrap(A):
    return np.remainder(A + np.pi, 2 * np.pi) - np.pi


def wilson_flow_step(lat: Lattice, U: np.ndarray, A: np.ndarray, eps: float):
    """One Runge-Kutta step of Luscher's scheme for SU(3) and for U(1)."""
    Z0 = eps * force_su3(lat, U)
    a0 = eps * force_u1(lat, A)
    U1 = expm_antihermitian(0.25 * Z0) @ U
    A1 = A + 0.25 * a0
    Z1 = eps * force_su3(lat, U1)
    a1 = eps * force_u1(lat, A1)
    U2 = expm_antihermitian(8.0 / 9.0 * Z1 - 17.0 / 36.0 * Z0) @ U1
    A2 = A1 + 8.0 / 9.0 * a1 - 17.0 / 36.0 * a0
    Z2 = eps * force_su3(lat, U2)
    a2 = eps * force_u1(lat, A2)
    U3 = expm_antihermitian(0.75 * Z2 - 8.0 / 9.0 * Z1 + 17.0 / 36.0 * Z0) @ U2
    A3 = A2 + 0.75 * a2 - 8.0 / 9.0 * a1 + 17.0 / 36.0 * a0
    return U3, _wrap(A3)


def wilson_flow(lat: Lattice, g: GaugeField, eps: float, nsteps: int) -> GaugeField:
    """The gauge field flowed to t = nsteps * eps (SU(3) and U(1))."""
    U, A = g.extended_arrays()
    U = np.array(U, dtype=np.complex128)
    A = np.array(A, dtype=np.float64)
    for _ in range(nsteps):
        U, A = wilson_flow_step(lat, U, A, eps)
    return GaugeField.from_extended(lat, U, A)


def wilson_action(lat: Lattice, U: np.ndarray) -> float:
    """g0^2 S_w = sum over oriented plaquettes Re tr(1 - U_p)
    = 2 sum over planes mu < nu and sites of Re tr(1 - U_munu(x))."""
    x = lat.all_sites()
    s = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            xm = lat.shift(x, mu, +1)
            xn = lat.shift(x, nu, +1)
            P = U[x, mu] @ U[xm, nu] @ dagger(U[xn, mu]) @ dagger(U[x, nu])
            s += 2.0 * np.sum(3.0 - np.trace(P, axis1=-2, axis2=-1).real)
    return s
