"""The gauge-observable and Wilson-flow oracle against closed forms and exact
properties (no GPU); planted mistakes are caught."""
import numpy as np
import pytest

from oracle import qxd_flow as F
import pins_flow as PF


def test_constant_flux_closed_forms():
    assert PF.pin_constant_flux() < 1e-12


def test_constant_flux_is_stationary_under_the_flow():
    assert PF.pin_constant_flux_is_stationary() < 1e-13


def test_unit_field():
    assert PF.pin_unit_field() < 1e-14


def test_gauge_invariance_and_flow_covariance():
    assert PF.pin_gauge_invariance_and_covariance() < 1e-12


def test_reflection_flips_the_topological_charge():
    assert PF.pin_reflection() < 1e-12


def test_action_derivative_matches_the_force():
    assert PF.pin_action_derivative() < 1e-4


def test_runge_kutta_is_third_order():
    assert PF.pin_runge_kutta_order() < 0.3


def test_action_decreases_along_the_flow():
    assert PF.pin_action_decreases() == 0.0


def test_mirror_half_repeats_the_physical_densities():
    assert PF.pin_mirror_densities() < 1e-12


# ---------------------------------------------------------------------------
# planted mistakes
# ---------------------------------------------------------------------------

CAUGHT = 1e-6


def _all_pins():
    checks = [(PF.pin_constant_flux, 1e-12), (PF.pin_unit_field, 1e-14),
              (PF.pin_reflection, 1e-12), (PF.pin_action_derivative, 1e-4),
              (PF.pin_gauge_invariance_and_covariance, 1e-12), (PF.pin_runge_kutta_order, 0.3),
              (PF.pin_action_decreases, 0.0), (PF.pin_constant_flux_is_stationary, 1e-13)]
    for fn, tol in checks:
        try:
            v = float(fn())
        except (AssertionError, FloatingPointError, np.linalg.LinAlgError):
            return True
        if not np.isfinite(v) or v > tol:
            return True
    return False


def _rk_coefficient(lat, U, A, eps):
    Z0 = eps * F.force_su3(lat, U)
    a0 = eps * F.force_u1(lat, A)
    U1 = F.expm_antihermitian(0.25 * Z0) @ U
    A1 = A + 0.25 * a0
    Z1 = eps * F.force_su3(lat, U1)
    a1 = eps * F.force_u1(lat, A1)
    U2 = F.expm_antihermitian(8.0 / 9.0 * Z1 - 17.0 / 32.0 * Z0) @ U1
    A2 = A1 + 8.0 / 9.0 * a1 - 17.0 / 32.0 * a0
    Z2 = eps * F.force_su3(lat, U2)
    a2 = eps * F.force_u1(lat, A2)
    U3 = F.expm_antihermitian(0.75 * Z2 - 8.0 / 9.0 * Z1 + 17.0 / 36.0 * Z0) @ U2
    A3 = A2 + 0.75 * a2 - 8.0 / 9.0 * a1 + 17.0 / 36.0 * a0
    return U3, A3


def _u1_backward_sign(lat, A):
    x = lat.all_sites()
    Z = np.zeros((lat.V, 4))
    for mu in range(4):
        for nu in range(4):
            if nu != mu:
                Z[:, mu] -= np.sin(F.plaquette_angle(lat, A, x, mu, nu))
                Z[:, mu] -= np.sin(F.plaquette_angle(lat, A, lat.shift(x, nu, -1), mu, nu))
    return Z


def _densities_e_sign(lat, g, q_el):
    e, u, q = _ORIG_DENS(lat, g, q_el)
    return -e, u, q


def _densities_q_abs_eps(lat, g, q_el):
    e, u, q = _ORIG_DENS(lat, g, q_el)
    # drops the sign of the Levi-Civita symbol
    op = F._plain_op(lat, g)
    idx = lat.all_sites()
    Fm = {(m, n): op.F_hat(idx, m, n) for m in range(4) for n in range(4) if m != n}
    q2 = np.zeros(lat.V)
    for (m, n, r_, s_), s in F.LEVI_CIVITA.items():
        q2 += np.einsum("nij,nji->n", Fm[m, n], Fm[r_, s_]).real
    return e, u, q2 / (32 * np.pi ** 2)


def _omega_wrong_staple(lat, U, mu):
    from oracle.qxd_oracle import dagger
    x = lat.all_sites()
    xp = lat.shift(x, mu, +1)
    st = np.zeros((lat.V, 3, 3), dtype=np.complex128)
    for nu in range(4):
        if nu == mu:
            continue
        xn = lat.shift(x, nu, +1)
        xmn = lat.shift(x, nu, -1)
        xpmn = lat.shift(xp, nu, -1)
        st += U[xp, nu] @ dagger(U[xn, mu]) @ dagger(U[x, nu])
        st += U[xpmn, nu] @ dagger(U[xmn, mu]) @ U[xmn, nu]   # missing dagger
    return U[x, mu] @ st


_ORIG_DENS = F.densities
_ORIG_FORCE = F.force_su3


def _force_flipped(lat, U):
    return -_ORIG_FORCE(lat, U)


MUTATIONS = {
    "force_sign": ("force_su3", _force_flipped),
    "rk_coefficient": ("wilson_flow_step", _rk_coefficient),
    "u1_backward_plaquette_sign": ("force_u1", _u1_backward_sign),
    "energy_sign": ("densities", _densities_e_sign),
    "levi_civita_sign_dropped": ("densities", _densities_q_abs_eps),
    "staple_missing_dagger": ("omega", _omega_wrong_staple),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(F, attr, fn)
    assert _all_pins()
