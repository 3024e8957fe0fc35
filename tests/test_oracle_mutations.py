"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins
catch every one of them: a pin that cannot fail pins nothing."""
import numpy as np
import pytest

import oracle as O
import pins as P

SMALL = O.Lattice(4, 2, 4, 2, 0b1110)
CAUGHT = 1e-6


def _run_all_pins(monkeypatch=None, dirac_cls=O.Dirac):
    """Largest deviation over all pins (an assertion inside a pin counts)."""
    worst = 0.0
    checks = [
        lambda: P.pin_plane_waves(SMALL, dirac_cls),
        lambda: P.pin_plane_waves(SMALL, dirac_cls, theta=np.array([0.3, -0.7, 1.1, 0.2]), qhat=-1),
        lambda: P.pin_clover_constant_field(dirac_cls),
        lambda: P.pin_gauge_covariance(SMALL, dirac_cls, admissible=True),
        lambda: P.pin_gauge_covariance(SMALL, dirac_cls, admissible=False),
        lambda: P.pin_gamma5_hermiticity(SMALL, dirac_cls),
        lambda: P.pin_transpose_identity(SMALL, dirac_cls),
        lambda: P.pin_mirror_identity(SMALL, dirac_cls),
        lambda: P.pin_antisymmetry(SMALL, dirac_cls),
        lambda: P.pin_theta_symmetry(SMALL, dirac_cls),
    ]
    for c in checks:
        try:
            worst = max(worst, float(c()))
        except AssertionError:
            return np.inf
    return worst


class BackwardNoDagger(O.Dirac):
    def nabla_star(self, mu, f):
        f = O.qxd_oracle._as_field_fn(f)

        def g(idx):
            dn = self.lat.shift(idx, mu, -1)
            return f(idx) - O.colour_mul(self.link(dn, mu), f(dn))
        return g


class BackwardPhaseSign(O.Dirac):
    def nabla_star(self, mu, f):
        f = O.qxd_oracle._as_field_fn(f)

        def g(idx):
            dn = self.lat.shift(idx, mu, -1)
            w = O.dagger(self.g.U(dn, mu)) * (self.g.z(dn, mu) ** self.qhat)[..., None, None]
            return f(idx) - O.colour_mul(w, f(dn))
        return g


class LaplacianSign(O.Dirac):
    def Dw_at(self, f, idx):
        f = O.qxd_oracle._as_field_fn(f)
        out = 0.0
        for mu in range(4):
            sym = self.nabla(mu, f)(idx) + self.nabla_star(mu, f)(idx)
            lap = self.nabla_star(mu, self.nabla(mu, f))(idx)
            out = out + 0.5 * (O.spin_mul(O.GAMMA[mu], sym) + lap)
        return out


class MissingLeaf(O.Dirac):
    def Q_leaves(self, idx, mu, nu):
        U, d = self.g.U, O.dagger
        p = self._plaquette_sites(idx, mu, nu)
        leaf1 = U(p["x"], mu) @ U(p["x+mu"], nu) @ d(U(p["x+nu"], mu)) @ d(U(p["x"], nu))
        leaf2 = U(p["x"], nu) @ d(U(p["x-mu+nu"], mu)) @ d(U(p["x-mu"], nu)) @ U(p["x-mu"], mu)
        leaf3 = d(U(p["x-mu"], mu)) @ d(U(p["x-mu-nu"], nu)) @ U(p["x-mu-nu"], mu) @ U(p["x-nu"], nu)
        return leaf1 + leaf2 + leaf3


class LeafOrder(O.Dirac):
    def Q_leaves(self, idx, mu, nu):
        U, d = self.g.U, O.dagger
        p = self._plaquette_sites(idx, mu, nu)
        leaf1 = U(p["x"], mu) @ U(p["x+mu"], nu) @ d(U(p["x+nu"], mu)) @ d(U(p["x"], nu))
        leaf2 = U(p["x"], nu) @ d(U(p["x-mu"], nu)) @ d(U(p["x-mu+nu"], mu)) @ U(p["x-mu"], mu)
        leaf3 = d(U(p["x-mu"], mu)) @ d(U(p["x-mu-nu"], nu)) @ U(p["x-mu-nu"], mu) @ U(p["x-nu"], nu)
        leaf4 = d(U(p["x-nu"], nu)) @ U(p["x-nu"], mu) @ U(p["x+mu-nu"], nu) @ d(U(p["x"], mu))
        return leaf1 + leaf2 + leaf3 + leaf4


class SymmetricF(O.Dirac):
    def F_hat(self, idx, mu, nu):
        return (self.Q_leaves(idx, mu, nu) + self.Q_leaves(idx, nu, mu)) / 8.0


class U1TensorHalf(O.Dirac):
    def qA_hat(self, idx, mu, nu):
        return 0.5 * super().qA_hat(idx, mu, nu)


class U1TensorOnePlaquette(O.Dirac):
    def qA_hat(self, idx, mu, nu):
        return self.qhat * 0.25j * np.imag(4 * self.z_plaquette(idx, mu, nu))


class NoMass(O.Dirac):
    def apply_at(self, psi, idx):
        f = O.qxd_oracle._as_field_fn(psi)
        return super().apply_at(psi, idx) - self.m0 * f(np.asarray(idx))


DIRAC_MUTANTS = [BackwardNoDagger, BackwardPhaseSign, LaplacianSign, MissingLeaf,
                 LeafOrder, SymmetricF, U1TensorHalf, U1TensorOnePlaquette, NoMass]


def test_unmutated_oracle_passes_all_pins():
    assert _run_all_pins() < 1e-11


@pytest.mark.parametrize("mutant", DIRAC_MUTANTS, ids=lambda c: c.__name__)
def test_dirac_mutant_is_caught(mutant):
    assert _run_all_pins(dirac_cls=mutant) > CAUGHT


def test_mirror_without_conjugation_is_caught(monkeypatch):
    orig = O.GaugeField.U

    def U(self, idx, mu):
        if not self.physical:
            return orig(self, idx, mu)
        p, mirror = self._physical_site(idx)
        return self.su3[p, mu]
    monkeypatch.setattr(O.GaugeField, "U", U)
    assert _run_all_pins() > CAUGHT


def test_mirror_without_photon_sign_is_caught(monkeypatch):
    def A(self, idx, mu):
        if not self.physical:
            return self.angle[idx, mu]
        p, mirror = self._physical_site(idx)
        return self.angle[p, mu]
    monkeypatch.setattr(O.GaugeField, "A", A)
    assert _run_all_pins() > CAUGHT


def test_unshifted_cstar_boundary_is_caught(monkeypatch):
    def shift(self, idx, mu, sign):
        c = self.coords(idx)
        c[..., mu] = (c[..., mu] + sign) % self.N[mu]
        return self.index(c)
    monkeypatch.setattr(O.Lattice, "shift", shift)
    assert _run_all_pins() > CAUGHT


def test_shift_by_wrong_amount_is_caught(monkeypatch):
    def shift(self, idx, mu, sign):
        c = self.coords(idx)
        new = c[..., mu] + sign
        if mu >= 2 and self.cstar[mu]:
            crossed = (new == self.L[mu]) | (new == -1)
            c[..., 1] = np.where(crossed, (c[..., 1] + 1) % self.N[1], c[..., 1])
            c[..., mu] = new % self.L[mu]
        else:
            c[..., mu] = new % self.N[mu]
        return self.index(c)
    monkeypatch.setattr(O.Lattice, "shift", shift)
    assert _run_all_pins() > CAUGHT
