"""Plain FP64 CPU oracle for the openQ*D Dirac operator with C* boundaries.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and
its Python binding) may import, call or link this module. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and its
``--impl reference`` arm) use it, to produce the values the GPU results are
compared with. It shares no code with the GPU path; only the seeded input
generators of ``synth`` feed both.

What it computes, and where each piece comes from (the paper is the openQ*D
proceedings, arXiv:1710.08839):

* ``Lattice``      -- the extended lattice (Sec. 2.1, Eq. (1)), periodicity
  2 L1 in direction 1 (Eq. (10)) and the shifted boundaries of the C*
  directions 2, 3 (Eq. (11), Fig. 1).
* ``GaugeField``   -- SU(3) links U and photon field A, z = exp(iA) (Eq. (3));
  the mirror half is built from the physical half by the orbifold constraint
  U(x + L1 e1) = U(x)^*, A(x + L1 e1) = -A(x) (Eq. (4a)).
* ``Dirac``        -- D = m0 + Dw + dDsw (Sec. 2.3, Eq. (16), periodic time so
  dDb = 0); Dw from the covariant derivatives on the compound links
  U z^qhat (Eqs. (18)-(20)); the SW term (Eq. (21)) with the U(1) clover of
  Eqs. (22)-(23) and the SU(3) clover of Luscher et al. (1996), which the
  paper cites but does not print (reading: F = (Q_munu - Q_numu)/8 with
  Q the four plaquette leaves through x, no traceless projection).
* ``EvenOdd``      -- the block form of D and D_hat = Dee - Deo Doo^-1 Doe
  (Sec. 2.4, Eqs. (29)-(30)).
* ``dense_matrix`` -- D as a dense matrix on tiny lattices (for LU and for the
  exact identities of Sec. 2.4, Eqs. (25)-(28)).
* ``gcr``          -- plain restarted GCR in FP64 (no preconditioner); the
  paper names GCR but does not specify it, this is the textbook algorithm.

Readings where the paper is silent (gamma basis, sigma_munu, C, q_el):
chiral basis with gamma5 = diag(1, 1, -1, -1); sigma_munu = (i/2)[g_mu, g_nu];
C = gamma0 gamma2; q * A_hat = qhat * (i/4) Im{...} since q = qhat q_el.

Pins (tests/test_oracle_*.py): free-field plane waves with the momenta of the
shifted torus, constant abelian phase, closed-form clover for constant
abelian field strength, Fig. 1's identifications (tests/golden), gauge
covariance, gamma5-hermiticity, the transpose, mirror and antisymmetry
identities of Sec. 2.4, the antilinear symmetry derived from them, dense LU,
the even-odd determinant identity, and the reductions q=0 / csw=0 / U=1.
Every function here is pinned by at least one of them.

Field conventions: a spinor field is an array ``(..., V, 4, 3)`` complex128
(spin major, colour minor), V sites in lexicographic order of
(x0, x1, x2, x3) with x3 fastest; any leading batch dimensions are allowed.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# Dirac algebra (the paper gives no basis; chiral basis, gamma5 diagonal)
# ---------------------------------------------------------------------------

PAULI = np.array(
    [[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128
)


def _gamma_matrices() -> np.ndarray:
    i2 = np.eye(2, dtype=np.complex128)
    z2 = np.zeros((2, 2), dtype=np.complex128)
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    g[0] = np.block([[z2, -i2], [-i2, z2]])
    for k in range(3):
        g[k + 1] = np.block([[z2, -1j * PAULI[k]], [1j * PAULI[k], z2]])
    return g


GAMMA = _gamma_matrices()
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ID4 = np.eye(4, dtype=np.complex128)
ID3 = np.eye(3, dtype=np.complex128)


def sigma(mu: int, nu: int) -> np.ndarray:
    """sigma_munu = (i/2) [gamma_mu, gamma_nu] (Hermitian)."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


# Charge conjugation: fixed in Sec. 2.1 (Eq. (5)) only by its properties.
CHARGE_C = GAMMA[0] @ GAMMA[2]
CHARGE_C_INV = np.linalg.inv(CHARGE_C)


def spin_mul(m: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a 4x4 spin matrix to a spinor field (..., n, 4, 3)."""
    return np.einsum("st,...ntc->...nsc", m, psi)


def colour_mul(w: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply per-site 3x3 colour matrices w (n, 3, 3) to a field (..., n, 4, 3)."""
    return np.einsum("nab,...nsb->...nsa", w, psi)


def dagger(w: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(w, -1, -2))


# ---------------------------------------------------------------------------
# Geometry: extended lattice and its global topology (Sec. 2.1, Fig. 1)
# ---------------------------------------------------------------------------


class Lattice:
    """The simulated lattice.

    ``cstar_mask`` bit k (k = 1, 2, 3) marks direction k as a C* direction.
    If any bit is set, bit 1 must be set: the lattice is then doubled in
    direction 1 (x1 in [0, 2 L1), Eq. (1)), periodic in it (Eq. (10)), and a
    C* direction k = 2, 3 gets the shifted boundary of Eq. (11): the site
    beyond x_k = L_k - 1 is (x1 + L1 mod 2 L1, x_k = 0). Time and the
    periodic directions wrap plainly. With ``cstar_mask = 0`` the lattice is
    the plain periodic torus L0 x L1 x L2 x L3.
    """

    def __init__(self, T: int, L1: int, L2: int, L3: int, cstar_mask: int = 0b1110):
        if cstar_mask & ~0b1110:
            raise ValueError("cstar_mask may only use bits 1..3")
        if cstar_mask and not (cstar_mask & 2):
            raise ValueError("C* in direction 2 or 3 needs C* in direction 1")
        self.L = (T, L1, L2, L3)
        self.cstar = [False, bool(cstar_mask & 2), bool(cstar_mask & 4), bool(cstar_mask & 8)]
        self.cstar_mask = cstar_mask
        self.N = (T, 2 * L1 if self.cstar[1] else L1, L2, L3)
        self.V = int(np.prod(self.N))

    # lexicographic index <-> coordinates, x3 fastest
    def coords(self, idx) -> np.ndarray:
        idx = np.asarray(idx, dtype=np.int64)
        c = np.empty(idx.shape + (4,), dtype=np.int64)
        r = idx.copy()
        for mu in (3, 2, 1, 0):
            c[..., mu] = r % self.N[mu]
            r //= self.N[mu]
        return c

    def index(self, c) -> np.ndarray:
        c = np.asarray(c, dtype=np.int64)
        N = self.N
        return ((c[..., 0] * N[1] + c[..., 1]) * N[2] + c[..., 2]) * N[3] + c[..., 3]

    def all_sites(self) -> np.ndarray:
        return np.arange(self.V, dtype=np.int64)

    def shift(self, idx, mu: int, sign: int) -> np.ndarray:
        """Index of the nearest neighbour x + sign * mu_hat (sign = +1 or -1)."""
        c = self.coords(idx)
        new = c[..., mu] + sign
        if mu >= 2 and self.cstar[mu]:
            L1, Lk = self.L[1], self.L[mu]
            crossed = (new == Lk) | (new == -1)
            # Eq. (11): leaving through the x_k boundary lands at x + L1 e1
            c[..., 1] = np.where(crossed, (c[..., 1] + L1) % (2 * L1), c[..., 1])
            c[..., mu] = new % Lk
        else:
            c[..., mu] = new % self.N[mu]
        return self.index(c)

    def parity(self, idx) -> np.ndarray:
        return self.coords(idx).sum(axis=-1) % 2

    def translate(self, idx) -> np.ndarray:
        """Site T(x) of the translation operator of Eq. (7): x1 -> x1 + L1 mod 2 L1."""
        if not self.cstar[1]:
            raise ValueError("the translation operator needs C* in direction 1")
        c = self.coords(idx)
        c[..., 1] = (c[..., 1] + self.L[1]) % (2 * self.L[1])
        return self.index(c)

    def is_physical(self, idx) -> np.ndarray:
        return self.coords(idx)[..., 1] < self.L[1]


# ---------------------------------------------------------------------------
# Gauge field (Sec. 2.1, Eqs. (3)-(4a))
# ---------------------------------------------------------------------------


class GaugeField:
    """SU(3) links U(x, mu) and photon field A(x, mu) on the simulated lattice.

    ``from_physical`` takes the physical half (x1 < L1), shapes
    (T, L1, L2, L3, 4, 3, 3) and (T, L1, L2, L3, 4), and builds the mirror half
    by Eq. (4a). ``from_extended`` takes arrays over the whole simulated
    lattice (V, 4, 3, 3) and (V, 4) as they are (no admissibility implied).
    """

    def __init__(self, lat: Lattice, su3, angle, physical: bool):
        self.lat = lat
        self.su3 = np.asarray(su3)
        self.angle = np.asarray(angle, dtype=np.float64)
        self.physical = physical

    @classmethod
    def from_physical(cls, lat: Lattice, su3, angle) -> "GaugeField":
        T, L1, L2, L3 = lat.L
        su3 = np.asarray(su3, dtype=np.complex128).reshape(T * L1 * L2 * L3, 4, 3, 3)
        angle = np.asarray(angle, dtype=np.float64).reshape(T * L1 * L2 * L3, 4)
        return cls(lat, su3, angle, physical=True)

    @classmethod
    def from_extended(cls, lat: Lattice, su3, angle) -> "GaugeField":
        su3 = np.asarray(su3, dtype=np.complex128).reshape(lat.V, 4, 3, 3)
        angle = np.asarray(angle, dtype=np.float64).reshape(lat.V, 4)
        return cls(lat, su3, angle, physical=False)

    def _physical_site(self, idx):
        lat = self.lat
        c = lat.coords(idx)
        mirror = c[..., 1] >= lat.L[1]
        c[..., 1] = np.where(mirror, c[..., 1] - lat.L[1], c[..., 1])
        T, L1, L2, L3 = lat.L
        p = ((c[..., 0] * L1 + c[..., 1]) * L2 + c[..., 2]) * L3 + c[..., 3]
        return p, mirror

    def U(self, idx, mu: int) -> np.ndarray:
        if not self.physical:
            return self.su3[idx, mu]
        p, mirror = self._physical_site(idx)
        u = self.su3[p, mu]
        # Eq. (4a): U(x + L1 e1, mu) = U(x, mu)^*
        return np.where(mirror[..., None, None], np.conj(u), u)

    def A(self, idx, mu: int) -> np.ndarray:
        if not self.physical:
            return self.angle[idx, mu]
        p, mirror = self._physical_site(idx)
        a = self.angle[p, mu]
        # Eq. (4a): A(x + L1 e1, mu) = -A(x, mu)
        return np.where(mirror, -a, a)

    def z(self, idx, mu: int) -> np.ndarray:
        """U(1) link z = exp(i A) (Eq. (3))."""
        return np.exp(1j * self.A(idx, mu))

    def extended_arrays(self):
        """(U, A) over the whole simulated lattice, shapes (V, 4, 3, 3), (V, 4)."""
        s = self.lat.all_sites()
        U = np.stack([self.U(s, mu) for mu in range(4)], axis=1)
        A = np.stack([self.A(s, mu) for mu in range(4)], axis=1)
        return U, A

    def conjugated(self) -> "GaugeField":
        """The field with U -> U^*, z -> z^* (A -> -A), as used in Eqs. (25)-(26)."""
        return GaugeField(self.lat, np.conj(self.su3), -self.angle, self.physical)


# ---------------------------------------------------------------------------
# The Dirac operator (Sec. 2.3)
# ---------------------------------------------------------------------------


def _as_field_fn(psi):
    """Wrap a full-lattice array (..., V, 4, 3) as a function of site indices."""
    if callable(psi):
        return psi
    psi = np.asarray(psi)
    return lambda idx: psi[..., idx, :, :]


# lattices up to this many sites keep the SW matrices of all sites
_SW_CACHE_SITES = 1 << 16


class Dirac:
    """D = m0 + Dw + dDsw for one quark of integer charge qhat (Eq. (16)-(23)).

    Fields are functions ``f(idx) -> (..., len(idx), 4, 3)`` or full arrays.
    ``apply_at(psi, idx)`` returns (D psi)(x) at the sites ``idx`` only;
    ``apply(psi)`` at every site.
    """

    def __init__(self, lat: Lattice, gauge: GaugeField, m0: float, csw: float,
                 cswU1: float, qhat: int):
        self.lat, self.g = lat, gauge
        self.m0, self.csw, self.cswU1, self.qhat = float(m0), float(csw), float(cswU1), int(qhat)

    # compound hopping link U(x, mu) z(x, mu)^qhat (Eq. (19))
    def link(self, idx, mu: int) -> np.ndarray:
        zq = self.g.z(idx, mu) ** self.qhat
        return self.g.U(idx, mu) * zq[..., None, None]

    # Eq. (19): nabla_mu psi(x) = U(x,mu) z(x,mu)^q psi(x+mu) - psi(x)
    def nabla(self, mu: int, f):
        f = _as_field_fn(f)
        op = self

        def g(idx):
            up = op.lat.shift(idx, mu, +1)
            return colour_mul(op.link(idx, mu), f(up)) - f(idx)

        return g

    # Eq. (20): nabla*_mu psi(x) = psi(x) - U(x-mu,mu)^+ z(x-mu,mu)^-q psi(x-mu)
    def nabla_star(self, mu: int, f):
        f = _as_field_fn(f)
        op = self

        def g(idx):
            dn = op.lat.shift(idx, mu, -1)
            return f(idx) - colour_mul(dagger(op.link(dn, mu)), f(dn))

        return g

    # Eq. (18): Dw = sum_mu (1/2) { gamma_mu (nabla_mu + nabla*_mu) - nabla*_mu nabla_mu }
    def Dw_at(self, f, idx) -> np.ndarray:
        f = _as_field_fn(f)
        out = 0.0
        for mu in range(4):
            sym = self.nabla(mu, f)(idx) + self.nabla_star(mu, f)(idx)
            lap = self.nabla_star(mu, self.nabla(mu, f))(idx)
            out = out + 0.5 * (spin_mul(GAMMA[mu], sym) - lap)
        return out

    # --- clover field tensors ------------------------------------------------

    def _plaquette_sites(self, idx, mu, nu):
        s = self.lat.shift
        return {
            "x": idx,
            "x+mu": s(idx, mu, +1),
            "x+nu": s(idx, nu, +1),
            "x-mu": s(idx, mu, -1),
            "x-nu": s(idx, nu, -1),
            "x-mu+nu": s(s(idx, mu, -1), nu, +1),
            "x+mu-nu": s(s(idx, mu, +1), nu, -1),
            "x-mu-nu": s(s(idx, mu, -1), nu, -1),
        }

    def Q_leaves(self, idx, mu: int, nu: int) -> np.ndarray:
        """Sum of the four oriented mu-nu plaquettes that start and end at x."""
        U = self.g.U
        p = self._plaquette_sites(idx, mu, nu)
        d = dagger
        leaf1 = U(p["x"], mu) @ U(p["x+mu"], nu) @ d(U(p["x+nu"], mu)) @ d(U(p["x"], nu))
        leaf2 = U(p["x"], nu) @ d(U(p["x-mu+nu"], mu)) @ d(U(p["x-mu"], nu)) @ U(p["x-mu"], mu)
        leaf3 = d(U(p["x-mu"], mu)) @ d(U(p["x-mu-nu"], nu)) @ U(p["x-mu-nu"], mu) @ U(p["x-nu"], nu)
        leaf4 = d(U(p["x-nu"], nu)) @ U(p["x-nu"], mu) @ U(p["x+mu-nu"], nu) @ d(U(p["x"], mu))
        return leaf1 + leaf2 + leaf3 + leaf4

    def F_hat(self, idx, mu: int, nu: int) -> np.ndarray:
        """SU(3) clover field tensor (1/8)(Q_munu - Q_numu), anti-Hermitian."""
        return (self.Q_leaves(idx, mu, nu) - self.Q_leaves(idx, nu, mu)) / 8.0

    # Eq. (23): z_munu(x) = z(x,mu) z(x+mu,nu) z(x+nu,mu)^* z(x,nu)^*
    def z_plaquette(self, idx, mu: int, nu: int) -> np.ndarray:
        z, s = self.g.z, self.lat.shift
        return z(idx, mu) * z(s(idx, mu, +1), nu) * np.conj(z(s(idx, nu, +1), mu)) * np.conj(z(idx, nu))

    def qA_hat(self, idx, mu: int, nu: int) -> np.ndarray:
        """q * A_hat_munu(x) of Eq. (22) with q = qhat q_el, so q_el cancels:
        qhat * (i/4) Im{ z_munu(x) + z_munu(x-mu) + z_munu(x-nu) + z_munu(x-mu-nu) }."""
        s = self.lat.shift
        xm, xn = s(idx, mu, -1), s(idx, nu, -1)
        xmn = s(xm, nu, -1)
        tot = (self.z_plaquette(idx, mu, nu) + self.z_plaquette(xm, mu, nu)
               + self.z_plaquette(xn, mu, nu) + self.z_plaquette(xmn, mu, nu))
        return self.qhat * 0.25j * np.imag(tot)

    def sw_matrix(self, idx) -> np.ndarray:
        """dDsw(x) of Eq. (21) as per-site 12x12 matrices (index 3*spin + colour).

        The matrices of the whole lattice are computed once and kept."""
        idx = np.asarray(idx, dtype=np.int64)
        cached = getattr(self, "_sw_all", None)
        if cached is None and self.lat.V <= _SW_CACHE_SITES:
            # small lattice: build every site's matrix once, index it after
            cached = self._sw_all = self._sw_matrix(self.lat.all_sites())
        if cached is not None:
            return cached[idx]
        full = idx.shape == (self.lat.V,) and idx[0] == 0 and idx[-1] == self.lat.V - 1
        out = self._sw_matrix(idx)
        if full and np.array_equal(idx, self.lat.all_sites()):
            self._sw_all = out
        return out

    def _sw_matrix(self, idx) -> np.ndarray:
        out = np.zeros(idx.shape + (12, 12), dtype=np.complex128)
        for mu in range(4):
            for nu in range(4):
                if mu == nu:
                    continue  # sigma_mumu = 0
                s = sigma(mu, nu)
                F = self.F_hat(idx, mu, nu)
                a = self.qA_hat(idx, mu, nu)
                out += self.csw * 0.25j * np.einsum("st,nab->nsatb", s, F).reshape(-1, 12, 12)
                out += self.cswU1 * 0.25j * np.einsum(
                    "st,n,ab->nsatb", s, a, ID3).reshape(-1, 12, 12)
        return out

    # --- the operator ------------------------------------------------------

    def apply_at(self, psi, idx) -> np.ndarray:
        """(D psi)(x) = m0 psi(x) + (Dw psi)(x) + dDsw(x) psi(x) at sites idx."""
        f = _as_field_fn(psi)
        idx = np.asarray(idx, dtype=np.int64)
        here = f(idx)
        sw = self.sw_matrix(idx)
        swpsi = np.einsum("nij,...nj->...ni", sw, here.reshape(here.shape[:-2] + (12,)))
        return self.m0 * here + self.Dw_at(f, idx) + swpsi.reshape(here.shape)

    def apply(self, psi) -> np.ndarray:
        return self.apply_at(psi, self.lat.all_sites())

    def conjugate_fields(self) -> "Dirac":
        """D[U^*, z^*] with the same parameters (Sec. 2.4, Eqs. (25)-(26))."""
        return Dirac(self.lat, self.g.conjugated(), self.m0, self.csw, self.cswU1, self.qhat)


# ---------------------------------------------------------------------------
# Dense form, even-odd blocks, solvers
# ---------------------------------------------------------------------------


def dense_matrix(op: Dirac) -> np.ndarray:
    """D as a dense (12V x 12V) matrix, column j = D e_j (tiny lattices only)."""
    V = op.lat.V
    n = 12 * V
    if n > 4096:
        raise ValueError("dense_matrix is for tiny lattices (12V <= 4096)")
    e = np.eye(n, dtype=np.complex128).reshape(n, V, 4, 3)
    cols = op.apply(e).reshape(n, n)
    return cols.T


class EvenOdd:
    """Even-odd block form of D (Sec. 2.4, Eqs. (29)-(30)).

    A site is even when x0 + x1 + x2 + x3 is even on the simulated lattice.
    Half-lattice fields are arrays (..., V/2, 4, 3) in increasing site order.
    """

    def __init__(self, op: Dirac):
        self.op = op
        lat = op.lat
        par = lat.parity(lat.all_sites())
        self.even = np.nonzero(par == 0)[0]
        self.odd = np.nonzero(par == 1)[0]
        # Doo is diagonal in the lattice index (Sec. 2.4): its 12x12 block at
        # each odd site is read off by applying D to the 12 spin-colour unit
        # fields supported on all odd sites at once.
        self.Doo_blocks = self._diag_blocks(self.odd)
        self.Dee_blocks = self._diag_blocks(self.even)

    def _diag_blocks(self, sites):
        lat = self.op.lat
        n = len(sites)
        blocks = np.empty((n, 12, 12), dtype=np.complex128)
        for j in range(12):
            f = np.zeros((lat.V, 4, 3), dtype=np.complex128)
            f[sites, j // 3, j % 3] = 1.0
            blocks[:, :, j] = self.op.apply(f)[sites].reshape(n, 12)
        return blocks

    def _full(self, fe=None, fo=None):
        shape = (fe if fe is not None else fo).shape[:-3]
        f = np.zeros(shape + (self.op.lat.V, 4, 3), dtype=np.complex128)
        if fe is not None:
            f[..., self.even, :, :] = fe
        if fo is not None:
            f[..., self.odd, :, :] = fo
        return f

    def D_ee(self, fe):
        return self.op.apply_at(self._full(fe=fe), self.even)

    def D_eo(self, fo):
        return self.op.apply_at(self._full(fo=fo), self.even)

    def D_oe(self, fe):
        return self.op.apply_at(self._full(fe=fe), self.odd)

    def D_oo(self, fo):
        return self.op.apply_at(self._full(fo=fo), self.odd)

    @staticmethod
    def _block_solve(blocks, f):
        sh = f.shape
        rhs = f.reshape(sh[:-3] + (sh[-3], 12))
        rhs = np.moveaxis(rhs, -2, 0)  # (n, ..., 12)
        x = np.linalg.solve(blocks[:, None, :, :], rhs.reshape(sh[-3], -1, 12)[..., None])[..., 0]
        x = x.reshape(rhs.shape)
        return np.moveaxis(x, 0, -2).reshape(sh)

    def D_oo_inv(self, fo):
        return self._block_solve(self.Doo_blocks, fo)

    def D_ee_inv(self, fe):
        return self._block_solve(self.Dee_blocks, fe)

    def D_hat(self, fe):
        """D_hat = Dee - Deo Doo^-1 Doe (Eq. (30))."""
        return self.D_ee(fe) - self.D_eo(self.D_oo_inv(self.D_oe(fe)))

    def prepare_source(self, b):
        """b_hat_e = b_e - Deo Doo^-1 b_o, so that D_hat x_e = b_hat_e."""
        return b[..., self.even, :, :] - self.D_eo(self.D_oo_inv(b[..., self.odd, :, :]))

    def reconstruct(self, xe, b):
        """Full solution from x_e: x_o = Doo^-1 (b_o - Doe x_e)."""
        xo = self.D_oo_inv(b[..., self.odd, :, :] - self.D_oe(xe))
        return self._full(fe=xe, fo=xo)


def vdot(a, b) -> complex:
    return complex(np.vdot(a.ravel(), b.ravel()))


def norm(a) -> float:
    return float(np.linalg.norm(a.ravel()))


def gcr(apply, b, tol: float = 1e-13, nkv: int = 16, max_iter: int = 20000, x0=None):
    """Plain restarted GCR(nkv) in FP64 for A x = b (no preconditioner).

    The paper names GCR (Sec. 1-2) without giving it; this is the textbook
    generalised conjugate residual method of Eisenstat, Elman and Schultz:
    each new direction p = r is made A-orthogonal to the previous ones
    (modified Gram-Schmidt on q = A p), x and r are updated along it, and the
    residual is recomputed from scratch at every restart.
    Returns (x, iterations, final true relative residual).
    """
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    bn = norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    r = b - apply(x) if x0 is not None else b.copy()
    it = 0
    while it < max_iter:
        ps, qs = [], []
        for _ in range(nkv):
            p = r.copy()
            q = apply(p)
            for pj, qj in zip(ps, qs):
                a = vdot(qj, q)
                q = q - a * qj
                p = p - a * pj
            qn = norm(q)
            q, p = q / qn, p / qn
            alpha = vdot(q, r)
            x = x + alpha * p
            r = r - alpha * q
            ps.append(p)
            qs.append(q)
            it += 1
            if norm(r) <= tol * bn or it >= max_iter:
                break
        r = b - apply(x)
        if norm(r) <= tol * bn:
            break
    return x, it, norm(b - apply(x)) / bn


# ---------------------------------------------------------------------------
# Schwarz alternating procedure (the preconditioner of the GCR solver)
# ---------------------------------------------------------------------------


def block_mr(A, c, block_id, nblocks: int, nmr: int, mask):
    """nmr minimal-residual steps on A y = c from y = 0, rho = c, on every
    block at once (A maps fields supported on `mask` to such fields and does
    not couple blocks). Step: w = A rho, omega_b = <w, rho>_b / <w, w>_b with
    the inner products summed over block b (omega_b = 0 where w vanishes on
    b), y += omega rho, rho -= omega w. That omega minimises the block norm
    of rho - omega w, so the new rho is orthogonal to w on every block, and
    rho = c - A y throughout. Returns (y, rho). This is the block solve of
    the Schwarz method below, which the paper names without giving it."""
    y = np.zeros_like(c)
    rho = c.copy()

    def restrict(f):
        g = np.zeros_like(f)
        g[mask] = f[mask]
        return g

    for _ in range(nmr):
        w = A(rho)
        wr = np.einsum("nsc,nsc->n", np.conj(w), rho)
        ww = np.einsum("nsc,nsc->n", np.conj(w), w).real
        num = np.bincount(block_id, weights=wr.real, minlength=nblocks) + \
            1j * np.bincount(block_id, weights=wr.imag, minlength=nblocks)
        den = np.bincount(block_id, weights=ww, minlength=nblocks)
        with np.errstate(invalid="ignore", divide="ignore"):
            om = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
        omega = om[block_id][:, None, None]
        y = restrict(y + omega * rho)
        rho = restrict(rho - omega * w)
    return y, rho


def sap(op: Dirac, eta, ncy: int, nmr: int, bs: int = 4):
    """SAP(eta): multiplicative Schwarz method on bs^4 blocks.

    The paper names the SAP preconditioner (Sec. 1-2) without giving it; this
    is the standard method. The lattice is cut into bs^4 blocks, coloured by
    the parity of their block coordinates. Starting from psi = 0, each of the
    ncy cycles visits colour 0, then colour 1. For the blocks B of a colour:
      r = eta - D psi                                  (whole lattice)
      delta_B ~ D_B^-1 r_B by nmr minimal-residual steps (block_mr) on the
               even-odd form D_hat_B = D_ee - D_eo D_oo^-1 D_oe of D_B
      psi_B += delta_B
    where D_B is D restricted to B with the hops leaving B dropped. Blocks of
    one colour never touch, so D restricted to all of them is the direct sum
    of their D_B, and all of them are handled at once here.
    """
    lat = op.lat
    V = lat.V
    c = lat.coords(lat.all_sites())
    for mu in range(4):
        if lat.N[mu] % (2 * bs):
            raise ValueError("every extent must be a multiple of 2 bs")
    for k in (2, 3):
        # across a shifted boundary the block coordinate b_k jumps by
        # -(N_k/bs - 1) and b_1 by L1/bs: the colouring stays a checkerboard
        # only if N_k/bs + L1/bs is even
        if lat.cstar[k] and (lat.L[1] % bs or (lat.N[k] // bs + lat.L[1] // bs) % 2):
            raise ValueError("block colouring inconsistent across the shifted boundary")
    B = c // bs
    nb = [lat.N[mu] // bs for mu in range(4)]
    block_id = ((B[:, 0] * nb[1] + B[:, 1]) * nb[2] + B[:, 2]) * nb[3] + B[:, 3]
    colour = B.sum(axis=1) % 2
    parity = c.sum(axis=1) % 2
    eo = EvenOdd(op)
    Doo_inv = np.linalg.inv(eo.Doo_blocks)  # per odd site
    inv_full = np.zeros((V, 12, 12), dtype=np.complex128)
    inv_full[eo.odd] = Doo_inv
    eta = np.asarray(eta, dtype=np.complex128)
    psi = np.zeros_like(eta)

    def restrict(f, mask):
        g = np.zeros_like(f)
        g[mask] = f[mask]
        return g

    def site_mul(mats, f):
        return np.einsum("nij,nj->ni", mats, f.reshape(V, 12)).reshape(V, 4, 3)

    for _ in range(ncy):
        for col in (0, 1):
            inb = colour == col
            even_b = inb & (parity == 0)
            odd_b = inb & (parity == 1)

            def D_B(f):  # D restricted to the blocks of this colour
                return restrict(op.apply(restrict(f, inb)), inb)

            def D_B_eo(f, rows, cols):  # block of D_B from the `cols` to the `rows` sites
                return restrict(D_B(restrict(f, cols)), rows)

            def Doo_inv_B(f):
                return restrict(site_mul(inv_full, f), odd_b)

            def D_hat_B(f):
                return D_B_eo(f, even_b, even_b) - D_B_eo(Doo_inv_B(D_B_eo(f, odd_b, even_b)), even_b, odd_b)

            r = restrict(eta - op.apply(psi), inb)
            # even-odd source: c_e = r_e - D_eo D_oo^-1 r_o
            ce = restrict(r, even_b) - D_B_eo(Doo_inv_B(r), even_b, odd_b)
            y, _ = block_mr(D_hat_B, ce, block_id, int(np.prod(nb)), nmr, even_b)
            # odd part: y_o = D_oo^-1 (r_o - D_oe y_e)
            yo = Doo_inv_B(restrict(r, odd_b) - D_B_eo(y, odd_b, even_b))
            psi = psi + y + yo
    return psi
