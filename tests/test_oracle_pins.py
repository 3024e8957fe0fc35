"""The FP64 oracle against what the paper and mathematics fix (no GPU)."""
import numpy as np
import pytest

import oracle as O
import pins as P

TOL = 1e-11

# small lattices: (T, L1, L2, L3, cstar_mask)
CSTAR3 = (4, 2, 4, 2, 0b1110)      # C* in x, y, z
CSTAR12 = (4, 4, 2, 4, 0b0110)     # C* in x, y; z periodic
CSTAR1 = (2, 4, 2, 4, 0b0010)      # C* in x only
PERIODIC = (4, 2, 4, 4, 0)         # plain torus
LATTICES = [CSTAR3, CSTAR12, CSTAR1, PERIODIC]
TINY = [(2, 2, 2, 2, 0b1110), (4, 2, 2, 2, 0b1110)]   # 64 and 128 sites


def lat_of(t):
    return O.Lattice(*t)


def test_gamma_matrices_clifford_and_basis():
    # {g_mu, g_nu} = 2 delta, Hermitian; gamma5 = g0 g1 g2 g3 = diag(1,1,-1,-1)
    for mu in range(4):
        assert np.allclose(O.GAMMA[mu], P.GAMMA_HAND[mu])
        assert np.allclose(O.GAMMA[mu], O.GAMMA[mu].conj().T)
        for nu in range(4):
            ac = O.GAMMA[mu] @ O.GAMMA[nu] + O.GAMMA[nu] @ O.GAMMA[mu]
            assert np.allclose(ac, 2 * (mu == nu) * np.eye(4))
    assert np.allclose(O.GAMMA5, np.diag([1, 1, -1, -1]))


def test_sigma_chiral_blocks():
    hand = {(0, 1): P.SIGMA_01, (0, 2): P.SIGMA_02, (0, 3): P.SIGMA_03,
            (1, 2): P.SIGMA_12, (1, 3): P.SIGMA_13, (2, 3): P.SIGMA_23}
    for (mu, nu), s in hand.items():
        assert np.allclose(O.sigma(mu, nu), s)
        assert np.allclose(O.sigma(nu, mu), -s)


def test_charge_conjugation_properties():
    # Eq. (5): C^T = -C, C^+ = C^-1, C g_mu C^-1 = -g_mu^T
    C = O.CHARGE_C
    assert np.allclose(C, P._hand_C())
    assert np.allclose(C.T, -C)
    assert np.allclose(C.conj().T, np.linalg.inv(C))
    for mu in range(4):
        assert np.allclose(C @ O.GAMMA[mu] @ np.linalg.inv(C), -O.GAMMA[mu].T)


def _fig1_rows():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "fig1_geometry.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            d, col, ex1, exk, sx1, sxk = line.split()
            rows.append((d, col, int(ex1), int(exk), int(sx1), int(sxk)))
    return rows


@pytest.mark.parametrize("k", [2, 3])
def test_fig1_identifications(k):
    """Fig. 1: the empty circles beyond the boundary are the solid circles of
    the same colour (top: k is C*, bottom: k is periodic)."""
    rows = _fig1_rows()
    assert len(rows) == 36
    for diagram in ("cstar", "periodic"):
        mask = 0b0010 | ((1 << k) if diagram == "cstar" else 0)
        L = [2, 6, 2, 2]
        L[k] = 6
        lat = O.Lattice(*L, cstar_mask=mask)
        for d, col, ex1, exk, sx1, sxk in rows:
            if d != diagram:
                continue
            # the empty circle is reached by one step from an inner site
            if ex1 == 12:
                inner, mu = (11, exk), 1
            else:
                inner, mu = (ex1, exk - 1), k
            c = [1, 0, 1, 1]
            c[1], c[k] = inner
            got = lat.coords(lat.shift(lat.index(np.array(c)), mu, +1))
            assert (got[1], got[k]) == (sx1, sxk), (d, col, ex1, exk)
            # and back again
            c2 = [1, 0, 1, 1]
            c2[1], c2[k] = sx1, sxk
            back = lat.coords(lat.shift(lat.index(np.array(c2)), mu, -1))
            assert (back[1], back[k]) == inner


@pytest.mark.parametrize("t", LATTICES)
def test_free_field_plane_waves(t):
    assert P.pin_plane_waves(lat_of(t)) < TOL


@pytest.mark.parametrize("t", LATTICES)
def test_constant_abelian_phase(t):
    assert P.pin_plane_waves(lat_of(t), theta=np.array([0.3, -0.7, 1.1, 0.2]), qhat=-1) < TOL


def test_clover_constant_field_closed_form():
    assert P.pin_clover_constant_field() < TOL


def test_u1_tensor_matches_su3_leaf_formula():
    """The paper's U(1) tensor (Eqs. (22)-(23)) and the SU(3) clover leaves are
    written independently; on abelian links both must give (i/4) Im Q."""
    r = P.rng(11)
    lat = lat_of(CSTAR3)
    g = P.random_physical_gauge(r, lat)
    U, A = g.extended_arrays()
    Ud = np.exp(1j * A)[..., None, None] * np.eye(3)  # abelian "SU(3)" links diag(z,z,z)
    op_su3 = O.Dirac(lat, O.GaugeField.from_extended(lat, Ud, A), 0, 1, 1, 1)
    s = lat.all_sites()
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            F = op_su3.F_hat(s, mu, nu)
            a = op_su3.qA_hat(s, mu, nu)
            assert np.abs(F - a[:, None, None] * np.eye(3)).max() < 1e-13


@pytest.mark.parametrize("t", [CSTAR3, CSTAR12, PERIODIC])
@pytest.mark.parametrize("admissible", [True, False])
def test_gauge_covariance(t, admissible):
    lat = lat_of(t)
    if admissible and not lat.cstar[1]:
        pytest.skip("admissibility needs C* in direction 1")
    assert P.pin_gauge_covariance(lat, admissible=admissible) < TOL


@pytest.mark.parametrize("t", LATTICES)
def test_gamma5_hermiticity(t):
    assert P.pin_gamma5_hermiticity(lat_of(t)) < TOL


@pytest.mark.parametrize("t", [CSTAR3, CSTAR12, CSTAR1])
def test_transpose_identity(t):
    assert P.pin_transpose_identity(lat_of(t)) < TOL


def test_transpose_identity_dense():
    """Eq. (25) as a matrix identity on a tiny lattice."""
    r = P.rng(12)
    lat = lat_of(TINY[0])
    g = P.random_physical_gauge(r, lat)
    op = O.Dirac(lat, g, 0.2, 1.0, 1.0, -1)
    M = O.dense_matrix(op)
    Mc = O.dense_matrix(op.conjugate_fields())
    C = np.kron(np.eye(lat.V), np.kron(P._hand_C(), np.eye(3)))
    assert np.abs(M.T - C @ Mc @ np.linalg.inv(C)).max() < TOL


@pytest.mark.parametrize("t", [CSTAR3, CSTAR12, CSTAR1])
def test_mirror_identity(t):
    assert P.pin_mirror_identity(lat_of(t)) < TOL


@pytest.mark.parametrize("t", [CSTAR3, CSTAR12, CSTAR1])
def test_antisymmetry(t):
    assert P.pin_antisymmetry(lat_of(t)) < TOL


@pytest.mark.parametrize("t", [CSTAR3, CSTAR12, CSTAR1])
def test_theta_symmetry(t):
    assert P.pin_theta_symmetry(lat_of(t)) < TOL


def test_pfaffian_structure_dense():
    """Sec. 2.4: C T D is antisymmetric as a matrix, and |Det D| = |Det(C T D)|
    (det C = det T = 1, Eq. (28))."""
    r = P.rng(13)
    lat = lat_of(TINY[0])
    g = P.random_physical_gauge(r, lat)
    op = O.Dirac(lat, g, 0.2, 1.0, 1.0, 2)
    M = O.dense_matrix(op)
    n = 12 * lat.V
    Tm = np.zeros((lat.V, lat.V))
    Tm[np.arange(lat.V), lat.translate(lat.all_sites())] = 1.0
    CT = np.kron(Tm, np.kron(P._hand_C(), np.eye(3)))
    A = CT @ M
    assert np.abs(A + A.T).max() < TOL
    assert abs(np.linalg.det(CT) - 1) < 1e-12
    s1, l1 = np.linalg.slogdet(M)
    s2, l2 = np.linalg.slogdet(A)
    assert abs(l1 - l2) < 1e-9 and n == A.shape[0]


@pytest.mark.parametrize("t", TINY)
def test_dense_lu_vs_gcr(t):
    assert P.pin_dense_lu_vs_gcr(lat_of(t)) < 1e-10


@pytest.mark.parametrize("t", TINY)
def test_even_odd_block_form(t):
    assert P.pin_even_odd(lat_of(t)) < 1e-10


@pytest.mark.parametrize("t", [CSTAR3, PERIODIC])
def test_reductions(t):
    assert P.pin_reductions(lat_of(t)) < TOL


def test_parity_is_well_defined_on_shifted_torus():
    """Every hop connects sites of opposite parity (needs T, L1..L3 even)."""
    for t in LATTICES:
        lat = lat_of(t)
        s = lat.all_sites()
        for mu in range(4):
            for sg in (+1, -1):
                assert np.all(lat.parity(lat.shift(s, mu, sg)) != lat.parity(s))


def test_neighbour_map_is_a_bijection():
    for t in LATTICES:
        lat = lat_of(t)
        s = lat.all_sites()
        for mu in range(4):
            up = lat.shift(s, mu, +1)
            assert len(np.unique(up)) == lat.V
            assert np.all(lat.shift(up, mu, -1) == s)
