"""Pins of the FP64 oracle: statements fixed by the paper or by mathematics.

Each ``pin_*`` function builds its own inputs, runs one oracle computation and
returns the largest deviation from what the paper (or a closed form derived
from it) fixes. ``test_oracle_pins.py`` checks that every deviation is at
rounding level; ``test_oracle_mutations.py`` plants plausible mistakes in the
oracle and checks that at least one pin catches each of them.

The closed forms here are derived by hand from the paper's definitions and
written out independently of the oracle's code (explicit chiral-basis
matrices, explicit momenta of the shifted torus), so a pin is not the oracle
checked against itself.
"""
from __future__ import annotations

import numpy as np

import oracle as O

RNG_SEED = 12345

# chiral-basis matrices written out by hand (gamma5 = diag(1,1,-1,-1))
S1 = np.array([[0, 1], [1, 0]], dtype=complex)
S2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
S3 = np.array([[1, 0], [0, -1]], dtype=complex)
Z2 = np.zeros((2, 2), dtype=complex)
I2 = np.eye(2, dtype=complex)


def _blockdiag(a, b):
    return np.block([[a, Z2], [Z2, b]])


# sigma_0k = diag(s_k, -s_k); sigma_ij = -eps_ijk diag(s_k, s_k)
SIGMA_01 = _blockdiag(S1, -S1)
SIGMA_02 = _blockdiag(S2, -S2)
SIGMA_03 = _blockdiag(S3, -S3)
SIGMA_12 = -_blockdiag(S3, S3)
SIGMA_13 = _blockdiag(S2, S2)
SIGMA_23 = -_blockdiag(S1, S1)
GAMMA_HAND = np.array([
    np.block([[Z2, -I2], [-I2, Z2]]),
    np.block([[Z2, -1j * S1], [1j * S1, Z2]]),
    np.block([[Z2, -1j * S2], [1j * S2, Z2]]),
    np.block([[Z2, -1j * S3], [1j * S3, Z2]]),
])


def rng(seed=RNG_SEED):
    return np.random.default_rng(seed)


def random_su3(r, n):
    """Random SU(3) matrices (QR of complex Gaussians, det fixed to 1)."""
    z = r.normal(size=(n, 3, 3)) + 1j * r.normal(size=(n, 3, 3))
    q, rr = np.linalg.qr(z)
    d = np.diagonal(rr, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[:, None, None]


def random_spinor(r, shape):
    return r.normal(size=shape + (4, 3)) + 1j * r.normal(size=shape + (4, 3))


def random_physical_gauge(r, lat, eps=0.5, sigma=0.6):
    """Admissible gauge field: random physical half (mirror built by the oracle)."""
    T, L1, L2, L3 = lat.L
    n = T * L1 * L2 * L3 * 4
    # links near the identity: U = exp(i eps H), H random Hermitian traceless
    H = r.normal(size=(n, 3, 3)) + 1j * r.normal(size=(n, 3, 3))
    H = 0.5 * (H + np.conj(np.swapaxes(H, -1, -2)))
    H -= np.trace(H, axis1=-2, axis2=-1)[:, None, None] * np.eye(3) / 3
    w, v = np.linalg.eigh(H)
    U = np.einsum("nij,nj,nkj->nik", v, np.exp(1j * eps * w), np.conj(v))
    A = sigma * r.normal(size=n)
    A = np.remainder(A + np.pi, 2 * np.pi) - np.pi
    return O.GaugeField.from_physical(lat, U.reshape(T, L1, L2, L3, 4, 3, 3),
                                      A.reshape(T, L1, L2, L3, 4))


def random_extended_gauge(r, lat):
    """Unconstrained gauge field over the whole simulated lattice."""
    U = random_su3(r, lat.V * 4).reshape(lat.V, 4, 3, 3)
    A = r.uniform(-np.pi, np.pi, size=(lat.V, 4))
    return O.GaugeField.from_extended(lat, U, A)


def unit_gauge(lat):
    U = np.broadcast_to(np.eye(3, dtype=complex), (lat.V, 4, 3, 3)).copy()
    return O.GaugeField.from_extended(lat, U, np.zeros((lat.V, 4)))


# ---------------------------------------------------------------------------
# P1 / P2: plane waves on the shifted torus
# ---------------------------------------------------------------------------


def allowed_momentum(lat, n):
    """Momentum p = (p0, p1, p2, p3) of the plane waves of the simulated torus.

    Periodic directions: p = 2 pi n / N. With C* in direction 1 the x1 extent
    is 2 L1, so p1 = pi n1 / L1; a C* direction k (shifted boundary) needs
    exp(i p_k L_k) = exp(i p1 L1), i.e. p_k = (2 pi n_k + pi n1) / L_k.
    """
    T, L1, L2, L3 = lat.L
    p = np.zeros(4)
    p[0] = 2 * np.pi * n[0] / T
    p[1] = (np.pi * n[1] / L1) if lat.cstar[1] else (2 * np.pi * n[1] / L1)
    for k in (2, 3):
        if lat.cstar[k]:
            p[k] = (2 * np.pi * n[k] + np.pi * n[1]) / lat.L[k]
        else:
            p[k] = 2 * np.pi * n[k] / lat.L[k]
    return p


def plane_wave(lat, p, u):
    c = lat.coords(lat.all_sites())
    ph = np.exp(1j * (c @ p))
    return ph[:, None, None] * u[None, :, :]


def free_symbol(p, m0):
    """m0 + sum_mu (1 - cos p_mu + i gamma_mu sin p_mu) (Dw on plane waves, U = 1)."""
    M = m0 * np.eye(4, dtype=complex)
    for mu in range(4):
        M += (1 - np.cos(p[mu])) * np.eye(4) + 1j * np.sin(p[mu]) * GAMMA_HAND[mu]
    return M


def pin_plane_waves(lat, dirac_cls=O.Dirac, ntrial=4, m0=0.3, qhat=2, theta=None, seed=1):
    """Max |D pw - symbol pw| over random allowed momenta; U = 1.

    With ``theta`` (4 angles) the U(1) links are the constant phases
    exp(i theta_mu) (not admissible; P2), which shift p_mu by qhat theta_mu.
    """
    r = rng(seed)
    g = unit_gauge(lat)
    if theta is not None:
        g = O.GaugeField.from_extended(lat, g.su3, np.broadcast_to(theta, (lat.V, 4)).copy())
    op = dirac_cls(lat, g, m0, 1.3, 0.7, qhat)
    err = 0.0
    for _ in range(ntrial):
        n = r.integers(-5, 6, size=4)
        p = allowed_momentum(lat, n)
        u = r.normal(size=(4, 3)) + 1j * r.normal(size=(4, 3))
        psi = plane_wave(lat, p, u)
        peff = p + (qhat * np.asarray(theta) if theta is not None else 0.0)
        expect = plane_wave(lat, p, free_symbol(peff, m0) @ u)
        err = max(err, np.abs(op.apply(psi) - expect).max())
    return err


# ---------------------------------------------------------------------------
# Clover: closed form for constant abelian field strength (plain torus)
# ---------------------------------------------------------------------------


def constant_flux_angles(N0, N1, nflux):
    """Photon field with plaquette angle theta = 2 pi nflux / (N0 N1) on every
    (0,1) plaquette of an N0 x N1 torus, zero in all other planes.

    A(x,1) = theta x0; A(x,0) = -theta N0 x1 on the slice x0 = N0 - 1, else 0.
    Returns (theta, A0(x0,x1), A1(x0,x1)).
    """
    theta = 2 * np.pi * nflux / (N0 * N1)
    x0, x1 = np.meshgrid(np.arange(N0), np.arange(N1), indexing="ij")
    A1 = theta * x0
    A0 = np.where(x0 == N0 - 1, -theta * N0 * x1, 0.0)
    return theta, A0, A1


def pin_clover_constant_field(dirac_cls=O.Dirac, m0=0.1, csw=1.7, cswU1=0.9, qhat=-2):
    """dDsw for constant abelian field strength in the (0,1) plane.

    Hand derivation: every (0,1) plaquette is exp(i theta) (and the (1,0) one
    its conjugate), so A_hat_01 = i sin(theta) q_el^-1 and F_hat_01 =
    diag(i sin theta_a); the sum over mu, nu of (i/4) sigma_munu X_munu is
    then -(1/2) sigma_01 X'_01 with X' = sin. Hence
        dDsw = -(csw/2) sigma_01 (x) diag(sin theta_a)
               -(qhat cswU1 / 2) sin(theta) sigma_01 (x) 1.
    Returns the max deviation of the oracle's 12x12 SW matrices from that.
    """
    lat = O.Lattice(4, 6, 2, 2, cstar_mask=0)
    N0, N1 = lat.N[0], lat.N[1]
    c = lat.coords(lat.all_sites())
    fluxes = (1, 2, -3)  # three abelian fields on the SU(3) diagonal
    th_a, U = [], np.zeros((lat.V, 4, 3, 3), dtype=complex)
    for a, nf in enumerate(fluxes):
        th, A0, A1 = constant_flux_angles(N0, N1, nf)
        th_a.append(th)
        U[:, 0, a, a] = np.exp(1j * A0[c[:, 0], c[:, 1]])
        U[:, 1, a, a] = np.exp(1j * A1[c[:, 0], c[:, 1]])
        U[:, 2, a, a] = 1.0
        U[:, 3, a, a] = 1.0
    thq, B0, B1 = constant_flux_angles(N0, N1, 1)
    A = np.zeros((lat.V, 4))
    A[:, 0] = B0[c[:, 0], c[:, 1]]
    A[:, 1] = B1[c[:, 0], c[:, 1]]
    g = O.GaugeField.from_extended(lat, U, A)
    op = dirac_cls(lat, g, m0, csw, cswU1, qhat)
    sw = op.sw_matrix(lat.all_sites())
    expect = (-(csw / 2) * np.kron(SIGMA_01, np.diag(np.sin(th_a)))
              - (qhat * cswU1 / 2) * np.sin(thq) * np.kron(SIGMA_01, np.eye(3)))
    return np.abs(sw - expect[None]).max()


# ---------------------------------------------------------------------------
# Gauge covariance, gamma5-hermiticity, Sec. 2.4 identities
# ---------------------------------------------------------------------------


def pin_gauge_covariance(lat, dirac_cls=O.Dirac, admissible=True, qhat=2, seed=2):
    """D[U', z'](w^q L psi) = w^q L (D[U,z] psi) for a random local transform
    L(x) in SU(3), w(x) = exp(i alpha(x)), U' = L U L(x+mu)^+,
    A' = A + alpha(x) - alpha(x+mu). With ``admissible`` the transform obeys
    L(T x) = L(x)^*, alpha(T x) = -alpha(x), so U', A' stay admissible."""
    r = rng(seed)
    V = lat.V
    if admissible:
        g = random_physical_gauge(r, lat)
    else:
        g = random_extended_gauge(r, lat)
    U, A = g.extended_arrays()
    Lam = random_su3(r, V)
    alpha = r.uniform(-np.pi, np.pi, size=V)
    if admissible:
        s = lat.all_sites()
        phys = lat.is_physical(s)
        tr = lat.translate(s)
        Lam[~phys] = np.conj(Lam[tr[~phys]])
        alpha[~phys] = -alpha[tr[~phys]]
    Up = np.empty_like(U)
    Ap = np.empty_like(A)
    for mu in range(4):
        up = lat.shift(lat.all_sites(), mu, +1)
        Up[:, mu] = Lam @ U[:, mu] @ O.dagger(Lam[up])
        Ap[:, mu] = A[:, mu] + alpha - alpha[up]
    if admissible:
        T_, L1, L2, L3 = lat.L
        ph = lat.is_physical(lat.all_sites())
        gp = O.GaugeField.from_physical(lat, Up[ph].reshape(T_, L1, L2, L3, 4, 3, 3),
                                        Ap[ph].reshape(T_, L1, L2, L3, 4))
        # the transformed mirror half must equal the one Eq. (4a) builds
        Ue, Ae = gp.extended_arrays()
        assert np.abs(Ue - Up).max() < 1e-12
        assert np.abs(np.exp(1j * Ae) - np.exp(1j * Ap)).max() < 1e-12
    else:
        gp = O.GaugeField.from_extended(lat, Up, Ap)
    op = dirac_cls(lat, g, 0.15, 1.1, 0.8, qhat)
    opp = dirac_cls(lat, gp, 0.15, 1.1, 0.8, qhat)
    psi = random_spinor(r, (V,))
    wq = np.exp(1j * qhat * alpha)
    tpsi = wq[:, None, None] * O.colour_mul(Lam, psi)
    lhs = opp.apply(tpsi)
    rhs = wq[:, None, None] * O.colour_mul(Lam, op.apply(psi))
    return np.abs(lhs - rhs).max() / np.abs(rhs).max()


def pin_gamma5_hermiticity(lat, dirac_cls=O.Dirac, seed=3):
    """<chi, g5 D phi> = <g5 D chi, phi> for random chi, phi (g5 D Hermitian)."""
    r = rng(seed)
    g = random_physical_gauge(r, lat)
    op = dirac_cls(lat, g, 0.05, 1.2, 0.9, -1)
    chi, phi = random_spinor(r, (lat.V,)), random_spinor(r, (lat.V,))
    G5 = np.diag([1, 1, -1, -1]).astype(complex)
    a = np.vdot(chi, O.spin_mul(G5, op.apply(phi)))
    b = np.vdot(O.spin_mul(G5, op.apply(chi)), phi)
    return abs(a - b) / abs(a)


def _bilinear(a, b):
    return np.sum(a * b)


def pin_transpose_identity(lat, dirac_cls=O.Dirac, seed=4):
    """Eq. (25): D[U,z]^T = C D[U^*, z^*] C^-1, checked as the bilinear
    chi^T D phi = phi^T C D[U^*,z^*] C^-1 chi for random chi, phi."""
    r = rng(seed)
    g = random_physical_gauge(r, lat)
    op = dirac_cls(lat, g, 0.07, 1.4, 0.6, 2)
    opc = op.conjugate_fields()
    chi, phi = random_spinor(r, (lat.V,)), random_spinor(r, (lat.V,))
    C, Ci = _hand_C(), np.linalg.inv(_hand_C())
    lhs = _bilinear(chi, op.apply(phi))
    rhs = _bilinear(phi, O.spin_mul(C, opc.apply(O.spin_mul(Ci, chi))))
    return abs(lhs - rhs) / abs(lhs)


def _hand_C():
    """C = gamma0 gamma2 written out in the chiral basis: diag(-i s2, i s2),
    real and antisymmetric."""
    return np.block([[np.array([[0, -1], [1, 0]]), Z2],
                     [Z2, np.array([[0, 1], [-1, 0]])]]).astype(complex)


def _translate_field(lat, f):
    return f[..., lat.translate(lat.all_sites()), :, :]


def pin_mirror_identity(lat, dirac_cls=O.Dirac, seed=5):
    """Eq. (26): T D[U^*, z^*] T^-1 = D[U, z] for admissible fields."""
    r = rng(seed)
    g = random_physical_gauge(r, lat)
    op = dirac_cls(lat, g, 0.2, 1.0, 1.0, -1)
    opc = op.conjugate_fields()
    phi = random_spinor(r, (lat.V,))
    lhs = _translate_field(lat, opc.apply(_translate_field(lat, phi)))  # T^-1 = T
    rhs = op.apply(phi)
    return np.abs(lhs - rhs).max() / np.abs(rhs).max()


def pin_antisymmetry(lat, dirac_cls=O.Dirac, seed=6):
    """Sec. 2.4: C T D is antisymmetric: chi^T C T D phi = -phi^T C T D chi."""
    r = rng(seed)
    g = random_physical_gauge(r, lat)
    op = dirac_cls(lat, g, 0.2, 1.3, 0.5, 2)
    C = _hand_C()
    chi, phi = random_spinor(r, (lat.V,)), random_spinor(r, (lat.V,))

    def ctd(f):
        return O.spin_mul(C, _translate_field(lat, op.apply(f)))

    a = _bilinear(chi, ctd(phi))
    b = _bilinear(phi, ctd(chi))
    return abs(a + b) / abs(a)


def pin_theta_symmetry(lat, dirac_cls=O.Dirac, seed=7):
    """Antilinear map Theta phi(x) = g5 C^-1 phi(T x)^* (derived from
    Eqs. (25)-(26) and gamma5-hermiticity): D Theta = Theta D, Theta^2 = -1."""
    r = rng(seed)
    g = random_physical_gauge(r, lat)
    op = dirac_cls(lat, g, 0.1, 1.1, 1.2, -1)
    G5 = np.diag([1, 1, -1, -1]).astype(complex)
    K = G5 @ np.linalg.inv(_hand_C())

    def theta(f):
        return O.spin_mul(K, np.conj(_translate_field(lat, f)))

    phi = random_spinor(r, (lat.V,))
    e1 = np.abs(op.apply(theta(phi)) - theta(op.apply(phi))).max() / np.abs(op.apply(phi)).max()
    e2 = np.abs(theta(theta(phi)) + phi).max() / np.abs(phi).max()
    return max(e1, e2)


# ---------------------------------------------------------------------------
# Dense LU, even-odd, reductions
# ---------------------------------------------------------------------------


def pin_dense_lu_vs_gcr(lat, dirac_cls=O.Dirac, seed=8):
    """GCR to 1e-13 against numpy's dense LU solve (tiny lattice)."""
    r = rng(seed)
    g = random_physical_gauge(r, lat)
    op = dirac_cls(lat, g, 0.2, 1.0, 1.0, -1)
    M = O.dense_matrix(op)
    b = random_spinor(r, (lat.V,))
    x_lu = np.linalg.solve(M, b.ravel()).reshape(b.shape)
    x_gcr, _, res = O.gcr(op.apply, b, tol=1e-13)
    return max(np.linalg.norm(x_gcr - x_lu) / np.linalg.norm(x_lu), res * 1e-3)


def pin_even_odd(lat, dirac_cls=O.Dirac, seed=9):
    """Sec. 2.4 (Eqs. (29)-(31)): Det D = Det Doo Det D_hat, and the solve via
    D_hat plus reconstruction equals the dense solve of D."""
    r = rng(seed)
    g = random_physical_gauge(r, lat)
    op = dirac_cls(lat, g, 0.1, 1.2, 0.8, 2)
    eo = O.EvenOdd(op)
    M = O.dense_matrix(op)
    ne = len(eo.even)
    Dhat = eo.D_hat(np.eye(12 * ne, dtype=complex).reshape(12 * ne, ne, 4, 3)).reshape(12 * ne, 12 * ne).T
    s_full, ld_full = np.linalg.slogdet(M)
    s_oo, ld_oo = np.linalg.slogdet(eo.Doo_blocks)
    s_hat, ld_hat = np.linalg.slogdet(Dhat)
    e1 = abs(ld_full - (ld_oo.sum() + ld_hat)) / abs(ld_full)
    e2 = abs(s_full - np.prod(s_oo) * s_hat)
    b = random_spinor(r, (lat.V,))
    bh = eo.prepare_source(b)
    xe = np.linalg.solve(Dhat, bh.ravel()).reshape(bh.shape)
    x = eo.reconstruct(xe, b)
    x_ref = np.linalg.solve(M, b.ravel()).reshape(b.shape)
    e3 = np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
    return max(e1, e2, e3)


def pin_reductions(lat, dirac_cls=O.Dirac, seed=10):
    """qhat = 0: D does not depend on A. csw = cswU1 = 0: D is m0 + Dw.
    U = 1 with random z: D acts identically on the three colours."""
    r = rng(seed)
    g = random_physical_gauge(r, lat)
    psi = random_spinor(r, (lat.V,))
    # (a) qhat = 0 -> independent of the photon field
    g2 = O.GaugeField.from_physical(lat, g.su3.reshape(lat.L + (4, 3, 3)),
                                    r.uniform(-np.pi, np.pi, size=lat.L + (4,)))
    a = dirac_cls(lat, g, 0.1, 1.0, 1.0, 0).apply(psi)
    b = dirac_cls(lat, g2, 0.1, 1.0, 1.0, 0).apply(psi)
    e1 = np.abs(a - b).max()
    # (b) csw = cswU1 = 0: (m0 + 4) psi - 1/2 sum of the hops
    op = dirac_cls(lat, g, 0.1, 0.0, 0.0, 2)
    hop = np.zeros_like(psi)
    s = lat.all_sites()
    U, A = g.extended_arrays()
    for mu in range(4):
        up, dn = lat.shift(s, mu, +1), lat.shift(s, mu, -1)
        W = U[:, mu] * np.exp(2j * A[:, mu])[:, None, None]
        fwd = O.colour_mul(W, psi[up])
        bwd = O.colour_mul(O.dagger(W[dn]), psi[dn])
        hop += O.spin_mul(np.eye(4) - GAMMA_HAND[mu], fwd) + O.spin_mul(np.eye(4) + GAMMA_HAND[mu], bwd)
    e2 = np.abs(op.apply(psi) - (4.1 * psi - 0.5 * hop)).max()
    # (c) U = 1, random z: colour-diagonal, identical on each colour
    T_, L1, L2, L3 = lat.L
    gu = O.GaugeField.from_physical(
        lat, np.broadcast_to(np.eye(3), lat.L + (4, 3, 3)).astype(complex),
        r.uniform(-np.pi, np.pi, size=lat.L + (4,)))
    opu = dirac_cls(lat, gu, 0.3, 1.0, 1.5, -1)
    chi = random_spinor(r, (lat.V,))[..., :1]
    chi3 = np.repeat(chi, 3, axis=-1)
    out = opu.apply(chi3)
    e3 = np.abs(out - out[..., :1]).max()
    return max(e1, e2, e3)
