"""The local-deflation oracle against exact relations and the free-field
coarse operator (no GPU); planted mistakes are caught."""
import numpy as np
import pytest

from oracle import qxd_dfl as DF
import pins_dfl as PD


def test_block_qr():
    assert PD.pin_block_qr() < 1e-12


def test_free_field_little_operator_is_the_coarse_wilson_operator():
    assert PD.pin_free_little_operator() < 1e-12


def test_prolong_restrict_and_little_operator_definition():
    assert PD.pin_prolong_restrict() < 1e-12


def test_deflated_preconditioner_exact_on_the_deflation_image():
    assert PD.pin_preconditioner_exact_on_DS() < 1e-10


def test_little_system_splits_by_block_colour():
    assert PD.pin_little_even_odd() < 1e-10
    assert PD.pin_little_even_odd(planted_colouring=True) > 1e-3


_ORIG_LITTLE = DF.little_operator
_ORIG_ORTH = DF.block_orthonormalize
_ORIG_PRE = DF.deflated_preconditioner


def _little_adjoint(op, phi, bs=4):
    return _ORIG_LITTLE(op, phi, bs).conj().T


def _orth_no_sign(lat, psi, bs=4):
    phi = _ORIG_ORTH(lat, psi, bs)
    phi[0] = -phi[0]
    return phi


def _pre_no_coarse(op, phi, A, eta, ncy, nmr, bs=4):
    from oracle.qxd_oracle import sap
    return sap(op, eta, ncy, nmr, bs)


def _restrict_no_conj(lat, phi, eta, bs=4):
    bid = DF.block_index(lat, bs)
    nblk = bid.max() + 1
    w = np.einsum("kxsc,xsc->kx", phi, eta)
    c = np.zeros((nblk, phi.shape[0]), dtype=np.complex128)
    for k in range(phi.shape[0]):
        c[:, k] = np.bincount(bid, weights=w[k].real, minlength=nblk) + \
            1j * np.bincount(bid, weights=w[k].imag, minlength=nblk)
    return c


MUTATIONS = {
    "little_operator_adjoint": ("little_operator", _little_adjoint),
    "orthonormalize_sign": ("block_orthonormalize", _orth_no_sign),
    "preconditioner_without_coarse_step": ("deflated_preconditioner", _pre_no_coarse),
    "restrict_without_conjugate": ("restrict", _restrict_no_conj),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(DF, attr, fn)
    worst = 0.0
    for pin in (PD.pin_block_qr, PD.pin_free_little_operator, PD.pin_prolong_restrict,
                PD.pin_preconditioner_exact_on_DS):
        try:
            worst = max(worst, float(pin()))
        except AssertionError:
            worst = np.inf
        if worst > 1e-6:
            break
    assert worst > 1e-6
