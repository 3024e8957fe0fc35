"""Shared set-up of the GPU parity tests: seeded inputs from ``synth`` feed
both the CUDA path (through the C ABI) and the FP64 oracle."""
from __future__ import annotations

import numpy as np
import torch

import oracle as O
import synth


def rel_max(a, b):
    """Relative max error: max|a - b| / max|b| over all reals."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


def rel_norm(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


class Case:
    """Physical lattice, C* mask, generator widths and quark parameters."""

    def __init__(self, T, L1, L2, L3, mask=0b1110, eps=0.3, sigma=0.3, m0=0.2, csw=1.0,
                 cswqed=1.0, qhat=-1, seed=0, device="cpu"):
        self.T, self.L1, self.L2, self.L3, self.mask = T, L1, L2, L3, mask
        self.m0, self.csw, self.cswqed, self.qhat = m0, csw, cswqed, qhat
        self.N1 = synth.extended_extent(L1, mask)
        self.V = T * self.N1 * L2 * L3
        self.su3 = synth.su3_field(T, L1, L2, L3, eps, synth.SEED_GAUGE + seed, device=device)
        self.ang = synth.u1_field(T, L1, L2, L3, sigma, synth.SEED_GAUGE + 500 + seed, device=device)
        self.psi = synth.spinor_field(T, self.N1, L2, L3, synth.SEED_SOURCE + seed,
                                      device=device).reshape(self.V, 4, 3)

    def oracle(self, su3=None, ang=None):
        lat = O.Lattice(self.T, self.L1, self.L2, self.L3, self.mask)
        su3 = (self.su3 if su3 is None else su3)
        ang = (self.ang if ang is None else ang)
        su3 = su3.cpu().numpy() if torch.is_tensor(su3) else su3
        ang = ang.cpu().numpy() if torch.is_tensor(ang) else ang
        g = O.GaugeField.from_physical(lat, su3, ang)
        return O.Dirac(lat, g, self.m0, self.csw, self.cswqed, self.qhat)

    def lattice(self):
        from paper_1710_08839_gb300 import qxd
        lat = qxd.Lattice(self.T, self.L1, self.L2, self.L3, self.mask)
        lat.set_gauge(self.su3.cuda(), self.ang.cuda())
        lat.set_params(self.m0, self.csw, self.cswqed, self.qhat)
        lat.sw_build()
        return lat
