"""Seeded synthetic inputs for the C*-boundary Wilson-clover operator.

This module is shared by the FP64 oracle (``oracle/``), the tests and the
benchmark. It holds no arithmetic of the Dirac operator itself: it only draws
gauge fields, photon fields and spinor sources. The orbifold (mirror) half of
the gauge field is NOT built here: the generators return the physical half
``0 <= x1 < L1`` only, and each side builds the mirror half on its own.

Recipe (the paper's ensembles are not available; these stand in for them):

* SU(3) link: ``U = exp(i * eps * H)`` with ``H = sum_a h_a lambda_a / 2``,
  ``h_a ~ N(0, 1)`` and ``lambda_a`` the Gell-Mann matrices (Hermitian,
  traceless). Rows 0 and 1 are then re-orthonormalised (Gram-Schmidt) and row
  2 is set to ``conj(row0 x row1)``, so that ``det U = 1`` to rounding.
* U(1) angle: ``A = sigma * theta`` with ``theta ~ N(0, 1)``, wrapped to
  ``[-pi, pi)`` (Sec. 2.1: the photon field is restricted to that interval).
* Spinor source: every real and imaginary part ``~ N(0, 1)`` on every site of
  the extended lattice (the pseudofermion field is unrestricted there, Sec. 2.4).
* Point sources: the 12 spin-colour unit vectors at one seeded site.

Array shapes (all lexicographic, x3 fastest):

* ``su3``   : ``(T, L1, L2, L3, 4, 3, 3)`` complex128, physical half.
* ``angle`` : ``(T, L1, L2, L3, 4)`` float64, physical half.
* spinor    : ``(T, N1, L2, L3, 4, 3)`` complex128, ``N1 = 2 L1`` with C*
  boundaries, ``L1`` without.

Normals come from a CPU ``torch.Generator`` seeded with ``seed``, drawn in
fixed-size chunks so the stream does not depend on the device that does the
matrix exponentials. Large fields can be finished on a CUDA device
(``device='cuda'``); the result is the same up to rounding of the exponential.
"""
from __future__ import annotations

import math

import torch

__all__ = [
    "gell_mann",
    "su3_field",
    "u1_field",
    "spinor_field",
    "spinor_field_device",
    "point_source",
    "extended_extent",
    "SEED_GAUGE",
    "SEED_SOURCE",
]

# Seed rule of the benchmark workloads: gauge = 1000 + workload id,
# source = 2000 + workload id + request id, arrivals = 3000.
SEED_GAUGE = 1000
SEED_SOURCE = 2000

_CHUNK = 1 << 22  # normals drawn per generator call (fixed: keeps streams stable)


def extended_extent(L1: int, cstar_mask: int) -> int:
    """x1 extent of the simulated lattice: 2 L1 when direction 1 is C*."""
    return 2 * L1 if (cstar_mask & 2) else L1


def _normals(n: int, seed: int) -> torch.Tensor:
    """``n`` standard normals (float64, CPU) from one seeded stream."""
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    out = torch.empty(n, dtype=torch.float64)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        buf = torch.randn(_CHUNK, dtype=torch.float64, generator=g)
        out[s:e] = buf[: e - s]
    return out


def gell_mann(device="cpu") -> torch.Tensor:
    """The eight Gell-Mann matrices, shape (8, 3, 3) complex128."""
    lam = torch.zeros(8, 3, 3, dtype=torch.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1] = -1j
    lam[1, 1, 0] = 1j
    lam[2, 0, 0] = 1
    lam[2, 1, 1] = -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2] = -1j
    lam[4, 2, 0] = 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2] = -1j
    lam[6, 2, 1] = 1j
    lam[7, 0, 0] = lam[7, 1, 1] = 1 / math.sqrt(3)
    lam[7, 2, 2] = -2 / math.sqrt(3)
    return lam.to(device)


def _reunitarise(u: torch.Tensor) -> torch.Tensor:
    r0 = u[..., 0, :]
    r0 = r0 / torch.linalg.vector_norm(r0, dim=-1, keepdim=True)
    r1 = u[..., 1, :]
    r1 = r1 - (r0.conj() * r1).sum(-1, keepdim=True) * r0
    r1 = r1 / torch.linalg.vector_norm(r1, dim=-1, keepdim=True)
    r2 = torch.stack(
        [
            r0[..., 1] * r1[..., 2] - r0[..., 2] * r1[..., 1],
            r0[..., 2] * r1[..., 0] - r0[..., 0] * r1[..., 2],
            r0[..., 0] * r1[..., 1] - r0[..., 1] * r1[..., 0],
        ],
        dim=-1,
    ).conj()
    return torch.stack([r0, r1, r2], dim=-2)


def su3_field(T: int, L1: int, L2: int, L3: int, eps: float, seed: int,
              device="cpu", chunk_links: int = 1 << 21) -> torch.Tensor:
    """Physical-half SU(3) links ``exp(i eps H)``, shape (T, L1, L2, L3, 4, 3, 3).

    ``eps = 0`` gives unit links.
    """
    nl = T * L1 * L2 * L3 * 4
    out = torch.empty(nl, 3, 3, dtype=torch.complex128, device=device)
    h = _normals(8 * nl, seed).view(nl, 8)
    lam = gell_mann(device)
    for s in range(0, nl, chunk_links):
        e = min(nl, s + chunk_links)
        hc = h[s:e].to(device)
        H = torch.einsum("na,aij->nij", hc.to(torch.complex128), lam) * 0.5
        u = torch.linalg.matrix_exp(1j * eps * H)
        out[s:e] = _reunitarise(u)
    return out.view(T, L1, L2, L3, 4, 3, 3)


def u1_field(T: int, L1: int, L2: int, L3: int, sigma: float, seed: int,
             device="cpu") -> torch.Tensor:
    """Physical-half photon field ``A`` in ``[-pi, pi)``, shape (T, L1, L2, L3, 4)."""
    n = T * L1 * L2 * L3 * 4
    a = sigma * _normals(n, seed).to(device)
    a = torch.remainder(a + math.pi, 2 * math.pi) - math.pi
    return a.view(T, L1, L2, L3, 4)


def spinor_field(T: int, N1: int, L2: int, L3: int, seed: int,
                 device="cpu") -> torch.Tensor:
    """Gaussian spinor on the whole simulated lattice, shape (T, N1, L2, L3, 4, 3)."""
    n = T * N1 * L2 * L3 * 12
    z = _normals(2 * n, seed).view(n, 2)
    psi = torch.complex(z[:, 0], z[:, 1]).to(device)
    return psi.view(T, N1, L2, L3, 4, 3)


def spinor_field_device(T: int, N1: int, L2: int, L3: int, seed: int, device="cuda") -> torch.Tensor:
    """Gaussian spinor drawn directly on `device` from a generator of that
    device seeded with `seed` (a different stream from spinor_field; used when
    many large sources are needed quickly)."""
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    n = T * N1 * L2 * L3 * 12
    z = torch.randn(n, 2, dtype=torch.float64, device=device, generator=g)
    return torch.complex(z[:, 0], z[:, 1]).view(T, N1, L2, L3, 4, 3)


def point_source(T: int, N1: int, L2: int, L3: int, seed: int,
                 device="cpu") -> tuple[tuple[int, int, int, int], torch.Tensor]:
    """The 12 spin-colour unit sources at one seeded site.

    Returns ``(site, src)`` with ``src`` of shape (12, T, N1, L2, L3, 4, 3);
    source ``k = 3 * spin + colour`` is 1 at ``site`` in that component.
    """
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    site = tuple(int(torch.randint(0, n, (1,), generator=g)) for n in (T, N1, L2, L3))
    src = torch.zeros(12, T, N1, L2, L3, 4, 3, dtype=torch.complex128, device=device)
    for k in range(12):
        src[(k,) + site + (k // 3, k % 3)] = 1.0
    return site, src
