"""Seeded synthetic SU(3) gauge fields (input generator only).

This module builds inputs; it contains none of the gauge-fixing arithmetic.
Both the CUDA library's tests/benchmarks and the CPU oracle's tests take their
fields from here.

Recipe (the stand-in for the paper's beta = 6.1 Monte-Carlo ensembles, whose
links live in SU(3) as U = exp(i a g A), Sec. 1 eq. 2):

1. Every link is drawn independently as V = exp(i s H), H = sum_a xi_a lambda_a/2
   with xi_a ~ N(0, 1) i.i.d. and lambda_a the Gell-Mann matrices.
2. The scale s is fixed so that the expected average plaquette equals the
   target.  H's law is invariant under SU(3) conjugation, so E[V] = c(s) 1 with
   c(s) = E[Re tr V]/3, and for independent links E[plaquette] = c(s)^4.  c(s)
   is estimated once from a fixed-seed sample of eigenvalues of H and s is
   found by bisection.
3. V is projected back onto SU(3) (one Newton-Schulz polar step and a
   determinant phase), to remove rounding of the matrix exponential.
4. The field is rotated by a Haar-random gauge transformation g(x) (QR of a
   complex Gaussian matrix with R's diagonal made positive, Mezzadri 2007,
   computed as Gram-Schmidt on its columns, then divided by a cube root of
   its determinant):
   U_mu(x) = g(x) V_mu(x) g(x + mu)^dagger.
5. The pure-gauge input takes V = 1: U_mu(x) = g(x) g(x + mu)^dagger.

Fields are complex128 tensors of shape (Lt, Lz, Ly, Lx, 4, 3, 3); dims are
(Lx, Ly, Lz, Lt).  The generator runs on any torch device; a given seed gives
the same field on every run on the same device type.
"""
from __future__ import annotations

import functools
import math

import numpy as np
import torch

_PLAQ_SAMPLE = 200_000


def gell_mann(device="cpu") -> torch.Tensor:
    """The eight Gell-Mann matrices, shape (8, 3, 3), complex128."""
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


def _generator(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed))
    return g


def _algebra(xi: torch.Tensor) -> torch.Tensor:
    """H = sum_a xi_a lambda_a / 2 for xi of shape (..., 8)."""
    lam = gell_mann(xi.device)
    return torch.einsum("...a,aij->...ij", xi.to(torch.complex128), lam) * 0.5


def _det3(M: torch.Tensor) -> torch.Tensor:
    """Determinant of (..., 3, 3) matrices by cofactor expansion (vectorised)."""
    return (M[..., 0, 0] * (M[..., 1, 1] * M[..., 2, 2] - M[..., 1, 2] * M[..., 2, 1])
            - M[..., 0, 1] * (M[..., 1, 0] * M[..., 2, 2] - M[..., 1, 2] * M[..., 2, 0])
            + M[..., 0, 2] * (M[..., 1, 0] * M[..., 2, 1] - M[..., 1, 1] * M[..., 2, 0]))


def _remove_det_phase(U: torch.Tensor) -> torch.Tensor:
    return U / torch.exp(1j * torch.angle(_det3(U)) / 3)[..., None, None]


def _project_su3(U: torch.Tensor) -> torch.Tensor:
    """Nearest-unitary Newton-Schulz step, then remove the determinant phase."""
    eye = torch.eye(3, dtype=U.dtype, device=U.device)
    U = U @ (3 * eye - U.mH @ U) * 0.5
    return _remove_det_phase(U)


@functools.lru_cache(maxsize=None)
def _eigs_sample() -> np.ndarray:
    xi = torch.randn(_PLAQ_SAMPLE, 8, dtype=torch.float64, generator=_generator(0, "cpu"))
    return torch.linalg.eigvalsh(_algebra(xi)).numpy()


def link_mean_trace(scale: float) -> float:
    """c(s) = E[Re tr exp(i s H)]/3 estimated on the fixed sample."""
    w = _eigs_sample()
    return float(np.cos(scale * w).sum(axis=1).mean() / 3.0)


@functools.lru_cache(maxsize=None)
def link_scale_for_plaquette(plaquette: float) -> float:
    """Scale s with c(s)^4 = plaquette (bisection, c decreasing on [0, 2.5])."""
    if not 0.0 < plaquette <= 1.0:
        raise ValueError("plaquette must be in (0, 1]")
    target = plaquette ** 0.25
    lo, hi = 0.0, 2.5
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if link_mean_trace(mid) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def random_links(shape, scale: float, seed: int, device="cpu") -> torch.Tensor:
    """exp(i s sum_a xi_a lambda_a/2) for every entry of shape (i.i.d.)."""
    gen = _generator(seed, device)
    xi = torch.randn(*shape, 8, dtype=torch.float64, generator=gen, device=device)
    V = torch.linalg.matrix_exp(1j * scale * _algebra(xi))
    return _project_su3(V)


def haar_su3(shape, seed: int, device="cpu") -> torch.Tensor:
    """Haar-distributed SU(3) matrices of the given batch shape."""
    gen = _generator(seed, device)
    re = torch.randn(*shape, 3, 3, dtype=torch.float64, generator=gen, device=device)
    im = torch.randn(*shape, 3, 3, dtype=torch.float64, generator=gen, device=device)
    Z = torch.complex(re, im) / math.sqrt(2.0)
    # Q of the QR factorisation with a positive real diagonal of R (Mezzadri's
    # phase fix) is the Gram-Schmidt orthonormalisation of Z's columns
    # (two projection passes per column keep it orthogonal to rounding).
    cols = []
    for j in range(3):
        v = Z[..., :, j]
        for _ in range(2):
            for q in cols:
                v = v - (q.conj() * v).sum(-1, keepdim=True) * q
        cols.append(v / torch.linalg.vector_norm(v, dim=-1, keepdim=True))
    Q = torch.stack(cols, dim=-1)
    return _remove_det_phase(Q)


# axis of the (Lt, Lz, Ly, Lx) site block that direction mu runs along
_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


def rotate_field(U: torch.Tensor, g: torch.Tensor) -> torch.Tensor:
    """U_mu(x) -> g(x) U_mu(x) g(x+mu)^dagger (input construction only)."""
    out = torch.empty_like(U)
    for mu in range(4):
        g_fwd = torch.roll(g, shifts=-1, dims=_AXIS[mu])
        out[..., mu, :, :] = g @ U[..., mu, :, :] @ g_fwd.mH
    return out


def make_field(dims, plaquette: float = 0.60, field_seed: int = 1, gauge_seed: int = 2,
               pure_gauge: bool = False, device="cpu") -> torch.Tensor:
    """Seeded near-identity field at the target plaquette, Haar-rotated.

    dims = (Lx, Ly, Lz, Lt); returns complex128 (Lt, Lz, Ly, Lx, 4, 3, 3).
    """
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    sites = (Lt, Lz, Ly, Lx)
    if pure_gauge:
        V = torch.eye(3, dtype=torch.complex128, device=device).expand(*sites, 4, 3, 3)
    else:
        V = random_links(sites + (4,), link_scale_for_plaquette(plaquette), field_seed, device)
    g = haar_su3(sites, gauge_seed, device)
    return rotate_field(V.contiguous(), g).contiguous()


def batched_plaquettes(n: int = 64, seed: int = 99, lo: float = 0.55, hi: float = 0.62):
    """Target plaquettes of the uneven-volume batch, uniform in [lo, hi]."""
    return np.random.default_rng(seed).uniform(lo, hi, n).tolist()


def as_numpy(U: torch.Tensor) -> np.ndarray:
    """A C-contiguous complex128 numpy array (host copy when on a device)."""
    return np.ascontiguousarray(U.detach().cpu().numpy())
