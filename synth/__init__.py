"""Seeded synthetic inputs for the Wilson-Clover operator and its solvers.

This module only draws random numbers and shapes them into gauge links,
gauge transformations, su(3) directions and source spinors.  It holds none of
the operator's arithmetic (no hopping term, clover term, projector or solver):
the CPU oracle and the CUDA library both receive what it produces as inputs.

Canonical layouts (numpy complex128, C order):
  * gauge field  U[V, 4, 3, 3]   site-major, mu = x,y,z,t, then row, column
  * spinor       psi[V, 4, 3]    site-major, then spin, colour
with site = x + Lx*(y + Ly*(z + Lz*t)).

The paper benchmarks on synthetic lattices (Sec. 3): no gauge ensemble is
read anywhere.  Recipes:
  * exp links:  U = exp(i*eps*H), H = sum_a w_a lambda_a / 2, w ~ N(0,1),
    lambda the Gell-Mann matrices; computed as V diag(exp(i eps h)) V^+.
  * Haar-like:  complex Gaussian 3x3 -> QR -> fix column phases by
    diag(R)/|diag(R)| -> multiply row 3 by conj(det) to land in SU(3).
  * sources:    point (site 0, given spin/colour), real Z2 (+-1 per complex
    component), complex Gaussian (N(0,1) real and imaginary parts).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "volume", "gell_mann", "exp_links", "haar_links", "pool_links", "unit_links",
    "random_su3", "random_su3_algebra", "point_source", "z2_source",
    "gaussian_source", "config_inputs", "CONFIGS",
]


def volume(dims) -> int:
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1], lam[1, 1, 0] = -1j, 1j
    lam[2, 0, 0], lam[2, 1, 1] = 1, -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2], lam[4, 2, 0] = -1j, 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2], lam[6, 2, 1] = -1j, 1j
    lam[7, 0, 0] = lam[7, 1, 1] = 1 / np.sqrt(3)
    lam[7, 2, 2] = -2 / np.sqrt(3)
    return lam


def _hermitian_from_normals(w: np.ndarray) -> np.ndarray:
    """sum_a w[..., a] * lambda_a / 2 for w of shape (..., 8)."""
    return np.einsum("...a,aij->...ij", w, gell_mann() / 2)


def exp_links(dims, eps: float, seed: int) -> np.ndarray:
    """SU(3) links U = exp(i*eps*H) with Gaussian traceless Hermitian H."""
    n = volume(dims) * 4
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n, 8))
    h = _hermitian_from_normals(w)
    evals, evecs = np.linalg.eigh(h)
    phase = np.exp(1j * eps * evals)
    u = np.einsum("nij,nj,nkj->nik", evecs, phase, evecs.conj())
    return np.ascontiguousarray(u.reshape(volume(dims), 4, 3, 3))


def random_su3(n: int, rng: np.random.Generator) -> np.ndarray:
    """n Haar-distributed SU(3) matrices via QR of complex Gaussians."""
    z = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q[:, 2, :] *= np.conj(det)[:, None]
    return q


def haar_links(dims, seed: int) -> np.ndarray:
    """Haar-like SU(3) links (reunitarised Gaussian matrices)."""
    rng = np.random.default_rng(seed)
    u = random_su3(volume(dims) * 4, rng)
    return np.ascontiguousarray(u.reshape(volume(dims), 4, 3, 3))


def pool_links(dims, seed: int, pool: int = 4096) -> np.ndarray:
    """Haar-like SU(3) links drawn (seeded) from a pool of `pool` random
    matrices: every link is a valid SU(3) matrix and neighbouring links
    differ, at a generation cost independent of the volume's 3x3 algebra
    (for very large lattices)."""
    rng = np.random.default_rng(seed)
    base = random_su3(pool, rng)
    idx = rng.integers(0, pool, size=volume(dims) * 4)
    return np.ascontiguousarray(base[idx].reshape(volume(dims), 4, 3, 3))


def unit_links(dims) -> np.ndarray:
    u = np.zeros((volume(dims), 4, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1
    return u


def random_su3_algebra(shape, rng: np.random.Generator) -> np.ndarray:
    """Random traceless anti-Hermitian 3x3 matrices i*sum_a w_a lambda_a/2."""
    w = rng.standard_normal(tuple(shape) + (8,))
    return 1j * _hermitian_from_normals(w)


def point_source(dims, spin: int = 0, colour: int = 0, site: int = 0) -> np.ndarray:
    psi = np.zeros((volume(dims), 4, 3), dtype=np.complex128)
    psi[site, spin, colour] = 1.0
    return psi


def z2_source(dims, seed: int) -> np.ndarray:
    """Real Z2 noise: every complex component is +1 or -1 with probability 1/2."""
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2, size=(volume(dims), 4, 3))
    return (2.0 * bits - 1.0).astype(np.complex128)


def gaussian_source(dims, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = volume(dims)
    return rng.standard_normal((v, 4, 3)) + 1j * rng.standard_normal((v, 4, 3))


# The five benchmark workloads: lattice, gauge recipe, csw, kappa, time boundary
# condition and source.  Seeds: gauge 1000+n, source 2000+n; batched instance i
# draws its gauge field from seed 1100+10*i.
CONFIGS = {
    1: dict(dims=(8, 8, 8, 8), gauge=("exp", 0.3), csw=1.0, kappa=0.12, tbc=-1,
            source="point"),
    2: dict(dims=(24, 24, 24, 32), gauge=("haar",), csw=1.0, kappa=0.125, tbc=-1,
            source="z2"),
    3: dict(dims=(32, 32, 32, 64), gauge=("exp", 0.25), csw=1.6, kappa=0.128, tbc=-1,
            source="gaussian"),
    4: dict(dims=[(24, 24, 24, 48), (16, 16, 16, 32), (32, 32, 32, 32)],
            gauge=("exp", 0.3), csw=1.0, kappa=0.124, tbc=-1, source="point12"),
    5: dict(dims=(16, 16, 16, 32), gauge=("exp", 0.3), csw=1.0, kappa=0.12, tbc=-1,
            source="gaussian"),
}


def gauge_for(recipe, dims, seed: int) -> np.ndarray:
    if recipe[0] == "exp":
        return exp_links(dims, recipe[1], seed)
    if recipe[0] == "haar":
        return haar_links(dims, seed)
    if recipe[0] == "unit":
        return unit_links(dims)
    raise ValueError(f"unknown gauge recipe {recipe!r}")


def source_for(kind: str, dims, seed: int) -> np.ndarray:
    if kind == "point":
        return point_source(dims)
    if kind == "z2":
        return z2_source(dims, seed)
    if kind == "gaussian":
        return gaussian_source(dims, seed)
    raise ValueError(f"unknown source kind {kind!r}")


def config_inputs(n: int, dims=None):
    """(dims, U, source, csw, kappa, tbc) for workload n, optionally at other dims."""
    c = CONFIGS[n]
    d = tuple(dims) if dims is not None else tuple(c["dims"])
    u = gauge_for(c["gauge"], d, 1000 + n)
    src = source_for(c["source"], d, 2000 + n)
    return d, u, src, c["csw"], c["kappa"], c["tbc"]
