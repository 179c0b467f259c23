"""Even-odd (Schur complement) reference, in plain numpy FP64 (test infrastructure).

The paper's double-precision solver and its single-precision inner solver
both work on the even-odd site preconditioned Wilson-Clover matrix (Sec. 2);
the paper gives no formula, so this follows the textbook definition.  Order
the sites by parity (even: x+y+z+t even).  The hopping term only links sites
of opposite parity, so with A = 1 + T (site-diagonal)

    M = [[A_ee, -k H_eo], [-k H_oe, A_oo]],

and eliminating the odd sites leaves the Schur complement on the even sites

    M^ = A_ee - k^2 H_eo A_oo^-1 H_oe.

A solve of M x = b then reads: b^_e = b_e + k H_eo A_oo^-1 b_o,
M^ x_e = b^_e, x_o = A_oo^-1 (b_o + k H_oe x_e).  Fields here are full-volume
psi[V,4,3] arrays whose entries off the relevant parity are zero.  The
hopping term and the clover field come from the C oracle; A_oo^-1 is a
library solve of each site's 12x12 block.
"""
from __future__ import annotations

import numpy as np

from . import apply_hop, gamma, volume


def parity(dims) -> np.ndarray:
    """(x+y+z+t) mod 2 for every site, site = x + Lx(y + Ly(z + Lz t))."""
    lx, ly, lz, lt = (int(d) for d in dims)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return ((x + y + z + t) % 2).reshape(-1)


def _restrict(psi, mask):
    out = np.zeros_like(psi)
    out[mask] = psi[mask]
    return out


def _site_mul(A, psi, mask):
    """A psi on the sites in mask (A[V,12,12], psi[V,4,3]), zero elsewhere."""
    out = np.zeros_like(psi)
    out[mask] = np.einsum("sij,sj->si", A[mask], psi[mask].reshape(-1, 12)).reshape(-1, 4, 3)
    return out


def _site_solve(A, psi, mask):
    """A^-1 psi on the sites in mask, zero elsewhere."""
    out = np.zeros_like(psi)
    out[mask] = np.linalg.solve(A[mask], psi[mask].reshape(-1, 12, 1)).reshape(-1, 4, 3)
    return out


def _gamma5(psi):
    return np.einsum("ab,sbc->sac", gamma(4), psi)


class EvenOdd:
    """Schur complement of M = (1 + T) - k H on the even sites."""

    def __init__(self, dims, tbc: int, kappa: float, U, T):
        self.dims = tuple(int(d) for d in dims)
        self.tbc, self.kappa = int(tbc), float(kappa)
        self.U = np.ascontiguousarray(U, dtype=np.complex128)
        self.A = np.eye(12, dtype=np.complex128)[None] + np.asarray(T, dtype=np.complex128)
        par = parity(self.dims)
        self.even, self.odd = par == 0, par == 1
        assert len(par) == volume(self.dims)

    def hop(self, psi, to_mask):
        return _restrict(apply_hop(self.dims, self.tbc, self.U, psi), to_mask)

    def schur(self, psi, dagger: bool = False):
        """M^ psi_e (or M^+ psi_e = gamma5 M^ gamma5 psi_e: A commutes with
        gamma5 and gamma5 H gamma5 = H^+); zero on the odd sites."""
        if dagger:
            return _gamma5(self.schur(_gamma5(psi)))
        pe = _restrict(psi, self.even)
        t = _site_solve(self.A, self.hop(pe, self.odd), self.odd)
        return _site_mul(self.A, pe, self.even) - self.kappa ** 2 * self.hop(t, self.even)

    def prepare(self, b):
        """b^_e = b_e + k H_eo A_oo^-1 b_o."""
        t = _site_solve(self.A, b, self.odd)
        return _restrict(b, self.even) + self.kappa * self.hop(t, self.even)

    def reconstruct(self, x_e, b):
        """Full solution from x_e: x_o = A_oo^-1 (b_o + k H_oe x_e)."""
        xe = _restrict(x_e, self.even)
        xo = _site_solve(self.A, _restrict(b, self.odd) + self.kappa * self.hop(xe, self.odd), self.odd)
        return xe + xo
