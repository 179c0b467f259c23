"""Overlapped RAS on block Schur complements, in plain numpy FP64 (test
infrastructure: only the tests may import it).

The paper's single-precision inner solver is preconditioned by even-odd site
ordering and by overlapped Restricted Additive Schwarz (Sec. 2).  The paper
gives no formula for how the two combine; this module reads it as RAS
applied to the even-odd system itself.  For an extended block B (core
block[mu] sites tiled from the origin, grown by delta sites on every face,
periodically) let M_B be M restricted to the sites of B with every hop that
leaves B dropped.  Its Schur complement on the even sites of B,

    M^_B = A_ee - kappa^2 H^B_eo A_oo^-1 H^B_oe,

(H^B the hopping term with both ends in B, A = 1 + T site-diagonal) is the
block operator; the preconditioner is

    z_e = sum_B Rtilde_B^T MR_k(M^_B, R_B v_e),

R_B the restriction of an even-site vector to the even sites of B, MR_k k
minimal-residual steps from zero (q = M^_B r, alpha = <q, r> / <q, q>,
x += alpha r, r -= alpha q; alpha = 0 when q = 0), Rtilde_B^T the write-back
of the even sites of B's core.  Parity is the global one: (x+y+z+t) mod 2.
M^+ uses the projectors of M^+ = gamma5 M gamma5.  Fields are full-volume
arrays psi[V,4,3]; the odd sites of the result are zero.
"""
from __future__ import annotations

import numpy as np

from . import gamma


def block_geometry(dims, block, delta: int, bc):
    """Sites of the extended block with block coordinates bc: global site,
    global coordinates and local coordinates of every local site (x
    fastest), and the local extents.  Checks the same fit rule as the full
    RAS: L % b == 0 and L > b + 2 delta."""
    L = [int(d) for d in dims]
    b = [int(x) for x in block]
    for mu in range(4):
        if b[mu] <= 0 or L[mu] % b[mu] != 0 or L[mu] <= b[mu] + 2 * delta or delta < 0:
            raise ValueError(f"RAS block {tuple(block)} / overlap {delta} does not fit {tuple(dims)}")
    e = [b[mu] + 2 * delta for mu in range(4)]
    lt, lz, ly, lx = np.meshgrid(*(np.arange(e[m]) for m in (3, 2, 1, 0)), indexing="ij")
    lc = np.stack([lx.reshape(-1), ly.reshape(-1), lz.reshape(-1), lt.reshape(-1)], axis=1)
    gc = (lc + np.array([bc[m] * b[m] - delta for m in range(4)])) % np.array(L)
    gsite = gc[:, 0] + L[0] * (gc[:, 1] + L[1] * (gc[:, 2] + L[2] * gc[:, 3]))
    return gsite, gc, lc, e


def _proj(mu: int, s: int, psi):
    return psi + s * np.einsum("ab,sbc->sac", gamma(mu), psi)


def block_hop(dims, tbc: int, U, gsite, gc, lc, e, psi, dagger: bool = False):
    """H^B psi on the local sites of a block (psi[ne,4,3] local): forward and
    backward hops whose target lies inside the extended block, the time
    boundary factor on hops across the global t boundary."""
    sf, sb = (1, -1) if dagger else (-1, 1)
    L = [int(d) for d in dims]
    es = [1, e[0], e[0] * e[1], e[0] * e[1] * e[2]]
    out = np.zeros_like(psi)
    idx = np.arange(len(gsite))
    for mu in range(4):
        fw = lc[:, mu] + 1 < e[mu]
        src = idx[fw] + es[mu]
        term = np.einsum("sab,sqb->sqa", U[gsite[fw], mu], _proj(mu, sf, psi[src]))
        if mu == 3:
            term[gc[fw, 3] == L[3] - 1] *= tbc
        out[fw] += term
        bw = lc[:, mu] >= 1
        src = idx[bw] - es[mu]
        term = np.einsum("sba,sqb->sqa", U[gsite[src], mu].conj(), _proj(mu, sb, psi[src]))
        if mu == 3:
            term[gc[bw, 3] == 0] *= tbc
        out[bw] += term
    return out


def block_schur_apply(dims, tbc: int, kappa: float, U, A, gsite, gc, lc, e, psi, dagger: bool = False):
    """M^_B psi for psi on the local sites of a block (entries on the odd
    sites are ignored; the result is zero there)."""
    par = gc.sum(axis=1) % 2
    ev, od = par == 0, par == 1
    pe = np.where(ev[:, None, None], psi, 0.0)
    h = block_hop(dims, tbc, U, gsite, gc, lc, e, pe, dagger)
    t = np.zeros_like(psi)
    t[od] = np.linalg.solve(A[gsite[od]], h[od].reshape(-1, 12, 1)).reshape(-1, 4, 3)
    h2 = block_hop(dims, tbc, U, gsite, gc, lc, e, t, dagger)
    out = np.zeros_like(psi)
    out[ev] = (np.einsum("sij,sj->si", A[gsite[ev]], pe[ev].reshape(-1, 12)).reshape(-1, 4, 3)
               - kappa ** 2 * h2[ev])
    return out


def ras_schur(dims, tbc: int, kappa: float, U, T, block, delta: int, k: int, v, dagger: bool = False,
              blocks=None):
    """z_e = sum_B Rtilde_B^T MR_k(M^_B, R_B v_e); zero on the odd sites.
    blocks: optional list of block coordinates (bx, by, bz, bt) to compute
    (the cores of the others stay zero)."""
    U = np.asarray(U, dtype=np.complex128)
    A = np.eye(12, dtype=np.complex128)[None] + np.asarray(T, dtype=np.complex128)
    v = np.asarray(v, dtype=np.complex128)
    L = [int(d) for d in dims]
    nb = [L[m] // int(block[m]) for m in range(4)]
    z = np.zeros_like(v)
    if blocks is None:
        blocks = [(bx, by, bz, bt) for bt in range(nb[3]) for bz in range(nb[2]) for by in range(nb[1])
                  for bx in range(nb[0])]
    for bc in blocks:
        gsite, gc, lc, e = block_geometry(dims, block, delta, bc)
        ev = gc.sum(axis=1) % 2 == 0
        r = np.where(ev[:, None, None], v[gsite], 0.0)
        x = np.zeros_like(r)
        for _ in range(k):
            q = block_schur_apply(dims, tbc, kappa, U, A, gsite, gc, lc, e, r, dagger)
            qq = np.vdot(q, q).real
            alpha = np.vdot(q, r) / qq if qq > 0 else 0.0
            x += alpha * r
            r -= alpha * q
        core = np.all((lc >= delta) & (lc < delta + np.array([int(c) for c in block])), axis=1)
        w = core & ev
        z[gsite[w]] = x[w]
    return z
