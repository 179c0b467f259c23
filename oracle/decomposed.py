"""Domain-decomposed Wilson-Clover apply with explicit face messages, in plain
numpy FP64 (test infrastructure: only the tests may import it).

The paper overlaps the halo exchange of its multi-node hopping
multiplication with computation (Sec. 2.2, communication-computation
overlapping): the lattice is cut into sub-domains, each process first
prepares the face data its neighbours need, computes the sites whose
neighbours are all local while the messages travel, and finishes the
surface sites once they arrive.  The paper prints no formula for the
messages; this is the textbook form of M = (1 + T) - kappa H with

    (H psi)(x) = sum_mu (1 + s_f gamma_mu) U_mu(x) psi(x + mu)
                      + (1 + s_b gamma_mu) U_mu(x - mu)^+ psi(x - mu),

s_f = -1, s_b = +1 for M and s_f = +1, s_b = -1 for M^+ = gamma5 M gamma5
(the clover term is Hermitian), the time-boundary factor t_bc on every hop
that crosses the global time boundary.  Across a cut face in direction mu a
sub-domain receives

    from the upper neighbour: (1 + s_f gamma_mu) psi(y) at the neighbour's
        lower-face sites y (the forward neighbours of this domain's upper
        face), to be multiplied by this domain's own link U_mu(x);
    from the lower neighbour: U_mu(y)^+ (1 + s_b gamma_mu) psi(y) at the
        neighbour's upper-face sites y (the backward neighbours of this
        domain's lower face), whose link lives with the sender.

Messages are full 4-spinors per face site (no two-spinor compression: that
is a detail of the GPU kernels), in the face's own site order.  Arrays are
shaped [Lt, Lz, Ly, Lx, ...] with local extents; mu = 0..3 is x, y, z, t,
i.e. array axis 3 - mu.
"""
from __future__ import annotations

import numpy as np

from . import gamma


def _axis(mu: int) -> int:
    return 3 - mu


def _grid(a, dims):
    """[V, ...] (site = x + Lx(y + Ly(z + Lz t))) -> [Lt, Lz, Ly, Lx, ...]."""
    lx, ly, lz, lt = (int(d) for d in dims)
    return a.reshape((lt, lz, ly, lx) + a.shape[1:])


def _proj(mu: int, s: int, psi):
    """(1 + s gamma_mu) psi on every site of psi[..., 4, 3]."""
    return psi + s * np.einsum("ab,...bc->...ac", gamma(mu), psi)


def _link_mul(U, psi, adjoint: bool):
    """U psi or U^+ psi per site, U[..., 3, 3], psi[..., 4, 3]."""
    if adjoint:
        return np.einsum("...ba,...sb->...sa", U.conj(), psi)
    return np.einsum("...ab,...sb->...sa", U, psi)


def _face(a, mu: int, upper: bool):
    ax = _axis(mu)
    idx = [slice(None)] * a.ndim
    idx[ax] = -1 if upper else 0
    return a[tuple(idx)]


def face_messages(local_dims, U, psi, split, dagger: bool = False):
    """The messages this sub-domain sends: out[(mu, 'to_lower')] =
    (1 + s_f gamma_mu) psi on the lower face, out[(mu, 'to_upper')] =
    U_mu^+ (1 + s_b gamma_mu) psi on the upper face, for every cut
    direction mu (split[mu] true).  U[V,4,3,3], psi[V,4,3] local."""
    sf, sb = (1, -1) if dagger else (-1, 1)
    Ug, pg = _grid(np.asarray(U), local_dims), _grid(np.asarray(psi), local_dims)
    out = {}
    for mu in range(4):
        if not split[mu]:
            continue
        out[(mu, "to_lower")] = _proj(mu, sf, _face(pg, mu, upper=False))
        up = _face(pg, mu, upper=True)
        out[(mu, "to_upper")] = _link_mul(_face(Ug, mu, upper=True)[..., mu, :, :], _proj(mu, sb, up), True)
    return out


def apply_local(local_dims, global_dims, offset, tbc: int, kappa: float, U, T, psi, split, recv,
                dagger: bool = False):
    """M psi (or M^+ psi) on the sites of one sub-domain.  Hops inside the
    domain use the local psi (periodically within the domain along uncut
    directions, whose local extent is the global one); hops across a cut face
    use recv[(mu, 'from_upper')] (the upper neighbour's 'to_lower') and
    recv[(mu, 'from_lower')] (the lower neighbour's 'to_upper').  T[V,12,12]
    is the clover term of the local sites, offset the global coordinate of
    local site 0."""
    sf, sb = (1, -1) if dagger else (-1, 1)
    lx, ly, lz, lt = (int(d) for d in local_dims)
    V = lx * ly * lz * lt
    Ug, pg = _grid(np.asarray(U), local_dims), _grid(np.asarray(psi), local_dims)
    hop = np.zeros_like(pg)
    tglob = offset[3] + np.arange(lt)   # global t of each local slice
    for mu in range(4):
        ax = _axis(mu)
        Lmu = int(local_dims[mu])
        # forward: psi(x + mu), the last slice from the upper neighbour when cut
        fwd = np.roll(pg, -1, axis=ax)
        if split[mu]:
            idx = [slice(None)] * pg.ndim
            idx[ax] = Lmu - 1
            fwd[tuple(idx)] = 0.0
        term = _link_mul(Ug[..., mu, :, :], _proj(mu, sf, fwd), False)
        if split[mu]:
            idx = [slice(None)] * pg.ndim
            idx[ax] = Lmu - 1
            term[tuple(idx)] = _link_mul(_face(Ug, mu, upper=True)[..., mu, :, :], recv[(mu, "from_upper")], False)
        if mu == 3:
            cross = (tglob == int(global_dims[3]) - 1)   # forward hop leaves the global time range
            term[cross] *= tbc
        hop += term
        # backward: U_mu(x - mu)^+ psi(x - mu), the first slice from the lower neighbour when cut
        bwd = np.roll(pg, 1, axis=ax)
        Ub = np.roll(Ug[..., mu, :, :], 1, axis=ax)
        term = _link_mul(Ub, _proj(mu, sb, bwd), True)
        if split[mu]:
            idx = [slice(None)] * pg.ndim
            idx[ax] = 0
            term[tuple(idx)] = recv[(mu, "from_lower")]
        if mu == 3:
            cross = (tglob == 0)
            term[cross] *= tbc
        hop += term
    Tpsi = np.einsum("sij,sj->si", np.asarray(T), np.asarray(psi).reshape(V, 12)).reshape(V, 4, 3)
    return np.asarray(psi) + Tpsi - kappa * hop.reshape(V, 4, 3)


def subdomains(global_dims, grid):
    """Offsets and local extents of a Cartesian cut of the lattice into
    grid[mu] equal parts per direction, in rank order (x fastest)."""
    local = tuple(int(g) // int(n) for g, n in zip(global_dims, grid))
    out = []
    for t in range(grid[3]):
        for z in range(grid[2]):
            for y in range(grid[1]):
                for x in range(grid[0]):
                    c = (x, y, z, t)
                    out.append(tuple(c[m] * local[m] for m in range(4)))
    return local, out


def restrict(global_dims, a, offset, local_dims):
    """The sub-box [offset, offset + local_dims) of a [V, ...] field."""
    g = _grid(np.asarray(a), global_dims)
    sl = tuple(slice(offset[m], offset[m] + local_dims[m]) for m in (3, 2, 1, 0))
    sub = g[sl]
    return sub.reshape((-1,) + np.asarray(a).shape[1:])


def neighbour(grid, rank: int, mu: int, step: int) -> int:
    """Rank of the sub-domain one step along mu (periodic in the grid)."""
    c, r = [], rank
    for m in range(4):
        c.append(r % grid[m])
        r //= grid[m]
    c[mu] = (c[mu] + step) % grid[mu]
    return c[0] + grid[0] * (c[1] + grid[1] * (c[2] + grid[2] * c[3]))


def restrict_periodic(global_dims, a, start, extents):
    """The box [start, start + extents) of a [V, ...] field, coordinates taken
    periodically (start may be negative): e.g. a sub-domain's gauge field
    with its one-site halo across the cut faces."""
    g = _grid(np.asarray(a), global_dims)
    for m in range(4):
        idx = (np.arange(int(start[m]), int(start[m]) + int(extents[m])) % int(global_dims[m]))
        g = np.take(g, idx, axis=_axis(m))
    return np.ascontiguousarray(g).reshape((-1,) + np.asarray(a).shape[1:])


def embed(global_dims, full, sub, offset, local_dims):
    """Write the sub-domain field sub[V_local, ...] into full[V, ...] at
    [offset, offset + local_dims)."""
    g = _grid(full, global_dims)
    sl = tuple(slice(offset[m], offset[m] + local_dims[m]) for m in (3, 2, 1, 0))
    g[sl] = _grid(np.asarray(sub), local_dims)
    return full


def exchange(grid, msgs, split):
    """The messages each rank receives, from the list of every rank's sent
    messages (face_messages), for an in-process run of all sub-domains."""
    recv = []
    for r in range(len(msgs)):
        d = {}
        for mu in range(4):
            if split[mu]:
                d[(mu, "from_upper")] = msgs[neighbour(grid, r, mu, +1)][(mu, "to_lower")]
                d[(mu, "from_lower")] = msgs[neighbour(grid, r, mu, -1)][(mu, "to_upper")]
        recv.append(d)
    return recv
