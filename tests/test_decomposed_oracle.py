"""The domain-decomposed oracle apply (face messages + local apply, the
paper's overlapped multi-node MULT, Sec. 2.2) against the undivided oracle
operator: every sub-domain's sites, computed from local data and the
messages of its neighbours, equal M psi (and M^+ psi) of the whole lattice.
CPU only; all sub-domains run in this process (the gloo test runs them as
separate ranks)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import decomposed as dd


def split_apply(gdims, grid, tbc, kappa, U, T, psi, dagger):
    local, offs = dd.subdomains(gdims, grid)
    split = [g > 1 for g in grid]
    Us = [dd.restrict(gdims, U, o, local) for o in offs]
    Ts = [dd.restrict(gdims, T, o, local) for o in offs]
    ps = [dd.restrict(gdims, psi, o, local) for o in offs]
    msgs = [dd.face_messages(local, Us[r], ps[r], split, dagger) for r in range(len(offs))]
    recv = dd.exchange(grid, msgs, split)
    out = np.zeros_like(psi)
    for r, o in enumerate(offs):
        part = dd.apply_local(local, gdims, o, tbc, kappa, Us[r], Ts[r], ps[r], split, recv[r], dagger)
        dd.embed(gdims, out, part, o, local)
    return out


@pytest.mark.parametrize("gdims,grid", [
    ((4, 4, 4, 8), (1, 1, 1, 2)),
    ((4, 6, 4, 4), (1, 2, 1, 1)),
    ((4, 4, 6, 8), (1, 1, 2, 2)),
    ((4, 4, 4, 6), (2, 2, 2, 2)),
    ((6, 4, 4, 9), (1, 1, 1, 3)),
])
@pytest.mark.parametrize("tbc", [-1, 1])
@pytest.mark.parametrize("dagger", [False, True])
def test_decomposed_apply_equals_whole_lattice(gdims, grid, tbc, dagger):
    kappa, csw = 0.124, 1.3
    U = synth.haar_links(gdims, 11 + sum(gdims))
    psi = synth.gaussian_source(gdims, 12)
    op = oracle.Operator(gdims, U, csw, kappa, tbc)
    ref = op.Mdag(psi) if dagger else op.M(psi)
    out = split_apply(gdims, grid, tbc, kappa, U, op.T, psi, dagger)
    assert np.max(np.abs(out - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_decomposed_apply_needs_the_messages():
    """Dropping one direction's messages changes exactly the sites on that
    cut face (the messages carry the hops across it and nothing else)."""
    gdims, grid, tbc, kappa = (4, 4, 4, 8), (1, 1, 1, 2), -1, 0.12
    U = synth.haar_links(gdims, 3)
    psi = synth.gaussian_source(gdims, 4)
    T = oracle.clover_field(gdims, 1.0, kappa, U)
    local, offs = dd.subdomains(gdims, grid)
    split = [g > 1 for g in grid]
    Us = [dd.restrict(gdims, U, o, local) for o in offs]
    ps = [dd.restrict(gdims, psi, o, local) for o in offs]
    msgs = [dd.face_messages(local, Us[r], ps[r], split) for r in range(2)]
    recv = dd.exchange(grid, msgs, split)
    good = dd.apply_local(local, gdims, offs[0], tbc, kappa, Us[0], dd.restrict(gdims, T, offs[0], local), ps[0],
                          split, recv[0])
    bad_recv = dict(recv[0])
    bad_recv[(3, "from_upper")] = np.zeros_like(bad_recv[(3, "from_upper")])
    bad = dd.apply_local(local, gdims, offs[0], tbc, kappa, Us[0], dd.restrict(gdims, T, offs[0], local), ps[0],
                         split, bad_recv)
    diff = np.abs(bad - good).reshape(local[3], -1).max(axis=1)
    assert diff[-1] > 0 and np.all(diff[:-1] == 0)


def test_restrict_periodic_is_the_halo_box():
    gdims = (4, 4, 4, 6)
    a = np.arange(synth.volume(gdims), dtype=float)
    box = dd.restrict_periodic(gdims, a, (0, 0, 0, -1), (4, 4, 4, 5))
    g = a.reshape(6, 4, 4, 4)
    assert np.array_equal(box.reshape(5, 4, 4, 4), g[[5, 0, 1, 2, 3]])
