"""The overlapped (domain-decomposed) MULT on one GPU: a lattice is cut into
virtual sub-domains (paper Sec. 2.2: the pre-communication step packs the
face data, the interior sites are computed while it travels, the surface
sites after it arrived).  Here the "network" is a device copy from each
sub-domain's send buffers into its neighbours' receive buffers.  The
assembled result is compared bit for bit with the undivided FP32 operator
and elementwise with the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import make_lattice, wc
from oracle import decomposed as dd

pytestmark = pytest.mark.gpu


def run_split(gdims, grid, tbc, kappa, csw, U, psi, dagger, two_streams=False):
    import torch
    w = wc()
    local, offs = dd.subdomains(gdims, grid)
    split = [g > 1 for g in grid]
    main = torch.cuda.current_stream()
    subs, fin, fout, send, recv = [], [], [], [], []
    for o in offs:
        start = [o[m] - int(split[m]) for m in range(4)]
        ext = [local[m] + 2 * int(split[m]) for m in range(4)]
        s = w.SubDomain(local, gdims, o, tbc, stream=main)
        s.load_gauge(dd.restrict_periodic(gdims, U, start, ext)).load_clover(csw, kappa)
        subs.append(s)
        fin.append(s.field(w.F32).load(np.ascontiguousarray(dd.restrict(gdims, psi, o, local))))
        fout.append(s.field(w.F32))
        sb, rb = [None] * 8, [None] * 8
        for mu in range(4):
            nb = s.halo_bytes(mu)
            assert (nb > 0) == split[mu]
            if nb:
                for d in range(2):
                    sb[2 * mu + d] = torch.empty(nb // 4, dtype=torch.float32, device="cuda")
                    rb[2 * mu + d] = torch.full((nb // 4,), float("nan"), dtype=torch.float32, device="cuda")
        send.append(sb)
        recv.append(rb)
    side = torch.cuda.Stream() if two_streams else main
    # pre: pack; in: interior (on a second stream when asked, overlapping the
    # exchange); exchange: device copies; post: surface
    for r, s in enumerate(subs):
        s.halo_pack(fin[r], send[r], dagger)
    if two_streams:
        side.wait_stream(main)
        for r, s in enumerate(subs):
            s.set_stream(side)
            s.apply_interior(fout[r], fin[r], dagger)
            s.set_stream(main)
    else:
        for r, s in enumerate(subs):
            s.apply_interior(fout[r], fin[r], dagger)
    for r in range(len(subs)):
        for mu in range(4):
            if split[mu]:
                recv[r][2 * mu + 1].copy_(send[dd.neighbour(grid, r, mu, +1)][2 * mu])
                recv[r][2 * mu].copy_(send[dd.neighbour(grid, r, mu, -1)][2 * mu + 1])
    main.wait_stream(side)
    for r, s in enumerate(subs):
        s.apply_surface(fout[r], fin[r], recv[r], dagger)
    torch.cuda.synchronize()
    out = np.zeros_like(psi)
    for r, o in enumerate(offs):
        dd.embed(gdims, out, fout[r].store(np.zeros((synth.volume(local), 4, 3), complex)), o, local)
    return out


@pytest.mark.parametrize("gdims,grid", [
    ((8, 8, 8, 8), (1, 1, 1, 2)),
    ((6, 8, 4, 12), (1, 2, 1, 3)),
    ((8, 4, 6, 6), (2, 1, 1, 1)),
    ((4, 6, 4, 6), (2, 2, 2, 2)),
    ((12, 12, 12, 16), (1, 1, 2, 4)),
])
@pytest.mark.parametrize("tbc", [-1, 1])
@pytest.mark.parametrize("dagger", [False, True])
def test_split_equals_unsplit_bitwise_and_oracle(gdims, grid, tbc, dagger):
    kappa, csw = 0.125, 1.0
    U = synth.haar_links(gdims, 31 + sum(gdims))
    psi = synth.z2_source(gdims, 32) if tbc < 0 else synth.gaussian_source(gdims, 33)
    out = run_split(gdims, grid, tbc, kappa, csw, U, psi, dagger, two_streams=(grid[3] > 1 and not dagger))
    lat = make_lattice(gdims, U, csw, kappa, tbc)
    w = wc()
    a, b = lat.field(w.F32).load(psi), lat.field(w.F32)
    (lat.apply_Mdag if dagger else lat.apply_M)(b, a)
    whole = b.store(np.zeros_like(psi))
    assert np.array_equal(out, whole), np.max(np.abs(out - whole))
    op = oracle.Operator(gdims, U, csw, kappa, tbc)
    ref = op.Mdag(psi) if dagger else op.M(psi)
    assert np.max(np.abs(out - ref)) <= 1e-5 * np.max(np.abs(ref))
    assert np.linalg.norm(out - ref) <= 1e-5 * np.linalg.norm(ref)


def test_subdomain_rejects_whole_lattice_calls_and_bad_buffers():
    import torch
    w = wc()
    gdims, local, o = (8, 8, 8, 8), (8, 8, 8, 4), (0, 0, 0, 4)
    U = synth.haar_links(gdims, 1)
    s = w.SubDomain(local, gdims, o, -1)
    s.load_gauge(dd.restrict_periodic(gdims, U, (0, 0, 0, 3), (8, 8, 8, 6))).load_clover(1.0, 0.12)
    a, b = s.field(w.F32), s.field(w.F32)
    with pytest.raises(w.WCError) as e:
        s.apply_M(b, a)
    assert e.value.status == 1 and "sub-domain" in str(e.value)
    h = s.field(w.F16)
    with pytest.raises(w.WCError) as e:
        s.apply_interior(h, a)
    assert e.value.status == 1
    with pytest.raises(w.WCError) as e:
        s.halo_pack(a, [None] * 8)
    assert e.value.status == 1
    nb = s.halo_bytes(3)
    assert nb == 8 * 8 * 8 * 48 and s.halo_bytes(0) == 0
    buf = torch.empty(nb // 4 + 1, dtype=torch.float32, device="cuda")
    bad = [None] * 6 + [buf[1:], buf[:-1]]   # 4-byte offset: misaligned
    with pytest.raises(w.WCError) as e:
        s.halo_pack(a, bad)
    assert e.value.status == 1 and "aligned" in str(e.value)
