"""The decomposed oracle apply on two CPU ranks (gloo, one process per rank,
rendezvous on 127.0.0.1): each rank holds one half of the lattice (cut in
t), sends its face messages to the other rank with explicit point-to-point
messages, applies M (and M^+) to its sites, and the two halves together
equal the undivided oracle operator.  This is the message pattern of the
paper's overlapped multi-node MULT (Sec. 2.2): messages are posted before
the local work and received before the surface sites are finished."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


GDIMS, GRID, TBC, KAPPA, CSW = (4, 4, 6, 8), (1, 1, 1, 2), -1, 0.125, 1.2


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    from oracle import decomposed as dd

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # every rank draws the same seeded global inputs and keeps its own part
    U = synth.haar_links(GDIMS, 21)
    psi = synth.gaussian_source(GDIMS, 22)
    T = oracle.clover_field(GDIMS, CSW, KAPPA, U)
    local, offs = dd.subdomains(GDIMS, GRID)
    split = [g > 1 for g in GRID]
    o = offs[rank]
    Ul, Tl, pl = (dd.restrict(GDIMS, a, o, local) for a in (U, T, psi))
    errs = []
    for dagger in (False, True):
        msgs = dd.face_messages(local, Ul, pl, split, dagger)
        up, dn = dd.neighbour(GRID, rank, 3, +1), dd.neighbour(GRID, rank, 3, -1)
        # post both sends, then receive (gloo isend/irecv; with two ranks the
        # upper and lower neighbour are the same rank, tags tell them apart)
        shape = msgs[(3, "to_lower")].shape
        send_lo = torch.from_numpy(np.ascontiguousarray(msgs[(3, "to_lower")]).view(np.float64))
        send_up = torch.from_numpy(np.ascontiguousarray(msgs[(3, "to_upper")]).view(np.float64))
        recv_from_up, recv_from_dn = torch.empty_like(send_lo), torch.empty_like(send_up)
        reqs = [dist.isend(send_lo, dn, tag=1), dist.isend(send_up, up, tag=2),
                dist.irecv(recv_from_up, up, tag=1), dist.irecv(recv_from_dn, dn, tag=2)]
        for r in reqs:
            r.wait()
        recv = {(3, "from_upper"): recv_from_up.numpy().view(np.complex128).reshape(shape),
                (3, "from_lower"): recv_from_dn.numpy().view(np.complex128).reshape(shape)}
        out = dd.apply_local(local, GDIMS, o, TBC, KAPPA, Ul, Tl, pl, split, recv, dagger)
        ref_full = oracle.apply_Mdag(GDIMS, TBC, KAPPA, U, T, psi) if dagger else \
            oracle.apply_M(GDIMS, TBC, KAPPA, CSW, U, psi, T=T)
        ref = dd.restrict(GDIMS, ref_full, o, local)
        errs.append(float(np.max(np.abs(out - ref)) / np.max(np.abs(ref))))
    q.put((rank, errs))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_undivided_operator():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for _, errs in out:
        assert max(errs) <= 1e-13, errs
