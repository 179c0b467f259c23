"""GPU parity of the Wilson-Clover operator against the CPU oracle.

M, M^+ and H through the C ABI in FP64, FP32 and FP16 storage, compared
element by element with the oracle on the same seeded inputs.  Tolerances:
FP64 1e-12 (rounding order only), FP32 1e-5 and FP16 storage 5e-3 relative
(the accuracy bars of the FP32 and FP16 applies).  Lattices cover several
thread blocks with a ragged tail, odd extents, the 2^4 degenerate lattice
(forward and backward neighbour coincide) and both time boundary conditions;
the full 24^3x32 and 32^3x64 workloads are checked on sampled sites.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import assert_elementwise, gpu_apply, make_lattice, rel_err, wc

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 5e-3}
CASES = [((4, 4, 4, 4), -1), ((6, 4, 8, 10), -1), ((3, 5, 4, 7), 1), ((2, 2, 2, 2), -1),
         ((5, 3, 2, 6), -1)]


@pytest.mark.parametrize("dims,tbc", CASES)
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_apply_M_matches_oracle(dims, tbc, prec):
    kappa, csw = 0.124, 1.3
    U = synth.exp_links(dims, 0.4, 100 + sum(dims))
    psi = synth.gaussian_source(dims, 200 + sum(dims))
    lat = make_lattice(dims, U, csw, kappa, tbc)
    ref = oracle.apply_M(dims, tbc, kappa, csw, U, psi)
    assert_elementwise(gpu_apply(lat, psi, prec, "M"), ref, TOL[prec])


@pytest.mark.parametrize("dims,tbc", CASES[:3])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_apply_Mdag_matches_oracle(dims, tbc, prec):
    kappa, csw = 0.13, 1.0
    U = synth.haar_links(dims, 300 + sum(dims))
    psi = synth.gaussian_source(dims, 400 + sum(dims))
    lat = make_lattice(dims, U, csw, kappa, tbc)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    assert_elementwise(gpu_apply(lat, psi, prec, "Mdag"), op.Mdag(psi), TOL[prec])


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_apply_hop_matches_oracle(prec):
    dims, tbc = (6, 4, 8, 10), -1
    U = synth.exp_links(dims, 0.3, 5)
    psi = synth.z2_source(dims, 6)
    lat = make_lattice(dims, U, 1.0, 0.12, tbc)
    ref = oracle.apply_hop(dims, tbc, U, psi)
    assert_elementwise(gpu_apply(lat, psi, prec, "hop"), ref, TOL[prec])


def test_free_field_plane_wave_on_gpu():
    """Unit links: M e^{ipx} u = e^{ipx} M~(p) u (antiperiodic p_t), FP64."""
    dims, kappa, tbc = (4, 6, 4, 8), 0.13, -1
    U = synth.unit_links(dims)
    V = synth.volume(dims)
    s = np.arange(V)
    c = np.stack([s % 4, (s // 4) % 6, (s // 24) % 4, s // 96], axis=1)
    p = np.array([2 * np.pi / 4, 4 * np.pi / 6, 0.0, 3 * np.pi / 8])
    u = np.random.default_rng(1).standard_normal((4, 3)) + 0j
    psi = np.exp(1j * (c @ p))[:, None, None] * u[None]
    lat = make_lattice(dims, U, 2.0, kappa, tbc)
    g = [oracle.gamma(m) for m in range(4)]
    Mp = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + sum(2j * kappa * np.sin(p[m]) * g[m] for m in range(4))
    expect = np.exp(1j * (c @ p))[:, None, None] * (Mp @ u)[None]
    assert np.allclose(gpu_apply(lat, psi, 0, "M"), expect, atol=1e-13)


def test_import_export_round_trip_and_fp16_scale():
    dims = (4, 4, 4, 6)
    lat = make_lattice(dims, synth.unit_links(dims), 1.0, 0.1, -1)
    psi = synth.gaussian_source(dims, 3) * np.logspace(-20, 3, synth.volume(dims))[:, None, None]
    out = lat.field(0).load(psi).store(np.zeros_like(psi))
    assert np.array_equal(out, psi)
    out32 = lat.field(1).load(psi).store(np.zeros_like(psi))
    assert np.array_equal(out32, psi.real.astype(np.float32) + 1j * psi.imag.astype(np.float32))
    # FP16 with a per-site scale keeps every site to ~2^-11 of its own maximum
    out16 = lat.field(2).load(psi).store(np.zeros_like(psi))
    site_max = np.max(np.abs(np.stack([psi.real, psi.imag])), axis=(0, 2, 3))
    err = np.max(np.abs(np.stack([(out16 - psi).real, (out16 - psi).imag])), axis=(0, 2, 3))
    assert np.all(err <= 2.0 ** -11 * site_max * 1.0001)


def test_import_export_memory_kinds():
    """Pageable (numpy), page-locked (pinned torch) and device (CUDA torch)
    buffers give identical imports and exports."""
    import torch
    dims = (6, 4, 4, 6)
    lat = make_lattice(dims, synth.unit_links(dims), 1.0, 0.1, -1)
    psi = synth.gaussian_source(dims, 4)
    for prec in (0, 1, 2):
        ref = lat.field(prec).load(psi).store(np.zeros_like(psi))
        pinned = torch.from_numpy(psi).pin_memory()
        out_pinned = torch.zeros_like(pinned).pin_memory()
        lat.field(prec).load(pinned).store(out_pinned)
        assert np.array_equal(out_pinned.numpy(), ref)
        dev = torch.from_numpy(psi).cuda()
        out_dev = torch.zeros_like(dev)
        lat.field(prec).load(dev).store(out_dev)
        torch.cuda.synchronize()
        assert np.array_equal(out_dev.cpu().numpy(), ref)


def test_import_export_complex64():
    """complex64 import/export (wc_field_import_f32 / _export_f32): exact
    for FP32 fields, widening into FP64 and rounding out of it, the same
    FP16 rounding as from complex128, on host and device buffers."""
    import torch
    dims = (4, 6, 4, 6)
    lat = make_lattice(dims, synth.unit_links(dims), 1.0, 0.1, -1)
    psi = synth.gaussian_source(dims, 5) * np.logspace(-8, 3, synth.volume(dims))[:, None, None]
    p32 = psi.astype(np.complex64)
    # FP32 field: bit-exact round trip of complex64 data
    assert np.array_equal(lat.field(1).load(p32).store(np.zeros_like(p32)), p32)
    # FP64 field: widened exactly; complex128 export returns the widened values
    f64 = lat.field(0).load(p32)
    assert np.array_equal(f64.store(np.zeros_like(psi)), p32.astype(np.complex128))
    # complex64 export of FP64 data rounds to nearest
    assert np.array_equal(lat.field(0).load(psi).store(np.zeros_like(p32)), p32)
    # FP16 field: same stored values whichever width the import came in
    a = lat.field(2).load(p32).store(np.zeros_like(psi))
    b = lat.field(2).load(p32.astype(np.complex128)).store(np.zeros_like(psi))
    assert np.array_equal(a, b)
    # device and pinned buffers
    dev = torch.from_numpy(p32).cuda()
    out = torch.zeros_like(dev)
    lat.field(1).load(dev).store(out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), p32)
    pin = torch.from_numpy(p32).pin_memory()
    outp = torch.zeros_like(pin).pin_memory()
    lat.field(1).load(pin).store(outp)
    assert np.array_equal(outp.numpy(), p32)
    with pytest.raises(ValueError):
        lat.field(1).load(p32[:-1])


def test_async_import_export_pipeline():
    """wc_field_import_async / export_async: a pipelined loop over several
    inputs (page-locked complex64 and complex128 host buffers, CUDA
    tensors) gives exactly the outputs of the synchronous calls; pageable
    host memory is refused before anything is queued."""
    import torch
    w = wc()
    dims = (4, 6, 4, 6)
    U = synth.exp_links(dims, 0.3, 2101)
    lat = make_lattice(dims, U, 1.0, 0.12, -1)
    srcs = [synth.gaussian_source(dims, 2102 + i) for i in range(7)]   # the two copy-out buffers alternate
    fin, fout = lat.field(1), lat.field(1)
    for dt in (np.complex64, np.complex128):
        ref = []
        for s in srcs:
            fin.load(s.astype(dt))
            lat.apply_M(fout, fin)
            ref.append(fout.store(np.zeros(s.shape, dt)))
        hins = [torch.from_numpy(s.astype(dt)).pin_memory() for s in srcs]
        houts = [torch.zeros_like(h).pin_memory() for h in hins]
        for hi, ho in zip(hins, houts):
            fin.load_async(hi)
            lat.apply_M(fout, fin)
            fout.store_async(ho)
        lat.sync()
        for r, ho in zip(ref, houts):
            assert np.array_equal(ho.numpy(), r)
    dev = torch.from_numpy(srcs[1]).cuda()
    out = torch.zeros_like(dev)
    fin.load_async(dev)
    lat.apply_M(fout, fin)
    fout.store_async(out)
    lat.sync()
    fin.load(srcs[1])
    lat.apply_M(fout, fin)
    assert np.array_equal(out.cpu().numpy(), fout.store(np.zeros_like(srcs[1])))
    for call in (lambda: fin.load_async(srcs[0]), lambda: fout.store_async(np.zeros_like(srcs[0]))):
        with pytest.raises(w.WCError) as e:
            call()
        assert e.value.status == 1


def test_gpu_gauge_covariance():
    dims, kappa, csw, tbc = (4, 6, 4, 6), 0.12, 1.5, -1
    U = synth.exp_links(dims, 0.5, 11)
    g = synth.random_su3(synth.volume(dims), np.random.default_rng(12))
    V = synth.volume(dims)
    s = np.arange(V)
    c = np.stack([s % dims[0], (s // dims[0]) % dims[1], (s // (dims[0] * dims[1])) % dims[2],
                  s // (dims[0] * dims[1] * dims[2])], axis=1)
    Up = np.empty_like(U)
    for mu in range(4):
        cf = c.copy()
        cf[:, mu] = (cf[:, mu] + 1) % dims[mu]
        sf = cf[:, 0] + dims[0] * (cf[:, 1] + dims[1] * (cf[:, 2] + dims[2] * cf[:, 3]))
        Up[:, mu] = g @ U[:, mu] @ g[sf].conj().transpose(0, 2, 1)
    psi = synth.gaussian_source(dims, 13)
    psip = np.einsum("vab,vsb->vsa", g, psi)
    a = gpu_apply(make_lattice(dims, U, csw, kappa, tbc), psi, 0, "M")
    b = gpu_apply(make_lattice(dims, Up, csw, kappa, tbc), psip, 0, "M")
    assert np.allclose(b, np.einsum("vab,vsb->vsa", g, a), atol=1e-12)


@pytest.mark.parametrize("cfg,prec,tol", [(2, 1, 1e-5), (3, 2, 5e-3), (3, 1, 1e-5)])
def test_full_size_sampled(cfg, prec, tol):
    """The 24^3x32 (FP32) and 32^3x64 (FP16 storage) workloads in the launch
    configuration the benchmark times, checked on 3000 sampled sites."""
    dims, U, src, csw, kappa, tbc = synth.config_inputs(cfg)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    out = gpu_apply(lat, src, prec, "M")
    V = synth.volume(dims)
    rng = np.random.default_rng(cfg)
    sites = np.concatenate([[0, V - 1], rng.choice(V, 3000, replace=False)])
    ref = oracle.apply_M(dims, tbc, kappa, csw, U, src, sites=sites)
    assert rel_err(out[sites], ref) <= tol
    assert np.max(np.abs(out[sites] - ref)) <= tol * np.max(np.abs(ref))


def test_apply_argument_errors():
    w = wc()
    dims = (4, 4, 4, 4)
    lat = w.Lattice(dims, -1)
    a, b = lat.field(1), lat.field(1)
    with pytest.raises(w.WCError) as e:
        lat.apply_M(b, a)       # no gauge field yet
    assert e.value.status == 3
    lat.load_gauge(synth.unit_links(dims))
    with pytest.raises(w.WCError) as e:
        lat.apply_M(b, a)       # no clover yet
    assert e.value.status == 3
    lat.load_clover(1.0, 0.1)
    with pytest.raises(w.WCError) as e:
        lat.apply_M(a, a)
    assert e.value.status == 1
    with pytest.raises(w.WCError) as e:
        lat.apply_M(lat.field(0), a)
    assert e.value.status == 1


N_SHAPES = 24


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_every_launch_shape_matches_oracle(prec):
    """Each candidate launch shape of the autotuner (lexicographic and tiled
    site maps, register caps) computes the same operator."""
    w = wc()
    dims, kappa, csw, tbc = (8, 8, 4, 4), 0.124, 1.2, -1
    U = synth.exp_links(dims, 0.4, 61)
    psi = synth.gaussian_source(dims, 62)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    ref = oracle.apply_M(dims, tbc, kappa, csw, U, psi)
    refd = oracle.Operator(dims, U, csw, kappa, tbc).Mdag(psi)
    tested = 0
    for i in range(N_SHAPES):
        try:
            lat.apply_shape(prec, 0, force=i)
            lat.apply_shape(prec, 1, force=i)
        except w.WCError:
            continue
        assert_elementwise(gpu_apply(lat, psi, prec, "M"), ref, TOL[prec])
        assert_elementwise(gpu_apply(lat, psi, prec, "Mdag"), refd, TOL[prec])
        tested += 1
    assert tested == (11 if prec == 0 else 24)   # FP64 takes no register-capped shape
    with pytest.raises(w.WCError):
        lat.apply_shape(prec, 0, force=N_SHAPES)


@pytest.mark.parametrize("shape", [16, 17, 18, 19, 20, 21])
def test_persistent_launch_walks_all_blocks(shape):
    """Persistent shapes launch fewer CTAs than there are site blocks (16^3x32:
    1024 blocks of 128 sites, 512 of 256, against at most 152 x resident
    CTAs), also as programmatic dependent launches; every site must still be
    computed (also with a volume that is not a multiple of the CTA size)."""
    kappa, csw, tbc = 0.12, 1.0, -1
    for dims in ((16, 16, 16, 32), (6, 5, 7, 9)):
        U = synth.exp_links(dims, 0.3, 71)
        psi = synth.gaussian_source(dims, 72)
        lat = make_lattice(dims, U, csw, kappa, tbc)
        lat.apply_shape(1, 0, force=shape)
        out = gpu_apply(lat, psi, 1, "M")
        V = synth.volume(dims)
        sites = np.concatenate([np.arange(0, V, 97), [V - 1]])
        ref = oracle.apply_M(dims, tbc, kappa, csw, U, psi, sites=sites)
        assert rel_err(out[sites], ref) <= 1e-5
        assert np.count_nonzero(np.all(out.reshape(V, -1) == 0, axis=1)) == 0


def test_large_lattice_48x48x48x64_sampled():
    """A 48^3x64 lattice (7.1 M sites; the FP64 link and clover arrays hold
    255 M 16-byte elements, 4 GB each): FP64, FP32 and FP16 applies on
    sampled sites against the oracle, so that no index or plane offset
    overflows at this size."""
    dims, kappa, csw, tbc = (48, 48, 48, 64), 0.125, 1.2, -1
    U = synth.pool_links(dims, 77)
    psi = synth.z2_source(dims, 78)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    V = synth.volume(dims)
    sites = np.concatenate([np.random.default_rng(79).choice(V, 1000, replace=False), [0, V - 1]])
    ref = oracle.apply_M(dims, tbc, kappa, csw, U, psi, sites=sites)
    for prec in (0, 1, 2):
        out = gpu_apply(lat, psi, prec, "M")[sites]
        assert rel_err(out, ref) <= TOL[prec], prec
