"""GPU pseudofermion action and force.

Small lattices: S and F against the oracle's FP64 action and force.  At the
16^3x32 workload, where the oracle would take minutes: the force is
traceless anti-Hermitian and matches central finite differences of the
GPU's own action along random su(3) directions (a property that holds at any
size).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import make_lattice, wc

pytestmark = pytest.mark.gpu


def _expm_antiherm(L):
    w, v = np.linalg.eigh(1j * L)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(-1j * w), v.conj())


@pytest.mark.parametrize("dims,csw", [((4, 4, 4, 8), 1.0), ((3, 4, 5, 6), 1.7), ((4, 4, 4, 4), 0.0)])
def test_force_matches_oracle(dims, csw):
    kappa, tbc = 0.12, -1
    U = synth.exp_links(dims, 0.3, 51 + sum(dims))
    phi = synth.gaussian_source(dims, 52)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    S_ref, F_ref, _, _ = oracle.action_and_force(op, phi, tol=1e-14)
    lat = make_lattice(dims, U, csw, kappa, tbc)
    F = np.zeros((synth.volume(dims), 4, 3, 3), complex)
    S = lat.action_force(lat.field(0).load(phi), F, tol=1e-13)
    assert abs(S - S_ref) <= 1e-11 * S_ref
    assert np.max(np.abs(F - F_ref)) <= 1e-9 * np.max(np.abs(F_ref))


def test_force_finite_differences_16x16x16x32():
    dims, U, phi, csw, kappa, tbc = synth.config_inputs(5)
    w = wc()
    lat = make_lattice(dims, U, csw, kappa, tbc)
    V = synth.volume(dims)
    F = np.zeros((V, 4, 3, 3), complex)
    fphi = lat.field(0).load(phi)
    S0 = lat.action_force(fphi, F, tol=1e-13)
    assert np.allclose(F, -F.conj().transpose(0, 1, 3, 2), atol=1e-12 * np.max(np.abs(F)))
    assert np.allclose(np.trace(F, axis1=2, axis2=3), 0, atol=1e-12 * np.max(np.abs(F)))
    rng = np.random.default_rng(55)
    h = 1e-5
    scratch = np.zeros_like(F)
    for _ in range(8):
        Lam = synth.random_su3_algebra((V, 4), rng)
        Ss = []
        for sgn in (1, -1):
            Up = _expm_antiherm(sgn * h * Lam) @ U
            lp = make_lattice(dims, Up, csw, kappa, tbc)
            Ss.append(lp.action_force(lp.field(0).load(phi), scratch, tol=1e-13))
            lp.close()
        fd = (Ss[0] - Ss[1]) / (2 * h)
        an = np.real(np.einsum("lij,lji->", Lam.reshape(-1, 3, 3), F.reshape(-1, 3, 3)))
        assert abs(fd - an) <= 1e-5 * abs(an) + 1e-9 * S0, (fd, an)


def test_autograd_gradient_matches_oracle_and_tangent_derivative():
    """torch.autograd through the action: U.grad = -F U with the oracle's F,
    and the directional derivative along exp(h L) U matches finite
    differences of the forward."""
    import torch
    w = wc()
    dims, kappa, csw, tbc = (4, 4, 4, 8), 0.12, 1.0, -1
    U = synth.exp_links(dims, 0.3, 91)
    phi = synth.gaussian_source(dims, 92)
    lat = w.Lattice(dims, tbc)
    Ut = torch.from_numpy(U).cuda().requires_grad_(True)
    pt = torch.from_numpy(phi).cuda()
    S = w.pseudofermion_action(Ut, pt, lat, csw, kappa, tol=1e-13)
    S.backward()
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    S_ref, F_ref, _, _ = oracle.action_and_force(op, phi, tol=1e-14)
    assert abs(S.item() - S_ref) <= 1e-11 * S_ref
    g = Ut.grad.cpu().numpy()
    assert np.max(np.abs(g + F_ref @ U)) <= 1e-9 * np.max(np.abs(F_ref))
    rng = np.random.default_rng(93)
    Lam = synth.random_su3_algebra((synth.volume(dims), 4), rng)
    h = 1e-5
    Sp = w.pseudofermion_action(torch.from_numpy(_expm_antiherm(h * Lam) @ U).cuda(), pt, lat, csw, kappa,
                                tol=1e-13).item()
    Sm = w.pseudofermion_action(torch.from_numpy(_expm_antiherm(-h * Lam) @ U).cuda(), pt, lat, csw, kappa,
                                tol=1e-13).item()
    fd = (Sp - Sm) / (2 * h)
    an = np.real(np.sum(np.conj(g) * (Lam @ U)))
    assert abs(fd - an) <= 1e-6 * abs(an) + 1e-10 * S_ref


def test_force_times_links_kernel():
    """wc_force_times_links: scale * F U per link against numpy matmuls, and
    its argument checks (host pointers are rejected)."""
    import torch
    w = wc()
    dims = (4, 2, 2, 6)
    V = synth.volume(dims)
    rng = np.random.default_rng(7)
    F = (rng.standard_normal((V, 4, 3, 3)) + 1j * rng.standard_normal((V, 4, 3, 3)))
    U = synth.exp_links(dims, 0.5, 8)
    lat = w.Lattice(dims, -1)
    Ft, Ut = torch.from_numpy(F).cuda(), torch.from_numpy(U).cuda()
    out = torch.empty_like(Ut)
    lat.force_times_links(Ft, Ut, -2.5, out)
    torch.cuda.synchronize()
    ref = -2.5 * (F @ U)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-13 * np.max(np.abs(ref))
    with pytest.raises(ValueError):
        lat.force_times_links(torch.from_numpy(F), Ut, 1.0, out)
