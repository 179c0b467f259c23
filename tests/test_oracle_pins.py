"""Pins of the CPU oracle to facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, an invariant, a textbook
routine or brute force, chosen so that a dropped term, a wrong sign, a wrong
index or a transposed operand in the oracle fails at least one of them:

  * gamma algebra            Clifford relations, hermiticity, the chiral basis
  * free field plane waves   M~(p) = 1 - 2k sum cos p + 2ik sum gamma sin p
                             (catches kappa normalisation, projector signs, the
                             antiperiodic time phase and the hop direction)
  * free field spectrum      dense M on 2^4 and 2x3x4x5 vs the closed form
  * gamma5-hermiticity       <y, M x> = <g5 M g5 y, x>; dense M^+ = (dense M)^+
  * gauge covariance         catches U vs U^+ and link-site mix-ups in the
                             hopping and the clover leaves
  * clover zero / flux       T = 0 on unit links; T on a constant abelian flux
  * dense solve              BiCGStab vs numpy.linalg.solve
  * RAS brute force          MR on a block matrix cut out of the dense M
  * force                    central finite differences, covariance, TA form
"""
import os

import numpy as np
import pytest

import oracle
import synth

RNG = np.random.default_rng(12345)


def dense(apply, n_sites):
    """Dense matrix of a linear map on spinor fields, column by column."""
    n = 12 * n_sites
    D = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        D[:, j] = apply(e.reshape(n_sites, 4, 3)).ravel()
    return D


def chiral_gammas():
    s1 = np.array([[0, 1], [1, 0]], dtype=complex)
    s2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
    s3 = np.array([[1, 0], [0, -1]], dtype=complex)
    z = np.zeros((2, 2))
    g = [np.block([[z, 1j * s], [-1j * s, z]]) for s in (s1, s2, s3)]
    g.append(np.block([[z, np.eye(2)], [np.eye(2), z]]))
    return g


def coords(dims):
    V = synth.volume(dims)
    s = np.arange(V)
    x = s % dims[0]
    y = (s // dims[0]) % dims[1]
    z = (s // (dims[0] * dims[1])) % dims[2]
    t = s // (dims[0] * dims[1] * dims[2])
    return np.stack([x, y, z, t], axis=1)


# --------------------------------------------------------------------------
# gamma matrices
# --------------------------------------------------------------------------

def test_gamma_algebra_and_basis():
    g = [oracle.gamma(m) for m in range(4)]
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2.0 * (m == n) * np.eye(4))
    for m, ref in enumerate(chiral_gammas()):
        assert np.array_equal(g[m], ref)
    g5 = oracle.gamma(4)
    assert np.allclose(g5, g[0] @ g[1] @ g[2] @ g[3])
    assert np.allclose(g5, np.diag([-1, -1, 1, 1]))


# --------------------------------------------------------------------------
# free field: plane waves and the spectrum
# --------------------------------------------------------------------------

def free_symbol(p, kappa):
    g = chiral_gammas()
    m = (1 - 2 * kappa * np.sum(np.cos(p))) * np.eye(4, dtype=complex)
    for mu in range(4):
        m = m + 2j * kappa * np.sin(p[mu]) * g[mu]
    return m


@pytest.mark.parametrize("dims,tbc", [((4, 4, 4, 8), -1), ((3, 4, 5, 6), 1), ((3, 4, 5, 6), -1)])
def test_plane_wave_closed_form(dims, tbc):
    kappa = 0.13
    U = synth.unit_links(dims)
    c = coords(dims)
    for trial in range(4):
        n = RNG.integers(0, 7, size=4)
        p = 2 * np.pi * n / np.array(dims, dtype=float)
        if tbc == -1:
            p[3] = (2 * n[3] + 1) * np.pi / dims[3]
        u = RNG.standard_normal((4, 3)) + 1j * RNG.standard_normal((4, 3))
        phase = np.exp(1j * (c @ p))
        psi = phase[:, None, None] * u[None]
        for csw in (0.0, 1.7):  # the clover term vanishes on unit links
            out = oracle.apply_M(dims, tbc, kappa, csw, U, psi)
            expect = phase[:, None, None] * (free_symbol(p, kappa) @ u)[None]
            assert np.allclose(out, expect, atol=1e-13)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 3, 4, 5)])
def test_free_spectrum_dense(dims):
    kappa, tbc = 0.11, -1
    V = synth.volume(dims)
    U = synth.unit_links(dims)
    D = dense(lambda v: oracle.apply_M(dims, tbc, kappa, 1.0, U, v), V)
    ev = np.linalg.eigvals(D)
    expect = []
    for n in np.ndindex(*dims):
        p = 2 * np.pi * np.array(n, dtype=float) / np.array(dims)
        p[3] = (2 * n[3] + 1) * np.pi / dims[3]
        a = 1 - 2 * kappa * np.sum(np.cos(p))
        b = 2 * kappa * np.sqrt(np.sum(np.sin(p) ** 2))
        expect += [a + 1j * b] * 6 + [a - 1j * b] * 6
    expect = np.array(expect)
    key = lambda z: (np.round(z.real, 9), np.round(z.imag, 9))
    assert np.allclose(sorted(ev, key=key), sorted(expect, key=key), atol=1e-10)


# --------------------------------------------------------------------------
# gamma5-hermiticity and the independently written adjoint
# --------------------------------------------------------------------------

def test_gamma5_hermiticity_random_fields():
    dims, kappa, csw, tbc = (4, 3, 4, 6), 0.124, 1.3, -1
    U = synth.haar_links(dims, 7)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    g5 = np.diag([-1.0, -1.0, 1.0, 1.0]).astype(complex)
    x = synth.gaussian_source(dims, 8)
    y = synth.gaussian_source(dims, 9)
    G5 = lambda v: np.einsum("st,vtc->vsc", g5, v)
    lhs = np.vdot(y, op.M(x))
    rhs = np.vdot(G5(op.M(G5(y))), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # the scatter-form adjoint equals gamma5 M gamma5
    assert np.allclose(op.Mdag(y), G5(op.M(G5(y))), atol=1e-12)


def test_dense_adjoint_is_conjugate_transpose():
    dims, kappa, csw, tbc = (2, 3, 4, 5), 0.12, 1.0, -1
    U = synth.exp_links(dims, 0.3, 11)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    V = synth.volume(dims)
    D = dense(op.M, V)
    Dd = dense(op.Mdag, V)
    assert np.allclose(Dd, D.conj().T, atol=1e-13)
    # the clover block of every site is Hermitian
    assert np.allclose(op.T, op.T.conj().transpose(0, 2, 1), atol=1e-14)


# --------------------------------------------------------------------------
# gauge covariance
# --------------------------------------------------------------------------

def gauge_transform(dims, U, g):
    V = synth.volume(dims)
    c = coords(dims)
    Up = np.empty_like(U)
    for mu in range(4):
        cf = c.copy()
        cf[:, mu] = (cf[:, mu] + 1) % dims[mu]
        sf = cf[:, 0] + dims[0] * (cf[:, 1] + dims[1] * (cf[:, 2] + dims[2] * cf[:, 3]))
        Up[:, mu] = g @ U[:, mu] @ g[sf].conj().transpose(0, 2, 1)
    return Up


def test_gauge_covariance_of_M_and_clover():
    dims, kappa, csw, tbc = (3, 4, 4, 6), 0.12, 1.4, -1
    U = synth.exp_links(dims, 0.5, 21)
    g = synth.random_su3(synth.volume(dims), np.random.default_rng(22))
    Up = gauge_transform(dims, U, g)
    psi = synth.gaussian_source(dims, 23)
    psip = np.einsum("vab,vsb->vsa", g, psi)
    out = oracle.apply_M(dims, tbc, kappa, csw, U, psi)
    outp = oracle.apply_M(dims, tbc, kappa, csw, Up, psip)
    assert np.allclose(outp, np.einsum("vab,vsb->vsa", g, out), atol=1e-12)
    T = oracle.clover_field(dims, csw, kappa, U).reshape(-1, 4, 3, 4, 3)
    Tp = oracle.clover_field(dims, csw, kappa, Up).reshape(-1, 4, 3, 4, 3)
    rot = np.einsum("vab,vsbtc,vdc->vsatd", g, T, g.conj())
    assert np.allclose(Tp, rot, atol=1e-12)


# --------------------------------------------------------------------------
# clover term closed forms
# --------------------------------------------------------------------------

def test_free_field_zero_mode_at_kappa_one_eighth():
    """Unit links, fully periodic: H psi = 8 psi for a constant spinor (the
    eight hops each return psi and (1 - g) + (1 + g) = 2), so M = 1 - H/8 at
    kappa = 1/8 annihilates it -- the singular point the solvers' failure
    tests use.  With the time boundary antiperiodic it is not a zero mode."""
    dims = (4, 4, 4, 4)
    U = synth.unit_links(dims)
    const = np.tile(synth.gaussian_source((1, 1, 1, 1), 5), (synth.volume(dims), 1, 1))
    assert np.max(np.abs(oracle.apply_M(dims, 1, 0.125, 1.7, U, const))) <= 1e-14
    assert np.max(np.abs(oracle.apply_M(dims, -1, 0.125, 1.7, U, const))) > 0.1


def test_clover_vanishes_on_unit_links():
    dims = (3, 4, 2, 5)
    T = oracle.clover_field(dims, 2.3, 0.13, synth.unit_links(dims))
    assert np.count_nonzero(T) == 0


@pytest.mark.parametrize("k", [1, 2])
def test_clover_constant_abelian_flux(k):
    """Constant flux b in the xy plane: every xy plaquette equals exp(i b tau),
    tau = diag(1,-1,0), all other plaquettes are 1.  Then Fhat_xy = i sin(b) tau
    and, with sigma_xy = -diag(s3, s3) in the chiral basis,
    T = csw kappa sin(b) diag(1,-1,1,-1) (x) tau at every site."""
    dims = (4, 3, 3, 4)
    Lx, Ly = dims[0], dims[1]
    b = 2 * np.pi * k / (Lx * Ly)
    tau = np.array([1.0, -1.0, 0.0])
    U = synth.unit_links(dims)
    c = coords(dims)
    for s in range(synth.volume(dims)):
        x, y = c[s, 0], c[s, 1]
        U[s, 1] = np.diag(np.exp(1j * b * x * tau))
        if x == Lx - 1:
            U[s, 0] = np.diag(np.exp(-1j * b * Lx * y * tau))
    csw, kappa = 1.6, 0.128
    T = oracle.clover_field(dims, csw, kappa, U)
    expect = csw * kappa * np.sin(b) * np.kron(np.diag([1.0, -1.0, 1.0, -1.0]), np.diag(tau))
    for s in range(synth.volume(dims)):
        assert np.allclose(T[s], expect, atol=1e-13)
    # and the leaves themselves: Q_xy = 4 exp(i b tau), Q_xz = 4
    Q = oracle.leaf_sum(dims, U, 5, 0, 1)
    assert np.allclose(Q, 4 * np.diag(np.exp(1j * b * tau)), atol=1e-13)
    assert np.allclose(oracle.leaf_sum(dims, U, 5, 0, 2), 4 * np.eye(3), atol=1e-13)


def test_clover_random_abelian_field():
    """Diagonal links diag(exp(i phi_c)) with random phases (sum_c phi_c = 0):
    every plaquette is diagonal with per-colour phase
    Phi = phi_mu(y) + phi_nu(y+mu) - phi_mu(y+nu) - phi_nu(y), so
    Fhat_munu(x) = (i/4) sum over the four plaquettes touching x of sin(Phi),
    minus its colour trace / 3.  Distinguishes the four leaves."""
    dims = (3, 4, 3, 4)
    V = synth.volume(dims)
    rng = np.random.default_rng(81)
    ph = rng.uniform(-np.pi, np.pi, size=(V, 4, 3))
    ph[..., 2] = -ph[..., 0] - ph[..., 1]
    U = np.zeros((V, 4, 3, 3), dtype=complex)
    for c in range(3):
        U[:, :, c, c] = np.exp(1j * ph[..., c])
    c4 = coords(dims)

    def shift(s, mu, d):
        cc = c4[s].copy()
        cc[mu] = (cc[mu] + d) % dims[mu]
        return cc[0] + dims[0] * (cc[1] + dims[1] * (cc[2] + dims[2] * cc[3]))

    g = chiral_gammas()
    csw, kappa = 1.3, 0.12
    T = oracle.clover_field(dims, csw, kappa, U)
    for s in [0, 7, V - 1, 50]:
        expect = np.zeros((12, 12), dtype=complex)
        for mu in range(4):
            for nu in range(mu + 1, 4):
                f = np.zeros(3)
                for y in [s, shift(s, mu, -1), shift(shift(s, mu, -1), nu, -1), shift(s, nu, -1)]:
                    Phi = ph[y, mu] + ph[shift(y, mu, 1), nu] - ph[shift(y, nu, 1), mu] - ph[y, nu]
                    f += np.sin(Phi)
                F = 0.25j * (f - f.sum() / 3)
                sig = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
                expect += 1j * csw * kappa * np.kron(sig, np.diag(F))
        assert np.allclose(T[s], expect, atol=1e-13)


# --------------------------------------------------------------------------
# BiCGStab against a dense solve
# --------------------------------------------------------------------------

def test_bicgstab_matches_dense_solve():
    dims, kappa, csw, tbc = (2, 3, 4, 5), 0.12, 1.0, -1
    U = synth.exp_links(dims, 0.3, 31)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    V = synth.volume(dims)
    D = dense(op.M, V)
    b = synth.gaussian_source(dims, 32)
    x_ref = np.linalg.solve(D, b.ravel())
    res = oracle.bicgstab(op.M, b, tol=1e-13)
    assert res.converged and res.true_rel_resid <= 1e-13
    cond = np.linalg.cond(D)
    assert np.linalg.norm(res.x.ravel() - x_ref) <= 10 * 1e-13 * cond * np.linalg.norm(x_ref)


def test_bicgstab_point_source_8x8x8x8():
    """The plain FP64 solve at the 8^3x8 point-source workload certifies itself
    through its true residual."""
    dims, U, src, csw, kappa, tbc = synth.config_inputs(1)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    res = oracle.bicgstab(op.M, src, tol=1e-12)
    assert res.converged
    r = src - op.M(res.x)
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(src)


# --------------------------------------------------------------------------
# RAS against brute force
# --------------------------------------------------------------------------

def _block_sites(dims, origin, b, delta):
    """Global sites of an extended block in local lexicographic order, plus a
    mask of its core."""
    e = [bm + 2 * delta for bm in b]
    sites, core = [], []
    for lt in range(e[3]):
        for lz in range(e[2]):
            for ly in range(e[1]):
                for lx in range(e[0]):
                    lc = (lx, ly, lz, lt)
                    g = [(origin[m] - delta + lc[m]) % dims[m] for m in range(4)]
                    sites.append(g[0] + dims[0] * (g[1] + dims[1] * (g[2] + dims[2] * g[3])))
                    core.append(all(delta <= lc[m] < delta + b[m] for m in range(4)))
    return np.array(sites), np.array(core)


def _restricted_dense(op, sites):
    """Rows and columns of the dense M on the given set of sites."""
    n = len(sites)
    A = np.zeros((12 * n, 12 * n), dtype=np.complex128)
    for j in range(12 * n):
        v = np.zeros((synth.volume(op.dims), 4, 3), dtype=np.complex128)
        v[sites[j // 12], (j % 12) // 3, j % 3] = 1.0
        col = oracle.apply_M(op.dims, op.tbc, op.kappa, op.csw, op.U, v, T=op.T, sites=sites)
        A[:, j] = col.ravel()
    return A


@pytest.mark.parametrize("origin", [(0, 0, 0, 0), (2, 4, 2, 4)])
def test_ras_block_matches_dense_mr(origin):
    dims, kappa, csw, tbc = (6, 8, 6, 6), 0.12, 1.0, -1
    b, delta, k = (2, 2, 2, 2), 1, 4
    U = synth.haar_links(dims, 41)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    v = synth.gaussian_source(dims, 42)
    z = op.ras(v, block=b, delta=delta, k=k)
    sites, core = _block_sites(dims, origin, b, delta)
    A = _restricted_dense(op, sites)
    r = v[sites].ravel().copy()
    x = np.zeros_like(r)
    for _ in range(k):
        q = A @ r
        alpha = np.vdot(q, r) / np.vdot(q, q)
        x += alpha * r
        r -= alpha * q
    x = x.reshape(-1, 4, 3)
    assert np.allclose(z[sites[core]], x[core], atol=1e-13)
    # many MR steps converge to the block inverse: pins the Dirichlet cut
    zinf = op.ras(v, block=b, delta=delta, k=300)
    xinf = np.linalg.solve(A, v[sites].ravel()).reshape(-1, 4, 3)
    assert np.allclose(zinf[sites[core]], xinf[core], atol=1e-9)


def test_ras_without_overlap_is_block_jacobi():
    dims, kappa, csw, tbc = (4, 4, 4, 4), 0.11, 1.0, -1
    b = (2, 2, 2, 2)
    U = synth.exp_links(dims, 0.3, 51)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    v = synth.gaussian_source(dims, 52)
    z = op.ras(v, block=b, delta=0, k=400)
    for origin in [(0, 0, 0, 0), (2, 0, 2, 2)]:
        sites, core = _block_sites(dims, origin, b, 0)
        A = _restricted_dense(op, sites)
        xb = np.linalg.solve(A, v[sites].ravel()).reshape(-1, 4, 3)
        assert np.allclose(z[sites], xb, atol=1e-9)


def test_ras_rejects_blocks_that_do_not_fit():
    dims = (4, 4, 4, 4)
    op = oracle.Operator(dims, synth.unit_links(dims), 1.0, 0.1, -1)
    with pytest.raises(ValueError):
        op.ras(np.zeros((256, 4, 3), complex), block=(4, 4, 4, 4), delta=1, k=1)


# --------------------------------------------------------------------------
# force: finite differences, covariance, traceless anti-Hermitian
# --------------------------------------------------------------------------

def _expm_antiherm(L):
    """exp of anti-Hermitian 3x3 matrices via eigh of the Hermitian i*L."""
    w, v = np.linalg.eigh(1j * L)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(-1j * w), v.conj())


def _action(dims, U, csw, kappa, tbc, phi):
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    y = oracle.bicgstab(op.Mdag, phi, tol=1e-15, maxiter=5000)
    return float(np.real(np.vdot(y.x, y.x)))


@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_force_finite_differences(csw):
    dims, kappa, tbc = (3, 4, 3, 4), 0.12, -1
    U = synth.exp_links(dims, 0.3, 61)
    phi = synth.gaussian_source(dims, 62)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    S, F, X, Y = oracle.action_and_force(op, phi, tol=1e-15)
    assert abs(S - np.real(np.vdot(phi, X))) <= 1e-12 * S
    rng = np.random.default_rng(63)
    h = 1e-5
    for _ in range(3):
        Lam = synth.random_su3_algebra((synth.volume(dims), 4), rng)
        Sp = _action(dims, _expm_antiherm(h * Lam) @ U, csw, kappa, tbc, phi)
        Sm = _action(dims, _expm_antiherm(-h * Lam) @ U, csw, kappa, tbc, phi)
        fd = (Sp - Sm) / (2 * h)
        an = np.real(np.einsum("lij,lji->", Lam.reshape(-1, 3, 3), F.reshape(-1, 3, 3)))
        assert abs(fd - an) <= 2e-7 * max(abs(an), 1e-3 * S), (fd, an)


def test_force_is_traceless_antihermitian_and_covariant():
    dims, kappa, csw, tbc = (3, 4, 3, 4), 0.12, 1.2, -1
    U = synth.exp_links(dims, 0.4, 71)
    X = synth.gaussian_source(dims, 72)
    Y = synth.gaussian_source(dims, 73)
    F = oracle.force(dims, tbc, kappa, csw, U, X, Y)
    assert np.allclose(F, -F.conj().transpose(0, 1, 3, 2), atol=1e-13)
    assert np.allclose(np.trace(F, axis1=2, axis2=3), 0, atol=1e-13)
    g = synth.random_su3(synth.volume(dims), np.random.default_rng(74))
    Up = gauge_transform(dims, U, g)
    Xp = np.einsum("vab,vsb->vsa", g, X)
    Yp = np.einsum("vab,vsb->vsa", g, Y)
    Fp = oracle.force(dims, tbc, kappa, csw, Up, Xp, Yp)
    rot = np.einsum("vab,vmbc,vdc->vmad", g, F, g.conj())
    assert np.allclose(Fp, rot, atol=1e-12)


# --------------------------------------------------------------------------
# the synthetic inputs are SU(3)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["exp", "haar"])
def test_generated_links_are_su3(kind):
    dims = (4, 4, 4, 4)
    U = synth.exp_links(dims, 0.3, 1) if kind == "exp" else synth.haar_links(dims, 1)
    u = U.reshape(-1, 3, 3)
    assert np.allclose(u @ u.conj().transpose(0, 2, 1), np.eye(3), atol=1e-13)
    assert np.allclose(np.linalg.det(u), 1.0, atol=1e-13)


# --------------------------------------------------------------------------
# even-odd Schur complement (Sec. 2: the solvers act on the even-odd
# preconditioned matrix); pinned to the full operator, not to itself
# --------------------------------------------------------------------------
def _eo_setup(dims, seed, kappa=0.13, csw=1.2, tbc=-1):
    from oracle.evenodd import EvenOdd
    U = synth.exp_links(dims, 0.5, seed)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    return op, EvenOdd(dims, tbc, kappa, U, op.T)


def test_parity_mask_and_hopping_term_flip_parity():
    from oracle.evenodd import parity
    dims = (4, 2, 6, 4)
    par = parity(dims)
    xyz = coords(dims)
    assert np.array_equal(par, xyz.sum(axis=1) % 2)
    assert par.sum() * 2 == synth.volume(dims)
    op, eo = _eo_setup(dims, 31)
    psi = synth.gaussian_source(dims, 32)
    psi[par == 1] = 0
    h = oracle.apply_hop(dims, -1, op.U, psi)
    assert np.abs(h[par == 0]).max() == 0.0   # H maps even sites to odd only


def test_schur_block_elimination_against_full_M():
    """M (x_e + k A_oo^-1 H_oe x_e) = M^ x_e on the even sites, 0 on the odd
    ones: the lower block row of M vanishes by construction."""
    dims = (4, 4, 2, 6)
    op, eo = _eo_setup(dims, 41)
    xe = synth.gaussian_source(dims, 42)
    xe[eo.odd] = 0
    from oracle.evenodd import _site_solve
    xo = _site_solve(eo.A, op.kappa * eo.hop(xe, eo.odd), eo.odd)
    full = op.M(xe + xo)
    sch = eo.schur(xe)
    assert np.abs(full[eo.odd]).max() <= 1e-13 * np.abs(full).max()
    assert np.allclose(full[eo.even], sch[eo.even], atol=1e-13)
    assert np.abs(sch[eo.odd]).max() == 0.0


def test_schur_solve_reconstructs_full_solution():
    """prepare -> dense solve of M^ -> reconstruct gives M x = b."""
    dims = (4, 2, 2, 4)
    op, eo = _eo_setup(dims, 51)
    b = synth.gaussian_source(dims, 52)
    ev = np.flatnonzero(eo.even)
    n = len(ev)

    def schur_on_even(v):
        f = np.zeros((synth.volume(dims), 4, 3), dtype=np.complex128)
        f[ev] = v
        return eo.schur(f)[ev]

    D = dense(schur_on_even, n)
    bh = eo.prepare(b)
    xe = np.zeros_like(b)
    xe[ev] = np.linalg.solve(D, bh[ev].ravel()).reshape(n, 4, 3)
    x = eo.reconstruct(xe, b)
    assert np.allclose(op.M(x), b, atol=1e-11)


def test_full_residual_of_a_reconstruction_is_the_schur_residual():
    """For any x_e (not only a solution) and x_o = A_oo^-1 (b_o + k H_oe
    x_e), the full residual b - M x vanishes on the odd sites and equals
    the Schur residual b^_e - M^ x_e on the even sites: an even-odd solve's
    full true residual and its half solve's residual are one quantity."""
    dims = (4, 2, 4, 4)
    op, eo = _eo_setup(dims, 71)
    b = synth.gaussian_source(dims, 72)
    xe = synth.gaussian_source(dims, 73)
    xe[eo.odd] = 0
    x = eo.reconstruct(xe, b)
    r = b - op.M(x)
    rs = eo.prepare(b) - eo.schur(xe)
    scale = np.abs(b).max() + np.abs(op.M(x)).max()
    assert np.abs(r[eo.odd]).max() <= 1e-13 * scale
    assert np.abs(r[eo.even] - rs[eo.even]).max() <= 1e-13 * scale
    assert np.abs(rs[eo.even]).max() > 1e-2 * scale   # x_e is far from a solution


def test_schur_determinant_identity_and_adjoint():
    """det M = det A_oo det M^, and M^+ is the conjugate transpose of M^."""
    dims = (2, 2, 2, 4)
    op, eo = _eo_setup(dims, 61, kappa=0.2)
    V = synth.volume(dims)
    ev = np.flatnonzero(eo.even)
    od = np.flatnonzero(eo.odd)

    def on_even(fn):
        def f(v):
            g = np.zeros((V, 4, 3), dtype=np.complex128)
            g[ev] = v
            return fn(g)[ev]
        return f

    D = dense(on_even(eo.schur), len(ev))
    Dd = dense(on_even(lambda g: eo.schur(g, dagger=True)), len(ev))
    assert np.allclose(Dd, D.conj().T, atol=1e-13)
    _, ld_full = np.linalg.slogdet(dense(op.M, V))
    _, ld_s = np.linalg.slogdet(D)
    ld_a = sum(np.linalg.slogdet(eo.A[s])[1] for s in od)
    assert abs(ld_full - (ld_s + ld_a)) <= 1e-9 * abs(ld_full)


def test_oracle_matches_stored_regression_values():
    """The oracle reproduces tests/golden/oracle_regression_4x4x4x4.json
    (written by tests/golden/make_golden.py from the oracle itself): a guard
    against unnoticed changes of the oracle's arithmetic, which every pin
    above and every GPU parity test relies on."""
    import importlib.util
    import json
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    stored = json.load(open(os.path.join(here, "oracle_regression_4x4x4x4.json")))
    now = mg.compute()
    assert stored["config"] == now["config"] and stored["sites"] == now["sites"]

    def close(a, b, rtol=1e-10):
        a, b = np.asarray(a, float), np.asarray(b, float)
        return np.max(np.abs(a - b)) <= rtol * max(np.max(np.abs(b)), 1e-300)

    for key in ("M_psi", "H_psi", "schur_psi"):
        for s in stored["sites"]:
            assert close(now[key][str(s)], stored[key][str(s)]), (key, s)
    for key in ("clover_block_site0", "force_link_site0_mu0"):
        assert close(now[key], stored[key]), key
    for key in ("norm2_M_psi", "action_S"):
        assert abs(now[key] - stored[key]) <= 1e-11 * abs(stored[key]), key
