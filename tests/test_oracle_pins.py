"""Pins of the CPU oracle against facts that do not come from the oracle
itself: textbook constants, closed forms, library routines, brute force,
finite differences and invariants the paper states.

Each test names the passage of the paper (Yang et al., arXiv:2004.12484) or
the mathematical fact it rests on.  A plausible slip in the oracle (a dropped
term, a wrong sign, a transposed index) fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "lattice_constants.json")))


# ------------------------------------------------------------------ FFT
@pytest.mark.parametrize("n", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft1d_matches_naive_dft(n, sign):
    """The oracle FFT equals the DFT sum written out (brute force)."""
    g = np.random.default_rng(n)
    x = g.normal(size=n) + 1j * g.normal(size=n)
    k = np.arange(n)
    naive = np.array([(x * np.exp(sign * 2j * np.pi * kk * k / n)).sum() for kk in k])
    assert np.allclose(O.fft1d(x, sign), naive, rtol=0, atol=1e-13 * max(1, n))


def test_fft3d_matches_numpy():
    """3D transform equals numpy.fft.fftn / n^3 ifftn (library routine)."""
    g = np.random.default_rng(3)
    a = g.normal(size=(16, 16, 16)) + 1j * g.normal(size=(16, 16, 16))
    assert np.abs(O.fft3d(a, -1) - np.fft.fftn(a)).max() < 1e-12
    assert np.abs(O.fft3d(a, +1) - np.fft.ifftn(a) * 16 ** 3).max() < 1e-12


# ------------------------------------------------------------------ window
def test_window_b_closed_form():
    """b = 2 sigma m / ((2 sigma - 1) pi): sigma = 2, m = 3 gives 4/pi."""
    assert abs(O.window_b(128, 32, 6) - 4.0 / np.pi) < 1e-15
    assert abs(O.window_b(64, 16, 4) - 8.0 / (3.0 * np.pi)) < 1e-15


def test_window_fourier_transform_by_quadrature():
    """M c(n) equals the numerically integrated Fourier transform of phi
    (the scaling step divides by it, Sec. 3.1)."""
    M, nc, p = 64, 16, 6
    b = O.window_b(M, nc, p)
    u = np.linspace(-30, 30, 60001)
    du = 60.0 / 60000
    phi = O.window(u, b)
    assert abs(phi.sum() * du - 1.0) < 1e-11  # unit mass
    for n in [0, 3, 8, 16]:
        ft = (phi * np.cos(2 * np.pi * n * u / M)).sum() * du
        assert abs(ft - O.window_hat([n], M, b)[0]) < 1e-12


def test_spread_interpolate_are_transposes():
    """sum_l g_l a_l = sum_j q_j (interpolated a)(x_j): spreading and
    interpolation use the same window with the same indices (Sec. 3.1)."""
    g = np.random.default_rng(7)
    N, M, p, nc = 40, 16, 6, 4
    L = np.array([5.0, 6.0, 7.0])
    pos = g.uniform(-3, 10, size=(N, 3))
    q = g.normal(size=N)
    grid = O.spread(pos, q, L, M, p, nc)
    a = g.normal(size=(M, M, M))
    # interpolate a through the structure of the oracle: potential of a single
    # unit charge is linear in the grid, so use the brute-force definition here
    b = O.window_b(M, nc, p)
    vals = []
    for j in range(N):
        u = M * np.mod(pos[j] / L, 1.0)
        f = np.floor(u).astype(int)
        s = 0.0
        for cz in range(p):
            for cy in range(p):
                for cx in range(p):
                    l = f - p // 2 + 1 + np.array([cx, cy, cz])
                    w = np.prod([O.window([u[t] - l[t]], b)[0] for t in range(3)])
                    s += w * a[l[2] % M, l[1] % M, l[0] % M]
        vals.append(s)
    assert abs((grid * a).sum() - (q * np.array(vals)).sum()) < 1e-12 * np.abs(q).sum()


def test_spread_mass_and_translation_by_cell():
    """The window has unit mass only approximately (truncation), but the
    spread grid of a particle moved by exactly one cell is the same grid
    rolled by one cell (periodicity, Eq. 18)."""
    M, p, nc = 16, 6, 4
    L = np.array([8.0, 8.0, 8.0])
    pos = np.array([[1.3, 2.7, 5.1]])
    g1 = O.spread(pos, [1.0], L, M, p, nc)
    g2 = O.spread(pos + np.array([[L[0] / M, 0, 0]]), [1.0], L, M, p, nc)
    assert np.abs(np.roll(g1, 1, axis=2) - g2).max() < 1e-14
    assert abs(g1.sum() - 1.0) < 1e-3


# ------------------------------------------------------------------ Madelung
def test_madelung_nacl_direct_and_nfft():
    """Rock salt: E = -(N/2) 1.747565 / r0 (Madelung check, Sec. 2.4.2);
    all forces vanish by symmetry."""
    pos, q, L = W.rock_salt(4)
    E_ref = -(len(q) / 2) * GOLD["nacl_madelung"] / (W.NACL_A / 2)
    r1 = O.direct_ewald(pos, q, L, alpha=0.5, rc=10.0, nmax=16, sphere=True)
    assert abs(r1.E / E_ref - 1) < 1e-6
    assert np.abs(r1.F).max() < 1e-10
    r2 = O.nfft_ewald(pos, q, L, alpha=0.45, rc=11.0, M=64, p=10, nc=16)
    assert abs(r2.E / E_ref - 1) < 1e-6
    assert np.abs(r2.F).max() < 1e-9


def test_madelung_cscl():
    pos, q, L = W.cesium_chloride(4, a=4.12)
    E_ref = -(len(q) / 2) * GOLD["cscl_madelung"] / (4.12 * np.sqrt(3) / 2)
    r1 = O.direct_ewald(pos, q, L, alpha=0.5, rc=8.0, nmax=16, sphere=True)
    assert abs(r1.E / E_ref - 1) < 1e-6


def test_wigner_background_term():
    """One ion with a neutralising background: E = -2.837297 q^2/(2L)
    (pins the uniform-background term for Q != 0)."""
    Lb = 10.0
    for a, rc, nm in [(0.6, 4.9, 14), (0.9, 4.9, 20)]:
        r = O.direct_ewald(np.zeros((1, 3)), np.ones(1), np.full(3, Lb), alpha=a, rc=rc, nmax=nm)
        assert abs(r.E / (-GOLD["wigner_sc"] / (2 * Lb)) - 1) < 1e-6


# ------------------------------------------------------------------ Ewald invariants
def test_alpha_independence_direct():
    """The total energy does not depend on alpha (Sec. 2.4.2)."""
    d = W.nacl()
    Es = []
    for a, rc, nm in [(0.3, 20.0, 14), (0.4, 15.0, 19), (0.5, 12.0, 24)]:
        Es.append(O.direct_ewald(d["pos"], d["q"], d["L"], alpha=a, rc=rc, nmax=nm, sphere=True).E)
    Es = np.array(Es)
    assert np.abs(Es / Es[0] - 1).max() < 1e-10


def test_image_sum_brute_force():
    """Spherical-order image sum (Eq. 1) converges to the Ewald energy plus
    the surface term 2 pi |sum q r|^2 / (3V) (tin-foil vs vacuum)."""
    g = np.random.default_rng(5)
    L = np.full(3, 6.0)
    pos = g.uniform(0, 6, size=(8, 3))
    q = np.array([1, -1, 1, -1, 1, -1, 1, -1.0])
    Md = (q[:, None] * pos).sum(0)
    ref = O.direct_ewald(pos, q, L, alpha=1.2, rc=2.9, nmax=12, sphere=True)
    e40 = O.image_sum(pos, q, L, 40)
    assert abs(e40 - (ref.E + 2 * np.pi / (3 * 216.0) * Md @ Md)) < 5e-8


def test_forces_are_minus_gradient_direct():
    """O1 forces (Eq. 29, 41 in textbook form) equal -dE/dr by central
    finite differences."""
    g = np.random.default_rng(11)
    L = np.array([9.0, 10.0, 11.0])
    N = 12
    pos = g.uniform(0, 10, size=(N, 3))
    q = g.normal(size=N); q -= q.mean()
    kw = dict(alpha=0.7, rc=4.4, nmax=9, sphere=False)
    r = O.direct_ewald(pos, q, L, **kw)
    h = 1e-5
    for i in [0, 5, 11]:
        for t in range(3):
            pp = pos.copy(); pp[i, t] += h
            pm = pos.copy(); pm[i, t] -= h
            fd = -(O.direct_ewald(pp, q, L, **kw).E - O.direct_ewald(pm, q, L, **kw).E) / (2 * h)
            assert abs(fd - r.F[i, t]) < 1e-7 * (1 + abs(r.F[i, t]))


def test_phi_is_dE_dq_direct_and_nfft():
    """E is quadratic in q, so a central difference in q_i is exact up to
    rounding and equals phi_i = dE/dq_i (Eq. 5)."""
    g = np.random.default_rng(12)
    L = np.full(3, 10.0)
    N = 20
    pos = g.uniform(0, 10, size=(N, 3))
    q = g.normal(size=N)
    for fn, kw in [(O.direct_ewald, dict(alpha=0.6, rc=4.9, nmax=8, sphere=False)),
                   (O.nfft_ewald, dict(alpha=0.6, rc=4.9, M=32, p=6, nc=8))]:
        r = fn(pos, q, L, **kw)
        h = 1e-3
        for i in [0, 7, 19]:
            qp = q.copy(); qp[i] += h
            qm = q.copy(); qm[i] -= h
            fd = (fn(pos, qp, L, **kw).E - fn(pos, qm, L, **kw).E) / (2 * h)
            assert abs(fd - r.phi[i]) < 1e-9 * (1 + abs(r.phi[i]))


def test_net_force_zero_and_translation():
    """Sum of forces vanishes (the momentum conservation the abstract claims) and the energy is
    translation invariant; O2 is exactly invariant under shifts by whole grid
    cells h = L/M (Eq. 18)."""
    d = W.nacl()
    pos, q, L = d["pos"], d["q"], d["L"]
    r1 = O.direct_ewald(pos, q, L, alpha=0.35, rc=9.0, nmax=10)
    scale = np.abs(r1.F).sum()
    assert np.abs(r1.F.sum(0)).max() < 1e-12 * scale
    shift = np.array([0.37, -1.91, 2.23])
    r1s = O.direct_ewald(pos + shift, q, L, alpha=0.35, rc=9.0, nmax=10)
    assert abs(r1s.E / r1.E - 1) < 1e-12
    assert np.abs(r1s.F - r1.F).max() < 1e-11 * np.abs(r1.F).max()
    kw = dict(alpha=0.35, rc=9.0, M=32, p=4, nc=8)
    r2 = O.nfft_ewald(pos, q, L, **kw)
    assert np.abs(r2.F.sum(0)).max() < 1e-12 * scale
    h = L / 32
    r2s = O.nfft_ewald(pos + np.array([3, -5, 7]) * h, q, L, **kw)
    assert abs(r2s.E / r2.E - 1) < 1e-12
    assert np.abs(r2s.F - r2.F).max() < 1e-10 * np.abs(r2.F).max()


def test_virial_trace_and_strain_derivative():
    """tr W = E for converged Ewald (Coulomb energy is homogeneous of degree
    -1), and each diagonal W_aa = -dE/d eps_aa under the strain L_a -> L_a
    (1 + eps), positions scaled with it."""
    d = W.nacl()
    pos, q, L = d["pos"], d["q"], d["L"]
    kw = dict(alpha=0.5, rc=11.0, nmax=24, sphere=True)
    r = O.direct_ewald(pos, q, L, **kw)
    assert abs(np.trace(r.virial) / r.E - 1) < 1e-9
    eps = 1e-5
    for a in range(3):
        s = np.ones(3); s[a] += eps
        ep = O.direct_ewald(pos * s, q, L * s, **kw).E
        s = np.ones(3); s[a] -= eps
        em = O.direct_ewald(pos * s, q, L * s, **kw).E
        assert abs(-(ep - em) / (2 * eps) - r.virial[a, a]) < 1e-6 * abs(r.E)
    assert np.abs(r.virial - r.virial.T).max() < 1e-12 * abs(r.E)


def test_reciprocal_virial_offdiagonal_by_strain():
    """Reciprocal virial, all nine components: under a general strain eps the
    structure factor is unchanged, k -> (1 - eps^T) k and V -> V (1 + tr eps);
    W^K_ab = -dE_K/d eps_ab by central differences of the energy sum."""
    g = np.random.default_rng(21)
    L = np.array([7.0, 8.0, 9.0])
    N = 10
    pos = g.uniform(0, 8, size=(N, 3))
    q = g.normal(size=N); q -= q.mean()
    alpha, nc = 0.6, 6
    EK, _, _, WK = O.kspace_direct(pos, q, L, alpha, nc, sphere=False)
    S = O.structure_factor_direct(pos, q, L, nc)
    n = np.stack(np.meshgrid(*[np.arange(-nc, nc + 1)] * 3, indexing="ij"), -1)[..., ::-1]  # [z,y,x] -> (nx,ny,nz)
    k0 = 2 * np.pi * n / L
    mask = np.any(n != 0, axis=-1)
    S2 = np.abs(S) ** 2

    def energy(e):
        k = k0 @ (np.eye(3) - e)  # k_b' = k_b - k_a e_ab
        V = np.prod(L) * (1 + np.trace(e))
        k2 = (k ** 2).sum(-1)[mask]
        return (2 * np.pi / V * np.exp(-k2 / (4 * alpha ** 2)) / k2 * S2[mask]).sum()

    assert abs(energy(np.zeros((3, 3))) / EK - 1) < 1e-12
    h = 1e-6
    for a in range(3):
        for b in range(3):
            e = np.zeros((3, 3)); e[a, b] = h
            fd = -(energy(e) - energy(-e)) / (2 * h)
            assert abs(fd - WK[a, b]) < 1e-6 * abs(EK)


# ------------------------------------------------------------------ NFFT
def test_structure_factor_nfft_error_decays_with_p():
    """The NFFT approximation error of S(n) falls exponentially with the
    window width at fixed oversampling (Sec. 2.2, Fig. 1 trend)."""
    d = W.nacl()
    Sd = O.structure_factor_direct(d["pos"], d["q"], d["L"], 8)
    errs = []
    for p in [2, 4, 6, 8, 10]:
        Sn = O.structure_factor_nfft(d["pos"], d["q"], d["L"], 32, p, 8)
        errs.append(np.sqrt((np.abs(Sn - Sd) ** 2).sum() / (np.abs(Sd) ** 2).sum()))
    errs = np.array(errs)
    assert np.all(errs[1:] < errs[:-1] / 4)
    assert errs[-1] < 5e-5


def test_structure_factor_additivity():
    """S(n) of a union is the sum of the subsets' S(n) (HP-ENUF, Sec. 3.3)."""
    d = W.nacl()
    pos, q, L = d["pos"], d["q"], d["L"]
    part = np.random.default_rng(9).integers(0, 3, size=len(q))
    Sfull = O.structure_factor_nfft(pos, q, L, 32, 6, 8)
    Ssum = sum(O.structure_factor_nfft(pos[part == i], q[part == i], L, 32, 6, 8) for i in range(3))
    assert np.abs(Sfull - Ssum).max() < 1e-11 * np.abs(q).sum()
    Sd = O.structure_factor_direct(pos, q, L, 4)
    Sds = sum(O.structure_factor_direct(pos[part == i], q[part == i], L, 4) for i in range(3))
    assert np.abs(Sd - Sds).max() < 1e-11 * np.abs(q).sum()


def test_direct_structure_factor_vs_recurrence_energy():
    """O1's recurrence-based reciprocal energy equals the energy from the
    plainly evaluated S(n) (two independent evaluations of Eq. 22)."""
    g = np.random.default_rng(4)
    L = np.array([6.0, 7.0, 8.0])
    pos = g.uniform(0, 8, size=(15, 3)); q = g.normal(size=15)
    alpha, nc = 0.8, 5
    EK = O.kspace_direct(pos, q, L, alpha, nc, sphere=False)[0]
    S = O.structure_factor_direct(pos, q, L, nc)
    n = np.stack(np.meshgrid(*[np.arange(-nc, nc + 1)] * 3, indexing="ij"), -1)[..., ::-1]
    k = 2 * np.pi * n / L
    k2 = (k ** 2).sum(-1)
    m = k2 > 0
    E2 = (2 * np.pi / np.prod(L) * np.exp(-k2[m] / (4 * alpha ** 2)) / k2[m] * np.abs(S[m]) ** 2).sum()
    assert abs(EK / E2 - 1) < 1e-12


def test_nfft_ewald_approaches_direct_with_p():
    """O2 energy and forces converge to O1 on the same cubic frequency set
    as the window widens (m >= 2 'negligible', Sec. 2.3.2)."""
    d = W.nacl()
    pos, q, L = d["pos"], d["q"], d["L"]
    kw = dict(alpha=0.35, rc=9.0)
    r1 = O.direct_ewald(pos, q, L, nmax=8, sphere=False, **kw)
    eE, eF = [], []
    for p in [4, 8, 12]:
        r2 = O.nfft_ewald(pos, q, L, M=32, p=p, nc=8, **kw)
        eE.append(abs(r2.E / r1.E - 1))
        eF.append(np.sqrt(((r2.F - r1.F) ** 2).sum() / (r1.F ** 2).sum()))
    assert eE[0] < 1e-4 and eE[2] < 1e-8
    assert eF[1] < eF[0] / 10 and eF[2] < eF[1] / 10
    assert eF[2] < 5e-6


def test_window_derivative_by_central_difference():
    """d phi/du of the Gaussian window against a central difference of the
    window itself (closed form -(2u/b) phi(u))."""
    b = O.window_b(32, 8, 8)
    u = np.linspace(-4.2, 4.3, 23)
    h = 1e-5
    fd = (O.window(u + h, b) - O.window(u - h, b)) / (2 * h)
    assert np.abs(O.window_deriv(u, b) - fd).max() < 1e-9


def _ad_system(seed=21, N=16):
    g = np.random.default_rng(seed)
    L = np.array([9.0, 10.0, 11.0])
    pos = g.uniform(0, 1, size=(N, 3)) * L
    q = g.normal(size=N); q -= q.mean()
    return pos, q, L


def test_ad_forces_are_minus_gradient_of_nfft_energy():
    """The analytic-differentiation forces are the exact gradient of the NFFT
    energy of Eq. 38 (the ik oracle's E, itself pinned against direct Ewald):
    a central difference of that energy reproduces them to rounding, for any
    window width, although they differ from the ik forces of Eq. 41-42."""
    pos, q, L = _ad_system()
    M, nc = 16, 5
    for p, alpha in [(4, 0.5), (6, 0.6)]:
        E, F, _, _ = O.kspace_nfft_ad(pos, q, L, alpha, M, p, nc)
        _, Fik, _, _ = O.kspace_nfft(pos, q, L, alpha, M, p, nc)
        h = 1e-5
        for i in [0, 7, 15]:
            for t in range(3):
                u = M * pos[i, t] / L[t]
                assert abs(u - np.round(u)) > 1e-3  # no window-support change inside the stencil
                pp = pos.copy(); pp[i, t] += h
                pm = pos.copy(); pm[i, t] -= h
                fd = -(O.kspace_nfft(pp, q, L, alpha, M, p, nc)[0] - O.kspace_nfft(pm, q, L, alpha, M, p, nc)[0]) / (2 * h)
                assert abs(fd - F[i, t]) < 1e-8 * (1 + np.abs(F).max())
        # the variant is a different discretisation: at p = 4 it measurably
        # differs from the ik forces
        if p == 4:
            assert np.abs(F - Fik).max() > 1e-6 * np.abs(F).max()


def test_ad_energy_virial_phi_equal_ik_oracle():
    """Only the forces differ between the two variants: E~ (Eq. 38), the
    virial and phi = dE/dq come from the same spectrum."""
    pos, q, L = _ad_system(seed=22, N=24)
    kw = dict(alpha=0.55, M=32, p=6, nc=8)
    Ea, _, pa, Wa = O.kspace_nfft_ad(pos, q, L, **kw)
    Ei, _, pi_, Wi = O.kspace_nfft(pos, q, L, **kw)
    assert abs(Ea / Ei - 1) < 1e-13
    assert np.abs(Wa - Wi).max() < 1e-13 * np.abs(Wi).max()
    assert np.abs(pa - pi_).max() < 1e-12 * np.abs(pi_).max()


def test_ad_forces_approach_direct_with_p_and_grid_shift_invariance():
    """With the window widened the analytic-differentiation forces converge to
    the direct reciprocal forces on the same cube (Eq. 41 summed exactly),
    and like O2 they are exactly invariant under shifts by whole grid cells
    (Eq. 18)."""
    d = W.nacl()
    pos, q, L = d["pos"], d["q"], d["L"]
    r1 = O.kspace_direct(pos, q, L, 0.35, 8, sphere=False)
    eF = []
    for p in [4, 8, 12]:
        _, F, _, _ = O.kspace_nfft_ad(pos, q, L, 0.35, 32, p, 8)
        eF.append(np.sqrt(((F - r1[1]) ** 2).sum() / (r1[1] ** 2).sum()))
    assert eF[1] < eF[0] / 10 and eF[2] < eF[1] / 10
    # (the ik forces reach 4.1e-6 here; the window derivative costs a factor
    # of 1.2-2 at every p)
    assert eF[2] < 1e-5
    _, F0, _, _ = O.kspace_nfft_ad(pos, q, L, 0.35, 32, 6, 8)
    h = np.asarray(L) / 32
    _, F1, _, _ = O.kspace_nfft_ad(pos + np.array([2, -3, 5]) * h, q, L, 0.35, 32, 6, 8)
    assert np.abs(F1 - F0).max() < 1e-10 * np.abs(F0).max()


def test_real_space_subset_matches_full():
    """The sampled evaluation path returns the same per-particle values as
    the full pair loop."""
    d = W.nacl()
    _, F, phi, _ = O.real_space(d["pos"], d["q"], d["L"], 0.35, 9.0)
    idx = [3, 100, 511]
    _, Fs, phis, _ = O.real_space(d["pos"], d["q"], d["L"], 0.35, 9.0, idx=idx)
    assert np.abs(Fs - F[idx]).max() < 1e-14 and np.abs(phis - phi[idx]).max() < 1e-14


# ------------------------------------------------------------------ ENUF-DPD (Slater-type charges)
LAMBDA_E = 6.954  # decay length of the method's smeared charges (beta = 1.125)


def test_slater_potential_solves_poisson_by_quadrature():
    """B_U(r)/r is the potential of the Slater density of Eq. 51 (Eq. 52):
    the density integrates to the charge, and the shell-theorem potential
    (enclosed charge / r plus the outer shells' 4 pi s rho ds), computed by
    quadrature, matches the oracle's factor."""
    from scipy.integrate import quad
    lam = LAMBDA_E
    rho = lambda s: np.exp(-2.0 * s / lam) / (np.pi * lam ** 3)
    total, _ = quad(lambda s: 4 * np.pi * s * s * rho(s), 0, np.inf, epsabs=1e-14)
    assert abs(total - 1.0) < 1e-12
    for r in [0.05, 1.0, 3.7, 6.954, 12.0, 23.5]:
        inner, _ = quad(lambda s: 4 * np.pi * s * s * rho(s), 0, r, epsabs=1e-15)
        outer, _ = quad(lambda s: 4 * np.pi * s * rho(s), r, np.inf, epsabs=1e-15)
        BU, _ = O.slater_factors(r, lam)
        assert abs(BU[0] / r - (inner / r + outer)) < 1e-11


def test_slater_force_factor_is_minus_derivative_and_limits():
    """B_F / r^2 = -d(B_U / r)/dr (Eq. 54 from Eq. 53, by central
    differences), the finite r -> 0 limits of Eq. 59-60 (energy beta/R_c =
    1/lambda_e, force 0) and B_U, B_F -> 1 far away."""
    lam = LAMBDA_E
    h = 1e-5
    for r in [0.3, 2.0, 7.0, 15.0, 23.0]:
        up, _ = O.slater_factors(r + h, lam)
        um, _ = O.slater_factors(r - h, lam)
        _, BF = O.slater_factors(r, lam)
        dU = ((up / (r + h)) - (um / (r - h))) / (2 * h)
        assert abs(BF[0] / r ** 2 + dU[0]) < 1e-9
    r = 1e-4
    BU, BF = O.slater_factors(r, lam)
    assert abs(BU[0] / r - 1.0 / lam) < 1e-4 / lam
    assert abs(BF[0] / r ** 2) < 1e-5
    BU, BF = O.slater_factors(40 * lam, lam)
    assert abs(BU[0] - 1) < 1e-15 and abs(BF[0] - 1) < 1e-15


def test_slater_real_space_pair_equals_quadrature_potential():
    """Two smeared charges alone within the cutoff, alpha -> 0 (erfc -> 1):
    the oracle's real-space energy is q1 q2 phi(r) with phi from the
    quadrature of Eq. 51, its force the central difference of that energy,
    its potentials q_j phi(r); coincident smeared charges carry the finite
    energy q1 q2 / lambda_e (Eq. 59) and no force (Eq. 60)."""
    from scipy.integrate import quad
    lam = LAMBDA_E
    rho = lambda s: np.exp(-2.0 * s / lam) / (np.pi * lam ** 3)

    def phi(r):
        inner, _ = quad(lambda s: 4 * np.pi * s * s * rho(s), 0, r, epsabs=1e-15)
        outer, _ = quad(lambda s: 4 * np.pi * s * rho(s), r, np.inf, epsabs=1e-15)
        return inner / r + outer

    L = np.full(3, 200.0)
    q = np.array([1.3, -0.7])
    for d in [0.5, 4.0, 11.0]:
        pos = np.array([[50.0, 60.0, 70.0], [50.0 + d * 0.6, 60.0 + d * 0.8, 70.0]])
        E, F, ph, W = O.real_space(pos, q, L, 1e-13, 30.0, slater=lam)
        assert abs(E - q[0] * q[1] * phi(d)) < 1e-9 * abs(q[0] * q[1] / d)
        assert abs(ph[0] - q[1] * phi(d)) < 1e-9 and abs(ph[1] - q[0] * phi(d)) < 1e-9
        h = 1e-5
        fd = -(q[0] * q[1] * (phi(d + h) - phi(d - h)) / (2 * h))  # radial force on particle 1
        unit = np.array([0.6, 0.8, 0.0])
        assert np.abs(F[1] - fd * unit).max() < 1e-7
        assert np.abs(F[0] + F[1]).max() < 1e-14
    pos = np.array([[50.0, 60.0, 70.0], [50.0, 60.0, 70.0]])
    E, F, ph, W = O.real_space(pos, q, L, 1e-13, 30.0, slater=lam)
    assert abs(E - q[0] * q[1] / lam) < 1e-12 and np.abs(F).max() == 0.0


def test_slater_reduces_to_point_charges_for_small_decay_length():
    """lambda_e -> 0 gives back the point-charge real-space sum."""
    g = np.random.default_rng(31)
    L = np.array([14.0, 15.0, 16.0])
    pos = g.uniform(0, 1, size=(40, 3)) * L
    q = g.normal(size=40)
    a = O.real_space(pos, q, L, 0.4, 6.0)
    b = O.real_space(pos, q, L, 0.4, 6.0, slater=1e-4)
    assert abs(a[0] / b[0] - 1) < 1e-12
    assert np.abs(a[1] - b[1]).max() < 1e-12 * np.abs(a[1]).max()
    assert np.abs(a[3] - b[3]).max() < 1e-12 * np.abs(a[3]).max()


# ------------------------------------------------------------------ time stepping (velocity Verlet)
def test_verlet_free_flight_and_constant_force_are_exact():
    """Without forces the trajectory is r0 + v t (wrapped); under a constant
    force velocity Verlet is exact: r0 + v0 t + a t^2 / 2, v0 + a t."""
    from oracle import md
    g = np.random.default_rng(40)
    L = np.array([5.0, 6.0, 7.0])
    r0 = g.uniform(0, 1, size=(10, 3)) * L
    v0 = g.normal(size=(10, 3))
    im = g.uniform(0.5, 2.0, size=10)
    dt, n = 0.01, 137
    pos, vel, _, _ = md.verlet(r0, v0, im, L, dt, n, lambda x: (0.0, np.zeros_like(x)))
    t = dt * n
    want = np.mod(r0 + v0 * t, L)
    d = np.abs(pos - want)
    assert np.minimum(d, L - d).max() < 1e-12 and np.abs(vel - v0).max() == 0.0
    f = g.normal(size=(10, 3))
    rc = r0 + 5e5  # in the middle of a box too large to wrap
    pos, vel, _, _ = md.verlet(rc, v0, im, np.full(3, 1e6), dt, n, lambda x: (0.0, f))
    a = im[:, None] * f
    assert np.abs(pos - (rc + v0 * t + 0.5 * a * t * t)).max() < 1e-8
    assert np.abs(vel - (v0 + a * t)).max() < 1e-12


def test_verlet_energy_error_is_second_order_on_a_harmonic_oscillator():
    """Velocity Verlet on x'' = -w^2 x: the energy error stays bounded and
    scales as dt^2 (halving dt divides it by 4)."""
    from oracle import md
    L = np.full(3, 1e6)
    k = 3.0
    forces = lambda x: (0.5 * k * ((x - 5e5) ** 2).sum(), -k * (x - 5e5))
    r0 = np.array([[5e5 + 1.0, 5e5, 5e5]])
    v0 = np.array([[0.0, 0.7, 0.0]])
    errs = []
    for dt in [0.02, 0.01]:
        n = int(round(20.0 / dt))
        _, _, _, en = md.verlet(r0, v0, [1.0], L, dt, n, forces)
        E0 = 0.5 * k * 1.0 + 0.5 * 0.49
        errs.append(np.abs(en[:, 2] - E0).max() / E0)
    assert errs[0] < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5
