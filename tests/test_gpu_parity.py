"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative): FP64 plans 1e-12 for E, F, phi and the virial;
mixed plans 1e-6 for E and 1e-5 for the RMS of F (and phi, virial).  Mixed
plans receive float32 inputs and the oracle the same float32 values.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2004_12484_b300 as P  # noqa: E402

DEV = torch.device("cuda", 0)
TOL = {"fp64": dict(E=1e-12, F=1e-12, phi=1e-12, W=1e-12), "mixed": dict(E=1e-6, F=1e-5, phi=1e-5, W=1e-5)}


def energy_scale(ref):
    """The size of the terms whose sum is E.  Float rounding is relative to
    these terms, so random-charge systems whose total is a cancellation of
    larger terms are measured against this scale; the workload checks use
    the total energy itself."""
    return max(abs(ref.E), abs(ref.E_real) + abs(ref.E_recip) + abs(ref.E_self) + abs(ref.E_background))


def rel_rms(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def run(pos, q, L, alpha, rc, M, p, nc, precision, phi=True, kspace_only=False):
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = P.Plan(L=L, N=len(q), alpha=alpha, r_c=rc, M=M, p=p, n_c=nc, precision=precision, device=DEV)
    tp = torch.tensor(pos, dtype=dt, device=DEV)
    tq = torch.tensor(q, dtype=dt, device=DEV)
    parts, F, Wv, ph = plan.energy_forces(tp, tq, phi=phi, kspace_only=kspace_only)
    return parts, F.cpu().double().numpy(), Wv, (ph.cpu().double().numpy() if ph is not None else None)


def inputs(pos, q, precision):
    return W.as_fp32(pos, q) if precision == "mixed" else (pos, q)


def check_full(pos, q, L, alpha, rc, M, p, nc, precision, escale=False):
    pos, q = inputs(pos, q, precision)
    parts, F, Wv, ph = run(pos, q, L, alpha, rc, M, p, nc, precision)
    ref = O.nfft_ewald(pos, q, L, alpha, rc, M, p, nc)
    t = TOL[precision]
    den = energy_scale(ref) if escale else abs(ref.E)
    assert abs(parts["E"] - ref.E) < t["E"] * den, (parts, ref.E, ref.E_real, ref.E_recip, ref.E_self)
    assert abs(parts["E_recip"] - ref.E_recip) < t["E"] * max(abs(ref.E_recip), den)
    assert abs(parts["E_real"] - ref.E_real) < t["E"] * max(abs(ref.E_real), den)
    if len(q) == 1:
        # a single ion: the force vanishes by symmetry
        assert np.abs(F).max() < (1e-14 if precision == "fp64" else 1e-6) * alpha ** 2
    else:
        assert rel_rms(F, ref.F) < t["F"]
    assert rel_rms(ph, ref.phi) < t["phi"]
    assert np.abs(Wv - ref.virial).max() < t["W"] * np.abs(ref.virial).max()
    return parts, ref


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nacl_config(precision):
    """512-ion rock salt, grid 32^3, p = 4 (the FP64 parity workload)."""
    d = W.nacl()
    check_full(d["pos"], d["q"], d["L"], d["alpha"], d["r_c"], d["M"], d["p"], d["n_c"], precision)


CASES = [
    # (N, L, alpha, rc, M, p, nc, seed)
    (300, (12.0, 13.0, 14.0), 0.5, 5.5, 16, 2, 0, 1),
    (300, (12.0, 13.0, 14.0), 0.5, 5.5, 32, 6, 7, 2),
    (700, (20.0, 20.0, 20.0), 0.35, 6.5, 32, 8, 10, 3),
    (1000, (25.0, 18.0, 30.0), 0.3, 8.0, 64, 10, 16, 4),
    (517, (16.0, 16.0, 16.0), 0.45, 5.0, 64, 12, 0, 5),
    (2000, (40.0, 40.0, 40.0), 0.3, 9.0, 8, 4, 3, 6),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_random_systems(case, precision):
    """Random neutral systems across grid sizes, window widths, cutoffs and
    anisotropic boxes, with positions outside the box (wrapping)."""
    N, L, alpha, rc, M, p, nc, seed = case
    g = np.random.default_rng(seed)
    L = np.array(L)
    pos = g.uniform(-1.0, 2.0, size=(N, 3)) * L
    q = g.normal(size=N)
    q -= q.mean()
    check_full(pos, q, L, alpha, rc, M, p, nc or M // 4, precision, escale=True)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_non_neutral_and_single_ion(precision):
    """Net charge: background term (and its potential shift); a single ion
    (Wigner lattice) is the degenerate N = 1 case."""
    g = np.random.default_rng(8)
    L = np.full(3, 15.0)
    pos = g.uniform(0, 15, size=(200, 3))
    q = g.normal(size=200) + 0.3
    check_full(pos, q, L, 0.5, 6.0, 32, 6, 8, precision, escale=True)
    parts, _ = check_full(np.array([[1.0, 2.0, 3.0]]), np.array([1.0]), np.full(3, 10.0), 0.6, 4.9, 32, 8, 8,
                          precision)
    assert abs(parts["E"] / (-2.837297 / 20.0) - 1) < 2e-4


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_all_particles_in_one_tile(precision):
    """Heavy-bin splitting: 3000 particles inside one 8^3 tile."""
    g = np.random.default_rng(9)
    L = np.full(3, 32.0)
    pos = 1.0 + g.uniform(0, 7.0, size=(3000, 3))
    q = g.normal(size=3000)
    q -= q.mean()
    check_full(pos, q, L, 0.4, 7.0, 32, 6, 8, precision, escale=True)


def test_rpm_config_kspace_full_size():
    """RPM electrolyte at full size (N = 65,536, grid 128^3, p = 6, mixed):
    reciprocal part element by element against the oracle."""
    d = W.rpm()
    pos, q = W.as_fp32(d["pos"], d["q"])
    parts, F, Wv, ph = run(pos, q, d["L"], d["alpha"], d["r_c"], d["M"], d["p"], d["n_c"], "mixed",
                           kspace_only=True)
    Ek, Fk, phik, Wk = O.kspace_nfft(pos, q, d["L"], d["alpha"], d["M"], d["p"], d["n_c"])
    assert abs(parts["E"] / Ek - 1) < 1e-6
    assert rel_rms(F, Fk) < 1e-5
    assert rel_rms(ph, phik) < 1e-5
    assert np.abs(Wv - Wk).max() < 1e-5 * np.abs(Wk).max()


def test_rpm_1e4_kspace_full_size():
    """The benchmark's workload (RPM electrolyte, N = 65,536, grid 128^3,
    p = 8, mixed) at full size in the launch configuration the benchmark
    times (16-cell tiles of 8^3 sub-tiles, staged interpolation): reciprocal
    part element by element against the oracle."""
    d = W.rpm_1e4()
    pos, q = W.as_fp32(d["pos"], d["q"])
    parts, F, Wv, ph = run(pos, q, d["L"], d["alpha"], d["r_c"], d["M"], d["p"], d["n_c"], "mixed",
                           kspace_only=True)
    Ek, Fk, phik, Wk = O.kspace_nfft(pos, q, d["L"], d["alpha"], d["M"], d["p"], d["n_c"])
    assert abs(parts["E"] / Ek - 1) < 1e-6
    assert rel_rms(F, Fk) < 1e-5
    assert rel_rms(ph, phik) < 1e-5
    assert np.abs(Wv - Wk).max() < 1e-5 * np.abs(Wk).max()


def check_kspace(pos, q, L, alpha, M, p, nc):
    """Mixed-precision reciprocal part (E, F, phi, virial) against the oracle."""
    pos, q = W.as_fp32(pos, q)
    parts, F, Wv, ph = run(pos, q, L, alpha, 0.45 * min(L), M, p, nc, "mixed", kspace_only=True)
    Ek, Fk, phik, Wk = O.kspace_nfft(pos, q, L, alpha, M, p, nc)
    assert abs(parts["E"] / Ek - 1) < 1e-6
    assert rel_rms(F, Fk) < 1e-5
    assert rel_rms(ph, phik) < 1e-5
    assert np.abs(Wv - Wk).max() < 1e-5 * np.abs(Wk).max()


@pytest.mark.parametrize("p", [2, 4, 6, 8])
def test_sixteen_cell_tiles_small_grid(p, monkeypatch):
    """16-cell tiles split into 8^3 sub-tiles (the layout of float grids of
    edge >= 128) forced on a 32^3 grid: a random system with wrapping, and a
    heavy tile whose sub-tiles are cut into several spreading items and
    whose tile into several interpolation items.  The reciprocal part is
    compared (the tile layout only concerns it; the real-space sum of these
    dense random systems carries the float error of its closest pairs)."""
    monkeypatch.setenv("ENUF_TILE", "16")
    g = np.random.default_rng(30 + p)
    L = np.array([22.0, 25.0, 27.0])
    pos = g.uniform(-1.0, 2.0, size=(2500, 3)) * L
    q = g.normal(size=2500)
    q -= q.mean()
    check_kspace(pos, q, L, 0.4, 32, p, 8)
    h = L / 32
    pos = (3.0 + g.uniform(0, 12.0, size=(1500, 3))) * h  # inside one 16-cell tile
    q = g.normal(size=1500)
    q -= q.mean()
    check_kspace(pos, q, L, 0.4, 32, p, 8)


def test_rpm_config_real_space_sampled():
    """Full RPM step: the real-space part on sampled particles (the oracle
    sums every pair for each sampled particle)."""
    d = W.rpm()
    pos, q = W.as_fp32(d["pos"], d["q"])
    parts, F, Wv, ph = run(pos, q, d["L"], d["alpha"], d["r_c"], d["M"], d["p"], d["n_c"], "mixed")
    _, Fk, _, phik = run(pos, q, d["L"], d["alpha"], d["r_c"], d["M"], d["p"], d["n_c"], "mixed", kspace_only=True)
    idx = np.random.default_rng(22).choice(len(q), 256, replace=False)
    _, Fr, phir, _ = O.real_space(pos, q, d["L"], d["alpha"], d["r_c"], idx=idx)
    assert rel_rms(F[idx] - Fk[idx], Fr) < 1e-5
    self_phi = -2 * d["alpha"] / np.sqrt(np.pi) * q[idx]
    assert rel_rms(ph[idx] - phik[idx], phir + self_phi) < 1e-5
    # E_real = 1/2 sum_i q_i phi_real,i (checked on the device output)
    phir_all = ph - phik - (-2 * d["alpha"] / np.sqrt(np.pi) * q)
    assert abs(0.5 * (q * phir_all).sum() / parts["E_real"] - 1) < 1e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_invariants_translation_and_net_force(precision):
    """Shift by whole grid cells leaves the result unchanged; the sum of the
    reciprocal forces vanishes (momentum conservation)."""
    d = W.rpm(N=4096, seed=12, M=32, p=6, r_c=10.0, alpha=0.3)
    pos, q = inputs(d["pos"], d["q"], precision)
    L = d["L"]
    a = run(pos, q, L, d["alpha"], d["r_c"], 32, 6, 8, precision, kspace_only=True)
    h = L[0] / 32
    b = run(pos + np.array([2, -3, 5]) * h, q, L, d["alpha"], d["r_c"], 32, 6, 8, precision, kspace_only=True)
    tol = 1e-12 if precision == "fp64" else 2e-5
    assert abs(a[0]["E"] / b[0]["E"] - 1) < tol
    assert rel_rms(a[1], b[1]) < tol * 10
    Fsum = np.abs(a[1].sum(0)).max()
    assert Fsum < (1e-12 if precision == "fp64" else 1e-6) * np.abs(a[1]).sum()


def test_remove_net_force_flag():
    d = W.rpm(N=4096, seed=13, M=32, p=6, r_c=10.0, alpha=0.3)
    plan = P.Plan(L=d["L"], N=4096, alpha=0.3, r_c=10.0, M=32, p=6, precision="fp64", device=DEV)
    tp = torch.tensor(d["pos"], dtype=torch.float64, device=DEV)
    tq = torch.tensor(d["q"], dtype=torch.float64, device=DEV)
    _, F0, _, _ = plan.energy_forces(tp, tq)
    _, F1, _, _ = plan.energy_forces(tp, tq, remove_net_force=True)
    F0 = F0.cpu().numpy(); F1 = F1.cpu().numpy()
    assert np.abs(F1.sum(0)).max() < 1e-10 * np.abs(F1).sum()
    assert np.abs((F0 - F1) - F0.mean(0)).max() < 1e-12 * np.abs(F0).max()


def test_fp64_determinism_and_graph_replay():
    """Two replays of the captured graph agree to rounding (atomics reorder
    sums), and a fresh capture for new buffers gives the same values."""
    d = W.rpm(N=8192, seed=14, M=64, p=8, r_c=10.0, alpha=0.3)
    plan = P.Plan(L=d["L"], N=8192, alpha=0.3, r_c=10.0, M=64, p=8, precision="fp64", device=DEV)
    tp = torch.tensor(d["pos"], dtype=torch.float64, device=DEV)
    tq = torch.tensor(d["q"], dtype=torch.float64, device=DEV)
    F = torch.empty((8192, 3), dtype=torch.float64, device=DEV)
    out = torch.empty(16, dtype=torch.float64, device=DEV)
    plan.compute(tp, tq, F=F, out=out)
    e1, f1 = out.clone(), F.clone()
    plan.compute(tp, tq, F=F, out=out)
    assert abs(float(out[0] / e1[0]) - 1) < 1e-13
    assert float((F - f1).abs().max() / f1.abs().max()) < 1e-13
    o2, F2, _ = plan.compute(tp.clone(), tq.clone())
    assert abs(float(o2[0] / e1[0]) - 1) < 1e-13


def test_nonfinite_input_is_reported():
    plan = P.Plan(L=(20.0,) * 3, N=64, alpha=0.4, r_c=8.0, M=16, p=4, precision="mixed", device=DEV)
    tp = torch.rand((64, 3), device=DEV) * 20
    tq = torch.ones(64, device=DEV)
    tp[5, 1] = float("nan")
    with pytest.raises(P.EnufError, match="NaN"):
        plan.energy_forces(tp, tq)
    # the plan stays usable
    tp[5, 1] = 1.0
    plan.energy_forces(tp, tq)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_reciprocal_part_is_linear_over_a_particle_partition(precision):
    """The spread grid, its spectrum and hence the reciprocal potential are
    linear in the charges (the structure factor is additive over any
    partition of the particles, which a particle-sharded multi-GPU run
    relies on): with the charges of two disjoint subsets evaluated
    separately (the other subset's charges zero), the reciprocal potentials
    sum to those of the whole system, and the energies satisfy
    E(A + B) = E(A) + E(B) + cross term with cross = sum_{i in B} q_i phi_A(i)."""
    g = np.random.default_rng(41)
    L = np.array([24.0, 26.0, 28.0])
    N = 3000
    pos = g.uniform(0, 1, size=(N, 3)) * L
    q = g.normal(size=N)
    q -= q.mean()
    pos, q = inputs(pos, q, precision)
    inA = g.random(N) < 0.4
    qA = np.where(inA, q, 0.0)
    qB = np.where(inA, 0.0, q)
    res = {}
    for name, qq in (("all", q), ("A", qA), ("B", qB)):
        parts, F, Wv, ph = run(pos, qq, L, 0.4, 8.0, 32, 6, 8, precision, kspace_only=True)
        res[name] = (parts["E"], ph)
    tol = 1e-11 if precision == "fp64" else 2e-6
    phi_sum = res["A"][1] + res["B"][1]
    assert rel_rms(phi_sum, res["all"][1]) < tol
    cross = float((qB * res["A"][1]).sum())
    E_sum = res["A"][0] + res["B"][0] + cross
    assert abs(E_sum - res["all"][0]) < tol * 10 * (abs(res["A"][0]) + abs(res["B"][0]) + abs(cross))


def test_host_buffer_entry_point_matches_device_call():
    d = W.rpm(N=4096, seed=15, M=32, p=6, r_c=10.0, alpha=0.3)
    pos, q = W.as_fp32(d["pos"], d["q"])
    plan = P.Plan(L=d["L"], N=4096, alpha=0.3, r_c=10.0, M=32, p=6, precision="mixed", device=DEV)
    ph = torch.tensor(pos, dtype=torch.float32).pin_memory()
    qh = torch.tensor(q, dtype=torch.float32).pin_memory()
    Fh = torch.empty((4096, 3), dtype=torch.float32).pin_memory()
    E, Wv = plan.energy_forces_host(ph, qh, F_host=Fh)
    parts, F, W2, _ = plan.energy_forces(ph.to(DEV), qh.to(DEV))
    # float atomics make the two calls differ at float rounding
    assert abs(E / parts["E"] - 1) < 1e-6
    assert float((Fh - F.cpu()).abs().max()) < 1e-5 * float(F.abs().max())
    assert np.abs(Wv - W2).max() < 1e-5 * np.abs(W2).max()


def test_host_buffer_entry_point_pageable_pinned_and_repeated():
    """Pageable host buffers (copies issued one by one) and pinned ones (the
    copies captured in the cached graph) give the same results; a second call
    on the same pinned buffers after the positions were rewritten in place
    sees the new positions (the graph copies at every launch)."""
    a = W.rpm(N=4096, seed=15, M=32, p=6, r_c=10.0, alpha=0.3)
    b = W.rpm(N=4096, seed=16, M=32, p=6, r_c=10.0, alpha=0.3)
    pos_a, q = W.as_fp32(a["pos"], a["q"])
    pos_b, _ = W.as_fp32(b["pos"], b["q"])
    plan = P.Plan(L=a["L"], N=4096, alpha=0.3, r_c=10.0, M=32, p=6, precision="mixed", device=DEV)
    F1 = np.empty((4096, 3), dtype=np.float32)
    phi1 = np.empty(4096, dtype=np.float32)
    E1, W1 = plan.energy_forces_host(np.ascontiguousarray(pos_a, dtype=np.float32),
                                     np.ascontiguousarray(q, dtype=np.float32), phi_host=phi1, F_host=F1)
    ph = torch.tensor(pos_a, dtype=torch.float32).pin_memory()
    qh = torch.tensor(q, dtype=torch.float32).pin_memory()
    Fh = torch.empty((4096, 3), dtype=torch.float32).pin_memory()
    phih = torch.empty(4096, dtype=torch.float32).pin_memory()
    E2, W2 = plan.energy_forces_host(ph, qh, phi_host=phih, F_host=Fh)
    assert abs(E2 / E1 - 1) < 1e-6
    assert rel_rms(Fh.double().numpy(), F1.astype(np.float64)) < 1e-5
    assert rel_rms(phih.double().numpy(), phi1.astype(np.float64)) < 1e-5
    assert np.abs(W2 - W1).max() < 1e-5 * np.abs(W1).max()
    ph.copy_(torch.tensor(pos_b, dtype=torch.float32))
    E3, W3 = plan.energy_forces_host(ph, qh, phi_host=phih, F_host=Fh)
    parts, F, Wd, phid = plan.energy_forces(ph.to(DEV), qh.to(DEV), phi=True)
    assert abs(E3 / parts["E"] - 1) < 1e-6 and abs(E3 / E2 - 1) > 1e-4
    assert rel_rms(Fh.double().numpy(), F.cpu().double().numpy()) < 1e-5
    assert rel_rms(phih.double().numpy(), phid.cpu().double().numpy()) < 1e-5
    assert np.abs(W3 - Wd).max() < 1e-5 * np.abs(Wd).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_unfused_fft_passes_match_fused(precision, monkeypatch):
    """Grids up to 256 use the fused x-y FFT kernels; the separate-pass
    kernels (used for 512 and below 32) are checked at the same size."""
    monkeypatch.setenv("ENUF_NO_FUSED_XY", "1")
    g = np.random.default_rng(16)
    L = np.array([30.0, 30.0, 30.0])
    pos = g.uniform(0, 30, size=(1500, 3))
    q = g.normal(size=1500)
    q -= q.mean()
    check_full(pos, q, L, 0.35, 8.0, 64, 6, 16, precision, escale=True)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_staged_gather_matches(precision, monkeypatch):
    """Small grids interpolate straight from L2-resident fields; the
    shared-memory staged kernel (used for large grids) is checked here on a
    small one."""
    monkeypatch.setenv("ENUF_STAGED_GATHER", "1")
    g = np.random.default_rng(17)
    L = np.array([26.0, 29.0, 31.0])
    pos = g.uniform(0, 30, size=(1800, 3))
    q = g.normal(size=1800)
    q -= q.mean()
    check_full(pos, q, L, 0.35, 8.0, 32, 8, 8, precision, escale=True)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_positions_on_cell_and_box_boundaries(precision):
    """Positions exactly on grid-cell faces, on the box faces (0 and L),
    just below L (float rounding can carry them to L), and several boxes
    away in both directions are wrapped and binned consistently."""
    g = np.random.default_rng(18)
    L = np.array([24.0, 24.0, 24.0])
    M = 32
    h = L[0] / M
    n = 600
    cells = g.integers(0, M, size=(n, 3)).astype(np.float64) * h
    pos = cells.copy()
    pos[: n // 4] += g.uniform(0, h, size=(n // 4, 3))
    pos[n // 4: n // 4 + 20, 0] = L[0] - 1e-7
    pos[n // 4 + 20: n // 4 + 40, 1] = 0.0
    pos[n // 4 + 40: n // 4 + 60] += 3 * L
    pos[n // 4 + 60: n // 4 + 80] -= 5 * L
    # drop exact duplicates (coincident charges have no finite energy)
    _, keep = np.unique(np.round(np.mod(pos, L), 9), axis=0, return_index=True)
    pos = pos[np.sort(keep)]
    q = g.normal(size=len(pos))
    q -= q.mean()
    check_full(pos, q, L, 0.4, 8.0, M, 6, 8, precision, escale=True)


@pytest.mark.parametrize("p", [2, 4, 6, 8])
def test_persistent_interpolation_forces_only(p, monkeypatch):
    """Forces without the potential on 16-cell tiles (for p = 8 and 6 the
    TMA-staged interpolation with z-accumulated window rows): a random system
    with wrapping and a heavy tile cut into several work items on a 32^3
    grid, against the oracle."""
    monkeypatch.setenv("ENUF_TILE", "16")
    g = np.random.default_rng(60 + p)
    L = np.array([22.0, 25.0, 27.0])
    for pos in (g.uniform(-1.0, 2.0, size=(2500, 3)) * L, (3.0 + g.uniform(0, 12.0, size=(2500, 3))) * (L / 32)):
        q = g.normal(size=len(pos))
        q -= q.mean()
        pos, q = W.as_fp32(pos, q)
        parts, F, Wv, _ = run(pos, q, L, 0.4, 0.45 * min(L), 32, p, 8, "mixed", phi=False, kspace_only=True)
        Ek, Fk, _, Wk = O.kspace_nfft(pos, q, L, 0.4, 32, p, 8)
        assert abs(parts["E"] / Ek - 1) < 1e-6
        assert rel_rms(F, Fk) < 1e-5


@pytest.mark.parametrize("workload", ["rpm_1e4", "rpm"])
def test_rpm_1e4_forces_only_full_size(workload):
    """The benchmark's call (k-space energy and forces, no potential) on its
    workload at full size, and on the RPM system's stated p = 6 settings that
    it times beside it: forces element by element against the oracle."""
    d = getattr(W, workload)()
    pos, q = W.as_fp32(d["pos"], d["q"])
    parts, F, Wv, _ = run(pos, q, d["L"], d["alpha"], d["r_c"], d["M"], d["p"], d["n_c"], "mixed", phi=False,
                          kspace_only=True)
    Ek, Fk, _, Wk = O.kspace_nfft(pos, q, d["L"], d["alpha"], d["M"], d["p"], d["n_c"])
    assert abs(parts["E"] / Ek - 1) < 1e-6
    assert rel_rms(F, Fk) < 1e-5
    assert np.abs(Wv - Wk).max() < 1e-5 * np.abs(Wk).max()


def test_plan_call_returns_energy_forces_virial():
    """plan(pos, q) -> (E, F, virial), the binding's short form, against the
    oracle on the rock-salt workload (FP64)."""
    d = W.nacl()
    plan = P.Plan(L=d["L"], N=len(d["q"]), alpha=d["alpha"], r_c=d["r_c"], M=d["M"], p=d["p"], n_c=d["n_c"],
                  precision="fp64", device=DEV)
    E, F, Wv = plan(torch.tensor(d["pos"], device=DEV), torch.tensor(d["q"], device=DEV))
    ref = O.nfft_ewald(d["pos"], d["q"], d["L"], d["alpha"], d["r_c"], d["M"], d["p"], d["n_c"])
    assert abs(E / ref.E - 1) < 1e-12
    assert rel_rms(F.cpu().numpy(), ref.F) < 1e-12
    assert np.abs(Wv - ref.virial).max() < 1e-12 * np.abs(ref.virial).max()


@pytest.mark.parametrize("env", [{"ENUF_TILE": "16", "ENUF_GATHER_FULL_TILE": "1"}, {"ENUF_FZ_W": "16"},
                                 {"ENUF_NO_PDL": "1"}, {"ENUF_NO_GRAPH": "1"},
                                 {"ENUF_TILE": "16", "ENUF_LEGACY_GATHER": "1"}])
def test_alternative_launch_configurations(env, monkeypatch):
    """The plan-creation switches that select other launch configurations
    (whole 16-cell interpolation tiles, another z-pass width, no
    programmatic dependent launch, direct launches instead of graphs, the
    generic interpolation kernel for p = 8 and 6 instead of their own) give
    the same results: forces only and with the potential, against the
    oracle."""
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    g = np.random.default_rng(70)
    L = np.array([22.0, 25.0, 27.0])
    pos = g.uniform(-1.0, 2.0, size=(2500, 3)) * L
    q = g.normal(size=2500)
    q -= q.mean()
    for p in (8, 6) if "ENUF_LEGACY_GATHER" in env else (8,):
        check_kspace(pos, q, L, 0.4, 32, p, 8)
        pos32, q32 = W.as_fp32(pos, q)
        parts, F, _, _ = run(pos32, q32, L, 0.4, 0.45 * min(L), 32, p, 8, "mixed", phi=False, kspace_only=True)
        Ek, Fk, _, _ = O.kspace_nfft(pos32, q32, L, 0.4, 32, p, 8)
        assert abs(parts["E"] / Ek - 1) < 1e-6
        assert rel_rms(F, Fk) < 1e-5
