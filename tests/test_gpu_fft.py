"""The hand-written forward 3D FFT against cuFFT, and the structure factor
(the transposed NFFT: spread, FFT, scaling) against the oracle.

cuFFT (through torch.fft) is used here only as a comparison, as the paper's
CU-NFFT pipeline calls it for its transforms (Sec. 3.1); the library never
calls it.  Each FFT is compared with an FP64 cuFFT transform of the same
grid, so the single-precision tolerance bounds each one's own rounding."""
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


def rel_rms(a, b):
    a = a.to(torch.complex128)
    b = b.to(torch.complex128)
    return float((a - b).abs().pow(2).sum().sqrt() / b.abs().pow(2).sum().sqrt())


def kept(full, nc):
    """The retained half cube [n_z + nc, n_y + nc, n_x] of an rfftn output
    indexed [k_z, k_y, k_x]."""
    M = full.shape[0]
    band = torch.tensor(list(range(M - nc, M)) + list(range(0, nc + 1)), device=full.device)
    return full.index_select(0, band).index_select(1, band)[:, :, : nc + 1]


@pytest.mark.parametrize("M", [32, 128, 256, 512])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_forward_fft_matches_cufft(M, precision):
    dt = torch.float64 if precision == "fp64" else torch.float32
    g = torch.Generator().manual_seed(M)
    grid64 = torch.randn((M, M, M), generator=g, dtype=torch.float64).to(DEV)
    grid = grid64.to(dt).contiguous()
    plan = P.Plan(L=(10.0, 10.0, 10.0), N=8, alpha=1.0, r_c=4.0, M=M, p=4, precision=precision, device=DEV)
    nc = plan.n_c
    mine = plan.fft_forward(grid)
    torch.cuda.synchronize()
    ref = kept(torch.fft.rfftn(grid.double(), dim=(0, 1, 2)), nc)  # the rounded input, transformed in FP64
    cu = kept(torch.fft.rfftn(grid, dim=(0, 1, 2)), nc)             # cuFFT in the plan's precision
    e_mine, e_cu = rel_rms(mine, ref), rel_rms(cu, ref)
    print(f"M={M} {precision}: hand FFT {e_mine:.2e}, cuFFT {e_cu:.2e} (relative RMS against FP64)")
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert e_mine < tol
    assert e_cu < tol
    # the grid buffer of the plan is left zeroed: a second call gives the same
    again = plan.fft_forward(grid)
    assert rel_rms(again, mine) < (1e-15 if precision == "fp64" else 1e-7)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("M,p", [(32, 6), (64, 8)])
def test_structure_factor_matches_oracle(precision, tol, M, p):
    g = np.random.default_rng(51)
    N, L = 700, np.array([21.0, 23.0, 25.0])
    pos = g.uniform(-0.5, 1.5, size=(N, 3)) * L
    q = g.normal(size=N)
    if precision == "mixed":
        pos, q = W.as_fp32(pos, q)
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = P.Plan(L=L, N=N, alpha=0.4, r_c=8.0, M=M, p=p, precision=precision, device=DEV)
    nc = plan.n_c
    S = plan.structure_factor(torch.tensor(pos, dtype=dt, device=DEV), torch.tensor(q, dtype=dt, device=DEV))
    ref = O.structure_factor_nfft(pos, q, L, M, p, nc)[:, :, nc:]
    assert rel_rms(S.cpu(), torch.from_numpy(ref)) < tol


def test_structure_factor_is_additive_and_checks_inputs():
    """S~ of a union is the sum of the partial structure factors (Sec. 3.3),
    to rounding in FP64; a NaN position is reported and the plan stays usable."""
    g = np.random.default_rng(52)
    N, L = 4000, np.full(3, 40.0)
    pos = g.uniform(0, 40.0, size=(N, 3))
    q = g.normal(size=N)
    kw = dict(L=L, alpha=0.3, r_c=10.0, M=64, p=8, precision="fp64", device=DEV)
    whole = P.Plan(N=N, **kw)
    a, b = 1500, N - 1500
    pa, pb = P.Plan(N=a, **kw), P.Plan(N=b, **kw)
    tp = torch.tensor(pos, dtype=torch.float64, device=DEV)
    tq = torch.tensor(q, dtype=torch.float64, device=DEV)
    S = whole.structure_factor(tp, tq)
    Sa = pa.structure_factor(tp[:a].contiguous(), tq[:a].contiguous())
    Sb = pb.structure_factor(tp[a:].contiguous(), tq[a:].contiguous())
    assert rel_rms(Sa + Sb, S) < 1e-12
    bad = tp.clone()
    bad[17, 1] = float("nan")
    with pytest.raises(P.EnufError):
        whole.structure_factor(bad, tq)
    again = whole.structure_factor(tp, tq)
    assert rel_rms(again, S) < 1e-13
    # an evaluation after the reported failure is unaffected
    parts, F, _, _ = whole.energy_forces(tp, tq)
    assert np.isfinite(parts["E"]) and torch.isfinite(F).all()


@pytest.mark.parametrize("M", [128, 256, 512])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-6)])
def test_wide_z_pass_matches_narrow(M, precision, tol, monkeypatch):
    """At M = 512 (and 128 and 256 in single precision) the z pass is k_fzw
    (radix 8, fields one after the other); ENUF_FZ_NARROW=1 selects k_fz, the z pass
    of the smaller grids, which the oracle checks at M <= 256.  Both give
    the same energy, forces, potentials and virial (a small system)."""
    g = np.random.default_rng(90)
    N, L = 3000, np.array([60.0, 64.0, 68.0])
    pos = g.uniform(0, 1, size=(N, 3)) * L
    q = g.normal(size=N)
    q -= q.mean()
    dt = torch.float64 if precision == "fp64" else torch.float32
    tp = torch.tensor(pos, dtype=dt, device=DEV)
    tq = torch.tensor(q, dtype=dt, device=DEV)
    res = []
    for narrow in (False, True):
        if narrow:
            monkeypatch.setenv("ENUF_FZ_NARROW", "1")
        plan = P.Plan(L=L, N=N, alpha=0.5, r_c=10.0, M=M, p=4, precision=precision, device=DEV)
        parts, F, Wv, ph = plan.energy_forces(tp, tq, phi=True, kspace_only=True)
        res.append((parts["E"], F.cpu().double(), Wv, ph.cpu().double()))
        del plan
        torch.cuda.empty_cache()
    (E0, F0, W0, p0), (E1, F1, W1, p1) = res
    assert abs(E0 / E1 - 1) < tol
    assert rel_rms(F0, F1) < tol
    assert rel_rms(p0, p1) < tol
    assert np.abs(W0 - W1).max() < tol * np.abs(W1).max()


@pytest.mark.parametrize("M", [128, 256, 512])
def test_energy_only_evaluation_on_the_wide_z_pass(M):
    """An evaluation without forces or potentials runs the z pass alone (no
    field transforms, no interpolation): its energy and virial equal those of
    a forces evaluation, before and after it (the grid is left cleared
    either way), and the k-space energy agrees with the oracle."""
    g = np.random.default_rng(93)
    N, L = 2000, np.array([60.0, 64.0, 68.0])
    pos = g.uniform(0, 1, size=(N, 3)) * L
    q = g.normal(size=N)
    q -= q.mean()
    pos32, q32 = W.as_fp32(pos, q)
    tp = torch.tensor(pos32, dtype=torch.float32, device=DEV)
    tq = torch.tensor(q32, dtype=torch.float32, device=DEV)
    plan = P.Plan(L=L, N=N, alpha=0.5, r_c=10.0, M=M, p=4, precision="mixed", device=DEV)
    e0, _, _ = plan.compute(tp, tq, forces=False, kspace_only=True)
    parts, F, Wv, _ = plan.energy_forces(tp, tq, kspace_only=True)
    e1, _, _ = plan.compute(tp, tq, forces=False, kspace_only=True)
    e0, e1 = e0.cpu().numpy(), e1.cpu().numpy()
    assert abs(e0[0] / parts["E"] - 1) < 1e-6 and abs(e1[0] / parts["E"] - 1) < 1e-6
    assert np.abs(e0[6:15] - Wv.reshape(-1)).max() < 1e-6 * np.abs(Wv).max()
    if M == 128:
        Ek, _, _, _ = O.kspace_nfft(pos32, q32, L, 0.5, M, 4, M // 4)
        assert abs(e0[2] / Ek - 1) < 1e-6  # the reciprocal energy
