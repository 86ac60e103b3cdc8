"""Parity of the ENUF-DPD real-space correction (smeared Slater-type charges,
Eq. 51-60: each real-space pair energy times B_U, each pair force times B_F)
with the FP64 CPU oracle, through the C ABI.

Tolerances as for point charges: FP64 plans 1e-12 relative, mixed plans
1e-6 for E and 1e-5 for the RMS of F, phi and the virial (float32 inputs;
the oracle gets the same float32 values).  Smeared charges may overlap, so
the systems include close pairs and coincident ones (finite energy, Eq. 59;
no force, Eq. 60).
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
BETA = 1.125  # R_c / lambda_e of the method's smeared charges


def rel_rms(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def run(pos, q, L, alpha, rc, M, p, nc, lam, precision, kspace_only=False):
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = P.Plan(L=L, N=len(q), alpha=alpha, r_c=rc, M=M, p=p, n_c=nc, precision=precision, device=DEV,
                  slater_lambda=lam)
    tp = torch.tensor(pos, dtype=dt, device=DEV)
    tq = torch.tensor(q, dtype=dt, device=DEV)
    parts, F, Wv, ph = plan.energy_forces(tp, tq, phi=True, kspace_only=kspace_only)
    return parts, F.cpu().double().numpy(), Wv, ph.cpu().double().numpy()


def check(pos, q, L, alpha, rc, M, p, nc, lam, precision):
    if precision == "mixed":
        pos, q = W.as_fp32(pos, q)
    parts, F, Wv, ph = run(pos, q, L, alpha, rc, M, p, nc, lam, precision)
    ref = O.nfft_ewald(pos, q, L, alpha, rc, M, p, nc, slater=lam)
    t = TOL[precision]
    scale = max(abs(ref.E), abs(ref.E_real) + abs(ref.E_recip) + abs(ref.E_self) + abs(ref.E_background))
    assert abs(parts["E"] - ref.E) < t["E"] * scale
    assert abs(parts["E_real"] - ref.E_real) < t["E"] * scale
    assert rel_rms(F, ref.F) < t["F"]
    assert rel_rms(ph, ref.phi) < t["phi"]
    assert np.abs(Wv - ref.virial).max() < t["W"] * np.abs(ref.virial).max()
    return parts, ref


def soft_system(seed, N, L, frac_close=0.2, n_dup=4):
    """Random positions with a share of close pairs (inside 0.05-1 A of
    another particle) and a few exact duplicates; charges normal, neutral."""
    g = np.random.default_rng(seed)
    L = np.asarray(L, dtype=np.float64)
    pos = g.uniform(-0.5, 1.5, size=(N, 3)) * L
    nclose = int(frac_close * N)
    src = g.integers(0, N - nclose, size=nclose)
    v = g.normal(size=(nclose, 3))
    v *= (g.uniform(0.05, 1.0, size=nclose) / np.linalg.norm(v, axis=1))[:, None]
    pos[N - nclose:] = pos[src] + v
    pos[N - nclose - n_dup:N - nclose] = pos[:n_dup]  # coincident with particles 0..n_dup-1
    q = g.normal(size=N)
    q -= q.mean()
    return pos, q


# (N, L, alpha, rc, M, p, nc, lambda_e, seed, stencil3): linked cells with
# the 5^3 stencil, the 3^3 stencil (forced), and the all-pairs kernel
CASES = [
    (1200, (40.0, 42.0, 44.0), 0.2, 12.0, 32, 4, 8, 6.954, 1, False),
    (800, (30.0, 30.0, 30.0), 0.25, 8.5, 32, 6, 8, 3.0, 2, True),
    (300, (16.0, 17.0, 18.0), 0.45, 7.9, 16, 4, 4, 1.5, 3, False),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dpd_random_soft_systems(case, precision, monkeypatch):
    """Random neutral systems with overlapping and coincident smeared
    charges, positions outside the box (wrapping), anisotropic boxes."""
    N, L, alpha, rc, M, p, nc, lam, seed, stencil3 = case
    if stencil3:
        monkeypatch.setenv("ENUF_CELL_STENCIL3", "1")
    pos, q = soft_system(seed, N, L)
    check(pos, q, np.array(L), alpha, rc, M, p, nc, lam, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dpd_coincident_pair_energy_and_no_force(precision):
    """Two opposite charges at one point and a third beyond the cutoff: the
    pair's real-space energy is q1 q2 erfc(0) / lambda_e (Eq. 59) and it
    exerts no force (Eq. 60)."""
    L = np.full(3, 30.0)
    pos = np.array([[10.0, 11.0, 12.0], [10.0, 11.0, 12.0], [22.0, 20.0, 18.0]])
    q = np.array([1.0, -1.0, 0.5])
    parts, ref = check(pos, q, L, 0.3, 9.0, 32, 6, 8, 2.0, precision)
    assert abs(parts["E_real"] - (-1.0 / 2.0)) < 1e-5


def test_dpd_polyelectrolyte_full_size_sampled():
    """The polyelectrolyte workload (N = 1,572,864, r_c = 3 sigma, the
    method's r_c = 3 R_c with R_c = sigma) with smeared charges of lambda_e =
    R_c / 1.125: the total minus the reciprocal part on sampled particles
    against the oracle's smeared real-space sum; the reciprocal part is the
    point-charge one."""
    d = W.polyelectrolyte()
    pos, q = W.as_fp32(d["pos"], d["q"])
    lam = 1.0 / BETA
    plan = P.Plan(L=d["L"], N=len(q), alpha=d["alpha"], r_c=d["r_c"], M=d["M"], p=d["p"], n_c=d["n_c"],
                  precision="mixed", device=DEV, slater_lambda=lam)
    tp = torch.tensor(pos, dtype=torch.float32, device=DEV)
    tq = torch.tensor(q, dtype=torch.float32, device=DEV)
    _, Fk, _, phik = plan.energy_forces(tp, tq, phi=True, kspace_only=True)
    _, F, _, ph = plan.energy_forces(tp, tq, phi=True)
    F, Fk = F.cpu().double().numpy(), Fk.cpu().double().numpy()
    ph, phik = ph.cpu().double().numpy(), phik.cpu().double().numpy()
    idx = np.random.default_rng(5).choice(len(q), 256, replace=False)
    _, Fr, phir, _ = O.real_space(pos, q, d["L"], d["alpha"], d["r_c"], idx=idx, slater=lam)
    assert rel_rms(F[idx] - Fk[idx], Fr) < 1e-5
    self_phi = -2 * d["alpha"] / np.sqrt(np.pi) * q[idx]
    assert rel_rms(ph[idx] - phik[idx], phir + self_phi) < 1e-5
    # the correction matters at this density: the point-charge real space differs
    _, Fr0, _, _ = O.real_space(pos, q, d["L"], d["alpha"], d["r_c"], idx=idx)
    assert rel_rms(Fr0, Fr) > 1e-2
