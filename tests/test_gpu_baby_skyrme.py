"""Baby Skyrme model (Table 1) on the CUDA path vs the FP64 oracle, through the C-ABI.

Same kernels as the other theories, with the mixed derivative of every component
(the Skyrme term) and the unit-vector projection of the chiral magnet. Tolerances
as in test_gpu_parity.py: FP64 1e-11 of the force scale, 1e-10 of the field after
tens of steps; FP32 3e-5 of the force scale and 2e-5 of the field; observables in
FP64 from the stored values 1e-12.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_24370_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BS = 3
PRM = (1.0, 0.7, 0.3)     # kappa, mu, nu
GRID = (79, 45, 0.2, 0.17)  # several 32-wide tiles, ragged, unequal spacings


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_24370_gb300 import build
    from paper_2603_24370_gb300 import soliton as S
    build.build()
    S.load_library()
    return S


def dtype_of(prec):
    return np.float64 if prec == 2 else np.float32


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_force_and_energy_match_oracle(S, prec):
    nx, ny, dx, dy = GRID
    f = I.smooth_field(BS, nx, ny, dx, dy, seed=111).astype(dtype_of(prec))
    with S.Solver(S.SS_BABY_SKYRME, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        G, E, gmax = s.force()
    f64 = f.astype(np.float64)
    Go = O.force(BS, PRM, f64, dx, dy)
    Eo = O.energy(BS, PRM, f64, dx, dy)
    scale = np.abs(Go).max()
    assert np.abs(G.astype(np.float64) - Go).max() <= (1e-11 if prec == 2 else 3e-5) * scale
    assert not G[:, :2, :].any() and not G[:, -2:, :].any() and not G[:, :, :2].any() and not G[:, :, -2:].any()
    esc = np.abs(O.energy_density(BS, PRM, f64, dx, dy)).sum() * dx * dy
    assert abs(E - Eo) <= (1e-12 if prec == 2 else 1e-6) * esc
    assert gmax == pytest.approx(dx * dy * scale, rel=(1e-11 if prec == 2 else 3e-5))


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_trajectory_matches_oracle(S, prec):
    """30 arrested-flow steps from a smooth field at rest: fields, velocity, energy and
    the arrest count against the oracle's RK4 + Eq. 4."""
    nx, ny, dx, dy = GRID
    n = 30
    f = I.smooth_field(BS, nx, ny, dx, dy, seed=222).astype(dtype_of(prec))
    with S.Solver(S.SS_BABY_SKYRME, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        st = s.step(n)
        fg = s.exact_fields() if prec == 1 else s.fields().astype(np.float64)
        vg = s.velocity().astype(np.float64)
    fo, vo = f.astype(np.float64), np.zeros(f.shape)
    E = O.energy(BS, PRM, fo, dx, dy)
    dt = O.time_step(dx, dy)
    arrests = 0
    for _ in range(n):
        fo, vo, E, a = O.anf_step(BS, PRM, fo, vo, dx, dy, dt, E)
        arrests += a
    tol = 1e-10 if prec == 2 else 2e-5
    assert np.abs(fg - fo).max() <= tol
    assert np.abs(vg - vo).max() <= tol / dt
    assert st["steps"] == n
    assert np.abs(np.sqrt((fg * fg).sum(axis=0)) - 1.0).max() < (1e-13 if prec == 2 else 1e-6)
    if prec == 2:
        assert st["arrests"] == arrests
        assert st["energy"] == pytest.approx(E, rel=1e-12)
    else:
        assert st["energy"] == pytest.approx(E, rel=1e-5)


@pytest.mark.parametrize("prec", [1, 2])
def test_descent_matches_oracle(S, prec):
    nx, ny, dx, dy = GRID
    f = I.smooth_field(BS, nx, ny, dx, dy, seed=333).astype(dtype_of(prec))
    with S.Solver(S.SS_BABY_SKYRME, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        s.set_method(S.SS_METHOD_GRADIENT)
        st = s.step(25)
        fg = s.exact_fields() if prec == 1 else s.fields()
    fo = f.astype(np.float64)
    E = O.energy(BS, PRM, fo, dx, dy)
    dtau = 0.8 * O.gd_step_limit(dx, dy)
    for _ in range(25):
        fo, E, _ = O.gd_step(BS, PRM, fo, dx, dy, dtau, E)
    assert np.abs(fg - fo).max() <= (1e-10 if prec == 2 else 2e-5)
    assert st["steps"] == 25 and st["energy"] == pytest.approx(E, rel=1e-12 if prec == 2 else 1e-5)


@pytest.mark.parametrize("prec", [1, 2])
def test_observables_match_oracle(S, prec):
    nx, ny, dx, dy = GRID
    sol = [[0.5, 0.2, 1, 2.0, 0.0], [-4.5, 0.0, 2, 1.8, 0.3]]
    for f in (I.smooth_field(BS, nx, ny, dx, dy, seed=444), O.ansatz(BS, sol, nx, ny, dx, dy)):
        f = f.astype(dtype_of(prec))
        with S.Solver(S.SS_BABY_SKYRME, PRM, nx, ny, dx, dy, prec) as s:
            s.set_fields(f)
            og = s.observables()
        oo = O.observables(BS, PRM, f.astype(np.float64), dx, dy)
        for k in ("energy", "charge", "flux", "grad_max", "grad_max_raw", "norm_dev"):
            assert og[k] == pytest.approx(oo[k], rel=1e-12, abs=1e-12), k
    with S.Solver(S.SS_BABY_SKYRME, PRM, nx, ny, dx, dy, prec) as s:
        s.init_ansatz(sol)
        assert s.observables()["charge"] == pytest.approx(-3.0, abs=1e-10)
        fd = torch.from_numpy(s.fields()).cuda()
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    if prec == 1:
        S.ss_observables_noalloc(BS, PRM, fd, nx, ny, dx, dy, S.SS_FP32, out)
        torch.cuda.synchronize()
        oo = O.observables(BS, PRM, fd.cpu().numpy().astype(np.float64), dx, dy)
        assert out[0].item() == pytest.approx(oo["energy"], rel=1e-12)
        assert out[1].item() == pytest.approx(-3.0, abs=1e-10)


def test_skyrmion_relaxes_like_the_oracle(S):
    """A compact charge-1 ansatz relaxed to dx dy max|G| < 1e-7 in FP64 on the GPU: the
    oracle's step count (+-1), arrests and energy; charge exact."""
    n, dx = 96, 0.2
    prm = (1.0, 0.7, 0.0)
    sol = [[0.0, 0.0, 1, 2.5, 0.0]]
    f = O.ansatz(BS, sol, n, n, dx, dx)
    ref = O.minimise(BS, prm, f, dx, dx, tol=1e-7, max_steps=20000)
    assert ref["converged"]
    with S.Solver(S.SS_BABY_SKYRME, prm, n, n, dx, dx, 2) as s:
        s.init_ansatz(sol)
        st = s.minimise(1e-7, 20000)
        o = s.observables()
    assert st["converged"] and abs(st["steps"] - ref["steps"]) <= 1
    assert o["energy"] == pytest.approx(ref["energy"], rel=1e-10)
    assert o["charge"] == pytest.approx(-1.0, abs=1e-10)
    assert 4 * np.pi < o["energy"]


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_problems_evolve_exactly_as_alone(S, prec):
    """Every problem of a batch follows the trajectory it follows alone: bitwise in FP64.
    In FP32 the single-problem kernels of this theory carry a register bound (3 blocks
    per SM) that the batched ones cannot take without spilling, so the two are compiled
    apart and may contract a product into an FMA differently: the fields agree to the
    FP32 trajectory tolerance, the step and arrest counts exactly."""
    rng = I.SplitMix64(41)
    probs = []
    for k in range(4):
        nx, ny = rng.choice((48, 64, 77)), rng.choice((40, 56, 64))
        kappa, mu = rng.uniform(0.5, 1.5), rng.uniform(0.3, 1.0)
        probs.append(I.Problem(BS, nx, ny, 0.2, 0.2, (kappa, mu, 0.2), [(0.0, 0.0, 1.0, 2.0, 0.0)]))
    b = S.ss_batch_create(S.SS_BABY_SKYRME, prec, probs)
    try:
        rc, st = S.ss_batch_step(b, 17)
        for k, p in enumerate(probs):
            got = np.empty((3, p.ny, p.nx), dtype=dtype_of(prec))
            S.ss_batch_get_fields(b, k, got)
            with S.Solver(S.SS_BABY_SKYRME, p.params, p.nx, p.ny, p.dx, p.dy, prec) as s:
                s.init_ansatz(p.solitons)
                st1 = s.step(17)
                ref = s.fields()
            if prec == 2:
                assert np.array_equal(got, ref), k
            else:
                assert np.abs(got.astype(np.float64) - ref).max() <= 2e-5, k
            assert st[k]["steps"] == 17 and st[k]["arrests"] == st1["arrests"]
    finally:
        S.ss_batch_destroy(b)
