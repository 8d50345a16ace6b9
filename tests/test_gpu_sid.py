"""s+id two-band superconductor (Table 1) on the CUDA path vs the FP64 oracle, through
the C-ABI: six planes (Delta_s, Delta_d, A), the d-wave mixed gradient, the gauge
field's mixed derivatives. Tolerances as in test_gpu_parity.py: FP64 1e-11 of the force
scale and 1e-10 of the field scale after tens of steps; FP32 3e-5 of the force scale
and 2e-5 of the field scale; observables in FP64 from the stored values 1e-12.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2603_24370_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SID = 5
PRM = (-1.0, -0.6, 0.5, 0.4, 0.3, 0.15, 0.35)  # a1, a2, b1, b2, b3, b4, nu
GRID = (77, 45, 0.25, 0.22)


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
    f = I.smooth_field(SID, nx, ny, dx, dy, seed=151).astype(dtype_of(prec))
    with S.Solver(S.SS_SID, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        G, E, gmax = s.force()
    f64 = f.astype(np.float64)
    Go = O.force(SID, PRM, f64, dx, dy)
    Eo = O.energy(SID, PRM, f64, dx, dy)
    scale = np.abs(Go).max()
    assert np.abs(G.astype(np.float64) - Go).max() <= (1e-11 if prec == 2 else 3e-5) * scale
    esc = np.abs(O.energy_density(SID, PRM, f64, dx, dy)).sum() * dx * dy
    assert abs(E - Eo) <= (1e-12 if prec == 2 else 1e-6) * esc
    assert gmax == pytest.approx(dx * dy * scale, rel=(1e-11 if prec == 2 else 3e-5))


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_trajectory_matches_oracle(S, prec):
    nx, ny, dx, dy = GRID
    n = 30
    f = I.smooth_field(SID, nx, ny, dx, dy, seed=262).astype(dtype_of(prec))
    with S.Solver(S.SS_SID, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        st = s.step(n)
        fg = s.exact_fields() if prec == 1 else s.fields().astype(np.float64)
        vg = s.velocity().astype(np.float64)
    fo, vo = f.astype(np.float64), np.zeros(f.shape)
    E = O.energy(SID, PRM, fo, dx, dy)
    dt = O.time_step(dx, dy)
    arrests = 0
    for _ in range(n):
        fo, vo, E, a = O.anf_step(SID, PRM, fo, vo, dx, dy, dt, E)
        arrests += a
    sc = max(1.0, np.abs(fo).max())
    tol = 1e-10 if prec == 2 else 2e-5
    assert np.abs(fg - fo).max() <= tol * sc
    assert np.abs(vg - vo).max() <= tol * sc / dt
    assert st["steps"] == n
    if prec == 2:
        assert st["arrests"] == arrests
        assert st["energy"] == pytest.approx(E, rel=1e-12)
    else:
        assert st["energy"] == pytest.approx(E, rel=1e-5)


@pytest.mark.parametrize("prec", [1, 2])
def test_descent_matches_oracle(S, prec):
    """The documented s+id descent step: 0.8 x the Laplacian limit / (1 + |nu|)."""
    nx, ny, dx, dy = GRID
    f = I.smooth_field(SID, nx, ny, dx, dy, seed=373).astype(dtype_of(prec))
    with S.Solver(S.SS_SID, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        s.set_method(S.SS_METHOD_GRADIENT)
        st = s.step(25)
        fg = s.exact_fields() if prec == 1 else s.fields()
    fo = f.astype(np.float64)
    E = O.energy(SID, PRM, fo, dx, dy)
    tau = 0.8 * O.gd_step_limit(dx, dy) / (1.0 + abs(PRM[6]))
    rises = 0
    for _ in range(25):
        fo, E, r = O.gd_step(SID, PRM, fo, dx, dy, tau, E)
        rises += r
    sc = max(1.0, np.abs(fo).max())
    assert np.abs(fg - fo).max() <= (1e-10 if prec == 2 else 2e-5) * sc
    assert st["steps"] == 25 and rises == 0


@pytest.mark.parametrize("prec", [1, 2])
def test_ansatz_and_observables_match_oracle(S, prec):
    nx, ny, dx, dy = GRID
    vort = [[0.8, 0.3, 1, 1.0, 0.0], [-2.5, -0.5, 2, 1.2, 0.4]]
    fo, (Smin, Dmin, phase) = O.ansatz_sid(PRM, vort, nx, ny, dx, dy)
    assert Smin == pytest.approx(1.0) and Dmin == pytest.approx(0.75) and phase == pytest.approx(math.pi / 2)
    with S.Solver(S.SS_SID, PRM, nx, ny, dx, dy, prec) as s:
        s.init_ansatz(vort)
        fg = s.fields()
        og = s.observables()
    if prec == 2:
        assert np.abs(fg - fo).max() <= 1e-13
    else:
        ulp = np.spacing(np.abs(fo).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(fg.astype(np.float64) - fo) <= ulp + 1e-15)
    oo = O.observables(SID, PRM, fg.astype(np.float64), dx, dy)
    for k in ("energy", "charge", "flux", "grad_max", "grad_max_raw", "norm_dev"):
        assert og[k] == pytest.approx(oo[k], rel=1e-12, abs=1e-12), k
    assert og["charge"] == pytest.approx(3.0, abs=1e-12)


def test_vortex_relaxes_like_the_oracle(S):
    """A charge-1 vortex on the s+id ground state relaxed to dx dy max|G| < 1e-4 in FP64:
    the oracle's step count (+-1) and energy, winding 1 and flux 2 pi. (Below ~1e-5 the
    flow creeps, every step arresting, in the oracle as well.)"""
    n, dx = 48, 0.3
    vort = [[0.0, 0.0, 1, 1.0, 0.0]]
    f, _ = O.ansatz_sid(PRM, vort, n, n, dx, dx)
    ref = O.minimise(SID, PRM, f, dx, dx, tol=1e-4, max_steps=20000)
    assert ref["converged"]
    with S.Solver(S.SS_SID, PRM, n, n, dx, dx, 2) as s:
        s.init_ansatz(vort)
        st = s.minimise(1e-4, 20000)
        o = s.observables()
    assert st["converged"] and abs(st["steps"] - ref["steps"]) <= 1
    assert o["energy"] == pytest.approx(ref["energy"], rel=1e-10)
    assert o["charge"] == pytest.approx(1.0, abs=1e-12)
    assert o["flux"] == pytest.approx(2 * math.pi, rel=1e-3)


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_problems_evolve_exactly_as_alone(S, prec):
    rng = I.SplitMix64(63)
    probs = []
    for k in range(4):
        nx, ny = rng.choice((40, 56, 64)), rng.choice((40, 48, 64))
        nu = rng.uniform(-0.5, 0.5)
        probs.append(I.Problem(SID, nx, ny, 0.3, 0.3, (-1.0, -0.6, 0.5, 0.4, 0.3, 0.15, nu),
                               [(0.2, -0.1, 1.0, 1.0, 0.0)]))
    b = S.ss_batch_create(S.SS_SID, prec, probs)
    try:
        rc, st = S.ss_batch_step(b, 15)
        for k, p in enumerate(probs):
            got = np.empty((6, p.ny, p.nx), dtype=dtype_of(prec))
            S.ss_batch_get_fields(b, k, got)
            with S.Solver(S.SS_SID, p.params, p.nx, p.ny, p.dx, p.dy, prec) as s:
                s.init_ansatz(p.solitons)
                st1 = s.step(15)
                ref = s.fields()
            assert np.array_equal(got, ref), k
            assert st[k]["steps"] == 15 and st[k]["arrests"] == st1["arrests"]
    finally:
        S.ss_batch_destroy(b)


def test_parameter_checks(S):
    bad = [(-1.0, -0.6, 0.5, 0.4, 0.3, 0.15, 1.2),   # |nu| >= 1
           (-1.0, -0.6, -0.5, 0.4, 0.3, 0.15, 0.3),  # b1 <= 0
           (-1.0, -0.6, 0.5, 0.4, 3.0, 0.15, 0.3)]   # unbounded quartic
    for prm in bad:
        with pytest.raises(S.SolitonError):
            S.Solver(S.SS_SID, prm, 32, 32, 0.3, 0.3, 2)
