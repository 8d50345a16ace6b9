"""Rotating trapped BEC (Table 1) on the CUDA path vs the FP64 oracle, through the C-ABI.

Grand-canonical form at chemical potential mu (the functional minimised is E - mu N);
the site positions enter the trap and rotation terms. Tolerances as in
test_gpu_parity.py: FP64 1e-11 of the force scale and 1e-10 of the field after tens
of steps; FP32 3e-5 of the force scale and 2e-5 of the field (relative to its scale);
observables in FP64 from the stored values 1e-12.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2603_24370_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BEC = 4
PRM = (1.3, 0.6, 2.0)        # g, Omega, mu
GRID = (77, 45, 0.2, 0.17)   # ragged tiles, unequal spacings, centre off the tile grid


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
    f = I.smooth_field(BEC, nx, ny, dx, dy, seed=121).astype(dtype_of(prec))
    with S.Solver(S.SS_BEC, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        G, E, gmax = s.force()
    f64 = f.astype(np.float64)
    Go = O.force(BEC, PRM, f64, dx, dy)
    Eo = O.energy(BEC, PRM, f64, dx, dy)
    scale = np.abs(Go).max()
    assert np.abs(G.astype(np.float64) - Go).max() <= (1e-11 if prec == 2 else 3e-5) * scale
    esc = np.abs(O.energy_density(BEC, PRM, f64, dx, dy)).sum() * dx * dy
    assert abs(E - Eo) <= (1e-12 if prec == 2 else 1e-6) * esc
    assert gmax == pytest.approx(dx * dy * scale, rel=(1e-11 if prec == 2 else 3e-5))


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_trajectory_matches_oracle(S, prec):
    nx, ny, dx, dy = GRID
    n = 30
    f = I.smooth_field(BEC, nx, ny, dx, dy, seed=232).astype(dtype_of(prec))
    with S.Solver(S.SS_BEC, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        st = s.step(n)
        fg = s.exact_fields() if prec == 1 else s.fields().astype(np.float64)
        vg = s.velocity().astype(np.float64)
    fo, vo = f.astype(np.float64), np.zeros(f.shape)
    E = O.energy(BEC, PRM, fo, dx, dy)
    dt = O.time_step(dx, dy)
    arrests = 0
    for _ in range(n):
        fo, vo, E, a = O.anf_step(BEC, PRM, fo, vo, dx, dy, dt, E)
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


def descent_tau(nx, ny, dx, dy, prm, factor=0.8):
    """The documented BEC descent step: factor x 2 / (Laplacian bound + trap + interaction + rotation)."""
    g, Om, mu = prm
    r2 = (0.5 * (nx - 1) * dx) ** 2 + (0.5 * (ny - 1) * dy) ** 2
    lam = 16.0 / 3.0 * (1 / dx**2 + 1 / dy**2) + r2 + 4 * abs(mu) + 2 * abs(Om) * math.sqrt(r2) * 1.3722 / min(dx, dy)
    return factor * 2.0 / lam


@pytest.mark.parametrize("prec", [1, 2])
def test_descent_matches_oracle(S, prec):
    nx, ny, dx, dy = GRID
    f = I.smooth_field(BEC, nx, ny, dx, dy, seed=343).astype(dtype_of(prec))
    with S.Solver(S.SS_BEC, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        s.set_method(S.SS_METHOD_GRADIENT)
        st = s.step(25)
        fg = s.exact_fields() if prec == 1 else s.fields()
    fo = f.astype(np.float64)
    E = O.energy(BEC, PRM, fo, dx, dy)
    tau = descent_tau(nx, ny, dx, dy, PRM)
    rises = 0
    for _ in range(25):
        fo, E, r = O.gd_step(BEC, PRM, fo, dx, dy, tau, E)
        rises += r
    sc = max(1.0, np.abs(fo).max())
    assert np.abs(fg - fo).max() <= (1e-10 if prec == 2 else 2e-5) * sc
    assert st["steps"] == 25 and st["energy"] == pytest.approx(E, rel=1e-12 if prec == 2 else 1e-5)
    assert rises == 0


@pytest.mark.parametrize("prec", [1, 2])
def test_ansatz_and_observables_match_oracle(S, prec):
    nx, ny, dx, dy = GRID
    vort = [[0.6, 0.2, 1, 0.5, 0.0], [-1.0, -0.4, -1, 0.6, 0.3], [1.4, -0.9, 2, 0.5, 1.1]]
    fo = O.ansatz_bec(PRM, vort, nx, ny, dx, dy)
    with S.Solver(S.SS_BEC, PRM, nx, ny, dx, dy, prec) as s:
        s.init_ansatz(vort)
        fg = s.fields()
        og = s.observables()
    if prec == 2:
        assert np.abs(fg - fo).max() <= 1e-13
    else:
        ulp = np.spacing(np.abs(fo).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(fg.astype(np.float64) - fo) <= ulp + 1e-15)
    oo = O.observables(BEC, PRM, fg.astype(np.float64), dx, dy)
    for k in ("energy", "charge", "flux", "grad_max", "grad_max_raw", "norm_dev", "atoms", "angular_momentum"):
        assert og[k] == pytest.approx(oo[k], rel=1e-12, abs=1e-12), k
    assert og["atoms"] > 1.0 and og["charge"] == 0.0


def test_ground_state_relaxes_like_the_oracle(S):
    """Omega = 0, mu = 10 from the Thomas-Fermi ansatz to dx dy max|G| < 1e-7 in FP64:
    the oracle's step count (+-1), energy and atom number (near pi mu^2 / g)."""
    n, dx = 81, 0.2
    prm = (1.0, 0.0, 10.0)
    f = O.ansatz_bec(prm, [], n, n, dx, dx)
    ref = O.minimise(BEC, prm, f, dx, dx, tol=1e-7, max_steps=20000)
    ro = O.observables(BEC, prm, ref["f"], dx, dx)
    with S.Solver(S.SS_BEC, prm, n, n, dx, dx, 2) as s:
        s.set_fields(f)
        st = s.minimise(1e-7, 20000)
        o = s.observables()
    assert st["converged"] and abs(st["steps"] - ref["steps"]) <= 1
    assert o["energy"] == pytest.approx(ro["energy"], rel=1e-10)
    assert o["atoms"] == pytest.approx(ro["atoms"], rel=1e-10)
    assert abs(o["atoms"] / (math.pi * 100.0) - 1.0) < 0.02


def test_rotation_nucleates_a_vortex_lattice_like_the_oracle(S):
    """Omega = 0.85, mu = 10 (about Omega R_TF^2 = 17 vortices expected): from a Thomas-Fermi
    profile seeded with five vortices, the FP64 flow to dx dy max|G| < 1e-4 takes the
    oracle's steps (+-2) to its energy and angular momentum (> 10 quanta per atom);
    compensated FP32 reaches the same lattice energy to 1e-6. (Below ~1e-5 the lattice
    flow creeps: nearly every step arrests, in the oracle as well.)"""
    n, dx = 96, 0.15
    prm = (1.0, 0.85, 10.0)
    vort = [[1.2 * math.cos(a), 1.2 * math.sin(a), 1, 0.4, 0.0] for a in np.linspace(0, 2 * math.pi, 6)[:-1]]
    f = O.ansatz_bec(prm, vort, n, n, dx, dx)
    ref = O.minimise(BEC, prm, f, dx, dx, tol=1e-4, max_steps=30000)
    ro = O.observables(BEC, prm, ref["f"], dx, dx)
    assert ref["converged"]
    res = {}
    for prec in (2, 1):
        with S.Solver(S.SS_BEC, prm, n, n, dx, dx, prec) as s:
            s.init_ansatz(vort)
            st = s.minimise(1e-4, 30000)
            res[prec] = (st, s.observables())
    st, o = res[2]
    assert st["converged"] and abs(st["steps"] - ref["steps"]) <= 2
    assert o["energy"] == pytest.approx(ro["energy"], rel=1e-9)
    assert o["angular_momentum"] == pytest.approx(ro["angular_momentum"], rel=1e-8)
    assert o["angular_momentum"] > 10 * o["atoms"]
    st32, o32 = res[1]
    assert st32["converged"] and o32["energy"] == pytest.approx(o["energy"], rel=1e-6)


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_problems_evolve_exactly_as_alone(S, prec):
    rng = I.SplitMix64(52)
    probs = []
    for k in range(4):
        nx, ny = rng.choice((48, 64, 77)), rng.choice((40, 56, 64))
        g, Om, mu = rng.uniform(0.5, 2.0), rng.uniform(0.0, 0.8), rng.uniform(1.0, 4.0)
        probs.append(I.Problem(BEC, nx, ny, 0.15, 0.15, (g, Om, mu), [(0.3, -0.2, 1.0, 0.5, 0.0)]))
    b = S.ss_batch_create(S.SS_BEC, prec, probs)
    try:
        rc, st = S.ss_batch_step(b, 19)
        for k, p in enumerate(probs):
            got = np.empty((2, p.ny, p.nx), dtype=dtype_of(prec))
            S.ss_batch_get_fields(b, k, got)
            with S.Solver(S.SS_BEC, p.params, p.nx, p.ny, p.dx, p.dy, prec) as s:
                s.init_ansatz(p.solitons)
                st1 = s.step(19)
                ref = s.fields()
            assert np.array_equal(got, ref), k
            assert st[k]["steps"] == 19 and st[k]["arrests"] == st1["arrests"]
    finally:
        S.ss_batch_destroy(b)
