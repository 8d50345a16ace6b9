"""Chiral magnet with demagnetisation (Eq. 6) on the CUDA path vs the FP64 oracle.

The GPU solves the 5-point Poisson problem of the magnetostatic potential with a
sine transform built on its own shared-memory FFTs (the test grids' boxes take
lengths 40, 42, 63, 70: radix 8, 5, 2, 3, 7 stages); the oracle with the transform
written out as plain sums. Tolerances as in test_gpu_parity.py (FP64 1e-11 of the force scale,
1e-10 of the field after tens of steps; FP32 3e-5 and 2e-5), with the potential
solved in the working precision.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2603_24370_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CMD = 6
PRM = (1.0, 1.0, 0.1, 0.6, 0.0, 0.8)  # J, D, K, h, dmi_type, mu_d
GRID = (71, 45, 0.2, 0.23)
# Dirichlet boxes: GRID pads x only (67 -> 69 sites, one below I); GRID_PAD pads both
# axes with a site below I (60 -> 62, 36 -> 39)
GRID_PAD = (64, 40, 0.21, 0.2)
# boxes whose transform lengths take radix 16 x 2 (35 -> Lx = 32) and 16 x 4 (67 -> Lx = 64)
# along x, 5 x 7 along y (36 -> Ly = 35); and 16 x 16 x 2 along x, 16 x 16 along y
# (515 -> Lx = 512, 259 -> Ly = 256)
GRID_R4 = (35, 36, 0.2, 0.22)
GRID_R8 = (67, 36, 0.19, 0.2)
GRID_R16 = (515, 259, 0.2, 0.2)


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


@pytest.mark.parametrize("grid", [GRID, GRID_PAD, GRID_R4, GRID_R8, GRID_R16])
@pytest.mark.parametrize("prec", [1, 2, 3])
def test_force_and_energy_match_oracle(S, prec, grid):
    nx, ny, dx, dy = grid
    f = I.smooth_field(CMD, nx, ny, dx, dy, seed=181).astype(dtype_of(prec))
    with S.Solver(S.SS_CHIRAL_MAGNET, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        G, E, gmax = s.force()
        o = s.observables()
    f64 = f.astype(np.float64)
    Go = O.force(CMD, PRM, f64, dx, dy)
    Eo = O.energy(CMD, PRM, f64, dx, dy)
    scale = np.abs(Go).max()
    assert np.abs(G.astype(np.float64) - Go).max() <= (1e-11 if prec == 2 else 3e-5) * scale
    esc = np.abs(O.energy_density(2, PRM[:5], f64, dx, dy)).sum() * dx * dy + abs(O.demag_energy(PRM, f64, dx, dy))
    assert abs(E - Eo) <= (1e-12 if prec == 2 else 1e-6) * esc
    assert o["energy"] == pytest.approx(Eo, rel=1e-12 if prec == 2 else 1e-6)
    # without demagnetisation the same field has the plain chiral-magnet force
    G0 = O.force(2, PRM[:5], f64, dx, dy)
    assert np.abs(G.astype(np.float64) - G0).max() > 1e-3 * scale


@pytest.mark.parametrize("grid", [GRID, GRID_PAD])
@pytest.mark.parametrize("prec", [1, 2, 3])
def test_trajectory_matches_oracle(S, prec, grid):
    """30 flow steps, the potential solved once per step for the step's starting field."""
    nx, ny, dx, dy = grid
    n = 30
    f = I.smooth_field(CMD, nx, ny, dx, dy, seed=282).astype(dtype_of(prec))
    with S.Solver(S.SS_CHIRAL_MAGNET, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        st = s.step(n)
        fg = s.exact_fields() if prec == 1 else s.fields().astype(np.float64)
        vg = s.velocity().astype(np.float64)
    fo, vo = f.astype(np.float64), np.zeros(f.shape)
    E = O.energy(CMD, PRM, fo, dx, dy)
    dt = O.time_step(dx, dy)
    arrests = 0
    for _ in range(n):
        fo, vo, E, a = O.anf_step(CMD, PRM, fo, vo, dx, dy, dt, E)
        arrests += a
    tol = 1e-10 if prec == 2 else 2e-5
    assert np.abs(fg - fo).max() <= tol
    assert np.abs(vg - vo).max() <= tol / dt
    assert st["steps"] == n
    assert np.abs(np.sqrt((fg * fg).sum(axis=0)) - 1.0).max() < (1e-13 if prec == 2 else 1e-6)
    if prec == 2:
        assert st["arrests"] == arrests
        assert st["energy"] == pytest.approx(E, rel=1e-12)


@pytest.mark.parametrize("prec", [1, 2])
def test_descent_matches_oracle(S, prec):
    nx, ny, dx, dy = GRID
    f = I.smooth_field(CMD, nx, ny, dx, dy, seed=383).astype(dtype_of(prec))
    with S.Solver(S.SS_CHIRAL_MAGNET, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        s.set_method(S.SS_METHOD_GRADIENT)
        st = s.step(20)
        fg = s.exact_fields() if prec == 1 else s.fields()
    fo = f.astype(np.float64)
    E = O.energy(CMD, PRM, fo, dx, dy)
    tau = 0.8 * O.gd_step_limit(dx, dy)
    for _ in range(20):
        fo, E, _ = O.gd_step(CMD, PRM, fo, dx, dy, tau, E)
    assert np.abs(fg - fo).max() <= (1e-10 if prec == 2 else 2e-5)
    assert st["steps"] == 20 and st["energy"] == pytest.approx(E, rel=1e-12 if prec == 2 else 1e-5)


def test_neel_skyrmion_relaxes_like_the_oracle(S):
    """A compact Neel skyrmion relaxed with demagnetisation to dx dy max|G| < 1e-6 in
    FP64: the oracle's step count (+-1) and energy, the charge kept, and a higher energy
    than without demagnetisation (the Neel texture carries magnetostatic charge)."""
    n, dx = 64, 0.2
    sol = [[0.0, 0.0, 1, 2.0, 0.0]]
    f = O.ansatz(2, sol, n, n, dx, dx)
    ref = O.minimise(CMD, PRM, f, dx, dx, tol=1e-6, max_steps=20000)
    assert ref["converged"]
    with S.Solver(S.SS_CHIRAL_MAGNET, PRM, n, n, dx, dx, 2) as s:
        s.init_ansatz(sol)
        st = s.minimise(1e-6, 20000)
        o = s.observables()
    assert st["converged"] and abs(st["steps"] - ref["steps"]) <= 1
    assert o["energy"] == pytest.approx(ref["energy"], rel=1e-10)
    assert o["charge"] == pytest.approx(-1.0, abs=1e-10)
    with S.Solver(S.SS_CHIRAL_MAGNET, PRM[:5], n, n, dx, dx, 2) as s:
        s.init_ansatz(sol)
        s.minimise(1e-6, 20000)
        o0 = s.observables()
    assert o["energy"] > o0["energy"] + 1e-3


def test_demag_is_single_context_only(S):
    from test_gpu_batch import cm_batch
    probs = cm_batch(count=2, seed=3)
    for p in probs:
        p.params = tuple(p.params) + (0.5,)
    with pytest.raises(S.SolitonError):
        S.ss_batch_create(S.SS_CHIRAL_MAGNET, 2, probs)
    with pytest.raises(S.SolitonError):
        S.Solver(S.SS_CHIRAL_MAGNET, (1.0, 1.0, 0.1, 0.6, 0.0, -1.0), 32, 32, 0.2, 0.2, 2)


def test_fp32_poisson_solve_at_1024_matches_the_fp64_solve(S):
    """The 1024^2 workload field (8 skyrmions, after 20 FP32 flow steps; the box takes
    radix 16 x 16 x 4 transforms): the FP32 solve's demagnetisation energy equals the
    FP64 solve's (oracle-pinned above) to 1e-6 of that energy. The rest of the energy
    is evaluated from the same field values in both contexts."""
    from paper_2603_24370_gb300 import inputs as I
    q = I.cm_skyrmions()
    prm = tuple(q.params) + (0.8,)
    with S.Solver(S.SS_CHIRAL_MAGNET, prm, q.nx, q.ny, q.dx, q.dy, S.SS_FP32) as s32:
        s32.init_ansatz(q.soliton_array())
        s32.step(20)
        f = s32.fields()
        s32.set_fields(f)  # no remainder: both contexts hold the same values
        e32 = s32.observables()["energy"]
    with S.Solver(S.SS_CHIRAL_MAGNET, prm, q.nx, q.ny, q.dx, q.dy, S.SS_FP64) as s64:
        s64.set_fields(f.astype(np.float64))
        e64 = s64.observables()["energy"]
    with S.Solver(S.SS_CHIRAL_MAGNET, tuple(q.params), q.nx, q.ny, q.dx, q.dy, S.SS_FP64) as s0:
        s0.set_fields(f.astype(np.float64))
        e0 = s0.observables()["energy"]
    demag = e64 - e0
    assert demag > 1.0
    assert abs(e32 - e64) <= 1e-6 * demag
