"""The rotating BEC at a fixed atom number on the CUDA path vs the FP64 oracle, through
the C-ABI.

Every new field is scaled to the atom number N on I, its velocity made tangent to the
constraint, and its step takes the force at the constraint's multiplier (held through
the step); the energy and Eq. 4 are at mu = 0. The refresh is compared after a new
field, the flow and gradient descent over tens of steps, and the relaxation to
convergence. Tolerances as in test_gpu_bec.py: FP64 1e-10 of the field after tens of
steps, FP32 2e-5 of the field scale; the multiplier and the atom number in FP64 to
1e-12 (relative), in FP32 to the working type's rounding.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2603_24370_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BEC = 4
G_OM = (1.3, 0.6)                # g, Omega
N0 = 9.0                         # atoms held
PRM = (G_OM[0], G_OM[1], 0.0, N0)  # {g, Omega, mu (ignored), N}
GRID = (77, 45, 0.2, 0.17)       # ragged tiles, unequal spacings, centre off the tile grid


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


def start_field(nx, ny, dx, dy, seed, prec):
    """A smooth complex field with a zero halo, in the context's storage type."""
    f = I.smooth_field(BEC, nx, ny, dx, dy, seed=seed)
    f[:, :2, :] = 0.0
    f[:, -2:, :] = 0.0
    f[:, :, :2] = 0.0
    f[:, :, -2:] = 0.0
    return f.astype(dtype_of(prec))


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_refresh_matches_oracle(S, prec):
    """A new field: scaled to N on I, its multiplier; the halo untouched."""
    nx, ny, dx, dy = GRID
    f = start_field(nx, ny, dx, dy, 11, prec)
    f[:, 0, 5] = 0.01  # a non-zero halo value keeps its value
    with S.Solver(S.SS_BEC, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        fg = s.exact_fields() if prec == 1 else s.fields().astype(np.float64)
        o = s.observables()
    fo, _, mu = O.bec_refresh(G_OM, N0, f.astype(np.float64), None, dx, dy)
    tol = 1e-14 if prec == 2 else (1e-7 if prec == 1 else 2e-7)  # compensated: value + remainder
    assert np.abs(fg - fo).max() <= tol * np.abs(fo).max()
    assert fg[0, 0, 5] == pytest.approx(0.01, rel=1e-7)
    assert o["atoms"] == pytest.approx(N0, rel=1e-12 if prec != 3 else 1e-6)
    assert o["chemical_potential"] == pytest.approx(mu, rel=1e-12 if prec == 2 else 2e-6)
    # the observables (FP64 from the stored field): the residual is the constrained one
    # at that multiplier, the energy that of mu = 0
    oo = O.observables(BEC, (G_OM[0], G_OM[1], o["chemical_potential"]), fg, dx, dy)
    assert o["grad_max"] == pytest.approx(oo["grad_max"], rel=1e-10)
    assert o["energy"] == pytest.approx(O.energy(BEC, (G_OM[0], G_OM[1], 0.0), fg, dx, dy), rel=1e-12)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_trajectory_matches_oracle(S, prec):
    """30 steps from rest: fields, velocity (tangent to the constraint), energy at
    mu = 0, the multiplier, the atom number and (FP64) the arrest count."""
    nx, ny, dx, dy = GRID
    n = 30
    f = start_field(nx, ny, dx, dy, 22, prec)
    with S.Solver(S.SS_BEC, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        st = s.step(n)
        fg = s.exact_fields() if prec == 1 else s.fields().astype(np.float64)
        vg = s.velocity().astype(np.float64)
        o = s.observables()
    fo, vo, mu = O.bec_refresh(G_OM, N0, f.astype(np.float64), np.zeros(f.shape), dx, dy)
    E = O.energy(BEC, (G_OM[0], G_OM[1], 0.0), fo, dx, dy)
    dt = O.time_step(dx, dy)
    arrests = 0
    for _ in range(n):
        fo, vo, E, mu, a = O.anf_step_fixed_n(G_OM, N0, fo, vo, dx, dy, dt, E, mu)
        arrests += a
    scale = np.abs(fo).max()
    tol = 1e-10 if prec == 2 else 2e-5
    assert np.abs(fg - fo).max() <= tol * scale
    assert np.abs(vg - vo).max() <= tol * scale / dt
    assert st["steps"] == n
    assert o["atoms"] == pytest.approx(N0, rel=1e-12 if prec != 3 else 1e-6)
    assert abs((vg * fg)[:, 2:-2, 2:-2].sum()) <= (1e-11 if prec == 2 else 1e-5) * (np.abs(vg) * np.abs(fg)).sum()
    if prec == 2:
        assert st["arrests"] == arrests
        assert st["energy"] == pytest.approx(E, rel=1e-12)
        assert o["chemical_potential"] == pytest.approx(mu, rel=1e-11)
    else:
        assert st["energy"] == pytest.approx(E, rel=1e-5)
        assert o["chemical_potential"] == pytest.approx(mu, rel=1e-4)


def descent_tau(nx, ny, dx, dy, factor=0.8):
    """The documented BEC descent step with the Thomas-Fermi mu of N atoms."""
    hx, hy = 0.5 * (nx - 1) * dx, 0.5 * (ny - 1) * dy
    r2 = hx * hx + hy * hy
    mu = math.sqrt(G_OM[0] * N0 / math.pi)
    lam = 16.0 / 3.0 * (1 / dx**2 + 1 / dy**2) + r2 + 4 * mu + 2 * abs(G_OM[1]) * math.sqrt(r2) * 1.3722 / min(dx, dy)
    return factor * 2.0 / lam


@pytest.mark.parametrize("prec", [1, 2])
def test_descent_matches_oracle(S, prec):
    nx, ny, dx, dy = GRID
    f = start_field(nx, ny, dx, dy, 33, prec)
    with S.Solver(S.SS_BEC, PRM, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        s.set_method(S.SS_METHOD_GRADIENT)
        st = s.step(25)
        fg = s.exact_fields() if prec == 1 else s.fields().astype(np.float64)
    ref = O.gd_minimise_fixed_n(G_OM, N0, f.astype(np.float64), dx, dy, -1.0, 25,
                                dtau=descent_tau(nx, ny, dx, dy))
    assert ref["steps"] == 25
    assert np.abs(fg - ref["f"]).max() <= (1e-10 if prec == 2 else 2e-5) * np.abs(ref["f"]).max()
    assert st["steps"] == 25
    assert st["energy"] == pytest.approx(ref["energy"], rel=1e-12 if prec == 2 else 1e-5)


def test_relaxes_like_the_oracle(S):
    """From the Thomas-Fermi ansatz with two vortices at Omega = 0.6, relaxed to
    dx dy max|G| < 1e-7 in FP64: the oracle's step count (+-1), energy and multiplier;
    N exact. Compensated FP32 reaches 3e-5 at the same energy (1e-6)."""
    n, dx = 64, 0.2
    g, Om, N = 1.0, 0.6, 40.0
    sol = [[1.2, 0.3, 1, 0.5, 0.0], [-1.0, -0.8, 1, 0.5, 0.0]]
    f = O.ansatz_bec((g, Om, math.sqrt(g * N / math.pi)), sol, n, n, dx, dx)
    ref = O.minimise_fixed_n((g, Om), N, f, dx, dx, tol=1e-7, max_steps=40000)
    assert ref["converged"]
    with S.Solver(S.SS_BEC, (g, Om, 0.0, N), n, n, dx, dx, 2) as s:
        s.init_ansatz(sol)
        assert np.abs(s.fields() - O.bec_refresh((g, Om), N, f, None, dx, dx)[0]).max() < 1e-12
        st = s.minimise(1e-7, 40000)
        o = s.observables()
    assert st["converged"] and abs(st["steps"] - ref["steps"]) <= 1
    assert o["energy"] == pytest.approx(ref["energy"], rel=1e-10)
    assert o["chemical_potential"] == pytest.approx(ref["mu"], rel=1e-9)
    assert o["atoms"] == pytest.approx(N, rel=1e-13)
    with S.Solver(S.SS_BEC, (g, Om, 0.0, N), n, n, dx, dx, 1) as s:
        s.init_ansatz(sol)
        st = s.minimise(3e-5, 40000)
        o = s.observables()
    assert st["converged"]
    assert o["energy"] == pytest.approx(ref["energy"], rel=1e-6)
    assert o["atoms"] == pytest.approx(N, rel=1e-12)


def test_fixed_n_limits(S):
    """Fixed N is single-context only and not available without a context; a field
    without atoms stops the flow as non-finite; N < 0 is rejected."""
    probs = [I.Problem(BEC, 48, 48, 0.2, 0.2, PRM, [(0.0, 0.0, 0.0, 1.0, 0.0)]) for _ in range(2)]
    with pytest.raises(S.SolitonError):
        S.ss_batch_create(S.SS_BEC, 2, probs)
    with pytest.raises(S.SolitonError):
        S.Solver(S.SS_BEC, (1.0, 0.0, 0.0, -1.0), 32, 32, 0.2, 0.2, 2)
    fd = torch.zeros((2, 32, 32), dtype=torch.float64, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SolitonError):
        S.ss_observables_noalloc(BEC, PRM, fd, 32, 32, 0.2, 0.2, S.SS_FP64, out)
    with S.Solver(S.SS_BEC, PRM, 32, 32, 0.2, 0.2, 2) as s:
        s.set_fields(np.zeros((2, 32, 32)))
        st = s.step(3, allow=(S.SS_ERR_NONFINITE,))
        assert st["rc"] == S.SS_ERR_NONFINITE
