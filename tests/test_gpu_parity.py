"""CUDA path vs the FP64 oracle, element by element, through the C-ABI.

Tolerances (written out per test):
* FP64 path: the kernels evaluate the same formulas in another rounding order, so
  fields/forces agree to ~1e-13 of their scale; tests allow 1e-11 relative (1e-10
  after tens of steps, where the flow's own sensitivity amplifies rounding).
* FP32 path: the oracle evaluates the FP32-rounded input in FP64. The FP32 force is
  bounded by the rounding of the stencil sums: |dG| <~ k eps32 (sum_w |w| / h^2) max|phi|
  with sum_w |w| = 64/12 per direction for Eq. 2 and eps32 = 2^-24, plus a few eps32 of
  the pointwise terms. Tests use 3e-5 of max|G| (about 250 eps32), fields 2e-5 after
  tens of steps, and energies 1e-6 relative (the stated FP32 target).
* Observables are evaluated in FP64 from the stored values on both sides: 1e-12.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2603_24370_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AH, CM = 1, 2
AH_PRM = (1.0, 1.0)
CM_PRM = (1.0, 1.0, 0.1, 0.6, 0.0)


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_24370_gb300 import build
    from paper_2603_24370_gb300 import soliton as S
    build.build()
    S.load_library()
    return S


def prm(theory):
    return AH_PRM if theory == AH else CM_PRM


def dtype_of(prec):
    return np.float64 if prec == 2 else np.float32


# grids spanning several 32x16 tiles with ragged edges, unequal spacings
GRIDS = {AH: (77, 45, 0.2, 0.17), CM: (83, 38, 0.2, 0.23)}
# FP32 rows of whole 16-byte units (nx % 4 == 0) take the vector staging at the grid's
# edges too: several tiles with a ragged last row of tiles, and grids narrower than
# one tile (every unit right of the grid outside it)
UNIT_GRIDS = {"units": {AH: (76, 45, 0.2, 0.17), CM: (84, 38, 0.2, 0.23)},
              "narrow": {AH: (12, 41, 0.2, 0.17), CM: (20, 9, 0.2, 0.23)}}


def grid_of(theory, kind):
    return GRIDS[theory] if kind == "ragged" else UNIT_GRIDS[kind][theory]


@pytest.mark.parametrize("theory", [AH, CM])
@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("kind", ["ragged", "units", "narrow"])
def test_force_and_energy_match_oracle(S, theory, prec, kind):
    nx, ny, dx, dy = grid_of(theory, kind)
    f = I.smooth_field(theory, nx, ny, dx, dy, seed=101).astype(dtype_of(prec))
    with S.Solver(theory, prm(theory), nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        G, E, gmax = s.force()
    f64 = f.astype(np.float64)
    Go = O.force(theory, prm(theory), f64, dx, dy)
    Eo = O.energy(theory, prm(theory), f64, dx, dy)
    scale = np.abs(Go).max()
    tol = 1e-11 if prec == 2 else 3e-5
    assert np.abs(G.astype(np.float64) - Go).max() <= tol * scale
    assert np.all(G[:, :2, :] == 0) and np.all(G[:, -2:, :] == 0) and np.all(G[:, :, :2] == 0) and np.all(G[:, :, -2:] == 0)
    esc = np.abs(O.energy_density(theory, prm(theory), f64, dx, dy)).sum() * dx * dy
    assert abs(E - Eo) <= (1e-12 if prec == 2 else 1e-6) * esc
    assert gmax == pytest.approx(dx * dy * scale, rel=(1e-11 if prec == 2 else 3e-5))


@pytest.mark.parametrize("theory", [AH, CM])
@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("kind", ["ragged", "units", "narrow"])
def test_trajectory_matches_oracle(S, theory, prec, kind):
    """30 flow steps from a smooth field at rest: fields, velocity, energy and the
    arrest count against the oracle's RK4 + Eq. 4 step by step."""
    nx, ny, dx, dy = grid_of(theory, kind)
    n = 30
    f = I.smooth_field(theory, nx, ny, dx, dy, seed=202).astype(dtype_of(prec))
    with S.Solver(theory, prm(theory), nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        st = s.step(n)
        fg = s.fields().astype(np.float64)
        vg = s.velocity().astype(np.float64)
    fo, vo = f.astype(np.float64), np.zeros(f.shape)
    E = O.energy(theory, prm(theory), fo, dx, dy)
    dt = O.time_step(dx, dy)
    arrests = 0
    for _ in range(n):
        E_prev = E
        fo, vo, E, a = O.anf_step(theory, prm(theory), fo, vo, dx, dy, dt, E)
        arrests += a
    tol = 1e-10 if prec == 2 else 2e-5
    assert np.abs(fg - fo).max() <= tol * max(1.0, np.abs(fo).max())
    assert np.abs(vg - vo).max() <= tol * max(1.0, np.abs(fo).max()) / dt
    assert st["steps"] == n
    if prec == 2:
        assert st["arrests"] == arrests
        assert st["energy"] == pytest.approx(E, rel=1e-12)
        # the arrest test's cancellation-free energy change vs the oracle's direct difference
        esc = np.abs(O.energy_density(theory, prm(theory), fo, dx, dy)).sum() * dx * dy
        assert abs(st["energy_change"] - (E - E_prev)) <= 1e-12 * esc
    else:
        assert st["energy"] == pytest.approx(E, rel=1e-5)


@pytest.mark.parametrize("theory", [AH, CM])
def test_fp32_pair_reductions_match_fp64_sums_of_the_stored_fields(S, theory):
    """The compensated-FP32 flow totals E_h and the arrest test's energy change in
    float-float pairs: after 20 and 21 steps, both equal the oracle's FP64 sums over
    the exactly stored fields (value + remainder), E to 1e-6 of sum |e| and the change
    to 1e-4 of itself; the arrest decision (change > 0) agrees."""
    nx, ny, dx, dy = GRIDS[theory]
    f = I.smooth_field(theory, nx, ny, dx, dy, seed=207).astype(np.float32)
    with S.Solver(theory, prm(theory), nx, ny, dx, dy, 1) as s:
        s.set_fields(f)
        s.step(20)
        fa = s.exact_fields()
        st = s.step(1)
        fb = s.exact_fields()
    Ea = O.energy(theory, prm(theory), fa, dx, dy)
    Eb = O.energy(theory, prm(theory), fb, dx, dy)
    esc = np.abs(O.energy_density(theory, prm(theory), fb, dx, dy)).sum() * dx * dy
    assert abs(st["energy"] - Eb) <= 1e-6 * esc
    dE = Eb - Ea
    assert abs(dE) > 1e-9 * esc  # a change the test can resolve
    assert abs(st["energy_change"] - dE) <= 1e-4 * abs(dE) + 1e-12 * esc
    assert (st["energy_change"] > 0) == (dE > 0)


@pytest.mark.parametrize("theory", [AH, CM])
@pytest.mark.parametrize("prec", [1, 2])
def test_ansatz_matches_oracle(S, theory, prec):
    nx, ny, dx, dy = 101, 66, 0.15, 0.2
    if theory == AH:
        sol = [[-1.0, 0.5, 1, 1.0, 0.0], [1.5, -0.8, 2, 1.2, 0.4], [0.2, 1.9, -1, 0.9, 0.0]]
    else:
        sol = [[-3.0, -1.0, 1, 2.0, 0.0], [3.5, 1.5, 1, 2.5, 0.7], [0.0, 4.0, -1, 1.5, 0.0]]
    with S.Solver(theory, prm(theory), nx, ny, dx, dy, prec) as s:
        s.init_ansatz(sol)
        fg = s.fields()
    fo = O.ansatz(theory, sol, nx, ny, dx, dy)
    if prec == 2:
        assert np.abs(fg - fo).max() <= 1e-13
    else:  # FP64 evaluation rounded once: within one FP32 ulp of the oracle's value (plus
        # 1e-15 absolute for values that are zero up to the FP64 rounding of sin/cos)
        ulp = np.spacing(np.abs(fo).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(fg.astype(np.float64) - fo) <= ulp + 1e-15)


@pytest.mark.parametrize("theory", [AH, CM])
@pytest.mark.parametrize("prec", [1, 2])
def test_observables_match_oracle(S, theory, prec):
    nx, ny, dx, dy = GRIDS[theory]
    cases = [I.smooth_field(theory, nx, ny, dx, dy, seed=303)]
    sol = [[0.4, -0.3, 1, 1.0, 0.0]] if theory == AH else [[0.5, 0.2, 1, 2.0, 0.0], [-5.0, 0.0, -1, 1.8, 0.0]]
    cases.append(O.ansatz(theory, sol, nx, ny, dx, dy))
    for f in cases:
        f = f.astype(dtype_of(prec))
        with S.Solver(theory, prm(theory), nx, ny, dx, dy, prec) as s:
            s.set_fields(f)
            og = s.observables()
        oo = O.observables(theory, prm(theory), f.astype(np.float64), dx, dy)
        for k in ("energy", "charge", "flux", "grad_max", "grad_max_raw", "norm_dev"):
            assert og[k] == pytest.approx(oo[k], rel=1e-12, abs=1e-12), k


def test_flow_is_deterministic_and_call_splitting_is_exact(S):
    nx, ny, dx, dy = GRIDS[AH]
    f = I.smooth_field(AH, nx, ny, dx, dy, seed=404).astype(np.float32)
    out = []
    for split in ([12], [5, 7], [1, 1, 10]):
        with S.Solver(AH, AH_PRM, nx, ny, dx, dy, 1) as s:
            s.set_fields(f)
            for k in split:
                st = s.step(k)
            out.append((s.fields(), st["energy"], st["arrests"]))
    for g, e, a in out[1:]:
        assert np.array_equal(g, out[0][0]) and e == out[0][1] and a == out[0][2]


def test_abelian_higgs_128_fp64_converges_like_the_oracle(S):
    """Abelian Higgs, lambda = 1, 128^2 (dx 0.1), one N = 1 vortex at the centre,
    FP64, relaxed to dx dy max|G| < 1e-6: E -> pi (Bogomolny), flux -> 2 pi, Q = 1."""
    p = I.ah_single_vortex()
    with S.Solver(AH, p.params, p.nx, p.ny, p.dx, p.dy, 2) as s:
        s.init_ansatz(p.soliton_array())
        st = s.minimise(1e-6, 20000)
        fg = s.fields()
        og = s.observables()
    assert st["rc"] == S.SS_OK and st["converged"]
    fo0 = O.ansatz(AH, p.soliton_array(), p.nx, p.ny, p.dx, p.dy)
    r = O.minimise(AH, p.params, fo0, p.dx, p.dy, 1e-6, 20000)
    assert r["converged"]
    assert st["steps"] == r["steps"] and st["arrests"] == r["arrests"]
    assert np.abs(fg - r["f"]).max() <= 1e-9
    assert og["energy"] == pytest.approx(r["energy"], rel=1e-10)
    assert abs(og["energy"] - math.pi) < 1e-3
    assert og["charge"] == pytest.approx(1.0, abs=1e-9)
    assert og["flux"] == pytest.approx(2 * math.pi, rel=2e-3)
    assert og["grad_max"] < 1e-6


def test_chiral_magnet_1024_fp32_relaxes_with_exact_charge(S):
    """Chiral magnet 1024^2 (dx 0.2), J = D = 1, h = 0.6, K = 0.1, 8 skyrmions,
    compensated FP32 fields, relaxed to dx dy max|G| < 1e-6. The FP64 oracle decides:
    its evaluation of the final field (value + remainder) is below 1e-6, and the
    energy is within 1e-6 (relative) of the oracle's own FP64 relaxation of the same
    workload (tests/golden/cm1024_relaxed.json, written by make_cm1024_relaxed.py)."""
    p = I.cm_skyrmions()
    with S.Solver(CM, p.params, p.nx, p.ny, p.dx, p.dy, 1) as s:
        s.init_ansatz(p.soliton_array())
        st = s.minimise(1e-6, 200000)
        f64 = s.exact_fields()  # value + remainder of the compensated FP32 field
        og = s.observables()
    assert st["converged"], st
    oo = O.observables(CM, p.params, f64, p.dx, p.dy)
    assert og["energy"] == pytest.approx(oo["energy"], rel=1e-12)
    assert st["energy"] == pytest.approx(oo["energy"], rel=1e-6)  # the flow's FP32-density energy
    assert abs(oo["charge"] + 8.0) <= 1e-4 and round(oo["charge"]) == -8
    assert oo["norm_dev"] <= 1e-6
    assert oo["grad_max"] < 1e-6  # converged by the oracle's FP64 evaluation
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cm1024_relaxed.json")))
    assert list(p.params) == golden["params"]
    assert golden["converged"] and round(golden["charge"]) == -8
    assert oo["energy"] == pytest.approx(golden["energy"], rel=1e-6)


@pytest.mark.parametrize("prec", [1, 2])
def test_sampled_one_step_parity_at_4096(S, prec):
    """The 4096^2 chiral-magnet workload (400 skyrmions): one flow step on the GPU, in
    the launch configuration the benchmark times (autotuned tile shape and grids), vs
    the oracle's step of 41x41 patches around sampled sites (a step reaches 8 sites
    out, so the central 11x11 of each patch is exact)."""
    p = I.cm_skyrmions(n=4096, count=400, seed=20264)
    with S.Solver(CM, p.params, p.nx, p.ny, p.dx, p.dy, prec) as s:
        s.init_ansatz(p.soliton_array())
        s.autotune(4)  # as bench.py does; the field is restored at rest
        f0 = s.fields().astype(np.float64)
        q = s.observables()["charge"]
        s.step(1)
        f1 = s.fields().astype(np.float64)
    assert abs(q + 400.0) < 1e-6
    rng = I.SplitMix64(99)
    centres = [(int(s_[0] / p.dx + (p.nx - 1) / 2), int(s_[1] / p.dy + (p.ny - 1) / 2)) for s_ in p.solitons[:6]]
    centres += [(int(rng.uniform(24, p.nx - 24)), int(rng.uniform(24, p.ny - 24))) for _ in range(6)]
    dt = O.time_step(p.dx, p.dy)
    tol = 1e-12 if prec == 2 else 2e-6
    for ci, cj in centres:
        ci = min(max(ci, 20), p.nx - 21)
        cj = min(max(cj, 20), p.ny - 21)
        patch = f0[:, cj - 20:cj + 21, ci - 20:ci + 21].copy()
        fo, _, _, _ = O.anf_step(CM, p.params, patch, np.zeros_like(patch), p.dx, p.dy, dt, float("inf"))
        got = f1[:, cj - 5:cj + 6, ci - 5:ci + 6]
        assert np.abs(got - fo[:, 15:26, 15:26]).max() <= tol


def test_minimal_and_thin_grids(S):
    for nx, ny in ((5, 5), (6, 37), (40, 5)):
        dx, dy = 0.3, 0.25
        f = I.smooth_field(AH, nx, ny, dx, dy, seed=nx * 100 + ny)
        with S.Solver(AH, AH_PRM, nx, ny, dx, dy, 2) as s:
            s.set_fields(f)
            s.step(3)
            fg = s.fields()
        fo, vo = f.copy(), np.zeros_like(f)
        E = O.energy(AH, AH_PRM, fo, dx, dy)
        for _ in range(3):
            fo, vo, E, _ = O.anf_step(AH, AH_PRM, fo, vo, dx, dy, O.time_step(dx, dy), E)
        assert np.abs(fg - fo).max() <= 1e-12


def test_step_budget_and_convergence_edges(S):
    nx, ny, dx, dy = GRIDS[AH]
    f = I.smooth_field(AH, nx, ny, dx, dy, seed=505)
    with S.Solver(AH, AH_PRM, nx, ny, dx, dy, 2) as s:
        s.set_fields(f)
        st = s.step(0)
        assert st["steps"] == 0 and st["energy"] == pytest.approx(O.energy(AH, AH_PRM, f, dx, dy), rel=1e-12)
        st = s.minimise(1e-14, 37)  # cannot converge: stops at exactly 37 steps
        assert st["rc"] == S.SS_ERR_NOT_CONVERGED and st["steps"] == 37 and not st["converged"]
        st = s.minimise(1e-14, 0)
        assert st["rc"] == S.SS_ERR_NOT_CONVERGED and st["steps"] == 37
        st = s.minimise(1e30, 10)  # already below the threshold: no step taken
        assert st["rc"] == S.SS_OK and st["converged"] and st["steps"] == 37
        s.set_fields(f)  # resume = new fields from rest
        assert s.step(0)["steps"] == 0
        assert np.abs(s.velocity()).max() == 0.0
    # vacuum converges immediately
    vac = np.zeros((4, ny, nx))
    vac[0] = 1.0
    with S.Solver(AH, AH_PRM, nx, ny, dx, dy, 1) as s:
        s.set_fields(vac.astype(np.float32))
        st = s.minimise(1e-6, 100)
        assert st["rc"] == S.SS_OK and st["steps"] == 0 and st["grad_max"] == 0.0


def test_nonfinite_field_stops_the_flow(S):
    nx, ny, dx, dy = GRIDS[CM]
    f = I.smooth_field(CM, nx, ny, dx, dy, seed=606).astype(np.float32)
    f[0, ny // 2, nx // 2] = np.nan
    with S.Solver(CM, CM_PRM, nx, ny, dx, dy, 1) as s:
        s.set_fields(f)
        with pytest.raises(S.SolitonError) as ei:
            s.step(5)
        assert ei.value.code == S.SS_ERR_NONFINITE
        st = s.step(5, allow=(S.SS_ERR_NONFINITE,))
        assert st["steps"] == 0


def test_call_order_and_argument_errors(S):
    ctx = S.ss_create_grid(32, 32, 0.1, 0.1, 1)
    try:
        with pytest.raises(S.SolitonError) as ei:
            S.ss_step(ctx, 1)
        assert ei.value.code == S.SS_ERR_STATE
        with pytest.raises(S.SolitonError) as ei:
            S.ss_set_theory(ctx, 7, [1.0])
        assert ei.value.code == S.SS_ERR_ARG
        with pytest.raises(S.SolitonError) as ei:
            S.ss_set_theory(ctx, S.SS_CHIRAL_MAGNET, [0.0, 1.0, 0.1, 0.6])
        assert ei.value.code == S.SS_ERR_ARG
        S.ss_set_theory(ctx, S.SS_ABELIAN_HIGGS, [1.0])
        with pytest.raises(S.SolitonError) as ei:
            S.ss_observables(ctx)
        assert ei.value.code == S.SS_ERR_STATE
        with pytest.raises(S.SolitonError) as ei:
            S.ss_init_ansatz(ctx, np.zeros((0, 5)))
        assert ei.value.code == S.SS_ERR_ARG
    finally:
        S.ss_destroy(ctx)


def test_device_pointers_and_torch_stream(S):
    """Fields in and out as torch CUDA tensors, work on a caller's stream."""
    nx, ny, dx, dy = GRIDS[AH]
    f = I.smooth_field(AH, nx, ny, dx, dy, seed=707).astype(np.float32)
    stream = torch.cuda.Stream()
    dev = torch.from_numpy(f).cuda()
    torch.cuda.synchronize()  # the copy ran on torch's stream, the library works on `stream`
    with S.Solver(AH, AH_PRM, nx, ny, dx, dy, 1, stream=stream) as s:
        s.set_fields(dev)
        s.step(4)
        out = torch.empty((4, ny, nx), dtype=torch.float32, device="cuda")
        S.ss_get_fields(s.ctx, out)
        host = s.fields()
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), host)


# Grids whose rows start on 16-byte boundaries (nx % 4 == 0) and which hold interior
# tiles: those tiles are staged in vector units (two sites per 8-byte load with
# compensated storage, four per 16-byte load in plain FP32); edge tiles keep the
# per-site staging. Every theory of the flow kernels, 20 steps against the oracle.
VEC_CASES = [
    (1, (1.0, 1.0), (104, 72, 0.2, 0.17)),
    (2, (1.0, 1.0, 0.1, 0.6, 0.0), (104, 72, 0.2, 0.23)),
    (3, (1.0, 0.7, 0.3), (104, 72, 0.2, 0.17)),
    (4, (1.3, 0.6, 2.0), (104, 72, 0.2, 0.17)),
    (5, (-1.0, -0.6, 0.5, 0.4, 0.3, 0.15, 0.35), (104, 72, 0.25, 0.22)),
]


@pytest.mark.parametrize("case", VEC_CASES, ids=["ah", "cm", "bs", "bec", "sid"])
@pytest.mark.parametrize("prec", [1, 3])
def test_vector_staged_tiles_match_oracle(S, case, prec):
    theory, params, (nx, ny, dx, dy) = case
    assert nx % 4 == 0
    n = 20
    f = I.smooth_field(theory, nx, ny, dx, dy, seed=909 + theory).astype(np.float32)
    with S.Solver(theory, params, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        st = s.step(n)
        fg = s.exact_fields() if prec == 1 else s.fields().astype(np.float64)
    fo, vo = f.astype(np.float64), np.zeros(f.shape)
    E = O.energy(theory, params, fo, dx, dy)
    dt = O.time_step(dx, dy)
    for _ in range(n):
        fo, vo, E, _ = O.anf_step(theory, params, fo, vo, dx, dy, dt, E)
    assert st["steps"] == n
    assert np.abs(fg - fo).max() <= 2e-5 * max(1.0, np.abs(fo).max())
    assert st["energy"] == pytest.approx(E, rel=1e-5)
