"""Batched relaxation (many uneven problems in the same launches) through the C-ABI.

Each problem of a batch must evolve exactly as it does alone (the same tiles, the
same per-problem reductions and decisions), match the FP64 oracle, and stop on its
own. Tolerances as in test_gpu_parity.py.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2603_24370_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_24370_gb300 import build
    from paper_2603_24370_gb300 import soliton as S
    build.build()
    S.load_library()
    return S


def mixed_batch(count=9, seed=77):
    """Small Abelian Higgs problems of uneven sizes, spacings, couplings and charges."""
    rng = I.SplitMix64(seed)
    out = []
    for k in range(count):
        nx = rng.choice((40, 56, 77, 96))
        ny = rng.choice((37, 64, 80))
        dx = rng.choice((0.15, 0.2, 0.25))
        lam = rng.uniform(0.5, 2.0)
        nv = rng.choice((1, 2, 3))
        Lx, Ly = nx * dx, ny * dx
        sol = [(rng.uniform(-Lx / 5, Lx / 5), rng.uniform(-Ly / 5, Ly / 5), 1.0, 1.0, 0.0) for _ in range(nv)]
        out.append(I.Problem(1, nx, ny, dx, dx, (lam, 1.0), sol))
    return out


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_problems_evolve_exactly_as_alone(S, prec):
    probs = mixed_batch()
    b = S.ss_batch_create(S.SS_ABELIAN_HIGGS, prec, probs)
    try:
        rc, st = S.ss_batch_step(b, 23)
        dt = np.float64 if prec == 2 else np.float32
        for k, p in enumerate(probs):
            got = np.empty((4, p.ny, p.nx), dtype=dt)
            S.ss_batch_get_fields(b, k, got)
            with S.Solver(S.SS_ABELIAN_HIGGS, p.params, p.nx, p.ny, p.dx, p.dy, prec) as s:
                s.init_ansatz(p.solitons)
                st1 = s.step(23)
                ref = s.fields()
            assert np.array_equal(got, ref), k
            assert st[k]["steps"] == 23 and st[k]["arrests"] == st1["arrests"]
            # the working-precision energy sums are grouped by the block that walks
            # the tiles, and a batch launch has its own grid: equal up to that rounding
            assert st[k]["energy"] == pytest.approx(st1["energy"], rel=1e-13 if prec == 2 else 1e-8)
    finally:
        S.ss_batch_destroy(b)


def test_batch_matches_oracle_fp64(S):
    probs = mixed_batch(count=4, seed=5)
    b = S.ss_batch_create(S.SS_ABELIAN_HIGGS, 2, probs)
    try:
        rc, st = S.ss_batch_step(b, 15)
        for k, p in enumerate(probs):
            got = np.empty((4, p.ny, p.nx))
            S.ss_batch_get_fields(b, k, got)
            f = O.ansatz(1, p.soliton_array(), p.nx, p.ny, p.dx, p.dy)
            v = np.zeros_like(f)
            E = O.energy(1, p.params, f, p.dx, p.dy)
            arrests = 0
            for _ in range(15):
                f, v, E, a = O.anf_step(1, p.params, f, v, p.dx, p.dy, O.time_step(p.dx, p.dy), E)
                arrests += a
            assert np.abs(got - f).max() <= 1e-10
            assert st[k]["arrests"] == arrests
            assert st[k]["energy"] == pytest.approx(E, rel=1e-12)
    finally:
        S.ss_batch_destroy(b)


def static_batch(count=12, seed=11):
    """Problems with a static minimum in the box: one unit vortex at the centre, with
    uneven grids, spacings and couplings.

    The boxes are kept several core radii wide: in a narrow box at large lambda the
    zero of the discretised force (Eq. 3 with the Eq. 2 stencils) lies O(h^4) above the
    minimum of the discretised energy, so close to it every step raises E_h and is
    arrested, and the flow creeps on from rest (the FP64 oracle, too, then needs
    more than 60000 steps to reach 1e-6)."""
    rng = I.SplitMix64(seed)
    out = []
    for _ in range(count):
        nx = rng.choice((56, 77, 96))
        ny = rng.choice((48, 64, 80))
        dx = rng.choice((0.2, 0.25))
        lam = rng.uniform(0.5, 1.5)
        out.append(I.Problem(1, nx, ny, dx, dx, (lam, 1.0), [(0.0, 0.0, 1.0, 1.0, 0.0)]))
    return out


def test_batch_minimise_stops_each_problem_on_its_own(S):
    """Compensated FP32 batch relaxed to dx dy max|G| < 1e-6: every problem stops on
    its own step, keeps its exact winding N, and its FP64-evaluated energy agrees with
    the oracle's evaluation of the same field."""
    probs = static_batch()
    b = S.ss_batch_create(S.SS_ABELIAN_HIGGS, 1, probs)
    try:
        rc, st = S.ss_batch_minimise(b, 1e-6, 60000)
        assert rc == S.SS_OK, [s["grad_max"] for s in st]
        steps = [s["steps"] for s in st]
        assert len(set(steps)) > 1  # problems stopped at different steps
        for k, p in enumerate(probs):
            assert st[k]["converged"] and st[k]["grad_max"] < 1e-6
            o = S.ss_batch_observables(b, k)
            assert o["charge"] == pytest.approx(p.solitons[0][2], abs=1e-9)
            got = np.empty((4, p.ny, p.nx), dtype=np.float32)
            S.ss_batch_get_fields(b, k, got)
            oo = O.observables(1, p.params, got.astype(np.float64), p.dx, p.dy)
            assert o["energy"] == pytest.approx(oo["energy"], rel=1e-6)  # remainder not included in `got`
            assert oo["grad_max"] < 2e-6
    finally:
        S.ss_batch_destroy(b)


def test_batch_rejects_bad_items(S):
    probs = mixed_batch(count=3)
    probs[1].nx = 3
    with pytest.raises(S.SolitonError) as ei:
        S.ss_batch_create(S.SS_ABELIAN_HIGGS, 1, probs)
    assert ei.value.code == S.SS_ERR_ARG and "item 1" in str(ei.value)


@pytest.mark.parametrize("prec", [1, 2])
def test_autotune_keeps_the_fields_and_the_trajectory(S, prec):
    """The tuner times the flow on the batch's own problems, then restores them: the
    tuned batch evolves exactly like an untuned one (the per-site update does not
    depend on the tile shape or the grid)."""
    probs = mixed_batch(count=5, seed=3)
    b = S.ss_batch_create(S.SS_ABELIAN_HIGGS, prec, probs)
    b2 = S.ss_batch_create(S.SS_ABELIAN_HIGGS, prec, probs)
    try:
        S.ss_batch_step(b, 7)  # tune from a state that is not the ansatz
        S.ss_batch_step(b2, 7)
        dt = np.float64 if prec == 2 else np.float32
        mid = [np.empty((4, p.ny, p.nx), dtype=dt) for p in probs]
        for k in range(len(probs)):
            S.ss_batch_get_fields(b2, k, mid[k])
            S.ss_batch_set_fields(b2, k, mid[k])  # the tuner restarts from rest: so does the reference
        choice = S.ss_batch_autotune(b, 3)
        assert choice["tile_shape"] in (0, 1) and min(choice["blocks"]) > 0
        for k in range(len(probs)):
            got = np.empty((4, probs[k].ny, probs[k].nx), dtype=dt)
            S.ss_batch_get_fields(b, k, got)
            if prec == 2:
                assert np.array_equal(got, mid[k])
        _, st = S.ss_batch_step(b, 15)
        _, st2 = S.ss_batch_step(b2, 15)
        for k, p in enumerate(probs):
            g1 = np.empty((4, p.ny, p.nx), dtype=dt)
            g2 = np.empty_like(g1)
            S.ss_batch_get_fields(b, k, g1)
            S.ss_batch_get_fields(b2, k, g2)
            assert st[k]["steps"] == st2[k]["steps"] == 15
            if prec == 2 and st[k]["arrests"] == st2[k]["arrests"]:
                assert np.array_equal(g1, g2), k
            else:  # compensated FP32: the reference restarted without the remainder planes
                assert np.abs(g1 - g2).max() <= 1e-5, k
    finally:
        S.ss_batch_destroy(b)
        S.ss_batch_destroy(b2)


def test_manual_launch_settings_do_not_change_the_flow(S):
    """The tile shape and grid only regroup the same per-site updates: FP64 fields are
    bitwise equal across launch settings (the arrest decisions agree here)."""
    probs = mixed_batch(count=4, seed=8)
    results = []
    for ts, blocks in ((1, None), (0, None), (0, [37, 55]), (1, [152, 152])):
        b = S.ss_batch_create(S.SS_ABELIAN_HIGGS, 2, probs)
        try:
            S.ss_batch_set_launch(b, ts, blocks)
            _, st = S.ss_batch_step(b, 19)
            fields = []
            for k, p in enumerate(probs):
                f = np.empty((4, p.ny, p.nx))
                S.ss_batch_get_fields(b, k, f)
                fields.append(f)
            results.append((st, fields))
        finally:
            S.ss_batch_destroy(b)
    st0, f0 = results[0]
    for st, f in results[1:]:
        for k in range(len(probs)):
            assert st[k]["arrests"] == st0[k]["arrests"]
            assert np.array_equal(f[k], f0[k]), k
    with pytest.raises(S.SolitonError):
        b = S.ss_batch_create(S.SS_ABELIAN_HIGGS, 2, probs)
        try:
            S.ss_batch_set_launch(b, 2)
        finally:
            S.ss_batch_destroy(b)


def cm_batch(count=5, seed=21):
    """Chiral-magnet problems of uneven sizes with 1..3 skyrmions each."""
    rng = I.SplitMix64(seed)
    out = []
    for _ in range(count):
        n = rng.choice((64, 77, 96))
        m = rng.choice((56, 64, 80))
        k = 1 + rng.next_u64() % 3
        half_x, half_y = 0.5 * (n - 1) * 0.2, 0.5 * (m - 1) * 0.2
        pts = I._separated_positions(rng, int(k), half_x, half_y, 2.5, 4.0)
        out.append(I.Problem(2, n, m, 0.2, 0.2, I.CM_DEFAULT, [(x, y, 1.0, 1.2, 0.0) for x, y in pts]))
    return out


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_chiral_magnet_batch_evolves_as_alone_and_keeps_unit_length(S, prec):
    probs = cm_batch()
    b = S.ss_batch_create(S.SS_CHIRAL_MAGNET, prec, probs)
    try:
        _, st = S.ss_batch_step(b, 17)
        dt = np.float64 if prec == 2 else np.float32
        for k, p in enumerate(probs):
            got = np.empty((3, p.ny, p.nx), dtype=dt)
            S.ss_batch_get_fields(b, k, got)
            with S.Solver(S.SS_CHIRAL_MAGNET, p.params, p.nx, p.ny, p.dx, p.dy, prec) as s:
                s.init_ansatz(p.solitons)
                st1 = s.step(17)
                ref = s.fields()
            assert np.array_equal(got, ref), k
            assert st[k]["arrests"] == st1["arrests"]
            norm = np.linalg.norm(got.astype(np.float64), axis=0)
            assert np.abs(norm - 1).max() < (1e-12 if prec == 2 else 1e-6)
            o = S.ss_batch_observables(b, k)
            assert round(o["charge"]) == -len(p.solitons)
    finally:
        S.ss_batch_destroy(b)


def test_chiral_magnet_batch_matches_the_oracle_fp64(S):
    probs = cm_batch(count=3, seed=4)
    b = S.ss_batch_create(S.SS_CHIRAL_MAGNET, 2, probs)
    try:
        _, st = S.ss_batch_step(b, 12)
        for k, p in enumerate(probs):
            got = np.empty((3, p.ny, p.nx))
            S.ss_batch_get_fields(b, k, got)
            f = O.ansatz(2, p.soliton_array(), p.nx, p.ny, p.dx, p.dy)
            v = np.zeros_like(f)
            E = O.energy(2, p.params, f, p.dx, p.dy)
            arrests = 0
            for _ in range(12):
                f, v, E, a = O.anf_step(2, p.params, f, v, p.dx, p.dy, O.time_step(p.dx, p.dy), E)
                arrests += a
            assert np.abs(got - f).max() <= 1e-10
            assert st[k]["arrests"] == arrests
    finally:
        S.ss_batch_destroy(b)


@pytest.mark.parametrize("prec", [1, 2])
def test_contexts_driven_from_two_threads_evolve_exactly_as_alone(S, prec):
    """Two solver contexts on their own streams, each driven from its own host thread
    (field in from pinned host memory, flow, field out: the overlapped end-to-end leg
    of the benchmark), end every round on the fields and status each reaches when run
    alone."""
    import threading
    cases = [(S.SS_CHIRAL_MAGNET, (1.0, 1.0, 0.1, 0.6, 0.0), 96, 84, 0.2, [[0.0, 0.0, -1, 2.0, 0.0]]),
             (S.SS_ABELIAN_HIGGS, (1.0, 1.0), 77, 64, 0.2, [[0.5, -0.3, 1, 1.0, 0.0], [-1.0, 0.8, 2, 1.0, 0.0]])]
    dt = np.float64 if prec == 2 else np.float32
    starts, refs = [], []
    for th, prm, nx, ny, dx, sol in cases:
        with S.Solver(th, prm, nx, ny, dx, dx, prec) as s:
            s.init_ansatz(sol)
            f0 = s.fields()
            s.set_fields(f0)  # the state the threads start from (no remainder part)
            st = s.step(40)
            refs.append((s.fields(), st["arrests"], st["energy"]))
        starts.append(f0)
    solvers = [S.Solver(th, prm, nx, ny, dx, dx, prec, stream=torch.cuda.Stream())
               for th, prm, nx, ny, dx, sol in cases]
    host_in = [torch.from_numpy(f).pin_memory() for f in starts]
    host_out = [torch.empty(f.shape, dtype=torch.float64 if prec == 2 else torch.float32).pin_memory()
                for f in starts]
    got, err = [[], []], []

    def drive(i):
        try:
            for _ in range(4):
                solvers[i].set_fields(host_in[i])
                st = solvers[i].step(40)
                S.ss_get_fields(solvers[i].ctx, host_out[i])
                got[i].append((host_out[i].numpy().copy(), st["arrests"], st["energy"]))
        except Exception as exc:
            err.append(exc)

    try:
        threads = [threading.Thread(target=drive, args=(i,)) for i in range(2)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not err, err
        for i in range(2):
            assert len(got[i]) == 4
            for f, arrests, energy in got[i]:
                assert f.dtype == dt and np.array_equal(f, refs[i][0]), i
                assert arrests == refs[i][1] and energy == refs[i][2]
    finally:
        for s in solvers:
            s.close()
