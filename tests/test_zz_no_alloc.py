"""ss_observables_noalloc against ss_observables, through the C-ABI.

The no-allocation entry point serves callers that cannot call cudaMalloc (device
memory owned by a framework allocator or a fixed arena, or code where an
allocation would synchronize the device or could fail). It keeps its scratch in a
fixed device array shared by all calls, so this test makes two calls in a row with
different theories and precisions and checks both against the context-based entry
point. This file is collected last on purpose: it must pass on its own in a fresh
process and after every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2603_24370_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AH_PRM = (1.0, 1.0)
CM_PRM = (1.0, 1.0, 0.1, 0.6, 0.0)
KEYS = ("energy", "charge", "flux", "grad_max", "grad_max_raw", "norm_dev")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_24370_gb300 import build
    from paper_2603_24370_gb300 import soliton as S
    build.build()
    S.load_library()
    return S


def reference(S, theory, params, f, dx, dy, prec):
    ny, nx = f.shape[1:]
    with S.Solver(theory, params, nx, ny, dx, dy, prec) as s:
        s.set_fields(f)
        return s.observables()


def noalloc(S, theory, params, f, dx, dy, prec):
    ny, nx = f.shape[1:]
    dev = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    S.ss_observables_noalloc(theory, params, dev, nx, ny, dx, dy, prec, out)
    torch.cuda.synchronize()
    return dict(zip(KEYS, out.cpu().numpy().tolist()))


def test_noalloc_matches_ss_observables_on_two_calls_in_a_row(S):
    cases = [
        (S.SS_ABELIAN_HIGGS, AH_PRM, I.smooth_field(1, 77, 45, 0.2, 0.17, seed=901), 0.2, 0.17, S.SS_FP64),
        (S.SS_CHIRAL_MAGNET, CM_PRM,
         O.ansatz(2, [[0.5, 0.2, 1, 2.0, 0.0], [-5.0, 0.0, -1, 1.8, 0.0]], 83, 38, 0.2, 0.23).astype(np.float32),
         0.2, 0.23, S.SS_FP32),
    ]
    for theory, params, f, dx, dy, prec in cases:
        got = noalloc(S, theory, params, f, dx, dy, prec)
        ref = reference(S, theory, params, f, dx, dy, prec)
        for k in KEYS:
            assert got[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-12), (theory, k)


def test_noalloc_plain_fp32_and_the_rules_of_ss_set_theory(S):
    """A single-plane FP32 field passes its own precision code; parameter sets that
    ss_set_theory rejects, and the two forms that need a context, are rejected."""
    f = I.smooth_field(1, 61, 40, 0.2, 0.2, seed=903).astype(np.float32)
    for _ in range(2):
        got = noalloc(S, S.SS_ABELIAN_HIGGS, AH_PRM, f, 0.2, 0.2, S.SS_FP32_PLAIN)
        ref = reference(S, S.SS_ABELIAN_HIGGS, AH_PRM, f, 0.2, 0.2, S.SS_FP32_PLAIN)
        for k in KEYS:
            assert got[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-12), k
    dev = torch.zeros((6, 16, 16), dtype=torch.float32, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    bad = [
        (S.SS_SID, (-1.0, -1.0, 1.0, 1.0, 3.0, 0.0, 0.1)),   # quartic unbounded below
        (S.SS_SID, (-1.0, -1.0, 1.0, 1.0, 0.5, 0.0, 1.5)),   # |nu| >= 1
        (S.SS_CHIRAL_MAGNET, (1.0, 1.0, 0.1, 0.6, 0.0, 0.5)),  # demagnetisation
        (S.SS_BEC, (1.0, 0.5, 10.0, 100.0)),                  # fixed atom number
    ]
    for theory, params in bad:
        with pytest.raises(S.SolitonError) as ei:
            S.ss_observables_noalloc(theory, params, dev, 16, 16, 0.2, 0.2, S.SS_FP32, out)
        assert ei.value.code == S.SS_ERR_ARG, (theory, params)


def test_noalloc_rejects_grids_beyond_the_maximum(S):
    dummy = ctypes.c_void_p(1)  # never dereferenced: the size check comes first
    p = np.array(AH_PRM)
    rc = S.load_library().ss_observables_noalloc(S.SS_ABELIAN_HIGGS, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                 2, dummy, 70000, 16, 0.1, 0.1, S.SS_FP32, dummy, None)
    assert rc == S.SS_ERR_ARG
    assert "maximum" in S.last_error()
