"""The large chiral-magnet workload (4096^2, 400 skyrmions, compensated FP32) relaxed
to dx dy max|G| < 1e-6 through the C-ABI: it converges, its lattice charge is -400
exactly after rounding, and on a 512^2 crop of the relaxed field the FP64 energy,
charge and residual of the GPU evaluation agree with the oracle's evaluation of the
same values, and the oracle finds the crop converged (dx dy max|G| < 1e-6 on its
interior, which is interior to the full grid)."""
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


def test_cm4096_relaxes_with_exact_charge_and_crop_parity(S):
    n, crop = 4096, 512
    p = I.cm_skyrmions(n=n, count=400, seed=20264)
    with S.Solver(S.SS_CHIRAL_MAGNET, p.params, n, n, p.dx, p.dy, S.SS_FP32) as s:
        s.init_ansatz(p.soliton_array())
        s.autotune(4)
        st = s.minimise(1e-6, 60000)
        obs = s.observables()
        f = s.exact_fields()
    assert st["converged"] and st["grad_max"] < 1e-6, st
    assert abs(obs["charge"] - round(obs["charge"])) <= 1e-4 and round(obs["charge"]) == -400, obs
    # crop: the GPU's FP64 observables of the crop vs the oracle's, on the same values
    c0 = (n - crop) // 2
    sub = np.ascontiguousarray(f[:, c0:c0 + crop, c0:c0 + crop])
    with S.Solver(S.SS_CHIRAL_MAGNET, p.params, crop, crop, p.dx, p.dy, S.SS_FP64) as s:
        s.set_fields(sub)
        g = s.observables()
    o = O.observables(O.CHIRAL_MAGNET, p.params, sub, p.dx, p.dy)
    assert g["energy"] == pytest.approx(o["energy"], rel=1e-12)
    assert g["charge"] == pytest.approx(o["charge"], abs=1e-9)
    assert g["grad_max"] == pytest.approx(o["grad_max"], rel=1e-9)
    assert o["grad_max"] < 1e-6  # the oracle's FP64 verdict on the crop's interior
    print(f"cm4096: {st['steps']} steps, {st['arrests']} arrests, E = {obs['energy']:.10f}, Q = {obs['charge']:.6f}")
