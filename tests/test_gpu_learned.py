"""What the trained initialiser gains over the plain ansatz, measured end to end on
the GPU: problems relaxed by the batched flow train the network (solver-generated
targets: the flow's state after 1000 steps), and on held-out problems the
network's start lies closer to that state than the ansatz does. The flow then
finishes both starts and finds the same topological charges, so the fallback
(flow from the ansatz) and the learned start agree on what they solve.

The gain measured here is the distance to the flow's own trajectory, with a margin
below what the network reached (0.21 vs 0.33 RMS at this size). The number of flow
steps to 1e-6 is not reduced by the network at this scale (see the learned-init
profile): the test records it and does not assert on it."""
import numpy as np
import pytest

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


def test_trained_start_is_closer_to_the_flow_than_the_ansatz(S):
    from paper_2603_24370_gb300 import learned as L
    probs = I.ah_learned_set(192 + 32, seed=20263, side=128)
    train_p, test_p = probs[:192], probs[192:]
    ansatz, target, cp, _ = L.relax_set(train_p, 1e-6, 20000, horizon=1000)
    net = S.ss_net_create(S.SS_ABELIAN_HIGGS, 128, 16, seed=20263)
    try:
        hist = L.train(net, ansatz, target, cp, epochs=20, batch=16, lr=2e-3, seed=1)
        ta, tr, tcp, _ = L.relax_set(test_p, 1e-6, 20000, horizon=1000)
        init = L.predict(net, ta, tcp, 16)
    finally:
        S.ss_net_destroy(net)
    assert hist[-1] < 0.6 * hist[0], hist
    rms_ansatz = float(((ta - tr) ** 2).mean().sqrt())
    rms_net = float(((init - tr) ** 2).mean().sqrt())
    assert rms_net < 0.8 * rms_ansatz, (rms_net, rms_ansatz)
    # the halo keeps the ansatz's Dirichlet values exactly
    assert torch.equal(init[..., :2, :], ta[..., :2, :]) and torch.equal(init[..., -2:], ta[..., -2:])
    # both starts relaxed by the flow: same charges
    _, st_p, ob_p = L.solve(test_p, 1e-5, 20000)
    _, st_n, ob_n = L.solve(test_p, 1e-5, 20000, init=init)
    for a, b, p in zip(ob_p, ob_n, test_p):
        assert round(a["charge"]) == round(b["charge"]) == len(p.solitons)
    print(f"RMS to the 1000-step state: ansatz {rms_ansatz:.3f}, network {rms_net:.3f}; mean steps to 1e-5: "
          f"plain {np.mean([s['steps'] for s in st_p]):.0f}, learned {np.mean([s['steps'] for s in st_n]):.0f}")
