"""The learned initialiser on the GPU against its CPU oracle (oracle/unet.py).

Convolutions: every tile width the network uses and every output width the kernels
are instantiated for, forward (all three epilogues) and weight gradient. The oracle
sums the same BF16 operands in float64; the GPU accumulates in FP32, so each output
may differ by the FP32 accumulation error, bounded here by 1e-5 times the sum of the
absolute values of its terms (K <= 1296 terms per output for the convolutions, FP32
unit roundoff 6e-8), and, where the output is stored in BF16, by one BF16 rounding
(2^-8 relative) on top.

Network, element by element, at S = 128 against the oracle with the same BF16
rounding points, in two settings:
- a network whose weights, biases and inputs are positive and whose target is zero,
  so every ReLU is active, every activation, output and gradient is a sum of positive
  terms, and a BF16 rounding that FP32 and float64 accumulation take differently can
  shift each value by at most its own rounding step: the output is held to 2^-8 of
  its value and every parameter gradient to 5e-4 of its value (a float32-accumulation
  replay of the oracle stays below 3e-4 and 1.3e-5);
- a general network (signed weights, dead and live ReLUs): every output within 2^-6
  of the sum of the absolute values of its terms in the last convolution (the
  replay: 2.5e-3), the median within 2^-10; every layer's gradients within 2e-2 in
  relative L2 norm and 95% of the entries within 1/8 of the sum of the absolute
  values of their terms (the replay: 99th percentiles up to 0.13 of those sums where
  a ReLU flips upstream; on GB300 at least 98% of every layer's entries). The loss
  within 1e-3.
Adam: the parameters and both moments after three updates from caller gradients,
element by element against the oracle's float64 updates.
"""
import os
import tempfile

import numpy as np
import pytest

from oracle import unet as U

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


def bf16_tensor(a):
    """Exact BF16 device tensor of the BF16-rounded values of a."""
    return torch.tensor(U.round_bf16(a), dtype=torch.float32).to(torch.bfloat16).cuda().contiguous()


CONV_CASES = [  # (N, H, W, Cin, Cout)
    (2, 16, 16, 16, 16),
    (1, 16, 32, 16, 32),
    (2, 8, 64, 32, 48),
    (1, 4, 128, 48, 80),
    (1, 2, 256, 16, 96),
    (2, 3, 128, 32, 16),
    (1, 3, 384, 16, 48),
    (2, 16, 16, 144, 48),
    (1, 8, 32, 80, 144),
    (1, 16, 8, 16, 16),
    (2, 4, 64, 48, 48),
]


@pytest.mark.parametrize("case", CONV_CASES)
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_conv_forward_matches_oracle(S, case, mode):
    N, H, W, Cin, Cout = case
    rng = np.random.default_rng(hash((case, mode)) % 2**32)
    x = U.round_bf16(rng.normal(size=(N, H, W, Cin)))
    w = U.round_bf16(rng.normal(size=(Cout, 9, Cin)) / np.sqrt(9 * Cin))
    b = rng.normal(size=Cout).astype(np.float32).astype(np.float64)
    ref = U.conv3x3(x, w) + (b if mode != 2 else 0.0)
    mag = U.conv3x3(np.abs(x), np.abs(w)) + np.abs(b if mode != 2 else 0.0)
    xd, wd = bf16_tensor(x), bf16_tensor(w.reshape(Cout, 9 * Cin))
    bd = torch.tensor(b, dtype=torch.float32, device="cuda")
    out = torch.zeros((N, H, W, Cout), dtype=torch.bfloat16 if mode == 0 else torch.float32, device="cuda")
    S.ss_conv3x3(xd, wd, bd, mode, out)
    got = out.float().cpu().numpy().astype(np.float64)
    if mode == 0:
        ref = np.maximum(ref, 0.0)
        tol = 2.0 ** -8 * np.abs(ref) + 1e-5 * mag + 1e-30
    else:
        tol = 1e-5 * mag + 1e-30
    err = np.abs(got - ref)
    assert np.all(err <= tol), (float(err.max()), float((err / (mag + 1e-30)).max()))


@pytest.mark.parametrize("case", [(2, 16, 16, 16, 16), (1, 8, 64, 32, 48), (1, 4, 128, 48, 96),
                                  (2, 16, 16, 144, 48), (2, 32, 32, 80, 32), (1, 8, 32, 96, 16),
                                  # rows of >= 64 pixels: 64-pixel swizzled K-blocks, all taps per CTA
                                  (2, 3, 128, 16, 16), (1, 4, 64, 80, 32), (1, 2, 64, 144, 48),
                                  (2, 2, 64, 96, 96), (1, 6, 256, 16, 48),
                                  # (tap, input channel) rows for 9 Cin <= 512
                                  (2, 4, 64, 16, 16), (1, 2, 128, 48, 16), (1, 3, 64, 32, 96)])
def test_conv_weight_gradient_matches_oracle(S, case):
    N, H, W, Cin, Cout = case
    rng = np.random.default_rng(sum(case))
    x = U.round_bf16(rng.normal(size=(N, H, W, Cin)))
    dy = rng.normal(size=(N, H, W, Cout)).astype(np.float32).astype(np.float64)
    ref = U.conv3x3_grad_weight(x, U.round_bf16(dy))
    mag = U.conv3x3_grad_weight(np.abs(x), np.abs(U.round_bf16(dy)))
    dw = torch.zeros((Cout, 9, Cin), dtype=torch.float32, device="cuda")
    S.ss_conv3x3_wgrad(torch.tensor(dy, dtype=torch.float32, device="cuda"), bf16_tensor(x), dw)
    err = np.abs(dw.cpu().numpy() - ref)
    assert np.all(err <= 1e-5 * mag + 1e-30), float(err.max())


def random_problem(rng, B, Sz, C=4, ncoup=1):
    """Smooth synthetic fields (sums of Gaussian bumps), couplings and targets."""
    yy, xx = np.meshgrid(np.linspace(-1, 1, Sz), np.linspace(-1, 1, Sz), indexing="ij")
    f = np.zeros((B, C, Sz, Sz))
    for b in range(B):
        for c in range(C):
            for _ in range(3):
                x0, y0, s = rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8), rng.uniform(0.1, 0.4)
                f[b, c] += rng.normal() * np.exp(-((xx - x0) ** 2 + (yy - y0) ** 2) / s ** 2)
    coup = rng.uniform(0.5, 2.0, size=(B, ncoup)) if ncoup else None
    target = 0.1 * np.roll(f, 3, axis=3) - 0.05 * f
    return f, coup, target


def test_network_loss_and_gradients_match_oracle(S):
    B, Sz = 2, 128
    rng = np.random.default_rng(7)
    net = S.ss_net_create(S.SS_ABELIAN_HIGGS, Sz, B, seed=3)
    try:
        n = S.ss_net_num_params(net)
        assert n == U.num_params()
        theta = S.ss_net_get_params(net).astype(np.float64)
        # give the (zero-initialised) last layer and the biases some weight so that every
        # path carries gradient; unused output channels stay zero
        sl = U.unflatten(theta)
        w14, b14 = sl[14]
        w14[:4] = rng.normal(size=w14[:4].shape) * 0.1
        for w, b in sl[:14]:
            b[:] = rng.normal(size=b.shape) * 0.05
        theta32 = theta.astype(np.float32)
        S.ss_net_set_params(net, theta32)
        f, coup, target = random_problem(rng, B, Sz)
        fd = torch.tensor(f, dtype=torch.float32, device="cuda")
        inp = torch.empty((B, Sz, Sz, 16), dtype=torch.bfloat16, device="cuda")
        S.ss_net_pack(net, fd, coup[:, 0], B, inp)
        x = U.pack_input(f.astype(np.float32).astype(np.float64), coup)
        assert np.array_equal(inp.float().cpu().numpy(), U.round_bf16(x))
        relaxed = (f + target).astype(np.float32)
        rd = torch.tensor(relaxed, dtype=torch.float32, device="cuda")
        g = torch.zeros(n, dtype=torch.float32, device="cuda")
        loss = S.ss_net_gradients(net, fd, coup[:, 0], rd, B, g)
        tgt = (relaxed - f.astype(np.float32)).astype(np.float64)  # formed in FP32 as on the GPU
        ref_loss, ref_g, ref_out = U.loss_and_grad(theta32.astype(np.float64), x, tgt, 4)
        assert loss == pytest.approx(ref_loss, rel=1e-3)
        out = torch.zeros((B, Sz, Sz, 16), dtype=torch.float32, device="cuda")
        S.ss_net_forward(net, fd, coup[:, 0], B, out)
        o = out.cpu().numpy()
        _, cache = U.forward(theta32.astype(np.float64), x)
        w14, b14 = cache["P"][14]
        mag = U.conv3x3(np.abs(cache["d1"]), np.abs(w14)) + np.abs(b14)
        rel = np.abs(o - ref_out) / (mag + 1e-30)
        assert rel.max() <= 2.0 ** -6, float(rel.max())
        assert np.median(rel[..., :4]) <= 2.0 ** -10, float(np.median(rel[..., :4]))
        _, gout = U.mse(ref_out, tgt, 4)
        _, gmag = U.backward(theta32.astype(np.float64), cache, gout, magnitudes=True)
        gg = g.cpu().numpy().astype(np.float64)
        k = 0
        for L, (ci, co) in enumerate(U.layer_shapes()):
            for part, size in (("W", 9 * ci * co), ("b", co)):
                a, r, m = gg[k:k + size], ref_g[k:k + size], gmag[k:k + size]
                k += size
                assert np.linalg.norm(a - r) <= 2e-2 * np.linalg.norm(r) + 1e-12, (L, part)
                assert np.mean(np.abs(a - r) <= m / 8 + 1e-12) >= 0.95, (L, part)
    finally:
        S.ss_net_destroy(net)


def positive_network(rng, n):
    """Parameters with every weight and bias positive, weights scaled so that each
    convolution averages its inputs (activations stay of order one)."""
    theta = np.zeros(n)
    k = 0
    for ci, co in U.layer_shapes():
        w = rng.uniform(0.5, 1.5, size=(co, 9, ci)) / (9 * ci)
        theta[k:k + w.size] = w.ravel()
        k += w.size
        theta[k:k + co] = rng.uniform(0.0, 0.2, size=co)
        k += co
    return theta.astype(np.float32)


def test_positive_network_output_and_gradients_elementwise(S):
    """All terms positive: no ReLU is inactive, nothing cancels, so each output and
    each gradient entry is checked against its own value."""
    B, Sz = 2, 128
    rng = np.random.default_rng(3)
    net = S.ss_net_create(S.SS_ABELIAN_HIGGS, Sz, B, seed=1)
    try:
        n = S.ss_net_num_params(net)
        theta32 = positive_network(rng, n)
        S.ss_net_set_params(net, theta32)
        f = rng.uniform(0.2, 1.0, size=(B, 4, Sz, Sz)).astype(np.float32)
        coup = rng.uniform(0.5, 2.0, size=B)
        fd = torch.tensor(f, device="cuda")
        g = torch.zeros(n, dtype=torch.float32, device="cuda")
        loss = S.ss_net_gradients(net, fd, coup, fd, B, g)  # relaxed = ansatz: the target is zero
        x = U.pack_input(f.astype(np.float64), coup[:, None])
        ref_loss, ref_g, ref_out = U.loss_and_grad(theta32.astype(np.float64), x, np.zeros((B, 4, Sz, Sz)), 4)
        assert loss == pytest.approx(ref_loss, rel=1e-3)
        out = torch.zeros((B, Sz, Sz, 16), dtype=torch.float32, device="cuda")
        S.ss_net_forward(net, fd, coup, B, out)
        o = out.cpu().numpy()
        assert ref_out.min() > 0.0
        err = np.abs(o - ref_out)
        assert np.all(err <= 2.0 ** -8 * ref_out), float((err / ref_out).max())
        gg = g.cpu().numpy().astype(np.float64)
        assert np.all(ref_g >= 0.0)
        gerr = np.abs(gg - ref_g)
        assert np.all(gerr <= 5e-4 * ref_g + 1e-30), float((gerr / (ref_g + 1e-30)).max())
    finally:
        S.ss_net_destroy(net)


def test_adam_updates_match_the_oracle_elementwise(S):
    """Three Adam updates from caller gradients (magnitudes 1e-6 .. 1e2, exact zeros,
    a changing learning rate as a schedule gives): parameters, first and second
    moments against the oracle's float64 Adam chained from the same start."""
    rng = np.random.default_rng(17)
    net = S.ss_net_create(S.SS_ABELIAN_HIGGS, 128, 1, seed=4)
    try:
        n = S.ss_net_num_params(net)
        theta = S.ss_net_get_params(net).astype(np.float64)
        m, v = np.zeros(n), np.zeros(n)
        # FP32 error budgets, element by element: a few roundings per operation,
        # relative to the absolute values of the terms (the moments' terms can cancel)
        tol_m, tol_v, tol_t = np.zeros(n), np.zeros(n), np.zeros(n)
        for t, lr in enumerate((1e-3, 7e-4, 2e-4), start=1):
            lr = float(np.float32(lr))  # the update is given an FP32 learning rate
            g = (rng.normal(size=n) * 10.0 ** rng.uniform(-6, 2, size=n)).astype(np.float32)
            g[rng.random(n) < 0.05] = 0.0
            S.ss_net_apply_gradients(net, torch.tensor(g, device="cuda"), lr)
            g64 = g.astype(np.float64)
            m0, v0 = m, v
            theta, m, v = U.adam_step(theta, m, v, g64, t, lr)
            c1, c2 = 1 - 0.9 ** t, 1 - 0.999 ** t
            tol_m = 0.9 * tol_m + 2.5e-7 * (0.9 * np.abs(m0) + 0.1 * np.abs(g64) + np.abs(m))
            tol_v = 0.999 * tol_v + 2.5e-7 * (0.999 * v0 + 0.001 * g64 * g64 + v)
            den = np.sqrt(v / c2) + 1e-8
            tol_t += 2.0 ** -24 * np.abs(theta) + lr * (tol_m / c1 / den +
                                                       np.abs(m / c1) / den * (1e-6 + tol_v / (2 * v + 1e-300)))
            gt = S.ss_net_get_params(net).astype(np.float64)
            gm, gv, steps = S.ss_net_get_optimizer_state(net)
            assert steps == t
            assert np.all(np.abs(gm - m) <= tol_m + 1e-45), float(np.abs(gm - m).max())
            assert np.all(np.abs(gv - v) <= tol_v + 1e-45), float(np.abs(gv - v).max())
            assert np.all(np.abs(gt - theta) <= tol_t + 1e-30), float(np.abs(gt - theta).max())
    finally:
        S.ss_net_destroy(net)


def test_training_steps_reduce_the_loss_on_a_fixed_batch(S):
    B, Sz = 4, 128
    rng = np.random.default_rng(11)
    net = S.ss_net_create(S.SS_ABELIAN_HIGGS, Sz, B, seed=5)
    try:
        f, coup, target = random_problem(rng, B, Sz)
        fd = torch.tensor(f, dtype=torch.float32, device="cuda")
        rd = torch.tensor(f + target, dtype=torch.float32, device="cuda")
        losses = [S.ss_net_train_step(net, fd, coup[:, 0], rd, B, 2e-3) for _ in range(60)]
        assert all(np.isfinite(losses))
        assert losses[-1] < 0.5 * losses[0], losses[::10]
    finally:
        S.ss_net_destroy(net)


def test_predict_keeps_the_halo_and_unit_length(S):
    rng = np.random.default_rng(2)
    for theory, C, ncoup in ((1, 4, 1), (2, 3, 0)):
        net = S.ss_net_create(theory, 128, 2, seed=9)
        try:
            theta = S.ss_net_get_params(net)
            sl = U.unflatten(theta.astype(np.float64))
            w14 = sl[14][0]
            w14[:C] = rng.normal(size=w14[:C].shape) * 0.05
            S.ss_net_set_params(net, np.concatenate([np.concatenate([w.ravel(), b]) for w, b in sl]))
            f, coup, _ = random_problem(rng, 2, 128, C, ncoup)
            if theory == 2:
                f /= np.linalg.norm(f, axis=1, keepdims=True) + 1e-12
            fd = torch.tensor(f, dtype=torch.float32, device="cuda")
            init = torch.zeros_like(fd)
            S.ss_net_predict(net, fd, coup[:, 0] if coup is not None else None, 2, init)
            g = init.cpu().numpy()
            a = fd.cpu().numpy()
            halo = np.ones((128, 128), bool)
            halo[2:-2, 2:-2] = False
            assert np.array_equal(g[..., halo], a[..., halo])
            assert np.abs(g[..., ~halo] - a[..., ~halo]).max() > 0  # the correction is applied
            if theory == 2:
                nrm = np.linalg.norm(g[..., 2:-2, 2:-2], axis=1)
                assert np.abs(nrm - 1).max() < 1e-6
        finally:
            S.ss_net_destroy(net)


def test_save_and_load_round_trip(S):
    net = S.ss_net_create(S.SS_ABELIAN_HIGGS, 128, 1, seed=1)
    net2 = S.ss_net_create(S.SS_ABELIAN_HIGGS, 128, 1, seed=2)
    try:
        with tempfile.TemporaryDirectory() as d:
            p = os.path.join(d, "net.bin")
            S.ss_net_save(net, p)
            assert not np.array_equal(S.ss_net_get_params(net), S.ss_net_get_params(net2))
            S.ss_net_load(net2, p)
            assert np.array_equal(S.ss_net_get_params(net), S.ss_net_get_params(net2))
        cm = S.ss_net_create(S.SS_CHIRAL_MAGNET, 128, 1)
        try:
            with tempfile.TemporaryDirectory() as d:
                p = os.path.join(d, "net.bin")
                S.ss_net_save(net, p)
                with pytest.raises(S.SolitonError):
                    S.ss_net_load(cm, p)
        finally:
            S.ss_net_destroy(cm)
    finally:
        S.ss_net_destroy(net)
        S.ss_net_destroy(net2)


def test_a_stalled_wait_times_out_and_the_device_stays_usable(S):
    """The kernels' bounded wait on a barrier nothing completes gives up after its
    limit and reports SS_ERR_TIMEOUT; a convolution afterwards still matches."""
    import time
    t0 = time.perf_counter()
    assert S.ss_wait_selftest(50000) == S.SS_ERR_TIMEOUT  # 50 ms limit
    assert time.perf_counter() - t0 < 5.0
    test_conv_forward_matches_oracle(S, CONV_CASES[0], 2)
