"""Learned initialisation workflow on top of the C-ABI.

1. ``relax_set``: relax a list of problems with the batched flow and keep, per
   problem, the ansatz it started from and the field it reached (device tensors,
   FP32 SoA [n][C][S][S]).
2. ``train``: fit the U-Net (soliton_net.h) to map each ansatz (and its couplings)
   to relaxed - ansatz, with Adam and a cosine learning-rate schedule.
3. ``solve``: relax problems with the batched flow from the ansatz, or from the
   network's prediction; the flow finishes every solve either way and its
   observables judge the result.

Everything that computes runs in libsoliton.so; this module only sequences calls
and owns device buffers (through PyTorch tensors).

Command line (one GPU):
    python -m paper_2603_24370_gb300.learned --count 2048 --epochs 40 --out ah256.net
    python -m paper_2603_24370_gb300.learned --theory cm --count 2048 --large   # + the 4096^2 workload
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs as I
from . import soliton as S


def _torch():
    import torch
    return torch


def relax_set(problems, tol: float, max_steps: int, chunk: int = 256, precision: int = S.SS_FP32,
              horizon: int = 0):
    """Ansatz and relaxed fields (device FP32 [n][C][S][S]) of problems of one size,
    their couplings (lambda for the Abelian Higgs) and per-problem statuses. With
    horizon > 0 the "relaxed" field is the flow's state after that many steps (or
    earlier convergence) instead of the converged one."""
    torch = _torch()
    theory = problems[0].theory
    C = 4 if theory == S.SS_ABELIAN_HIGGS else 3
    n, side = len(problems), problems[0].nx
    assert all(p.nx == side and p.ny == side for p in problems)
    ansatz = torch.empty((n, C, side, side), dtype=torch.float32, device="cuda")
    relaxed = torch.empty_like(ansatz)
    statuses = []
    for i0 in range(0, n, chunk):
        part = problems[i0:i0 + chunk]
        b = S.ss_batch_create(theory, precision, part)
        try:
            for k in range(len(part)):
                S.ss_batch_get_fields(b, k, ansatz[i0 + k])
            if horizon > 0:
                _, st = S.ss_batch_step(b, horizon)
            else:
                _, st = S.ss_batch_minimise(b, tol, max_steps)
            for k in range(len(part)):
                S.ss_batch_get_fields(b, k, relaxed[i0 + k])
            statuses += st
        finally:
            S.ss_batch_destroy(b)
    couplings = np.array([p.params[0] for p in problems]) if theory == S.SS_ABELIAN_HIGGS else None
    return ansatz, relaxed, couplings, statuses


def train(net, ansatz, relaxed, couplings, epochs: int, batch: int, lr: float, seed: int = 0, log=None):
    """Adam over contiguous mini-batches visited in a seeded random order each epoch;
    lr follows a cosine from `lr` to lr / 20. Returns the mean loss of every epoch."""
    n = ansatz.shape[0]
    starts = list(range(0, n - batch + 1, batch))
    rng = np.random.default_rng(seed)
    total, t, history = epochs * len(starts), 0, []
    for ep in range(epochs):
        losses = []
        for s0 in rng.permutation(starts):
            f = lr * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * t / max(total - 1, 1))))
            cp = couplings[s0:s0 + batch] if couplings is not None else None
            losses.append(S.ss_net_train_step(net, ansatz[s0:s0 + batch], cp, relaxed[s0:s0 + batch], batch, f))
            t += 1
        history.append(float(np.mean(losses)))
        if log:
            log(f"epoch {ep}: loss {history[-1]:.4e}")
    return history


def predict(net, ansatz, couplings, batch: int):
    """Network initial fields for every problem (device FP32, the layout of ansatz)."""
    torch = _torch()
    init = torch.empty_like(ansatz)
    n = ansatz.shape[0]
    for s0 in range(0, n, batch):
        b = min(batch, n - s0)
        cp = couplings[s0:s0 + b] if couplings is not None else None
        S.ss_net_predict(net, ansatz[s0:s0 + b], cp, b, init[s0:s0 + b])
    return init


def solve(problems, tol: float, max_steps: int, init=None, precision: int = S.SS_FP32):
    """Relax all problems in one batch, from the ansatz or from `init` (device fields of
    the batch's precision). Returns (wall seconds, statuses, observables)."""
    torch = _torch()
    b = S.ss_batch_create(problems[0].theory, precision, problems)
    try:
        if init is not None:
            for k in range(len(problems)):
                S.ss_batch_set_fields(b, k, init[k])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st = S.ss_batch_minimise(b, tol, max_steps)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        obs = [S.ss_batch_observables(b, k) for k in range(len(problems))]
    finally:
        S.ss_batch_destroy(b)
    return sec, st, obs


def large_start(net, a) -> dict:
    """The 4096^2, 400-skyrmion chiral magnet relaxed to a.tol from the ansatz and from
    the network's prediction (the trained weights applied at that size)."""
    torch = _torch()
    p = I.cm_skyrmions(n=4096, count=400, seed=20264)
    big = S.ss_net_create(S.SS_CHIRAL_MAGNET, 4096, 1, seed=0)
    try:
        S.ss_net_set_params(big, S.ss_net_get_params(net))
        out = {}
        for start in ("ansatz", "network"):
            with S.Solver(S.SS_CHIRAL_MAGNET, p.params, p.nx, p.ny, p.dx, p.dy, S.SS_FP32) as sv:
                sv.init_ansatz(p.soliton_array())
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if start == "network":
                    f = torch.empty((1, 3, p.ny, p.nx), dtype=torch.float32, device="cuda")
                    S.ss_get_fields(sv.ctx, f[0])
                    init = torch.empty_like(f)
                    S.ss_net_predict(big, f, None, 1, init)
                    sv.set_fields(init[0].contiguous())
                sv.autotune(4)
                st = sv.minimise(a.tol, 100000)
                torch.cuda.synchronize()
                o = sv.observables()
                out[start] = {"seconds": time.perf_counter() - t0, "steps": st["steps"],
                              "converged": bool(st["converged"]), "energy": o["energy"], "charge": o["charge"]}
        return out
    finally:
        S.ss_net_destroy(big)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--count", type=int, default=2048, help="training problems")
    ap.add_argument("--test", type=int, default=128, help="held-out problems")
    ap.add_argument("--side", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-steps", type=int, default=30000)
    ap.add_argument("--seed", type=int, default=20263)
    ap.add_argument("--out", default=None, help="save the trained parameters here")
    ap.add_argument("--report", default=None, help="write a JSON summary here")
    ap.add_argument("--horizon", type=int, default=0,
                    help="train on the flow's state after this many steps instead of the converged field")
    ap.add_argument("--theory", choices=("ah", "cm"), default="ah")
    ap.add_argument("--large", action="store_true",
                    help="chiral magnet: also start the 4096^2, 400-skyrmion workload from the network")
    a = ap.parse_args(argv)
    torch = _torch()
    torch.cuda.init()
    S.load_library()
    theory = S.SS_ABELIAN_HIGGS if a.theory == "ah" else S.SS_CHIRAL_MAGNET
    if theory == S.SS_ABELIAN_HIGGS:
        probs = I.ah_learned_set(a.count + a.test, a.seed, side=a.side)
    else:
        probs = I.cm_learned_set(a.count + a.test, a.seed + 2, side=a.side)
    train_p, test_p = probs[:a.count], probs[a.count:]
    t0 = time.perf_counter()
    ansatz, relaxed, cp, st = relax_set(train_p, a.tol, a.max_steps, horizon=a.horizon)
    t_data = time.perf_counter() - t0
    conv = sum(1 for s in st if s["converged"])
    print(f"relaxed {a.count} training problems in {t_data:.1f} s ({conv} converged)", flush=True)
    net = S.ss_net_create(theory, a.side, a.batch, seed=a.seed)
    try:
        t0 = time.perf_counter()
        hist = train(net, ansatz, relaxed, cp, a.epochs, a.batch, a.lr, seed=a.seed,
                     log=lambda m: print(m, flush=True))
        t_train = time.perf_counter() - t0
        if a.out:
            S.ss_net_save(net, a.out)
        # held-out: plain flow from the ansatz vs flow from the network's prediction
        ta, tr, tcp, _ = relax_set(test_p, a.tol, a.max_steps, horizon=a.horizon)
        init = predict(net, ta, tcp, a.batch)
        # distance of each start to the held-out reference state (RMS over all values)
        dist_plain = float(((ta - tr) ** 2).mean().sqrt())
        dist_net = float(((init - tr) ** 2).mean().sqrt())
        # looser tolerances first: where along the flow the prediction saves steps
        ladder = {}
        for tol in (1e-4, 1e-5):
            s_p, st_p, _ = solve(test_p, tol, a.max_steps)
            s_n, st_n, _ = solve(test_p, tol, a.max_steps, init=init)
            ladder[f"{tol:g}"] = {"plain_mean_steps": float(np.mean([s["steps"] for s in st_p])),
                                  "learned_mean_steps": float(np.mean([s["steps"] for s in st_n])),
                                  "plain_seconds": s_p, "learned_seconds": s_n}
        sec_plain, st_plain, ob_plain = solve(test_p, a.tol, a.max_steps)
        sec_net, st_net, ob_net = solve(test_p, a.tol, a.max_steps, init=init)
        large = large_start(net, a) if (a.large and theory == S.SS_CHIRAL_MAGNET) else None
    finally:
        S.ss_net_destroy(net)
    rep = {
        "train_problems": a.count, "test_problems": a.test, "side": a.side, "epochs": a.epochs,
        "horizon": a.horizon, "rms_to_reference": {"ansatz": dist_plain, "network": dist_net},
        "relax_seconds": t_data, "train_seconds": t_train, "loss_first_last": [hist[0], hist[-1]],
        "plain": {"seconds": sec_plain, "mean_steps": float(np.mean([s["steps"] for s in st_plain])),
                  "converged": sum(1 for s in st_plain if s["converged"])},
        "learned": {"seconds": sec_net, "mean_steps": float(np.mean([s["steps"] for s in st_net])),
                    "converged": sum(1 for s in st_net if s["converged"])},
        "max_rel_energy_diff": float(max(abs(x["energy"] - y["energy"]) / abs(y["energy"])
                                         for x, y in zip(ob_net, ob_plain))),
        "charges_equal": all(round(x["charge"]) == round(y["charge"]) for x, y in zip(ob_net, ob_plain)),
        "looser_tolerances": ladder,
        "large": large,
    }
    print(json.dumps(rep), flush=True)
    if a.report:
        with open(a.report, "w") as fh:
            json.dump(rep, fh, indent=1)


if __name__ == "__main__":
    main()
