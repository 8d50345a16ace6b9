"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle's tests.

This module only draws numbers: soliton positions, charges and couplings for the
workloads, and smooth test fields. It holds none of the method's arithmetic (no
stencil, energy, force, ansatz or flow): both sides receive the same arrays and
compute from them independently.

The generator is SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written from its published
definition, so the draws are identical on every machine.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_M64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform double in [lo, hi) from the top 53 bits."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def choice(self, options):
        return options[self.next_u64() % len(options)]


# theory ids (same numbering as the C-ABI and the oracle)
ABELIAN_HIGGS = 1
CHIRAL_MAGNET = 2
BABY_SKYRME = 3
BEC = 4
SID = 5
CM_DEMAG = 6

# Couplings of the workloads. Abelian Higgs: (lambda, u). Chiral magnet:
# (J, D, K, h, dmi_type) with interfacial DMI (type 0).
AH_CRITICAL = (1.0, 1.0)
CM_DEFAULT = (1.0, 1.0, 0.1, 0.6, 0.0)


@dataclass
class Problem:
    """One relaxation problem: grid, couplings and initial solitons."""
    theory: int
    nx: int
    ny: int
    dx: float
    dy: float
    params: tuple
    solitons: list = field(default_factory=list)  # rows (x, y, charge, size, phase)

    @property
    def interior_sites(self) -> int:
        return (self.nx - 4) * (self.ny - 4)

    def soliton_array(self) -> np.ndarray:
        return np.asarray(self.solitons, dtype=np.float64).reshape(-1, 5)


def ah_single_vortex(n: int = 128, dx: float = 0.1, lam: float = 1.0) -> Problem:
    """Abelian Higgs at critical coupling, one N=1 vortex at the centre (128^2, dx 0.1)."""
    return Problem(ABELIAN_HIGGS, n, n, dx, dx, (lam, 1.0), [(0.0, 0.0, 1.0, 1.0, 0.0)])


def _separated_positions(rng: SplitMix64, count: int, half_x: float, half_y: float, margin: float,
                         min_sep: float, max_tries: int = 1_000_000):
    """Rejection sampling: uniform in the box shrunk by ``margin``, pairwise >= min_sep."""
    pts: list[tuple[float, float]] = []
    tries = 0
    while len(pts) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place solitons with the requested separation")
        x = rng.uniform(-half_x + margin, half_x - margin)
        y = rng.uniform(-half_y + margin, half_y - margin)
        if all((x - a) ** 2 + (y - b) ** 2 >= min_sep * min_sep for a, b in pts):
            pts.append((x, y))
    return pts


def cm_skyrmions(n: int = 1024, count: int = 8, dx: float = 0.2, seed: int = 20261, radius: float = 2.0,
                 min_sep: float = 8.0, margin: float = 8.0, params=CM_DEFAULT) -> Problem:
    """Chiral magnet with ``count`` compact skyrmions (R = 2, helicity 0) at seeded
    uniform positions, minimum separation 8 and margin 8 from the edge."""
    rng = SplitMix64(seed)
    half = 0.5 * (n - 1) * dx
    pts = _separated_positions(rng, count, half, half, margin, min_sep)
    sol = [(x, y, 1.0, radius, 0.0) for x, y in pts]
    return Problem(CHIRAL_MAGNET, n, n, dx, dx, tuple(params), sol)


BS_DEFAULT = (1.0, 0.7, 0.0)  # kappa, mu, nu: standard potential


def bs_skyrmions(n: int = 2048, count: int = 100, dx: float = 0.2, seed: int = 20265, radius: float = 2.5,
                 min_sep: float = 10.0, margin: float = 8.0, params=BS_DEFAULT) -> Problem:
    """Baby Skyrme model with ``count`` compact charge-1 skyrmions (R = 2.5) at seeded
    uniform positions, minimum separation 10 and margin 8 from the edge."""
    rng = SplitMix64(seed)
    half = 0.5 * (n - 1) * dx
    pts = _separated_positions(rng, count, half, half, margin, min_sep)
    sol = [(x, y, 1.0, radius, 0.0) for x, y in pts]
    return Problem(BABY_SKYRME, n, n, dx, dx, tuple(params), sol)


def ah_batch(count: int = 256, seed: int = 20262, sides=(64, 128, 256, 512), dx: float = 0.1,
             lam_range=(0.5, 2.0), charges=(1, 2, 3, 4)) -> list[Problem]:
    """Batched Abelian Higgs set: side ~ U(sides), lambda ~ U[0.5, 2], N ~ U(charges),
    N unit vortices uniform in the central half [-L/4, L/4]^2."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        side = rng.choice(sides)
        lam = rng.uniform(*lam_range)
        nv = rng.choice(charges)
        L = side * dx
        sol = [(rng.uniform(-L / 4, L / 4), rng.uniform(-L / 4, L / 4), 1.0, 1.0, 0.0) for _ in range(nv)]
        out.append(Problem(ABELIAN_HIGGS, side, side, dx, dx, (lam, 1.0), sol))
    return out


def ah_learned_set(count: int = 20000, seed: int = 20263, side: int = 256, dx: float = 0.1,
                   lam_range=(0.5, 2.0), charges=(1, 2, 3, 4, 5, 6)) -> list[Problem]:
    """Training set of the learned initialiser: Abelian Higgs on side x side grids,
    lambda ~ U[0.5, 2], N ~ U{1..6} unit vortices uniform in the central half."""
    return ah_batch(count, seed, (side,), dx, lam_range, charges)


def cm_learned_set(count: int = 2048, seed: int = 20265, side: int = 256, dx: float = 0.2, max_count: int = 4,
                   radius: float = 2.0, min_sep: float = 8.0, margin: float = 8.0, params=CM_DEFAULT) -> list[Problem]:
    """Training set of the chiral-magnet initialiser: side x side grids with 1..max_count
    compact skyrmions (R = 2) at seeded positions, the separation and margin of the
    4096^2 workload, the same couplings."""
    rng = SplitMix64(seed)
    half = 0.5 * (side - 1) * dx
    out = []
    for _ in range(count):
        k = 1 + (rng.next_u64() % max_count)
        pts = _separated_positions(rng, k, half, half, margin, min_sep)
        sol = [(x, y, 1.0, radius, 0.0) for x, y in pts]
        out.append(Problem(CHIRAL_MAGNET, side, side, dx, dx, tuple(params), sol))
    return out


def smooth_field(theory: int, nx: int, ny: int, dx: float, dy: float, seed: int, bumps: int = 6,
                 amplitude: float = 0.3) -> np.ndarray:
    """A smooth random test field, float64 [C][ny][nx].

    Abelian Higgs: psi = (1 + s_1) + i s_2, A = (s_3, s_4), each s_c a sum of
    Gaussian bumps with seeded centres, widths and amplitudes. Chiral magnet and
    Baby Skyrme: a unit field from smooth angles, n = (sin T cos P, sin T sin P,
    cos T) with T, P sums of Gaussian bumps (unit length by construction, no
    normalisation). BEC: psi = env (1 + s_1) + i env s_2 with a Gaussian envelope
    env that is small at the edge of the box. s+id: Delta_s = (1 + s_1) + i s_2,
    Delta_d = (0.5 + s_3) + i (0.5 + s_4), A = (s_5, s_6).
    """
    rng = SplitMix64(seed)
    x = (np.arange(nx) - 0.5 * (nx - 1)) * dx
    y = (np.arange(ny) - 0.5 * (ny - 1)) * dy
    X, Y = np.meshgrid(x, y)
    Lx, Ly = 0.5 * (nx - 1) * dx, 0.5 * (ny - 1) * dy

    def bumpsum():
        s = np.zeros_like(X)
        for _ in range(bumps):
            cx, cy = rng.uniform(-0.6 * Lx, 0.6 * Lx), rng.uniform(-0.6 * Ly, 0.6 * Ly)
            w = rng.uniform(0.15, 0.35) * min(Lx, Ly)
            a = rng.uniform(-amplitude, amplitude)
            s += a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (w * w))
        return s

    if theory == ABELIAN_HIGGS:
        return np.stack([1.0 + bumpsum(), bumpsum(), bumpsum(), bumpsum()])
    if theory == BEC:
        env = np.exp(-(X * X + Y * Y) / (0.25 * min(Lx, Ly) ** 2))
        return np.stack([env * (1.0 + bumpsum()), env * bumpsum()])
    if theory == SID:
        return np.stack([1.0 + bumpsum(), bumpsum(), 0.5 + bumpsum(), 0.5 + bumpsum(), bumpsum(), bumpsum()])
    if theory in (CHIRAL_MAGNET, BABY_SKYRME, CM_DEMAG):
        T = 0.6 + 3.0 * bumpsum()
        P = 5.0 * bumpsum()
        return np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)])
    raise ValueError(f"unknown theory {theory}")


def smooth_velocity(theory: int, nx: int, ny: int, dx: float, dy: float, seed: int, amplitude: float = 0.05):
    """A smooth random velocity field, zero on the width-2 halo (for trajectory tests)."""
    rng = SplitMix64(seed)
    C = {ABELIAN_HIGGS: 4, BEC: 2, SID: 6}.get(theory, 3)
    x = (np.arange(nx) - 0.5 * (nx - 1)) * dx
    y = (np.arange(ny) - 0.5 * (ny - 1)) * dy
    X, Y = np.meshgrid(x, y)
    Lx, Ly = 0.5 * (nx - 1) * dx, 0.5 * (ny - 1) * dy
    v = np.zeros((C, ny, nx))
    for c in range(C):
        for _ in range(3):
            cx, cy = rng.uniform(-0.5 * Lx, 0.5 * Lx), rng.uniform(-0.5 * Ly, 0.5 * Ly)
            w = rng.uniform(0.2, 0.4) * min(Lx, Ly)
            v[c] += rng.uniform(-amplitude, amplitude) * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (w * w))
    v[:, :2, :] = 0.0
    v[:, -2:, :] = 0.0
    v[:, :, :2] = 0.0
    v[:, :, -2:] = 0.0
    return v
