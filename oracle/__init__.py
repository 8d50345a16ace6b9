"""FP64 CPU oracle of the soliton relaxation method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package. The CUDA product path never calls it and
shares no code with it (``soliton_oracle.cpp`` includes nothing of the product).

Every function follows the paper step by step (equation numbers in order of
appearance, see ``soliton_oracle.cpp``):

* ``derivatives``          -- Eq. 1, Eq. 2 and the composed mixed derivative (Sec. 3.1)
* ``energy`` / ``energy_density`` -- E_h of Table 1 (Abelian Higgs, Baby Skyrme, BEC, s+id)
  and Eq. 5 (chiral magnet, also with the magnetostatic term of Eq. 6: ``demag_*``)
* ``force``                -- Euler-Lagrange residual G driving Eq. 3
* ``energy_grad_exact``    -- exact dE_h/dphi, only for pinning ``force``
* ``anf_step`` / ``minimise`` -- arrested Newton flow, RK4 + Eq. 4 (Sec. 3.2)
* ``gd_step`` / ``gd_minimise`` / ``gd_step_limit`` -- the first-order gradient
  descent Sec. 3.2 names as the slower alternative (explicit Euler, see the C++)
* ``observables``          -- energy, topological charge, flux, residual, |n|-1
* ``ansatz`` / ``ansatz_bec`` / ``ansatz_sid`` -- initial data (Sec. 3.4; standard forms)

All functions are pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

ABELIAN_HIGGS = 1
CHIRAL_MAGNET = 2
BABY_SKYRME = 3
BEC = 4
SID = 5
CM_DEMAG = 6
HARMONIC_TEST = 99

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "soliton_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_STAMP = _LIB_PATH + ".arch"
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` in-tree with g++ (OpenMP when available)."""
    if (not force and os.path.exists(_LIB_PATH) and os.path.exists(_STAMP)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
            and open(_STAMP).read().strip() == platform.machine()):
        return _LIB_PATH
    base = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", _SRC, "-o", _LIB_PATH + ".tmp"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    with open(_STAMP, "w") as fh:
        fh.write(platform.machine())
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i, d, ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
            lib.or_num_threads.argtypes = []
            lib.or_num_threads.restype = i
            lib.or_ncomp.argtypes = [i]
            lib.or_ncomp.restype = i
            lib.or_time_step.argtypes = [d, d]
            lib.or_time_step.restype = d
            lib.or_derivatives.argtypes = [_D, i, i, d, d, _D, _D, _D, _D, _D]
            lib.or_derivatives.restype = None
            lib.or_energy_density.argtypes = [i, _D, _D, i, i, d, d, _D]
            lib.or_energy_density.restype = None
            lib.or_energy.argtypes = [i, _D, _D, i, i, d, d]
            lib.or_energy.restype = d
            lib.or_force.argtypes = [i, _D, _D, i, i, d, d, _D]
            lib.or_force.restype = None
            lib.or_energy_grad_exact.argtypes = [i, _D, _D, i, i, d, d, _D]
            lib.or_energy_grad_exact.restype = None
            lib.or_anf_step.argtypes = [i, _D, _D, _D, i, i, d, d, d, _D]
            lib.or_anf_step.restype = i
            lib.or_minimise.argtypes = [i, _D, _D, _D, i, i, d, d, d, d, ll, _D]
            lib.or_minimise.restype = i
            lib.or_gd_step.argtypes = [i, _D, _D, i, i, d, d, d, _D]
            lib.or_gd_step.restype = i
            lib.or_gd_step_limit.argtypes = [d, d]
            lib.or_gd_step_limit.restype = d
            lib.or_gd_minimise.argtypes = [i, _D, _D, i, i, d, d, d, d, ll, _D]
            lib.or_gd_minimise.restype = i
            lib.or_observables.argtypes = [i, _D, _D, i, i, d, d, _D]
            lib.or_observables.restype = None
            lib.or_ansatz.argtypes = [i, _D, i, _D, i, i, d, d]
            lib.or_ansatz_bec.argtypes = [_D, _D, i, _D, i, i, d, d]
            lib.or_demag_potential.argtypes = [_D, i, i, d, d, _D, _D]
            lib.or_demag_box.argtypes = [i, ctypes.POINTER(ctypes.c_int)]
            lib.or_demag_box.restype = None
            lib.or_demag_box_potential.argtypes = [_D, i, i, d, d, _D]
            lib.or_demag_box_potential.restype = None
            lib.or_demag_potential.restype = None
            lib.or_demag_energy.argtypes = [_D, _D, i, i, d, d]
            lib.or_demag_energy.restype = d
            lib.or_ansatz_sid.argtypes = [_D, _D, i, _D, i, i, d, d, _D]
            lib.or_ansatz_sid.restype = None
            lib.or_ansatz_bec.restype = None
            lib.or_ansatz.restype = None
            lib.or_bec_multiplier.argtypes = [_D, _D, i, i, d, d]
            lib.or_bec_multiplier.restype = d
            lib.or_bec_refresh.argtypes = [_D, d, _D, ctypes.c_void_p, i, i, d, d, _D]
            lib.or_bec_refresh.restype = i
            lib.or_anf_step_fixed_n.argtypes = [_D, d, _D, _D, i, i, d, d, d, _D, _D]
            lib.or_anf_step_fixed_n.restype = i
            lib.or_minimise_fixed_n.argtypes = [_D, d, _D, _D, i, i, d, d, d, d, ll, _D]
            lib.or_minimise_fixed_n.restype = i
            lib.or_gd_minimise_fixed_n.argtypes = [_D, d, _D, i, i, d, d, d, d, ll, _D]
            lib.or_gd_minimise_fixed_n.restype = i
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _params(params) -> np.ndarray:
    return _f64(np.asarray(params, dtype=np.float64).reshape(-1))


def num_threads() -> int:
    """Threads used by the oracle's parallel loops."""
    return _load().or_num_threads()


def ncomp(theory: int) -> int:
    return _load().or_ncomp(theory)


def time_step(dx: float, dy: float) -> float:
    """dt = C min(dx, dy), C = 0.5 (Sec. 3.1)."""
    return _load().or_time_step(dx, dy)


def derivatives(plane, dx: float, dy: float) -> dict:
    p = _f64(plane)
    ny, nx = p.shape
    outs = {k: np.zeros_like(p) for k in ("fx", "fy", "fxx", "fyy", "fxy")}
    _load().or_derivatives(_p(p), nx, ny, dx, dy, *(_p(outs[k]) for k in ("fx", "fy", "fxx", "fyy", "fxy")))
    return outs


def energy(theory: int, params, f, dx: float, dy: float) -> float:
    f = _f64(f)
    _, ny, nx = f.shape
    return _load().or_energy(theory, _p(_params(params)), _p(f), nx, ny, dx, dy)


def energy_density(theory: int, params, f, dx: float, dy: float) -> np.ndarray:
    f = _f64(f)
    _, ny, nx = f.shape
    e = np.zeros((ny, nx))
    _load().or_energy_density(theory, _p(_params(params)), _p(f), nx, ny, dx, dy, _p(e))
    return e


def force(theory: int, params, f, dx: float, dy: float) -> np.ndarray:
    f = _f64(f)
    _, ny, nx = f.shape
    G = np.zeros_like(f)
    _load().or_force(theory, _p(_params(params)), _p(f), nx, ny, dx, dy, _p(G))
    return G


def energy_grad_exact(theory: int, params, f, dx: float, dy: float) -> np.ndarray:
    f = _f64(f)
    _, ny, nx = f.shape
    g = np.zeros_like(f)
    _load().or_energy_grad_exact(theory, _p(_params(params)), _p(f), nx, ny, dx, dy, _p(g))
    return g


def anf_step(theory: int, params, f, v, dx: float, dy: float, dt: float, E: float):
    """One arrested-Newton-flow RK4 step. Returns (f_new, v_new, E_new, arrested)."""
    f = _f64(f).copy()
    v = _f64(v).copy()
    _, ny, nx = f.shape
    e = np.array([E], dtype=np.float64)
    arrested = _load().or_anf_step(theory, _p(_params(params)), _p(f), _p(v), nx, ny, dx, dy, dt, _p(e))
    return f, v, float(e[0]), bool(arrested)


def minimise(theory: int, params, f, dx: float, dy: float, tol: float, max_steps: int, v=None, dt=None) -> dict:
    """Arrested Newton flow from rest (unless ``v`` is given) until dx dy max|G| < tol."""
    f = _f64(f).copy()
    v = np.zeros_like(f) if v is None else _f64(v).copy()
    _, ny, nx = f.shape
    dt = time_step(dx, dy) if dt is None else dt
    out = np.zeros(4)
    conv = _load().or_minimise(theory, _p(_params(params)), _p(f), _p(v), nx, ny, dx, dy, dt, tol, int(max_steps),
                               _p(out))
    return {"f": f, "v": v, "energy": out[0], "grad_max": out[1], "steps": int(out[2]), "arrests": int(out[3]),
            "converged": bool(conv)}


def gd_step_limit(dx: float, dy: float) -> float:
    """Euler stability limit of gradient descent for the Eq. 2 Laplacian."""
    return _load().or_gd_step_limit(dx, dy)


def gd_step(theory: int, params, f, dx: float, dy: float, dtau: float, E: float):
    """One gradient-descent step phi - dtau G(phi). Returns (f_new, E_new, energy_rose)."""
    f = _f64(f).copy()
    _, ny, nx = f.shape
    e = np.array([E], dtype=np.float64)
    rose = _load().or_gd_step(theory, _p(_params(params)), _p(f), nx, ny, dx, dy, dtau, _p(e))
    return f, float(e[0]), bool(rose)


def gd_minimise(theory: int, params, f, dx: float, dy: float, tol: float, max_steps: int, dtau=None,
                step_factor: float = 0.8) -> dict:
    """Gradient descent until dx dy max|G| < tol; dtau defaults to step_factor x the stability limit."""
    f = _f64(f).copy()
    _, ny, nx = f.shape
    dtau = step_factor * gd_step_limit(dx, dy) if dtau is None else dtau
    out = np.zeros(4)
    conv = _load().or_gd_minimise(theory, _p(_params(params)), _p(f), nx, ny, dx, dy, dtau, tol, int(max_steps),
                                  _p(out))
    return {"f": f, "energy": out[0], "grad_max": out[1], "steps": int(out[2]), "rises": int(out[3]),
            "converged": bool(conv), "dtau": dtau}


def observables(theory: int, params, f, dx: float, dy: float) -> dict:
    f = _f64(f)
    _, ny, nx = f.shape
    out = np.zeros(8)
    _load().or_observables(theory, _p(_params(params)), _p(f), nx, ny, dx, dy, _p(out))
    return {"energy": out[0], "charge": out[1], "flux": out[2], "grad_max": out[3], "grad_max_raw": out[4],
            "norm_dev": out[5], "atoms": out[6], "angular_momentum": out[7]}


def bec_multiplier(params, f, dx: float, dy: float) -> float:
    """Lagrange multiplier of the atom-number constraint at a BEC field as it stands,
    sum_I G_0.psi / (2 sum_I |psi|^2) (params {g, Omega[, ...]}; see the C++)."""
    f = _f64(f)
    _, ny, nx = f.shape
    return _load().or_bec_multiplier(_p(_params(params)), _p(f), nx, ny, dx, dy)


def bec_refresh(params, atoms: float, f, v, dx: float, dy: float):
    """Fixed-atom-number refresh of a new BEC field: v tangent to N_h = const, psi scaled
    on I to N_h = atoms, the multiplier of the scaled field. Returns (f, v, mu); v may
    be None."""
    f = _f64(f).copy()
    v = None if v is None else _f64(v).copy()
    _, ny, nx = f.shape
    mu = np.zeros(1)
    rc = _load().or_bec_refresh(_p(_params(params)), atoms, _p(f), None if v is None else _p(v), nx, ny, dx, dy,
                                _p(mu))
    if rc != 0:
        raise ValueError("bec_refresh: the field has no atoms")
    return f, v, float(mu[0])


def anf_step_fixed_n(params, atoms: float, f, v, dx: float, dy: float, dt: float, E: float, mu: float):
    """One fixed-atom-number step from a refreshed (f, v) with multiplier mu and energy
    E (at mu = 0). Returns (f_new, v_new, E_new, mu_new, arrested)."""
    f = _f64(f).copy()
    v = _f64(v).copy()
    _, ny, nx = f.shape
    e, m = np.array([E]), np.array([mu])
    a = _load().or_anf_step_fixed_n(_p(_params(params)), atoms, _p(f), _p(v), nx, ny, dx, dy, dt, _p(e), _p(m))
    if a < 0:
        raise ValueError("anf_step_fixed_n: the field has no atoms")
    return f, v, float(e[0]), float(m[0]), bool(a)


def minimise_fixed_n(params, atoms: float, f, dx: float, dy: float, tol: float, max_steps: int, v=None,
                     dt=None) -> dict:
    """Arrested Newton flow of the BEC at fixed atom number (params {g, Omega[, ...]})."""
    f = _f64(f).copy()
    v = np.zeros_like(f) if v is None else _f64(v).copy()
    _, ny, nx = f.shape
    dt = time_step(dx, dy) if dt is None else dt
    out = np.zeros(5)
    conv = _load().or_minimise_fixed_n(_p(_params(params)), atoms, _p(f), _p(v), nx, ny, dx, dy, dt, tol,
                                       int(max_steps), _p(out))
    if conv < 0:
        raise ValueError("minimise_fixed_n: the field has no atoms")
    return {"f": f, "v": v, "energy": out[0], "grad_max": out[1], "steps": int(out[2]), "arrests": int(out[3]),
            "mu": out[4], "converged": bool(conv)}


def gd_minimise_fixed_n(params, atoms: float, f, dx: float, dy: float, tol: float, max_steps: int, dtau=None,
                        step_factor: float = 0.8) -> dict:
    """Gradient descent of the BEC at fixed atom number."""
    f = _f64(f).copy()
    _, ny, nx = f.shape
    dtau = step_factor * gd_step_limit(dx, dy) if dtau is None else dtau
    out = np.zeros(5)
    conv = _load().or_gd_minimise_fixed_n(_p(_params(params)), atoms, _p(f), nx, ny, dx, dy, dtau, tol,
                                          int(max_steps), _p(out))
    if conv < 0:
        raise ValueError("gd_minimise_fixed_n: the field has no atoms")
    return {"f": f, "energy": out[0], "grad_max": out[1], "steps": int(out[2]), "rises": int(out[3]),
            "mu": out[4], "converged": bool(conv), "dtau": dtau}


def demag_potential(f, dx: float, dy: float):
    """Magnetostatic charge and potential (rho, psi) of a field, Eq. 6 (see the C++)."""
    f = _f64(f)
    _, ny, nx = f.shape
    rho, psi = np.zeros((ny, nx)), np.zeros((ny, nx))
    _load().or_demag_potential(_p(f), nx, ny, dx, dy, _p(rho), _p(psi))
    return rho, psi


def demag_box(N: int):
    """The Dirichlet box of an axis with N interior sites: (N', sites added below I)."""
    out = (ctypes.c_int * 2)()
    _load().or_demag_box(int(N), out)
    return out[0], out[1]


def demag_box_potential(f, dx: float, dy: float) -> np.ndarray:
    """psi on the whole Dirichlet box, [Ny' + 2][Nx' + 2] with its zero outer nodes."""
    f = _f64(f)
    _, ny, nx = f.shape
    Nx, _ = demag_box(nx - 4)
    Ny, _ = demag_box(ny - 4)
    box = np.zeros((Ny + 2, Nx + 2))
    _load().or_demag_box_potential(_p(f), nx, ny, dx, dy, _p(box))
    return box


def demag_energy(params, f, dx: float, dy: float) -> float:
    f = _f64(f)
    _, ny, nx = f.shape
    return _load().or_demag_energy(_p(_params(params)), _p(f), nx, ny, dx, dy)


def ansatz_bec(params, vortices, nx: int, ny: int, dx: float, dy: float) -> np.ndarray:
    """Thomas-Fermi amplitude times vortex factors; ``vortices`` rows (x, y, n, size, phase)."""
    s = _f64(np.asarray(vortices, dtype=np.float64).reshape(-1, 5))
    f = np.zeros((2, ny, nx))
    _load().or_ansatz_bec(_p(_params(params)), _p(s), s.shape[0], _p(f), nx, ny, dx, dy)
    return f


def ansatz_sid(params, vortices, nx: int, ny: int, dx: float, dy: float):
    """s+id vortices on the uniform minimum; returns (field, (S, D, relative phase))."""
    s = _f64(np.asarray(vortices, dtype=np.float64).reshape(-1, 5))
    f = np.zeros((6, ny, nx))
    m = np.zeros(3)
    _load().or_ansatz_sid(_p(_params(params)), _p(s), s.shape[0], _p(f), nx, ny, dx, dy, _p(m))
    return f, tuple(m)


def ansatz(theory: int, solitons, nx: int, ny: int, dx: float, dy: float) -> np.ndarray:
    """``solitons``: rows (x, y, charge, size, phase)."""
    s = _f64(np.asarray(solitons, dtype=np.float64).reshape(-1, 5))
    f = np.zeros((ncomp(theory), ny, nx))
    _load().or_ansatz(theory, _p(s), s.shape[0], _p(f), nx, ny, dx, dy)
    return f
