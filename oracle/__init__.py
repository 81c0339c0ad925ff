"""FP64 CPU oracle of the NCI colour-gradient lattice Boltzmann step (arXiv:2003.11069).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers; the product path never imports this package.
The arithmetic lives in ``lbnci_oracle.c`` (plain nested loops, FP64, no FMA
contraction); this module compiles it with gcc and wraps it with ctypes.

Parity status of each function (what pins it is listed in ``tests/test_oracle_pins.py``):
every stage is pinned by an invariant, a closed form or a hand-derived case, except
the physics trend "dispersed flux grows with the forcing", which is a sanity check
only (parity unpinned for that trend; it is not a computed quantity of the step).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbnci_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liblbnci_oracle.so")
_lock = threading.Lock()
_lib = None

D2Q9, D3Q27 = 0, 1


class Params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("wall_y", ctypes.c_int), ("wall_z", ctypes.c_int),
        ("tau", ctypes.c_double), ("A_s", ctypes.c_double), ("beta", ctypes.c_double),
        ("A_h", ctypes.c_double), ("h_min", ctypes.c_double), ("h_max", ctypes.c_double),
        ("g_th", ctypes.c_double),
        ("force", ctypes.c_double * 3),
        ("forcing", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build (gcc, -O2, no FP contraction, OpenMP)."""
    with _lock:
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lbnci_oracle.h"))
        ):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(Params)
        dp = ctypes.c_void_p
        lib.orc_lattice.argtypes = [ctypes.c_int, dp, dp, dp]
        lib.orc_init.argtypes = [P, dp, dp, dp, dp]
        lib.orc_step.argtypes = [P, dp, ctypes.c_long, ctypes.c_int]
        lib.orc_fields.argtypes = [P, dp, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_observables.argtypes = [P, dp, dp]
        lib.orc_gradient.argtypes = [P, dp, dp]
        lib.orc_nci.argtypes = [P, dp, dp, dp]
        lib.orc_collide_site.argtypes = [P, dp, dp, dp, dp]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_params(lattice=D2Q9, nx=8, ny=8, nz=1, wall_y=0, wall_z=0, tau=1.0, A_s=0.0,
                beta=0.0, A_h=0.0, h_min=2.0, h_max=4.0, g_th=0.05, force=(0.0, 0.0, 0.0), forcing=0):
    p = Params()
    p.lattice, p.nx, p.ny, p.nz = lattice, nx, ny, nz
    p.wall_y, p.wall_z = wall_y, wall_z
    p.tau, p.A_s, p.beta, p.A_h = tau, A_s, beta, A_h
    p.h_min, p.h_max, p.g_th = h_min, h_max, g_th
    for a in range(3):
        p.force[a] = force[a]
    p.forcing = forcing
    return p


def Q_of(p) -> int:
    return 9 if p.lattice == D2Q9 else 27


def N_of(p) -> int:
    return p.nx * p.ny * p.nz


def lattice(lat: int):
    """Velocity set, weights and opposite indices as the oracle defines them."""
    c = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    opp = np.zeros(27, dtype=np.int32)
    Q = _load().orc_lattice(lat, _ptr(c), _ptr(w), _ptr(opp))
    if Q < 0:
        raise ValueError("unknown lattice")
    return c[:Q].copy(), w[:Q].copy(), opp[:Q].copy()


def init(p, rho1, rho2, u=None) -> np.ndarray:
    N, Q = N_of(p), Q_of(p)
    f = np.empty(2 * Q * N)
    r1, r2 = _f64(rho1).ravel(), _f64(rho2).ravel()
    uu = None if u is None else _f64(u).reshape(3 * N)
    if r1.size != N or r2.size != N:
        raise ValueError("field size does not match the lattice")
    rc = _load().orc_init(ctypes.byref(p), _ptr(r1), _ptr(r2), _ptr(uu), _ptr(f))
    if rc:
        raise RuntimeError(f"orc_init failed ({rc})")
    return f


def step(p, f, nsteps=1, nthreads=0) -> np.ndarray:
    """Advance a copy of the state by nsteps; returns the new state."""
    g = _f64(f).copy()
    rc = _load().orc_step(ctypes.byref(p), _ptr(g), int(nsteps), int(nthreads))
    if rc:
        raise RuntimeError(f"orc_step failed ({rc})")
    return g


def step_inplace(p, f, nsteps=1, nthreads=0) -> None:
    assert f.dtype == np.float64 and f.flags.c_contiguous
    rc = _load().orc_step(ctypes.byref(p), _ptr(f), int(nsteps), int(nthreads))
    if rc:
        raise RuntimeError(f"orc_step failed ({rc})")


def fields(p, f) -> dict:
    N = N_of(p)
    out = {k: np.empty(N) for k in ("rho1", "rho2", "psi")}
    out["grad"] = np.empty(3 * N)
    out["frep"] = np.empty(3 * N)
    out["u"] = np.empty(3 * N)
    out["hit"] = np.empty(N, dtype=np.int32)
    rc = _load().orc_fields(ctypes.byref(p), _ptr(_f64(f)), _ptr(out["rho1"]), _ptr(out["rho2"]),
                            _ptr(out["psi"]), _ptr(out["grad"]), _ptr(out["frep"]),
                            _ptr(out["hit"]), _ptr(out["u"]))
    if rc:
        raise RuntimeError(f"orc_fields failed ({rc})")
    for k in ("grad", "frep", "u"):
        out[k] = out[k].reshape(3, N)
    return out


def observables(p, f) -> dict:
    out = np.empty(7)
    rc = _load().orc_observables(ctypes.byref(p), _ptr(_f64(f)), _ptr(out))
    if rc:
        raise RuntimeError(f"orc_observables failed ({rc})")
    return {"mass": out[0:2].copy(), "momentum": out[2:5].copy(),
            "flow_rate": float(out[5]), "flow_rate_disp": float(out[6])}


def gradient(p, psi) -> np.ndarray:
    N = N_of(p)
    g = np.empty(3 * N)
    rc = _load().orc_gradient(ctypes.byref(p), _ptr(_f64(psi).ravel()), _ptr(g))
    if rc:
        raise RuntimeError("orc_gradient failed")
    return g.reshape(3, N)


def nci(p, psi):
    N = N_of(p)
    fr = np.empty(3 * N)
    hit = np.empty(N, dtype=np.int32)
    rc = _load().orc_nci(ctypes.byref(p), _ptr(_f64(psi).ravel()), _ptr(fr), _ptr(hit))
    if rc:
        raise RuntimeError("orc_nci failed")
    return fr.reshape(3, N), hit


def collide_site(p, fin, grad, F) -> np.ndarray:
    Q = Q_of(p)
    out = np.empty(2 * Q)
    rc = _load().orc_collide_site(ctypes.byref(p), _ptr(_f64(fin).ravel()),
                                  _ptr(_f64(grad).ravel()), _ptr(_f64(F).ravel()), _ptr(out))
    if rc:
        raise RuntimeError("orc_collide_site failed")
    return out
