"""ctypes binding of liblbnci.so (include/lbnci.h): argument marshalling only.

Every function keeps the C name and order of arguments. Arrays are numpy float64
(int32 for hit maps) on the host, or CUDA tensors (torch) on the device; the
``on_device`` flag passed to C follows from the array type. All arithmetic runs in
the library's CUDA kernels: if the library cannot be loaded, or no GPU is present,
these calls raise instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_ENUMERIC, LB_EUNSUPPORTED = range(6)
LB_D2Q9, LB_D3Q27 = 0, 1
LB_FP64, LB_FP32, LB_FP16DEV = 0, 1, 2
LB_FORCE_GUO, LB_FORCE_EDM_DISPERSED = 0, 1
STATUS = {0: "LB_OK", 1: "LB_EINVAL", 2: "LB_ENOMEM", 3: "LB_ECUDA", 4: "LB_ENUMERIC", 5: "LB_EUNSUPPORTED"}

# Every symbol include/lbnci.h declares.
EXPORTS = ("lb_workspace_size", "lb_create", "lb_init_fields", "lb_step", "lb_observables",
           "lb_fields", "lb_get_populations", "lb_set_populations", "lb_destroy",
           "lb_last_error", "lb_kernel_launches", "lb_step_path", "lb_state_form", "lb_observables_noalloc",
           "lb_ensemble_create", "lb_ensemble_member", "lb_ensemble_step", "lb_ensemble_tune",
           "lb_ensemble_tune_times", "lb_ensemble_tma_choice", "lb_ensemble_launches",
           "lb_ensemble_last_error", "lb_ensemble_destroy")


class lb_config(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("wall_y", ctypes.c_int), ("wall_z", ctypes.c_int),
        ("tau", ctypes.c_double), ("A_s", ctypes.c_double), ("beta", ctypes.c_double),
        ("A_h", ctypes.c_double), ("h_min", ctypes.c_double), ("h_max", ctypes.c_double),
        ("g_th", ctypes.c_double),
        ("force", ctypes.c_double * 3),
        ("precision", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("forcing", ctypes.c_int),
    ]


class lb_obs(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double * 2),
        ("momentum", ctypes.c_double * 3),
        ("flow_rate", ctypes.c_double),
        ("flow_rate_disp", ctypes.c_double),
        ("step", ctypes.c_longlong),
        ("n_interface", ctypes.c_longlong),
        ("n_nci", ctypes.c_longlong),
        ("n_bad", ctypes.c_longlong),
    ]

    def as_dict(self) -> dict:
        return {"mass": np.array(self.mass[:]), "momentum": np.array(self.momentum[:]),
                "flow_rate": self.flow_rate, "flow_rate_disp": self.flow_rate_disp,
                "step": self.step, "n_interface": self.n_interface, "n_nci": self.n_nci,
                "n_bad": self.n_bad}


class LBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load liblbnci.so (building it with nvcc first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, cfgp, simp = ctypes.c_void_p, ctypes.POINTER(lb_config), ctypes.c_void_p
    lib.lb_workspace_size.argtypes = [cfgp, ctypes.POINTER(ctypes.c_size_t)]
    lib.lb_create.argtypes = [cfgp, ctypes.POINTER(ctypes.c_void_p)]
    lib.lb_init_fields.argtypes = [simp, vp, vp, vp, ctypes.c_int]
    lib.lb_step.argtypes = [simp, ctypes.c_longlong]
    lib.lb_observables.argtypes = [simp, ctypes.POINTER(lb_obs), vp, vp, ctypes.c_int]
    lib.lb_fields.argtypes = [simp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int]
    lib.lb_get_populations.argtypes = [simp, vp, ctypes.c_int]
    lib.lb_set_populations.argtypes = [simp, vp, ctypes.c_int]
    lib.lb_destroy.argtypes = [simp]
    lib.lb_destroy.restype = None
    lib.lb_last_error.argtypes = [simp]
    lib.lb_last_error.restype = ctypes.c_char_p
    lib.lb_kernel_launches.argtypes = [simp]
    lib.lb_kernel_launches.restype = ctypes.c_longlong
    lib.lb_step_path.argtypes = [simp]
    lib.lb_step_path.restype = ctypes.c_int
    lib.lb_state_form.argtypes = [simp]
    lib.lb_state_form.restype = ctypes.c_int
    lib.lb_observables_noalloc.argtypes = [cfgp, vp, ctypes.POINTER(lb_obs)]
    lib.lb_ensemble_create.argtypes = [cfgp, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    lib.lb_ensemble_member.argtypes = [simp, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    lib.lb_ensemble_step.argtypes = [simp, ctypes.c_longlong]
    lib.lb_ensemble_tune.argtypes = [simp, ctypes.POINTER(ctypes.c_int)]
    lib.lb_ensemble_tune_times.argtypes = [simp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
    lib.lb_ensemble_tma_choice.argtypes = [simp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_float)]
    lib.lb_ensemble_launches.argtypes = [simp]
    lib.lb_ensemble_launches.restype = ctypes.c_longlong
    lib.lb_ensemble_last_error.argtypes = [simp]
    lib.lb_ensemble_last_error.restype = ctypes.c_char_p
    lib.lb_ensemble_destroy.argtypes = [simp]
    lib.lb_ensemble_destroy.restype = None
    for name in EXPORTS:
        fn = getattr(lib, name)
        if fn.restype is ctypes.c_int or name not in ("lb_destroy", "lb_last_error", "lb_kernel_launches",
                                                      "lb_ensemble_launches", "lb_ensemble_last_error",
                                                      "lb_ensemble_destroy"):
            fn.restype = ctypes.c_int
    _lib = lib
    return lib


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _arg(a, dtype=np.float64, writable=False):
    """(pointer, on_device, keepalive) for a numpy array, a CUDA tensor or None."""
    if a is None:
        return None, None, None
    if _is_torch(a):
        if not a.is_cuda or not a.is_contiguous():
            raise ValueError("device arrays must be contiguous CUDA tensors")
        want = {np.float64: "torch.float64", np.int32: "torch.int32"}[dtype]
        if str(a.dtype) != want:
            raise ValueError(f"device array must be {want}, got {a.dtype}")
        return ctypes.c_void_p(a.data_ptr()), 1, a
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        if writable:
            raise ValueError(f"host output arrays must be C-contiguous {np.dtype(dtype)}")
        a = np.ascontiguousarray(a, dtype=dtype)
    if writable and not a.flags.writeable:
        raise ValueError("host output array is read-only")
    return a.ctypes.data_as(ctypes.c_void_p), 0, a


def _on_device(*flags) -> int:
    fl = {f for f in flags if f is not None}
    if len(fl) > 1:
        raise ValueError("mixing host and device arrays in one call")
    return fl.pop() if fl else 0


def _check(st: int, sim=None) -> int:
    if st != LB_OK:
        msg = load().lb_last_error(sim)
        raise LBError(st, msg.decode() if msg else "")
    return st


def lb_config_make(lattice=LB_D2Q9, nx=64, ny=64, nz=1, wall_y=0, wall_z=0, tau=1.0, A_s=0.0,
                   beta=0.0, A_h=0.0, h_min=2.0, h_max=4.0, g_th=0.05, force=(0.0, 0.0, 0.0),
                   precision=LB_FP64, stream=None, workspace=None, workspace_bytes=0,
                   forcing=LB_FORCE_GUO) -> lb_config:
    c = lb_config()
    c.lattice, c.nx, c.ny, c.nz, c.wall_y, c.wall_z = lattice, nx, ny, nz, wall_y, wall_z
    c.tau, c.A_s, c.beta, c.A_h, c.h_min, c.h_max, c.g_th = tau, A_s, beta, A_h, h_min, h_max, g_th
    for a in range(3):
        c.force[a] = force[a]
    c.precision = precision
    c.stream = stream
    c.workspace = workspace
    c.workspace_bytes = workspace_bytes
    c.forcing = forcing
    return c


def lb_workspace_size(cfg: lb_config) -> int:
    n = ctypes.c_size_t(0)
    _check(load().lb_workspace_size(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def lb_create(cfg: lb_config):
    h = ctypes.c_void_p()
    _check(load().lb_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def lb_init_fields(sim, rho1, rho2, u=None) -> None:
    p1, d1, k1 = _arg(rho1)
    p2, d2, k2 = _arg(rho2)
    pu, du, ku = _arg(u)
    _check(load().lb_init_fields(sim, p1, p2, pu, _on_device(d1, d2, du)), sim)


def lb_step(sim, nsteps: int) -> None:
    _check(load().lb_step(sim, int(nsteps)), sim)


def lb_observables(sim, psi_out=None, u_out=None, allow_numeric=False) -> dict:
    o = lb_obs()
    pp, dp, kp = _arg(psi_out, writable=True)
    pu, du, ku = _arg(u_out, writable=True)
    st = load().lb_observables(sim, ctypes.byref(o), pp, pu, _on_device(dp, du))
    if not (allow_numeric and st == LB_ENUMERIC):
        _check(st, sim)
    return o.as_dict()


def lb_fields(sim, rho1=None, rho2=None, psi=None, grad=None, frep=None, hit=None, u=None,
              allow_numeric=False) -> int:
    args = [_arg(a, writable=True) for a in (rho1, rho2, psi, grad, frep)]
    ah = _arg(hit, dtype=np.int32, writable=True)
    au = _arg(u, writable=True)
    dev = _on_device(*[a[1] for a in args], ah[1], au[1])
    st = load().lb_fields(sim, *[a[0] for a in args], ah[0], au[0], dev)
    if not (allow_numeric and st == LB_ENUMERIC):
        _check(st, sim)
    return st


def lb_get_populations(sim, f) -> None:
    pf, df, kf = _arg(f, writable=True)
    _check(load().lb_get_populations(sim, pf, _on_device(df)), sim)


def lb_set_populations(sim, f) -> None:
    pf, df, kf = _arg(f)
    _check(load().lb_set_populations(sim, pf, _on_device(df)), sim)


def lb_destroy(sim) -> None:
    if sim:
        load().lb_destroy(sim)


def lb_last_error(sim=None) -> str:
    m = load().lb_last_error(sim)
    return m.decode() if m else ""


def lb_kernel_launches(sim) -> int:
    return int(load().lb_kernel_launches(sim))


LB_PATH_FUSED2D, LB_PATH_TMA2D, LB_PATH_D3Q27, LB_PATH_D3Q27_CARRY, LB_PATH_D3Q27_STREAM = 0, 1, 2, 3, 4


def lb_step_path(sim) -> int:
    return int(load().lb_step_path(sim))


LB_STATE_PAIRS, LB_STATE_TOTAL_RECOLOUR = 0, 1


def lb_state_form(sim) -> int:
    return int(load().lb_state_form(sim))


def lb_observables_noalloc(cfg: lb_config, f, allow_numeric=False) -> dict:
    """Observables of device populations f (a CUDA tensor of the storage dtype) with no
    allocation inside the library; see include/lbnci.h for its limits."""
    if not _is_torch(f) or not f.is_cuda or not f.is_contiguous():
        raise ValueError("f must be a contiguous CUDA tensor")
    o = lb_obs()
    st = load().lb_observables_noalloc(ctypes.byref(cfg), ctypes.c_void_p(f.data_ptr()), ctypes.byref(o))
    if not (allow_numeric and st == LB_ENUMERIC):
        _check(st, None)
    return o.as_dict()


class Sim:
    """Owning wrapper: lb_create on construction, lb_destroy on close().

    ``workspace="torch"`` hands the library device memory allocated by PyTorch
    (kept alive by this object) instead of letting it call cudaMalloc."""

    def __init__(self, cfg: lb_config, workspace=None):
        self._ws = None
        if workspace == "torch":
            import torch
            nbytes = lb_workspace_size(cfg)
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            ptr = self._ws.data_ptr()
            cfg.workspace = (ptr + 255) & ~255
            cfg.workspace_bytes = nbytes
        self.cfg = cfg
        self.h = lb_create(cfg)
        self.Q = 9 if cfg.lattice == LB_D2Q9 else 27
        self.N = cfg.nx * cfg.ny * cfg.nz

    def close(self):
        if self.h:
            lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def init_fields(self, rho1, rho2, u=None):
        lb_init_fields(self.h, rho1, rho2, u)

    def step(self, n=1):
        lb_step(self.h, n)

    def observables(self, psi_out=None, u_out=None, allow_numeric=False):
        return lb_observables(self.h, psi_out, u_out, allow_numeric)

    def fields(self) -> dict:
        N = self.N
        out = {k: np.empty(N) for k in ("rho1", "rho2", "psi")}
        out["grad"], out["frep"], out["u"] = np.empty(3 * N), np.empty(3 * N), np.empty(3 * N)
        out["hit"] = np.empty(N, dtype=np.int32)
        lb_fields(self.h, out["rho1"], out["rho2"], out["psi"], out["grad"], out["frep"],
                  out["hit"], out["u"])
        for k in ("grad", "frep", "u"):
            out[k] = out[k].reshape(3, N)
        return out

    def get_populations(self) -> np.ndarray:
        f = np.empty(2 * self.Q * self.N)
        lb_get_populations(self.h, f)
        return f

    def set_populations(self, f):
        lb_set_populations(self.h, f)

    def launches(self) -> int:
        return lb_kernel_launches(self.h)

    def step_path(self) -> int:
        return lb_step_path(self.h)

    def state_form(self) -> int:
        return lb_state_form(self.h)


def _echeck(st: int, ens=None) -> int:
    if st != LB_OK:
        msg = load().lb_ensemble_last_error(ens)
        raise LBError(st, msg.decode() if msg else "")
    return st


class Ensemble:
    """Owning wrapper of lb_ensemble_*: members are Sim-like views (no ownership)."""

    def __init__(self, cfgs):
        self.h = None
        arr = (lb_config * len(cfgs))(*cfgs)
        h = ctypes.c_void_p()
        _echeck(load().lb_ensemble_create(arr, len(cfgs), ctypes.byref(h)))
        self.h = h
        self.cfgs = list(cfgs)
        self.members = []
        for m, c in enumerate(cfgs):
            sh = ctypes.c_void_p()
            _echeck(load().lb_ensemble_member(self.h, m, ctypes.byref(sh)), self.h)
            self.members.append(_MemberView(sh, c))

    def step(self, n=1):
        _echeck(load().lb_ensemble_step(self.h, int(n)), self.h)

    def tune(self) -> int:
        v = ctypes.c_int(0)
        _echeck(load().lb_ensemble_tune(self.h, ctypes.byref(v)), self.h)
        return v.value

    def tune_times(self):
        a, b = ctypes.c_float(0), ctypes.c_float(0)
        _echeck(load().lb_ensemble_tune_times(self.h, ctypes.byref(a), ctypes.byref(b)), self.h)
        return a.value, b.value

    def tma_choice(self):
        """(L2 promotion bytes, static tiles per CTA, {(promotion, static tiles): ms per step})
        of the batched TMA kernel; the table is empty before any tune()."""
        pr, st = ctypes.c_int(0), ctypes.c_int(0)
        ms = (ctypes.c_float * 12)()
        _echeck(load().lb_ensemble_tma_choice(self.h, ctypes.byref(pr), ctypes.byref(st), ms), self.h)
        table = {(pb, 1 + i): float(ms[k * 3 + i]) for k, pb in enumerate((0, 64, 128, 256)) for i in range(3)}
        if not any(table.values()):
            table = {}
        return pr.value, st.value, table

    def launches(self) -> int:
        return int(load().lb_ensemble_launches(self.h))

    def close(self):
        if self.h:
            load().lb_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class _MemberView(Sim):
    """An ensemble member: a Sim whose handle belongs to the ensemble."""

    def __init__(self, h, cfg):  # noqa: D401 - no lb_create here
        self._ws = None
        self.cfg = cfg
        self.h = h
        self.Q = 9 if cfg.lattice == LB_D2Q9 else 27
        self.N = cfg.nx * cfg.ny * cfg.nz

    def close(self):
        self.h = None  # the ensemble releases it
