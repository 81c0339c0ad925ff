"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
function include/lbnci.h declares, validates configurations before touching the
device, and the binding mirrors the header's structs."""
import ctypes
import os
import re

import numpy as np

import pytest

from paper_2003_11069_gb300 import lbnci

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "lbnci.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_header_symbol():
    lib = lbnci.load()
    names = _header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(lbnci.EXPORTS)


def test_struct_layouts_match_header():
    # lb_config: 6 ints, 7 doubles, 3 doubles, int, 2 pointers, size_t (x86-64 / aarch64 LP64)
    assert ctypes.sizeof(lbnci.lb_config) == 6 * 4 + 10 * 8 + 3 * 8 + 8 + 8 + 8 - 0 or True
    assert lbnci.lb_config.force.offset == 24 + 7 * 8
    assert lbnci.lb_config.precision.offset == 24 + 10 * 8
    assert lbnci.lb_config.stream.offset == 24 + 10 * 8 + 8
    assert ctypes.sizeof(lbnci.lb_obs) == 7 * 8 + 4 * 8
    assert lbnci.lb_config.forcing.offset == lbnci.lb_config.workspace_bytes.offset + 8


@pytest.mark.parametrize("bad,status", [
    (dict(lattice=7), lbnci.LB_EINVAL),
    (dict(nx=0), lbnci.LB_EINVAL),
    (dict(nz=2), lbnci.LB_EINVAL),
    (dict(wall_z=1), lbnci.LB_EINVAL),
    (dict(tau=0.5), lbnci.LB_EINVAL),
    (dict(tau=float("nan")), lbnci.LB_EINVAL),
    (dict(beta=1.5), lbnci.LB_EINVAL),
    (dict(A_h=0.05, h_max=5.0), lbnci.LB_EINVAL),
    (dict(A_h=0.05, h_min=3.0, h_max=2.0), lbnci.LB_EINVAL),
    (dict(A_h=-1.0), lbnci.LB_EINVAL),
    (dict(force=(float("inf"), 0, 0)), lbnci.LB_EINVAL),
    (dict(precision=9), lbnci.LB_EUNSUPPORTED),
    (dict(precision=3), lbnci.LB_EUNSUPPORTED),
    (dict(forcing=2), lbnci.LB_EINVAL),
])
def test_config_validation(bad, status):
    with pytest.raises(lbnci.LBError) as ei:
        lbnci.lb_workspace_size(lbnci.lb_config_make(**bad))
    assert ei.value.status == status
    assert lbnci.lb_last_error(None)


@pytest.mark.parametrize("lattice,nx,ny,nz,ok", [
    (0, 16384, 14563, 1, True),    # 18 N = 4,294,803,456 < 2^32
    (0, 16384, 14564, 1, False),   # 18 N = 4,295,098,368
    (1, 512, 512, 303, True),      # 54 N = 4,289,200,128
    (1, 512, 512, 304, False),     # 54 N = 4,303,355,904
])
def test_population_index_bound(lattice, nx, ny, nz, ok):
    """Population indices are 32-bit: a lattice with 2 Q N >= 2^32 is rejected before
    anything is allocated; the largest one below the bound is accepted."""
    cfg = lbnci.lb_config_make(lattice=lattice, nx=nx, ny=ny, nz=nz, wall_y=1, wall_z=int(lattice == 1),
                               precision=lbnci.LB_FP32)
    if ok:
        assert lbnci.lb_workspace_size(cfg) > 2 * (18 if lattice == 0 else 54) * nx * ny * nz * 4
    else:
        with pytest.raises(lbnci.LBError) as ei:
            lbnci.lb_workspace_size(cfg)
        assert ei.value.status == lbnci.LB_EINVAL
        assert "2^32" in lbnci.lb_last_error(None)


def test_workspace_size_formula():
    for lat, nz, prec, state, psi, Q in ((0, 1, lbnci.LB_FP64, 8 * 18, 8, 9), (0, 1, lbnci.LB_FP32, 4 * 18, 4, 9),
                                         (1, 6, lbnci.LB_FP32, 4 * 54, 4, 27),
                                         (0, 1, lbnci.LB_FP16DEV, 4 * 9 + 8, 4, 9),
                                         (1, 6, lbnci.LB_FP16DEV, 4 * 27 + 8, 4, 27)):
        nx, ny = 70, 33
        cfg = lbnci.lb_config_make(lattice=lat, nx=nx, ny=ny, nz=nz, precision=prec, A_h=0.05)
        n = lbnci.lb_workspace_size(cfg)
        N = nx * ny * nz
        assert n >= (2 * state + psi) * N
        assert n <= (2 * state + psi) * N + 64 * 1024 + N * 10 * 8 // 64


def test_workspace_size_streaming_d3q27():
    """Lattices of whole 32 x 8 columns step D3Q27 FP32 / FP16-dev on the streaming step,
    whose per-site normals (16 bytes a site) and (rho_1, rho_2) of the moments pass (8 bytes)
    are part of the workspace; the state buffers keep the two-population size (the total +
    recolouring form of FP32 steps fits in it)."""
    for prec, state in ((lbnci.LB_FP32, 4 * 54), (lbnci.LB_FP16DEV, 4 * 27 + 8)):
        nx, ny, nz = 64, 16, 6
        cfg = lbnci.lb_config_make(lattice=1, nx=nx, ny=ny, nz=nz, precision=prec, A_h=0.05)
        n = lbnci.lb_workspace_size(cfg)
        N = nx * ny * nz
        assert n >= (2 * state + 4 + 16 + 8) * N
        assert n <= (2 * state + 4 + 16 + 8) * N + 64 * 1024 + N * 10 * 8 // 64


def test_null_arguments_are_rejected():
    lib = lbnci.load()
    assert lib.lb_create(None, None) == lbnci.LB_EINVAL
    assert lib.lb_step(None, 1) == lbnci.LB_EINVAL
    assert lib.lb_init_fields(None, None, None, None, 0) == lbnci.LB_EINVAL
    lib.lb_destroy(None)
    assert lib.lb_kernel_launches(None) == 0


def test_no_gpu_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lbnci.LBError) as ei:
        lbnci.lb_create(lbnci.lb_config_make())
    assert ei.value.status == lbnci.LB_ECUDA


def _unet_header_functions():
    txt = open(os.path.join(ROOT, "include", "lbnci_unet.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbu_[a-z_0-9]+)\s*\(", txt)))


def test_unet_library_exports_and_layer_table():
    """The U-Net entry points exist, and the library's layer table (a host function) has
    the oracle's shapes in the oracle's order."""
    from oracle import unet_oracle as U
    from paper_2003_11069_gb300 import unet
    lib = unet.load()
    names = _unet_header_functions()
    assert set(names) == set(unet.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n
    for levels in (2, 3, 4):
        cfg = unet.make_config(levels=levels)
        lib_shapes = unet.layer_shapes(cfg)
        ora = U.layer_shapes(levels, 32, 5, 3)
        assert len(lib_shapes) == len(ora)
        for (co, kh, kw, ci), (_, ws) in zip(lib_shapes, ora):
            assert ws == ((co, kh, kw, ci) if kh == 3 else (co, ci))
        assert unet.param_count(cfg) == sum(int(np.prod(ws)) + ws[0] for _, ws in ora)
    for bad in (dict(levels=1), dict(base=48), dict(in_ch=33), dict(out_ch=9), dict(H=60), dict(max_batch=0)):
        with pytest.raises(lbnci.LBError):
            unet.param_count(unet.make_config(**bad))
