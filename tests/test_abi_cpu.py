"""The C-ABI library without a GPU: it builds for sm_103a, loads, exports
every function include/cdi.h declares, and rejects bad arguments on the host
before touching the device."""
import ctypes
import math

import pytest

from paper_2412_16843_gb300 import build as cdi_build
from paper_2412_16843_gb300 import cdi


@pytest.fixture(scope="module")
def lib():
    cdi_build.build()
    return cdi.load()


def test_every_declared_function_is_exported(lib):
    names = cdi.header_functions()
    assert "cdi_step" in names and "cdi_init_grid" in names and len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def _init(lib, dim, nx, ny, nz, Lx, Ly, Lz, mask=3, prec=0):
    h = ctypes.c_void_p()
    st = lib.cdi_init_grid(ctypes.byref(h), dim, nx, ny, nz, Lx, Ly, Lz, mask, prec)
    return st, h


@pytest.mark.parametrize("args", [
    (4, 64, 32, 1, 1.0, 0.5, 0.0),     # bad dim
    (2, 63, 32, 1, 1.0, 0.5, 0.0),     # odd periodic extent
    (2, 64, 3, 1, 1.0, 3 / 64, 0.0),   # wall axis too short
    (2, 64, 32, 1, 1.0, 0.6, 0.0),     # non-uniform spacing
    (2, 96, 90, 1, 1.0, 90 / 96, 0.0),  # coarsest level too large
])
def test_init_grid_rejects_bad_arguments(lib, args):
    st, h = _init(lib, *args)
    assert st == 1 and not h.value
    assert len(lib.cdi_last_error(None)) > 0


def test_init_and_host_side_setters(lib):
    st, h = _init(lib, 2, 64, 32, 1, 1.0, 0.5, 0.0)
    assert st == 0 and h.value
    nbytes = ctypes.c_size_t()
    assert lib.cdi_workspace_bytes(h, ctypes.byref(nbytes)) == 0
    # 2D FP64: 6 cell fields + 5 x 2 face fields + 2 normals + MG hierarchy
    assert nbytes.value > 64 * 32 * 8 * 20
    assert lib.cdi_set_wall(h, 0, 1.0, 0.01, 0.0) == 2          # fluids first
    assert lib.cdi_set_fluids(h, 1.0, 1.0, 0.1, 0.1, 1.0, 1 / 64, 1.0) == 0
    assert lib.cdi_set_fluids(h, -1.0, 1.0, 0.1, 0.1, 1.0, 1 / 64, 1.0) == 1
    assert lib.cdi_set_wall(h, 2, math.radians(60), 1 / 64, 0.0) == 0
    assert lib.cdi_set_wall(h, 2, 4.0, 1 / 64, 0.0) == 1         # angle out of (0, pi)
    assert lib.cdi_set_wall_beta(h, 0, 1.0, float("inf")) == 1
    assert lib.cdi_set_model(h, 9) == 1
    assert lib.cdi_set_solver(h, 1e-10, 0, 0) == 1
    assert lib.cdi_set_smoothing(h, 0, 1) == 1 and lib.cdi_set_smoothing(h, 1, 5) == 1
    assert lib.cdi_set_smoothing(h, 1, 2) == 0
    for bad in ((0, 0), (1, 5), (-1, 1), (5, 0)):
        assert lib.cdi_set_coarse_smoothing(h, *bad) == 1, bad
    assert lib.cdi_set_coarse_smoothing(h, 0, 1) == 0 and lib.cdi_set_coarse_smoothing(h, -1, -1) == 0
    # no workspace bound yet: state calls refuse
    assert lib.cdi_step(h, 1e-4, 1) == 2
    m = ctypes.c_double()
    assert lib.cdi_mass(h, ctypes.byref(m)) == 2
    lib.cdi_destroy(h)
    lib.cdi_destroy(None)


def test_unet_host_side_checks(lib):
    n = ctypes.c_size_t()
    assert lib.cdi_unet_param_count(ctypes.byref(n)) == 0 and n.value == 726993
    u = ctypes.c_void_p()
    assert lib.cdi_unet_create(ctypes.byref(u), 12, 16, 16) == 1 and not u.value   # not a multiple of 8
    assert len(lib.cdi_unet_last_error(None)) > 0
    assert lib.cdi_unet_create(ctypes.byref(u), 16, 16, 8) == 0 and u.value
    nbytes = ctypes.c_size_t()
    assert lib.cdi_unet_workspace_bytes(u, ctypes.byref(nbytes)) == 0
    assert nbytes.value > 726993 * (4 * 4 + 2 * 2)  # FP32 weights, gradients, two Adam moments; two BF16 copies
    x = (ctypes.c_double * (16 * 16 * 8 * 2))()
    y = (ctypes.c_double * (16 * 16 * 8))()
    assert lib.cdi_unet_forward(u, x, y) == 2      # no workspace bound
    # the network attaches only to a 3D context of the same extents
    st, h2 = _init(lib, 2, 64, 32, 1, 1.0, 0.5, 0.0)
    assert st == 0 and lib.cdi_set_warm_unet(h2, u) == 1
    st, h3 = _init(lib, 3, 16, 16, 16, 1.0, 1.0, 1.0)
    assert st == 0 and lib.cdi_set_warm_unet(h3, u) == 1
    assert lib.cdi_set_warm_unet(h3, None) == 0
    assert lib.cdi_set_solver(h3, 1e-8, 10, 3) == 0   # CDI_WARM_UNET
    assert lib.cdi_set_solver(h3, 1e-8, 10, 4) == 1
    for h in (h2, h3):
        lib.cdi_destroy(h)
    lib.cdi_unet_destroy(u)
    lib.cdi_unet_destroy(None)
