"""cdi_mass_noalloc through the C ABI: the entry point for callers that cannot
allocate device memory (allocator callbacks, programs whose device memory is
reserved up front) and so cannot give a context its workspace.  Its scratch is
a fixed array inside the library; this test checks that two calls in a row,
on different inputs, agree with cdi_mass, and that sizes beyond the scratch
are refused.  The file name puts it last in collection order.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2412_16843_gb300 import cdi, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-13  # relative; both sums are FP64 in a fixed order, only the chunking differs


@pytest.fixture(scope="module")
def lib():
    from paper_2412_16843_gb300 import build
    build.build()
    lib = cdi.load()
    lib.cdi_mass_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]
    lib.cdi_mass_noalloc.restype = ctypes.c_int
    return lib


def _noalloc_mass(lib, phi_dev, cell_volume, out, stream):
    import torch
    err = ctypes.create_string_buffer(256)
    out.fill_(float("nan"))  # a stale output cannot pass
    st = lib.cdi_mass_noalloc(ctypes.c_void_p(phi_dev.data_ptr()), phi_dev.numel(), cell_volume,
                              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream), err, 256)
    assert st == 0, err.value
    torch.cuda.synchronize()
    return float(out.item())


def test_noalloc_mass_matches_cdi_mass_on_two_calls(lib):
    import torch
    wl = inputs.drop_2d(64, 32)
    s = cdi.from_workload(wl)
    s.step(wl.dt, 3)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    # first call: the drop after 3 steps; second call: a different, larger 3D field
    phi1, _, _ = s.get_fields()
    m1 = s.mass()
    got1 = _noalloc_mass(lib, torch.from_numpy(phi1).cuda(), wl.h ** 2, out, stream)
    assert abs(got1 - m1) <= TOL * abs(m1)
    n3 = (64, 64, 48)
    h3 = 1.0 / 64
    phi3 = inputs.add_noise(inputs.cap_phi_3d(*n3, h3, 0.3, math.radians(70), 0.5, 0.5, h3), 1e-3, 4)
    s3 = cdi.Solver(3, n3, tuple(x * h3 for x in n3))
    s3.set_fluids(1.0, 0.1, 0.05, 0.005, 1.0, h3, 1.0)
    s3.set_phi(phi3)
    m3 = s3.mass()
    got3 = _noalloc_mass(lib, torch.from_numpy(phi3).cuda(), h3 ** 3, out, stream)
    assert abs(got3 - m3) <= TOL * abs(m3)
    assert abs(got1 - got3) > 1e-3  # the two calls really saw different inputs


@pytest.mark.parametrize("n", [5 * 8192 + 1234, 33554432])
def test_noalloc_mass_ragged_and_largest_sizes(lib, n):
    """Several blocks with a partial last chunk, and the largest accepted size
    (every one of the 4096 scratch partials in use, 268 MB of FP64 input),
    against a float64 sum of the same values on the host."""
    import torch
    rng = np.random.default_rng(n)
    x = rng.uniform(0.0, 1.0, n)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    got = _noalloc_mass(lib, torch.from_numpy(x).cuda(), 0.5, out, torch.cuda.current_stream())
    ref = 0.5 * math.fsum(x.tolist()) if n < 100000 else 0.5 * float(np.sum(x, dtype=np.float64))
    assert abs(got - ref) <= TOL * abs(ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    import torch
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    err = ctypes.create_string_buffer(256)
    st = lib.cdi_mass_noalloc(ctypes.c_void_p(x.data_ptr()), 33554432 + 1, 1.0, ctypes.c_void_p(out.data_ptr()),
                              None, err, 256)
    assert st == 1 and b"outside" in err.value
    st = lib.cdi_mass_noalloc(ctypes.c_void_p(x.data_ptr()), 0, 1.0, ctypes.c_void_p(out.data_ptr()), None, err, 256)
    assert st == 1
