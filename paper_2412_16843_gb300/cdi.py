"""Thin Python binding of libcdi.so (C ABI in include/cdi.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of the library.  PyTorch provides the device workspace and the stream.  There
is no CPU fallback: if the library is missing or no GPU is present the calls
fail loudly.
"""
from __future__ import annotations

import ctypes
import math
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcdi.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "cdi.h")

STATUS = {0: "CDI_OK", 1: "CDI_EINVAL", 2: "CDI_ESTATE", 3: "CDI_ECUDA",
          4: "CDI_ENOCONV", 5: "CDI_ENAN", 6: "CDI_ETIMEOUT"}
FP64, FP32_MIXED = 0, 1
WALL_LO, WALL_HI, WALL_BOTH = 0, 1, 2
WARM_PREV, WARM_ZERO, WARM_EXTRAP, WARM_UNET = 0, 1, 2, 3
EXEC_PERSISTENT, EXEC_KERNELS, EXEC_AUTO = 0, 1, 2
SWEEP_AUTO, SWEEP_ONEPASS, SWEEP_COLOUR, SWEEP_ONEPASS_CPASYNC = 0, 1, 2, 3
MODELS = {"1A": 0, "1B": 1, "2A": 2, "2B": 3, "3A": 4, "3B": 5, "4A": 6, "4B": 7}

_lib = None


class CdiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, str(status)), msg))
        self.status = status


def header_functions() -> list:
    """Names of the functions include/cdi.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cdi_[a-z0-9_]+)\s*\(", text)))


def load(path: str = LIB_PATH):
    """Load libcdi.so and declare the signatures; raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libcdi.so is not built (%s); run "
                          "`python -m paper_2412_16843_gb300.build`" % path)
    lib = ctypes.CDLL(path)
    D, I, U = ctypes.c_double, ctypes.c_int, ctypes.c_uint
    P, S = ctypes.c_void_p, ctypes.c_size_t
    DP = ctypes.POINTER(ctypes.c_double)
    IP = ctypes.POINTER(ctypes.c_int)
    sig = {
        "cdi_init_grid": [ctypes.POINTER(P), I, I, I, I, D, D, D, U, I],
        "cdi_workspace_bytes": [P, ctypes.POINTER(S)],
        "cdi_bind_workspace": [P, P, S, P],
        "cdi_set_fluids": [P, D, D, D, D, D, D, D],
        "cdi_set_wall": [P, I, D, D, D],
        "cdi_set_wall_beta": [P, I, D, D],
        "cdi_set_wall_velocity": [P, I, D, D],
        "cdi_set_model": [P, I],
        "cdi_set_phi": [P, DP],
        "cdi_set_velocity": [P, DP, DP, DP],
        "cdi_set_solver": [P, D, I, I],
        "cdi_step": [P, D, I],
        "cdi_mass": [P, DP],
        "cdi_contact_angle": [P, I, DP, DP],
        "cdi_get_fields": [P, DP, DP, DP, DP, DP],
        "cdi_eval_rhs": [P, D, DP, DP, DP, DP],
        "cdi_eval_wall": [P, DP, DP],
        "cdi_solve_pressure": [P, DP, DP],
        "cdi_last_stats": [P, IP, DP, IP, IP],
        "cdi_set_exec": [P, I],
        "cdi_set_barrier_timeout": [P, ctypes.c_longlong],
        "cdi_set_smoothing": [P, I, I],
        "cdi_set_coarse_smoothing": [P, I, I],
        "cdi_set_relaxation": [P, D],
        "cdi_set_level0_sweep": [P, I],
        "cdi_launches_per_step": [P, ctypes.POINTER(ctypes.c_long)],
        "cdi_profile_start": [P, ctypes.c_char_p, I],
        "cdi_profile_stop": [P, DP, ctypes.POINTER(ctypes.c_long)],
    }
    sig.update({
        "cdi_batch_create": [ctypes.POINTER(P), I, ctypes.POINTER(P)],
        "cdi_batch_workspace_bytes": [P, ctypes.POINTER(S)],
        "cdi_batch_bind_workspace": [P, P, S, P],
        "cdi_batch_step": [P, DP, I],
        "cdi_batch_set_threads": [P, I],
        "cdi_batch_autotune": [P, DP, I, IP, ctypes.POINTER(S), DP],
        "cdi_batch_set_tail_budget": [P, S],
        "cdi_batch_stats": [P, I, IP, IP, IP, ctypes.POINTER(ctypes.c_float)],
        "cdi_unet_create": [ctypes.POINTER(P), I, I, I],
        "cdi_unet_workspace_bytes": [P, ctypes.POINTER(S)],
        "cdi_unet_bind_workspace": [P, P, S, P],
        "cdi_unet_param_count": [ctypes.POINTER(S)],
        "cdi_unet_set_params": [P, DP, S],
        "cdi_unet_get_params": [P, DP, S],
        "cdi_unet_forward": [P, DP, DP],
        "cdi_unet_forward_device": [P, P, P],
        "cdi_unet_set_conv_kernel": [P, I],
        "cdi_unet_train_step": [P, DP, DP, D, DP, DP],
        "cdi_set_warm_unet": [P, P],
        "cdi_last_pressure": [P, DP, DP],
    })
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = I
    lib.cdi_batch_last_error.argtypes = [P]
    lib.cdi_batch_last_error.restype = ctypes.c_char_p
    lib.cdi_batch_destroy.argtypes = [P]
    lib.cdi_batch_destroy.restype = None
    lib.cdi_unet_last_error.argtypes = [P]
    lib.cdi_unet_last_error.restype = ctypes.c_char_p
    lib.cdi_unet_destroy.argtypes = [P]
    lib.cdi_unet_destroy.restype = None
    lib.cdi_last_error.argtypes = [P]
    lib.cdi_last_error.restype = ctypes.c_char_p
    lib.cdi_destroy.argtypes = [P]
    lib.cdi_destroy.restype = None
    _lib = lib
    return lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Solver:
    """One CDI + GNBC problem on the GPU (see include/cdi.h for the semantics).

    dim 2: n = (nx, ny), walls on y.  dim 3: n = (nx, ny, nz), walls on z.
    Host arrays are numpy float64 in the C ABI layout (x fastest)."""

    def __init__(self, dim: int, n, L, precision: int = FP64, device=None, stream=None):
        import torch  # device memory and streams only

        self.lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("libcdi needs a CUDA device; there is no CPU path")
        self.dim = dim
        self.n = tuple(int(x) for x in n)
        self.precision = precision
        h = ctypes.c_void_p()
        nz = self.n[2] if dim == 3 else 1
        Lz = L[2] if dim == 3 else 0.0
        self._check(self.lib.cdi_init_grid(ctypes.byref(h), dim, self.n[0], self.n[1], nz,
                                           float(L[0]), float(L[1]), float(Lz), 3, precision), None)
        self.h = h
        nbytes = ctypes.c_size_t()
        self._check(self.lib.cdi_workspace_bytes(self.h, ctypes.byref(nbytes)))
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=dev)
        self.stream = torch.cuda.current_stream(dev) if stream is None else stream
        self._check(self.lib.cdi_bind_workspace(self.h, ctypes.c_void_p(self.workspace.data_ptr()),
                                                nbytes.value, ctypes.c_void_p(self.stream.cuda_stream)))
        self.mu = (0.0, 0.0)

    # ---- helpers ------------------------------------------------------------
    def _check(self, st, h="self"):
        if st != 0:
            hh = self.h if h == "self" else None
            msg = self.lib.cdi_last_error(hh)
            raise CdiError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.lib.cdi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def cell_shape(self):
        return self.n[::-1]

    def face_shape(self, a: int):
        s = list(self.n)
        if a == self.dim - 1:
            s[a] += 1
        return tuple(s[::-1])

    @property
    def plane(self):
        return (self.n[0],) if self.dim == 2 else (self.n[1], self.n[0])

    # ---- parameters ---------------------------------------------------------
    def set_fluids(self, rho1, rho2, mu1, mu2, sigma, eps, gamma):
        self._check(self.lib.cdi_set_fluids(self.h, rho1, rho2, mu1, mu2, sigma, eps, gamma))
        self.mu = (mu1, mu2)

    def set_wall(self, wall, theta_eq, slip_length, U_wall=0.0):
        self._check(self.lib.cdi_set_wall(self.h, wall, theta_eq, slip_length, U_wall))

    def set_wall_beta(self, wall, beta1, beta2):
        self._check(self.lib.cdi_set_wall_beta(self.h, wall, beta1, beta2))

    def set_wall_velocity(self, wall, Ux, Uy=0.0):
        self._check(self.lib.cdi_set_wall_velocity(self.h, wall, Ux, Uy))

    def set_model(self, name: str):
        self._check(self.lib.cdi_set_model(self.h, MODELS[name]))

    def set_solver(self, tol=1e-10, max_vcycles=100, warm=WARM_PREV):
        self._check(self.lib.cdi_set_solver(self.h, tol, max_vcycles, warm))

    # ---- state --------------------------------------------------------------
    def set_phi(self, phi):
        phi = _f64(phi)
        assert phi.shape == self.cell_shape
        self._check(self.lib.cdi_set_phi(self.h, _dp(phi)))

    def set_velocity(self, vel):
        vel = [_f64(v) for v in vel]
        for a in range(self.dim):
            assert vel[a].shape == self.face_shape(a)
        comps = vel + [None] * (3 - self.dim)
        self._check(self.lib.cdi_set_velocity(self.h, *[_dp(c) for c in comps]))

    def set_state(self, phi, vel=None):
        self.set_phi(phi)
        if vel is None:
            vel = [np.zeros(self.face_shape(a)) for a in range(self.dim)]
        self.set_velocity(vel)

    def get_fields(self, out=None):
        if out is None:
            out = (np.empty(self.cell_shape), [np.empty(self.face_shape(a)) for a in range(self.dim)],
                   np.empty(self.cell_shape))
        phi, vel, p = out
        comps = list(vel) + [None] * (3 - self.dim)
        self._check(self.lib.cdi_get_fields(self.h, _dp(phi), *[_dp(c) for c in comps], _dp(p)))
        return phi, vel, p

    def step(self, dt, nsteps=1):
        self._check(self.lib.cdi_step(self.h, dt, nsteps))

    def mass(self):
        m = ctypes.c_double()
        self._check(self.lib.cdi_mass(self.h, ctypes.byref(m)))
        return m.value

    def contact_angle(self, wall=0):
        th, L = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.cdi_contact_angle(self.h, wall, ctypes.byref(th), ctypes.byref(L)))
        return th.value, L.value

    def eval_rhs(self, gamma=-1.0):
        rphi = np.zeros(self.cell_shape)
        rv = [np.zeros(self.face_shape(a)) for a in range(self.dim)]
        comps = rv + [None] * (3 - self.dim)
        self._check(self.lib.cdi_eval_rhs(self.h, gamma, _dp(rphi), *[_dp(c) for c in comps]))
        return rphi, rv

    def eval_wall(self):
        t = self.dim - 1
        npl = int(np.prod(self.plane))
        uY = np.zeros(2 * t * npl)
        g = np.zeros(2 * t * npl)
        self._check(self.lib.cdi_eval_wall(self.h, _dp(uY), _dp(g)))
        sh = (2, t) + self.plane
        return uY.reshape(sh), g.reshape(sh)

    def solve_pressure(self, f, p0=None):
        f = _f64(f)
        p = np.zeros(self.cell_shape) if p0 is None else _f64(p0).copy()
        self._check(self.lib.cdi_solve_pressure(self.h, _dp(f), _dp(p)))
        return p

    def last_stats(self):
        c, r, m, t = ctypes.c_int(), ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.cdi_last_stats(self.h, ctypes.byref(c), ctypes.byref(r), ctypes.byref(m),
                                            ctypes.byref(t)))
        return {"cycles": c.value, "resid": r.value, "max_cycles_step": m.value, "total_cycles_call": t.value}

    def set_exec(self, mode: int):
        self._check(self.lib.cdi_set_exec(self.h, mode))

    def set_smoothing(self, npre: int, npost: int):
        self._check(self.lib.cdi_set_smoothing(self.h, npre, npost))

    def set_coarse_smoothing(self, npre: int, npost: int):
        self._check(self.lib.cdi_set_coarse_smoothing(self.h, npre, npost))

    def set_relaxation(self, omega: float):
        self._check(self.lib.cdi_set_relaxation(self.h, float(omega)))

    def set_level0_sweep(self, mode: int):
        self._check(self.lib.cdi_set_level0_sweep(self.h, mode))

    def set_barrier_timeout(self, ns: int):
        self._check(self.lib.cdi_set_barrier_timeout(self.h, int(ns)))

    def launches_per_step(self):
        n = ctypes.c_long()
        self._check(self.lib.cdi_launches_per_step(self.h, ctypes.byref(n)))
        return n.value


    def set_warm_unet(self, net):
        """Attach a Unet (None detaches) for WARM_UNET first guesses."""
        self._unet = net
        self._check(self.lib.cdi_set_warm_unet(self.h, None if net is None else net.h))

    def last_pressure(self):
        """(f, p) of the last pressure solve, cell layout."""
        f = np.empty(self.cell_shape)
        p = np.empty(self.cell_shape)
        self._check(self.lib.cdi_last_pressure(self.h, _dp(f), _dp(p)))
        return f, p

    def profile_start(self, kernel: str, max_launches: int = 4096):
        self._check(self.lib.cdi_profile_start(self.h, kernel.encode(), max_launches))

    def profile_stop(self):
        ms, n = ctypes.c_double(), ctypes.c_long()
        self._check(self.lib.cdi_profile_stop(self.h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value


class Batch:
    """Many Solvers advanced by one batched launch (cdi_batch_* in cdi.h)."""

    def __init__(self, solvers):
        import torch

        self.lib = load()
        self.solvers = list(solvers)
        n = len(self.solvers)
        arr = (ctypes.c_void_p * n)(*[s.h.value for s in self.solvers])
        h = ctypes.c_void_p()
        self._check(self.lib.cdi_batch_create(ctypes.byref(h), n, arr), None)
        self.h = h
        nbytes = ctypes.c_size_t()
        self._check(self.lib.cdi_batch_workspace_bytes(self.h, ctypes.byref(nbytes)))
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device="cuda")
        self.stream = self.solvers[0].stream
        self._check(self.lib.cdi_batch_bind_workspace(self.h, ctypes.c_void_p(self.workspace.data_ptr()),
                                                      nbytes.value, ctypes.c_void_p(self.stream.cuda_stream)))

    def _check(self, st, h="self"):
        if st != 0:
            msg = self.lib.cdi_batch_last_error(self.h if h == "self" else None)
            raise CdiError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.lib.cdi_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, dts, nsteps=1):
        d = np.ascontiguousarray(dts, dtype=np.float64)
        assert d.shape == (len(self.solvers),)
        self._check(self.lib.cdi_batch_step(self.h, _dp(d), nsteps))

    def set_threads(self, threads):
        self._check(self.lib.cdi_batch_set_threads(self.h, threads))

    def set_tail_budget(self, nbytes):
        self._check(self.lib.cdi_batch_set_tail_budget(self.h, int(nbytes)))

    def autotune(self, dts, trial_steps=1):
        """Returns (threads, tail budget in bytes, times in ms [budget][threads],
        -1 where a pair does not launch)."""
        d = np.ascontiguousarray(dts, dtype=np.float64)
        best = ctypes.c_int()
        tail = ctypes.c_size_t()
        ms = np.zeros(12)
        self._check(self.lib.cdi_batch_autotune(self.h, _dp(d), trial_steps, ctypes.byref(best), ctypes.byref(tail),
                                                _dp(ms)))
        return best.value, tail.value, ms.reshape(4, 3)

    def stats(self, i):
        st, mx, tot, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        self._check(self.lib.cdi_batch_stats(self.h, i, ctypes.byref(st), ctypes.byref(mx), ctypes.byref(tot),
                                             ctypes.byref(ms)))
        return {"status": st.value, "max_cycles": mx.value, "total_cycles": tot.value, "last_ms": ms.value}


class Unet:
    """Warm-start U-Net on the GPU (cdi_unet_* in cdi.h).  Arrays are
    channels-last (nz, ny, nx, C) float64; parameters are a flat vector in the
    order of cdi_unet_set_params."""

    def __init__(self, n, stream=None):
        import torch

        self.lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("libcdi needs a CUDA device; there is no CPU path")
        self.n = tuple(int(x) for x in n)
        h = ctypes.c_void_p()
        self._check(self.lib.cdi_unet_create(ctypes.byref(h), *self.n), None)
        self.h = h
        nbytes = ctypes.c_size_t()
        self._check(self.lib.cdi_unet_workspace_bytes(self.h, ctypes.byref(nbytes)))
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device="cuda")
        self.stream = torch.cuda.current_stream() if stream is None else stream
        self._check(self.lib.cdi_unet_bind_workspace(self.h, ctypes.c_void_p(self.workspace.data_ptr()),
                                                     nbytes.value, ctypes.c_void_p(self.stream.cuda_stream)))
        c = ctypes.c_size_t()
        self._check(self.lib.cdi_unet_param_count(ctypes.byref(c)))
        self.nparams = int(c.value)

    def _check(self, st, h="self"):
        if st != 0:
            msg = self.lib.cdi_unet_last_error(self.h if h == "self" else None)
            raise CdiError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.lib.cdi_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def set_params(self, flat):
        a = _f64(flat)
        assert a.shape == (self.nparams,)
        self._check(self.lib.cdi_unet_set_params(self.h, _dp(a), a.size))

    def get_params(self):
        a = np.empty(self.nparams)
        self._check(self.lib.cdi_unet_get_params(self.h, _dp(a), a.size))
        return a

    def forward(self, x):
        xa = _f64(x)
        assert xa.shape == self.shape + (2,)
        y = np.empty(self.shape)
        self._check(self.lib.cdi_unet_forward(self.h, _dp(xa), _dp(y)))
        return y

    def set_conv_kernel(self, tensor_core):
        """Convolutions and weight gradients on tcgen05 (True or 1, default),
        everything on mma.sync (False or 0), or tcgen05 convolutions with the
        mma.sync weight gradients (2)."""
        mode = tensor_core if isinstance(tensor_core, int) and not isinstance(tensor_core, bool) else (
            1 if tensor_core else 0)
        self._check(self.lib.cdi_unet_set_conv_kernel(self.h, mode))

    def forward_device(self, x, y):
        """Device forward pass: torch float32 tensors x (..., 2) and y (...) on
        the network's device; stream-ordered, no synchronisation."""
        import torch

        assert x.is_cuda and x.dtype == torch.float32 and y.dtype == torch.float32
        assert x.numel() == 2 * y.numel() == 2 * int(np.prod(self.n))
        assert x.is_contiguous() and y.is_contiguous()
        self._check(self.lib.cdi_unet_forward_device(self.h, ctypes.c_void_p(x.data_ptr()),
                                                     ctypes.c_void_p(y.data_ptr())))

    def train_step(self, x, target, lr=0.0, want_grads=False):
        """Loss before the update and (optionally) the flat gradients."""
        xa, ta = _f64(x), _f64(target)
        assert xa.shape == self.shape + (2,) and ta.size == xa.size // 2
        loss = ctypes.c_double()
        g = np.empty(self.nparams) if want_grads else None
        self._check(self.lib.cdi_unet_train_step(self.h, _dp(xa), _dp(ta), float(lr), ctypes.byref(loss), _dp(g)))
        return (loss.value, g) if want_grads else loss.value


def from_workload(wl, precision=FP64, tol=1e-10, max_vcycles=100):
    """Solver set up with a Workload from paper_2412_16843_gb300.inputs."""
    s = Solver(wl.dim, wl.n, wl.L, precision)
    s.set_fluids(wl.rho1, wl.rho2, wl.mu1, wl.mu2, wl.sigma, wl.eps, wl.gamma)
    s.set_wall(WALL_LO, wl.theta_eq, wl.slip_length, wl.U_lo)
    s.set_wall(WALL_HI, wl.theta_eq, wl.slip_length, wl.U_hi)
    s.set_solver(tol, max_vcycles, WARM_PREV)
    s.set_state(wl.phi0)
    return s
