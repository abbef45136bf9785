"""Python handle on the plain FP64 CPU oracle (oracle/cdi_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline leg of bench.py.  The product path (the CUDA library and its
binding) never imports this package.

Every function of the oracle follows a passage of the paper (see the header
of cdi_oracle.cpp).  Parity pins for each part live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cdi_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libcdi_oracle.so")
_lock = threading.Lock()
_lib = None

# slip models of Sec. 3
MODELS = {"1A": 0, "1B": 1, "2A": 2, "2B": 3, "3A": 4, "3B": 5, "4A": 6, "4B": 7}
STATUS = {0: "OK", 1: "EINVAL", 2: "ESTATE", 4: "ENOCONV", 5: "ENAN"}


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, no FP contraction, no -march)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D = ctypes.c_double
        I = ctypes.c_int
        P = ctypes.c_void_p
        DP = ctypes.POINTER(ctypes.c_double)
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [I, I, I, I, D, D, D]
        lib.orc_destroy.argtypes = [P]
        lib.orc_set_fluids.argtypes = [P, D, D, D, D, D, D, D]
        lib.orc_set_wall.argtypes = [P, I, D, D, D, D, D]
        lib.orc_set_model.argtypes = [P, I]
        lib.orc_set_solver.argtypes = [P, D, I, I]
        lib.orc_set_regularisation.argtypes = [P, D, D]
        lib.orc_set_state.argtypes = [P, DP, DP, DP, DP, DP]
        lib.orc_get_state.argtypes = [P, DP, DP, DP, DP, DP]
        lib.orc_step.argtypes = [P, D, I]
        lib.orc_project_final_only.argtypes = [P, I]
        lib.orc_mass.restype = D
        lib.orc_mass.argtypes = [P]
        lib.orc_contact_angle.argtypes = [P, I, DP, DP]
        lib.orc_last_stats.argtypes = [P, ctypes.POINTER(I), DP, ctypes.POINTER(I),
                                       ctypes.POINTER(ctypes.c_long)]
        lib.orc_eval_psi.argtypes = [P, DP] + [DP] * 10
        lib.orc_eval_wall.argtypes = [P, DP, DP, DP]
        lib.orc_eval_wall_columns.argtypes = [P, DP, DP]
        lib.orc_eval_rhs.argtypes = [P, D, DP, DP, DP, DP]
        lib.orc_poisson.argtypes = [P, DP, DP, ctypes.POINTER(I), DP]
        lib.orc_poisson_direct.argtypes = [P, DP, DP]
        lib.orc_apply_laplacian.argtypes = [P, DP, DP]
        lib.orc_divergence.argtypes = [P, DP]
        lib.orc_num_levels.argtypes = [P]
        _lib = lib
        return lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


class Oracle:
    """FP64 CPU solver with the same problem statement as the C ABI.

    dim 2: n = (nx, ny), walls at y = 0 and y = ny*h.
    dim 3: n = (nx, ny, nz), walls at z = 0 and z = nz*h.
    Spacing h = Lx / nx (uniform).
    """

    def __init__(self, dim: int, n, L):
        self.lib = _load()
        self.dim = dim
        self.n = tuple(int(x) for x in n)
        nz = self.n[2] if dim == 3 else 1
        Lz = L[2] if dim == 3 else 0.0
        self.h = L[0] / self.n[0]
        self.handle = self.lib.orc_create(dim, self.n[0], self.n[1], nz, L[0], L[1], Lz)
        if not self.handle:
            raise OracleError("invalid grid")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            self.lib.orc_destroy(h)
            self.handle = None

    # ---- shapes -----------------------------------------------------------
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

    # ---- parameters -------------------------------------------------------
    def set_fluids(self, rho1, rho2, mu1, mu2, sigma, eps, gamma):
        self.lib.orc_set_fluids(self.handle, rho1, rho2, mu1, mu2, sigma, eps, gamma)
        self.mu = (mu1, mu2)

    def set_wall(self, wall: int, theta, beta1, beta2, Ux=0.0, Uy=0.0):
        """wall 0 low, 1 high, 2 both; beta = inf means no slip."""
        self.lib.orc_set_wall(self.handle, wall, theta, beta1, beta2, Ux, Uy)

    def set_wall_slip_length(self, wall, theta, slip_length, Ux=0.0, Uy=0.0):
        """beta_i = mu_i / slip_length (Eq. u_slip_v: slip length mu / beta)."""
        if slip_length == 0:
            b1 = b2 = float("inf")
        else:
            b1, b2 = self.mu[0] / slip_length, self.mu[1] / slip_length
        self.set_wall(wall, theta, b1, b2, Ux, Uy)

    def set_model(self, name: str):
        self.lib.orc_set_model(self.handle, MODELS[name])

    def set_solver(self, tol=1e-10, maxcyc=200, warm=True):
        self.lib.orc_set_solver(self.handle, tol, maxcyc, 1 if warm else 0)

    def set_regularisation(self, delta=1e-6, tau=1e-6):
        self.lib.orc_set_regularisation(self.handle, delta, tau)

    def project_final_only(self, flag=True):
        self.lib.orc_project_final_only(self.handle, 1 if flag else 0)

    # ---- state ------------------------------------------------------------
    def set_state(self, phi, vel=None, p=None):
        phi = _c64(phi)
        if vel is None:
            vel = [np.zeros(self.face_shape(a)) for a in range(self.dim)]
        vel = [_c64(x) for x in vel]
        for a in range(self.dim):
            assert vel[a].shape == self.face_shape(a), (a, vel[a].shape)
        comps = vel + [None] * (3 - self.dim)
        pp = None if p is None else _c64(p)
        self.lib.orc_set_state(self.handle, _ptr(phi), *[_ptr(c) for c in comps], _ptr(pp))

    def get_state(self):
        phi = np.empty(self.cell_shape)
        vel = [np.empty(self.face_shape(a)) for a in range(self.dim)]
        p = np.empty(self.cell_shape)
        comps = vel + [None] * (3 - self.dim)
        self.lib.orc_get_state(self.handle, _ptr(phi), *[_ptr(c) for c in comps], _ptr(p))
        return phi, vel, p

    def step(self, dt, nsteps=1):
        st = self.lib.orc_step(self.handle, dt, nsteps)
        if st != 0:
            raise OracleError("step failed: " + STATUS.get(st, str(st)))

    def mass(self):
        return self.lib.orc_mass(self.handle)

    def contact_angle(self, wall=0):
        th = ctypes.c_double()
        L = ctypes.c_double()
        self.lib.orc_contact_angle(self.handle, wall, ctypes.byref(th), ctypes.byref(L))
        return th.value, L.value

    def last_stats(self):
        c = ctypes.c_int()
        r = ctypes.c_double()
        m = ctypes.c_int()
        t = ctypes.c_long()
        self.lib.orc_last_stats(self.handle, ctypes.byref(c), ctypes.byref(r),
                                ctypes.byref(m), ctypes.byref(t))
        return {"cycles": c.value, "resid": r.value, "max_cycles_step": m.value,
                "total_cycles": t.value}

    # ---- stage-level evaluations -----------------------------------------
    def eval_psi(self, phi):
        phi = _c64(phi)
        names = ["psi", "gx", "gy", "gz", "lap", "kappa", "muc", "nx", "ny", "nz"]
        out = {k: np.zeros(self.cell_shape) for k in names}
        self.lib.orc_eval_psi(self.handle, _ptr(phi), *[_ptr(out[k]) for k in names])
        return out

    def eval_wall(self):
        np_ = int(np.prod(self.plane))
        t = self.dim - 1
        uY = np.zeros((2, t, np_))
        g = np.zeros((2, t, np_))
        pw = np.zeros((2, np_))
        self.lib.orc_eval_wall(self.handle, _ptr(uY), _ptr(g), _ptr(pw))
        sh = (2, t) + self.plane
        return uY.reshape(sh), g.reshape(sh), pw.reshape((2,) + self.plane)

    def wall_columns(self):
        """Extrapolated psi_w and in-plane curvature kappa_p of every wall
        column, shape (2,) + wall plane (low wall first)."""
        np_ = int(np.prod(self.plane))
        psiw = np.zeros((2, np_))
        kpw = np.zeros((2, np_))
        self.lib.orc_eval_wall_columns(self.handle, _ptr(psiw), _ptr(kpw))
        sh = (2,) + self.plane
        return psiw.reshape(sh), kpw.reshape(sh)

    def eval_rhs(self, gamma=-1.0):
        rphi = np.zeros(self.cell_shape)
        rv = [np.zeros(self.face_shape(a)) for a in range(self.dim)]
        comps = rv + [None] * (3 - self.dim)
        self.lib.orc_eval_rhs(self.handle, gamma, _ptr(rphi), *[_ptr(c) for c in comps])
        return rphi, rv

    def poisson(self, f, p0=None):
        f = _c64(f)
        p = np.zeros(self.cell_shape) if p0 is None else _c64(p0).copy()
        cyc = ctypes.c_int()
        res = ctypes.c_double()
        st = self.lib.orc_poisson(self.handle, _ptr(f), _ptr(p), ctypes.byref(cyc), ctypes.byref(res))
        if st != 0:
            raise OracleError("poisson: " + STATUS.get(st, str(st)))
        return p, cyc.value, res.value

    def poisson_direct(self, f):
        f = _c64(f)
        p = np.zeros(self.cell_shape)
        st = self.lib.orc_poisson_direct(self.handle, _ptr(f), _ptr(p))
        if st != 0:
            raise OracleError("poisson_direct: " + STATUS.get(st, str(st)))
        return p

    def apply_laplacian(self, p):
        p = _c64(p)
        out = np.zeros(self.cell_shape)
        self.lib.orc_apply_laplacian(self.handle, _ptr(p), _ptr(out))
        return out

    def divergence(self):
        out = np.zeros(self.cell_shape)
        self.lib.orc_divergence(self.handle, _ptr(out))
        return out

    def num_levels(self):
        return self.lib.orc_num_levels(self.handle)


def from_workload(wl, tol=1e-10, maxcyc=200):
    """Oracle set up with a Workload from paper_2412_16843_gb300.inputs."""
    o = Oracle(wl.dim, wl.n, wl.L)
    o.set_fluids(wl.rho1, wl.rho2, wl.mu1, wl.mu2, wl.sigma, wl.eps, wl.gamma)
    o.set_wall_slip_length(0, wl.theta_eq, wl.slip_length, wl.U_lo)
    o.set_wall_slip_length(1, wl.theta_eq, wl.slip_length, wl.U_hi)
    o.set_solver(tol, maxcyc, True)
    o.set_state(wl.phi0)
    return o
