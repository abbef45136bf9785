"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds no step arithmetic of the method: only initial phase fields,
velocity fields and the workload parameter sets.  Both the CPU oracle and the
CUDA library receive the arrays built here, so the two sides never generate
their own inputs.

Layout of every array (the same as the C ABI): row-major with x fastest and no
halo.  Cell fields have shape (nz, ny, nx) in 3D and (ny, nx) in 2D.  The
velocity component normal to the walls (v in 2D, w in 3D) carries one extra
face plane, so its shape is (ny+1, nx) in 2D and (nz+1, ny, nx) in 3D.  The
walls sit on the low and high end of the last axis; all other axes are
periodic.

Initial conditions follow the paper:
  * prescribed equilibrium drop, Eq. (prescribed phase field) of Sec. 3.1, with
    the area-preserving radius of a circular segment (the printed radius
    formula is garbled: it only preserves the area at 90 degrees, which is
    what the paper says the formula is for);
  * two-interface Couette field, Eq. (couette flow initial phi) of Sec. 5.2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# --------------------------------------------------------------------------
# geometry helpers
# --------------------------------------------------------------------------

def cell_centres(n: int, h: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def cap_radius(R0: float, theta: float, dim: int = 2) -> float:
    """Radius of a wall-bound cap of contact angle theta with the area (2D) or
    volume (3D) of a half disc / hemisphere of radius R0 (Sec. 3.1).

    2D: circular segment area A(R, theta) = R^2 (theta - sin(theta) cos(theta)).
    3D: spherical cap volume V = pi R^3 (2 - 3 cos t + cos^3 t) / 3.
    """
    if dim == 2:
        A0 = 0.5 * math.pi * R0 * R0
        return math.sqrt(A0 / (theta - math.sin(theta) * math.cos(theta)))
    c = math.cos(theta)
    V0 = 2.0 * math.pi * R0 ** 3 / 3.0
    return (3.0 * V0 / (math.pi * (2.0 - 3.0 * c + c ** 3))) ** (1.0 / 3.0)


def cap_phi_2d(nx: int, ny: int, h: float, R: float, theta: float, xc: float,
               eps: float, wall: str = "lo") -> np.ndarray:
    """Tanh circular cap sitting on the low (or high) wall, contact angle theta.

    The circle centre is at distance -R cos(theta) from the wall (Sec. 3.1)."""
    x = cell_centres(nx, h)[None, :]
    y = cell_centres(ny, h)[:, None]
    Ly = ny * h
    if wall == "lo":
        yc = -R * math.cos(theta)
        r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    else:
        yc = Ly + R * math.cos(theta)
        r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    return 0.5 * (1.0 + np.tanh((R - r) / (2.0 * eps)))


def cap_phi_3d(nx: int, ny: int, nz: int, h: float, R: float, theta: float,
               xc: float, yc: float, eps: float) -> np.ndarray:
    x = cell_centres(nx, h)[None, None, :]
    y = cell_centres(ny, h)[None, :, None]
    z = cell_centres(nz, h)[:, None, None]
    zc = -R * math.cos(theta)
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2 + (z - zc) ** 2)
    return 0.5 * (1.0 + np.tanh((R - r) / (2.0 * eps)))


def couette_phi_2d(nx: int, ny: int, h: float, x1: float, x2: float,
                   eps: float) -> np.ndarray:
    """Two vertical tanh interfaces at x1 < x2, fluid 1 (phi = 1) between them
    (Eq. couette flow initial phi, with the interface positions as inputs)."""
    x = cell_centres(nx, h)[None, :]
    row = (0.5 * (1.0 + np.tanh((x - x1) / (2.0 * eps)))
           + 0.5 * (1.0 + np.tanh((x2 - x) / (2.0 * eps))) - 1.0)
    return np.repeat(row, ny, axis=0)


def tanh_profile_x(nx: int, ny: int, h: float, x0: float, eps: float) -> np.ndarray:
    x = cell_centres(nx, h)[None, :]
    return np.repeat(0.5 * (1.0 + np.tanh((x - x0) / (2.0 * eps))), ny, axis=0)


def add_noise(phi: np.ndarray, amplitude: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = phi + rng.uniform(-amplitude, amplitude, size=phi.shape)
    return np.clip(out, 0.0, 1.0)


def zero_velocity(shape_cells: tuple) -> tuple:
    """Zero face velocities for a cell shape (ny, nx) or (nz, ny, nx)."""
    if len(shape_cells) == 2:
        ny, nx = shape_cells
        return (np.zeros((ny, nx)), np.zeros((ny + 1, nx)))
    nz, ny, nx = shape_cells
    return (np.zeros((nz, ny, nx)), np.zeros((nz, ny, nx)), np.zeros((nz + 1, ny, nx)))


# --------------------------------------------------------------------------
# workload parameter sets
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    dim: int
    n: tuple            # (nx, ny) or (nx, ny, nz)
    L: tuple            # domain lengths
    rho1: float
    rho2: float
    mu1: float
    mu2: float
    sigma: float
    eps: float
    gamma: float
    theta_eq: float     # radians, both walls
    slip_length: float  # beta_i = mu_i / slip_length
    U_lo: float         # x velocity of the low wall
    U_hi: float         # x velocity of the high wall
    dt: float
    steps: int
    phi0: np.ndarray = field(repr=False, default=None)

    @property
    def h(self) -> float:
        return self.L[0] / self.n[0]

    @property
    def cells(self) -> int:
        return int(np.prod(self.n))


def drop_2d(nx: int = 64, ny: int = 32, theta_eq_deg: float = 60.0) -> Workload:
    """Equilibrium drop: 64x32 on [0,1]x[0,0.5], half disc R=0.2 at (0.5, 0),
    density and viscosity ratio 1, sigma=1, eps=dx, gamma=1, slip length dx,
    dt=1e-4."""
    Lx, Ly = 1.0, 0.5 * ny / (nx / 2)
    h = Lx / nx
    phi = cap_phi_2d(nx, ny, h, 0.2, math.pi / 2, 0.5, h)
    return Workload("drop2d_%dx%d" % (nx, ny), 2, (nx, ny), (Lx, ny * h),
                    1.0, 1.0, 0.1, 0.1, 1.0, h, 1.0, math.radians(theta_eq_deg),
                    h, 0.0, 0.0, 1e-4, 2000, phi)


def couette_2d(nx: int = 512, ny: int = 128, slip_factor: float = 1.0) -> Workload:
    """Two-phase Couette: 512x128 on [0,4]x[0,1], walls at +-U=0.1 (top moves
    +x), interfaces at x=1 and x=3, theta_eq=90 deg, slip length slip_factor*dx,
    viscosity ratio 1, Ca = mu U / sigma = 0.05, eps=dx, gamma = 2.5 U."""
    h = 1.0 / ny
    Lx = nx * h
    U = 0.1
    mu = 0.1
    sigma = mu * U / 0.05
    phi = couette_phi_2d(nx, ny, h, Lx / 4, 3 * Lx / 4, h)
    return Workload("couette2d_%dx%d_l%g" % (nx, ny, slip_factor), 2, (nx, ny),
                    (Lx, 1.0), 1.0, 1.0, mu, mu, sigma, h, 2.5 * U,
                    math.pi / 2, slip_factor * h, -U, U, 1.25e-4, 20000, phi)


def drop_3d(n: int = 256, theta_eq_deg: float = 60.0, seed: int = 12345,
            noise: float = 1e-3) -> Workload:
    """3D drop: n^3 on [0,1]^3, walls z, hemisphere R=0.25 at (0.5,0.5,0),
    density ratio 10, viscosity ratio 10, sigma=1, eps=dx, gamma=1, slip
    length dx, tanh profile plus seeded uniform noise clamped to [0,1]."""
    h = 1.0 / n
    phi = cap_phi_3d(n, n, n, h, 0.25, math.pi / 2, 0.5, 0.5, h)
    if noise > 0:
        phi = add_noise(phi, noise, seed)
    return Workload("drop3d_%d" % n, 3, (n, n, n), (1.0, 1.0, 1.0),
                    1.0, 0.1, 0.05, 0.005, 1.0, h, 1.0,
                    math.radians(theta_eq_deg), h, 0.0, 0.0, 3.5e-5, 5000, phi)


def drop_3d_wide(nx: int = 512, seed: int = 12345, noise: float = 1e-3) -> Workload:
    """Wide 3D drop: nx x nx/2 x nx/2 on [0,2]x[0,1]x[0,1], walls z, a 90 deg
    cap R = 0.25 at (1, 0.5, 0) relaxing on a 45 deg wall; density ratio 20
    (rho 1 / 0.05), viscosity ratio 10 (mu 0.05 / 0.005), sigma = 1, eps = dx,
    gamma = 1, slip length dx; dt = 3.0e-5 (the RK4 viscous limit of the
    lighter fluid, nu = 0.1, is 0.23 dx^2 / nu = 3.6e-5 at dx = 1/256);
    seeded uniform noise clamped to [0,1]."""
    ny = nx // 2
    h = 2.0 / nx
    phi = cap_phi_3d(nx, ny, ny, h, 0.25, math.pi / 2, 1.0, 0.5, h)
    if noise > 0:
        phi = add_noise(phi, noise, seed)
    return Workload("drop3d_%dx%dx%d" % (nx, ny, ny), 3, (nx, ny, ny), (2.0, 1.0, 1.0),
                    1.0, 0.05, 0.05, 0.005, 1.0, h, 1.0,
                    math.radians(45.0), h, 0.0, 0.0, 3.0e-5, 300, phi)


SWEEP_SIZES = (64, 96, 128, 192, 256, 384, 512)


def stable_dt(wl: Workload, safety: float = 0.4) -> float:
    """A step inside the explicit limits of the RK4 step: viscous
    (0.35 h^2 rho_min / mu_max in 2D, 0.23 h^2 rho_min / mu_max in 3D),
    capillary (sqrt((rho1+rho2) h^3 / (4 pi sigma))) and advective
    (h / (|U_wall| + 0.5)), times a safety factor."""
    h = wl.h
    rmin = min(wl.rho1, wl.rho2)
    mmax = max(wl.mu1, wl.mu2, 1e-30)
    visc = (0.35 if wl.dim == 2 else 0.23) * h * h * rmin / mmax
    cap = math.sqrt((wl.rho1 + wl.rho2) * h ** 3 / (4.0 * math.pi * max(wl.sigma, 1e-30)))
    adv = h / (max(abs(wl.U_lo), abs(wl.U_hi)) + 0.5)
    return safety * min(visc, cap, adv)


def sweep_2d(n_inst: int = 512, seed: int = 2024, steps: int = 2000) -> list:
    """Parameter sweep of uneven 2D instances (half drops, half Couette):
    nx drawn log-uniformly in [64, 512] and rounded (in log) to the nearest of
    SWEEP_SIZES (extents whose multigrid coarsens to at most 64 cells), ny =
    nx/2, h = 1/64; theta_eq ~ U[30, 150] deg, slip length ~ U[0.5, 4] h,
    Ca ~ U[0.01, 0.1], density ratio rho1/rho2 ~ U[1, 20] (rho2 = 1),
    mu = 0.1 in both fluids; Couette walls at -/+0.1 (sigma = mu U / Ca), drops
    with sigma = 1 start as a 90 deg cap of radius 0.3 Ly; per-instance dt =
    0.4 x the smallest explicit limit."""
    rng = np.random.default_rng(seed)
    logs = np.log(np.array(SWEEP_SIZES, dtype=float))
    out = []
    h = 1.0 / 64
    for i in range(n_inst):
        s = rng.uniform(math.log(64), math.log(512))
        nx = SWEEP_SIZES[int(np.argmin(np.abs(logs - s)))]
        ny = nx // 2
        th = math.radians(rng.uniform(30.0, 150.0))
        ell = rng.uniform(0.5, 4.0) * h
        ca = rng.uniform(0.01, 0.1)
        ratio = rng.uniform(1.0, 20.0)
        mu = 0.1
        Lx, Ly = nx * h, ny * h
        if i % 2 == 0:
            sigma, U, gamma = 1.0, 0.0, 1.0
            phi = cap_phi_2d(nx, ny, h, 0.3 * Ly, math.pi / 2, 0.5 * Lx, h)
            name = "sweep%03d_drop_%dx%d" % (i, nx, ny)
        else:
            U = 0.1
            sigma, gamma = mu * U / ca, 2.5 * U
            phi = couette_phi_2d(nx, ny, h, Lx / 4, 3 * Lx / 4, h)
            name = "sweep%03d_couette_%dx%d" % (i, nx, ny)
        wl = Workload(name, 2, (nx, ny), (Lx, Ly), ratio, 1.0, mu, mu, sigma, h, gamma, th, ell,
                      -U, U, 0.0, steps, phi)
        wl.dt = stable_dt(wl)
        out.append(wl)
    return out


def workload(name: str) -> Workload:
    table = {
        "drop2d_64x32": lambda: drop_2d(64, 32),
        "couette2d_512x128": lambda: couette_2d(512, 128, 1.0),
        "drop3d_256": lambda: drop_3d(256),
    }
    return table[name]()


# warm-start network: layer table (name, Cin, Cout, taps) and seeded initial
# parameters in the flat order of cdi_unet_set_params
UNET_LAYERS = (("e0", 2, 16, 27), ("e1", 16, 32, 27), ("e2", 32, 64, 27), ("b", 64, 128, 27),
               ("d2", 192, 64, 27), ("d1", 96, 32, 27), ("d0", 48, 16, 27), ("head", 16, 1, 1))


def unet_initial_params(seed: int = 0) -> np.ndarray:
    """He-normal weights (std sqrt(2 / (taps Cin))), zero biases; flat vector,
    per layer the weights [taps][Cout][Cin] then the biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for _, ci, co, t in UNET_LAYERS:
        parts.append((rng.standard_normal((t, co, ci)) * math.sqrt(2.0 / (t * ci))).ravel())
        parts.append(np.zeros(co))
    return np.concatenate(parts)


def unet_pair(f: np.ndarray, p: np.ndarray, phi: np.ndarray, rho1: float, rho2: float, h: float):
    """Network input (f / rms(f), rho / max(rho)) and target p / (rms(f) max(rho) h^2)
    for one pressure solve, channels last."""
    rms = float(np.sqrt(np.mean(f * f)))
    rmax = max(rho1, rho2)
    rho = (rho1 - rho2) * phi + rho2
    return np.stack([f / rms, rho / rmax], axis=-1), p / (rms * rmax * h * h)
