"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Per-call checks compare every element of a stage result; time-stepping checks
compare every field after many steps.  FP64 bar: 1e-12 relative per call and
1e-10 relative (max-norm difference over the field's max norm, p zero-mean)
after 1000 steps.  The two sides differ only in rounding order (fused
multiply-add, reduction order, libm).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2412_16843_gb300 import cdi, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_16843_gb300 import build
    build.build()
    cdi.load()


def rel(a, b):
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() / scale


def pair(wl, tol=1e-12, precision=cdi.FP64, exec_mode=cdi.EXEC_PERSISTENT):
    g = cdi.from_workload(wl, precision=precision, tol=tol)
    g.set_exec(exec_mode)
    o = oracle.from_workload(wl, tol=tol)
    return g, o


EXEC_MODES = pytest.mark.parametrize("exec_mode", [cdi.EXEC_PERSISTENT, cdi.EXEC_KERNELS],
                                     ids=["persistent", "kernels"])


def moving_state(wl, nsteps=5):
    """A state with a nonzero velocity: the oracle's state after a few steps."""
    o = oracle.from_workload(wl, tol=1e-12)
    o.step(wl.dt, nsteps)
    return o.get_state()


# ---------------------------------------------------------------------------
# per-call parity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("model", ["4A", "1A", "2B", "3B", "4B"])
def test_rhs_and_wall_parity_2d(model):
    wl = inputs.drop_2d(64, 32)
    phi, vel, p = moving_state(wl)
    g, o = pair(wl)
    g.set_model(model)
    o.set_model(model)
    g.set_state(phi, vel)
    o.set_state(phi, vel, p)
    rg, mg = g.eval_rhs(gamma=1.0)
    ro, mo = o.eval_rhs(gamma=1.0)
    assert rel(rg, ro) < 1e-12
    for a in range(2):
        assert rel(mg[a], mo[a]) < 1e-12, a
    uYg, ghg = g.eval_wall()
    uYo, gho, _ = o.eval_wall()
    assert rel(uYg, uYo) < 1e-12
    assert rel(ghg, gho) < 1e-12


@pytest.mark.parametrize("n", [(16, 8, 12), (64, 16, 16)], ids=["cellwise", "tiled"])
def test_rhs_and_wall_parity_3d(n):
    """Every element of the 3D stage right-hand side and wall rows against the
    oracle: on a grid the tiled kernels do not take (16 x 8 x 12) and on one
    they do (64 x 16 x 16: the tiled momentum kernel, 32 x 8 tiles, with
    periodic seams and both walls)."""
    h = 1.0 / 16
    L = tuple(x * h for x in n)
    rng = np.random.default_rng(11)
    phi = inputs.add_noise(inputs.cap_phi_3d(*n, h, 0.3, math.radians(80), 0.5, 0.25, 1.3 * h), 1e-3, 5)
    vel = [0.05 * rng.standard_normal((n[2], n[1], n[0])), 0.05 * rng.standard_normal((n[2], n[1], n[0])),
           0.05 * rng.standard_normal((n[2] + 1, n[1], n[0]))]
    vel[2][0] = 0.0
    vel[2][-1] = 0.0
    g = cdi.Solver(3, n, L)
    o = oracle.Oracle(3, n, L)
    for s in (g, o):
        s.set_fluids(1.0, 0.1, 0.05, 0.005, 1.0, 1.3 * h, 1.0)
    g.set_wall(cdi.WALL_LO, math.radians(60), h, 0.02)
    g.set_wall(cdi.WALL_HI, math.radians(120), 2 * h, -0.03)
    g.set_wall_velocity(cdi.WALL_LO, 0.02, 0.01)
    o.set_wall_slip_length(0, math.radians(60), h, 0.02, 0.01)
    o.set_wall_slip_length(1, math.radians(120), 2 * h, -0.03)
    g.set_state(phi, vel)
    o.set_state(phi, vel)
    rg, mg = g.eval_rhs(gamma=1.0)
    ro, mo = o.eval_rhs(gamma=1.0)
    assert rel(rg, ro) < 1e-12
    for a in range(3):
        assert rel(mg[a], mo[a]) < 1e-12, a
    uYg, ghg = g.eval_wall()
    uYo, gho, _ = o.eval_wall()
    assert rel(uYg, uYo) < 1e-12
    assert rel(ghg, gho) < 1e-12


def test_rhs_fp32_float4_kernels_vs_oracle():
    """FP32-mixed stage right-hand side of a 64 x 16 x 16 drop with a random
    velocity (periodic seams, both walls) through the float4 kernels (psi,
    normals and chemical potential, phi flux with the mass flux, then the tiled
    momentum kernel that reads them) against the FP64 oracle: every element
    within 1e-3 of the field's largest value.  A wrong neighbour or face in
    a kernel moves some elements by O(1) of it; FP32 rounding moves them by
    about 1e-6."""
    n = (64, 16, 16)
    h = 1.0 / 16
    L = tuple(x * h for x in n)
    rng = np.random.default_rng(12)
    phi = inputs.cap_phi_3d(*n, h, 0.3, math.radians(80), 2.0, 0.5, 1.3 * h)
    vel = [0.05 * rng.standard_normal((n[2], n[1], n[0])), 0.05 * rng.standard_normal((n[2], n[1], n[0])),
           0.05 * rng.standard_normal((n[2] + 1, n[1], n[0]))]
    vel[2][0] = 0.0
    vel[2][-1] = 0.0
    g = cdi.Solver(3, n, L, precision=cdi.FP32_MIXED)
    o = oracle.Oracle(3, n, L)
    for s_ in (g, o):
        s_.set_fluids(1.0, 0.1, 0.05, 0.005, 1.0, 1.3 * h, 1.0)
    g.set_wall(cdi.WALL_LO, math.radians(60), h, 0.02)
    g.set_wall(cdi.WALL_HI, math.radians(120), 2 * h, -0.03)
    o.set_wall_slip_length(0, math.radians(60), h, 0.02)
    o.set_wall_slip_length(1, math.radians(120), 2 * h, -0.03)
    g.set_state(phi, vel)
    o.set_state(phi, vel)
    rg, mg = g.eval_rhs(gamma=1.0)
    ro, mo = o.eval_rhs(gamma=1.0)
    errs = [rel(rg, ro)] + [rel(mg[a], mo[a]) for a in range(3)]
    print("FP32 RHS max error / max: phi %.2e, momentum %.2e %.2e %.2e" % tuple(errs))
    assert max(errs) < 1e-3, errs


@pytest.mark.parametrize("dim", [2, 3])
def test_pressure_solve_parity(dim):
    n = (64, 32) if dim == 2 else (16, 16, 8)
    h = 1.0 / n[0]
    L = tuple(x * h for x in n)
    rng = np.random.default_rng(2)
    phi = np.clip(rng.uniform(-0.2, 1.2, size=n[::-1]), 0, 1)
    f = rng.standard_normal(n[::-1])
    g = cdi.Solver(dim, n, L)
    o = oracle.Oracle(dim, n, L)
    for s in (g, o):
        s.set_fluids(20.0, 1.0, 0.1, 0.1, 0.0, h, 0.0)
    g.set_solver(1e-12, 100, cdi.WARM_ZERO)
    o.set_solver(1e-12, 100, False)
    g.set_state(phi)
    o.set_state(phi)
    pg = g.solve_pressure(f)
    po, cyc, _ = o.poisson(f)
    # the GPU solver (FP64 defect correction around FP32 V-cycles) and the
    # oracle's FP64 multigrid converge to the same solution of the same system
    assert rel(pg, po) < 1e-10
    fm = f - f.mean()
    assert np.linalg.norm(o.apply_laplacian(pg) - fm) <= 1.01e-12 * np.linalg.norm(fm)
    assert abs(pg.mean()) < 1e-12 * np.abs(pg).max()


# ---------------------------------------------------------------------------
# time-stepping parity
# ---------------------------------------------------------------------------

@EXEC_MODES
def test_step_parity_drop_1000_steps(exec_mode):
    """64x32 equilibrium drop (FP64 plain method), 1000 steps: every field
    within 1e-10 relative of the oracle; mass conserved to round-off."""
    wl = inputs.drop_2d(64, 32)
    g, o = pair(wl, tol=1e-12, exec_mode=exec_mode)
    m0 = g.mass()
    assert abs(m0 - o.mass()) < 1e-15
    g.step(wl.dt, 1000)
    o.step(wl.dt, 1000)
    phi_g, vel_g, p_g = g.get_fields()
    phi_o, vel_o, p_o = o.get_state()
    assert rel(phi_g, phi_o) < 1e-10
    for a in range(2):
        assert rel(vel_g[a], vel_o[a]) < 1e-10, a
    assert rel(p_g - p_g.mean(), p_o - p_o.mean()) < 1e-10
    assert abs(g.mass() - m0) / m0 < 1e-13
    tg, Lg = g.contact_angle(0)
    to, Lo = o.contact_angle(0)
    assert abs(tg - to) < 1e-9 and abs(Lg - Lo) < 1e-9


@EXEC_MODES
def test_step_parity_couette_cut(exec_mode):
    """128x32 cut of the two-phase Couette case (moving walls, slip length dx)."""
    wl = inputs.couette_2d(128, 32, 1.0)
    g, o = pair(wl, tol=1e-12, exec_mode=exec_mode)
    g.step(wl.dt, 100)
    o.step(wl.dt, 100)
    phi_g, vel_g, p_g = g.get_fields()
    phi_o, vel_o, p_o = o.get_state()
    assert rel(phi_g, phi_o) < 1e-11
    for a in range(2):
        assert rel(vel_g[a], vel_o[a]) < 1e-10, a


@EXEC_MODES
def test_step_parity_3d_drop(exec_mode):
    """16x16x12 3D drop with density ratio 10 and noise, 10 steps."""
    n = (16, 16, 12)
    h = 1.0 / 16
    L = tuple(x * h for x in n)
    phi = inputs.add_noise(inputs.cap_phi_3d(*n, h, 0.3, math.pi / 2, 0.5, 0.5, h), 1e-3, 12345)
    g = cdi.Solver(3, n, L)
    o = oracle.Oracle(3, n, L)
    for s in (g, o):
        s.set_fluids(1.0, 0.1, 0.05, 0.005, 1.0, h, 1.0)
        s.set_solver(1e-12, 100)
    g.set_wall(cdi.WALL_BOTH, math.radians(60), h, 0.0)
    g.set_exec(exec_mode)
    o.set_wall_slip_length(2, math.radians(60), h, 0.0)
    g.set_state(phi)
    o.set_state(phi)
    g.step(5e-5, 10)
    o.step(5e-5, 10)
    phi_g, vel_g, _ = g.get_fields()
    phi_o, vel_o, _ = o.get_state()
    assert rel(phi_g, phi_o) < 1e-11
    for a in range(3):
        assert rel(vel_g[a], vel_o[a]) < 1e-10, a


@pytest.mark.parametrize("sweep", [cdi.SWEEP_ONEPASS, cdi.SWEEP_COLOUR], ids=["onepass", "colour"])
@pytest.mark.parametrize("precision", [cdi.FP64, cdi.FP32_MIXED], ids=["fp64", "fp32_mixed"])
def test_step_parity_3d_level0_sweeps(precision, sweep):
    """64x16x16 3D drop (density ratio 10, noise) on the launch-per-kernel path
    with each level-0 smoother: one-pass red-black sweeps over 64 x 16 tiles
    marching along z (forced: on a grid this small the automatic choice takes
    the colour passes), and one launch per colour; 10 steps: FP64 within the
    FP64 bar of the oracle, FP32-mixed within its FP32-level bounds."""
    n = (64, 16, 16)
    h = 1.0 / 16
    L = tuple(x * h for x in n)
    phi = inputs.add_noise(inputs.cap_phi_3d(*n, h, 0.3, math.pi / 2, 2.0, 0.5, h), 1e-3, 99)
    g = cdi.Solver(3, n, L, precision=precision)
    o = oracle.Oracle(3, n, L)
    for s in (g, o):
        s.set_fluids(1.0, 0.1, 0.05, 0.005, 1.0, h, 1.0)
        s.set_solver(1e-12, 100)
    g.set_wall(cdi.WALL_BOTH, math.radians(60), h, 0.0)
    g.set_exec(cdi.EXEC_KERNELS)
    g.set_level0_sweep(sweep)
    o.set_wall_slip_length(2, math.radians(60), h, 0.0)
    g.set_state(phi)
    o.set_state(phi)
    g.step(5e-5, 10)
    o.step(5e-5, 10)
    assert g.last_stats()["resid"] <= 1e-12
    phi_g, vel_g, p_g = g.get_fields()
    phi_o, vel_o, p_o = o.get_state()
    tol_phi, tol_u = (1e-11, 1e-10) if precision == cdi.FP64 else (1e-5, 1e-3)
    assert rel(phi_g, phi_o) < tol_phi
    for a in range(3):
        assert rel(vel_g[a], vel_o[a]) < tol_u, a
    assert rel(p_g - p_g.mean(), p_o - p_o.mean()) < tol_u


def _drop3d_solver(n, precision, sweep, tol=1e-12):
    h = 1.0 / 16
    L = tuple(x * h for x in n)
    phi = inputs.add_noise(inputs.cap_phi_3d(*n, h, 0.3, math.pi / 2, 2.0, 0.5, h), 1e-3, 99)
    g = cdi.Solver(3, n, L, precision=precision)
    g.set_fluids(1.0, 0.1, 0.05, 0.005, 1.0, h, 1.0)
    g.set_solver(tol, 100)
    g.set_wall(cdi.WALL_BOTH, math.radians(60), h, 0.0)
    g.set_exec(cdi.EXEC_KERNELS)
    g.set_level0_sweep(sweep)
    g.set_state(phi)
    return g, phi, L


@pytest.mark.parametrize("precision", [cdi.FP64, cdi.FP32_MIXED], ids=["fp64", "fp32_mixed"])
def test_onepass_sweep_tma_staging_is_bitwise_cpasync(precision):
    """256x64x64 3D drop: 4 x 4 tiles of 64 x 16, of which the 2 x 2 whose
    halo lies inside the grid stage their planes with TMA boxes and the 12 on
    the periodic seams with cp.async (z in chunks of 8, so chunk edges are
    crossed too).  The same 4 steps with cp.async staging on every tile give
    bit-identical fields: the staging feeds the same arithmetic, and the
    cp.async form is the one held to the oracle above."""
    n = (256, 64, 64)
    out = []
    for sweep in (cdi.SWEEP_ONEPASS, cdi.SWEEP_ONEPASS_CPASYNC):
        g, _, _ = _drop3d_solver(n, precision, sweep)
        g.step(5e-5, 4)
        out.append(g.get_fields())
        assert g.last_stats()["resid"] <= 1e-12
    (phi_a, vel_a, p_a), (phi_b, vel_b, p_b) = out
    assert np.array_equal(phi_a, phi_b)
    for a in range(3):
        assert np.array_equal(vel_a[a], vel_b[a]), a
    assert np.array_equal(p_a, p_b)


@pytest.mark.parametrize("omega", [1.0, 1.2], ids=["gs", "sor1.2"])
@pytest.mark.parametrize("precision", [cdi.FP64, cdi.FP32_MIXED], ids=["fp64", "fp32_mixed"])
def test_onepass_sweep_is_bitwise_colour_passes(precision, omega):
    """The one-pass sweep (TMA and cp.async tiles, z chunks) computes each
    cell's update with the terms, order and rounding of the colour passes,
    with and without over-relaxation, so 4 steps of the 256x64x64 drop give
    bit-identical fields either way."""
    n = (256, 64, 64)
    out = []
    for sweep in (cdi.SWEEP_ONEPASS, cdi.SWEEP_COLOUR):
        g, _, _ = _drop3d_solver(n, precision, sweep)
        g.set_relaxation(omega)
        g.step(5e-5, 4)
        out.append(g.get_fields())
    (phi_a, vel_a, p_a), (phi_b, vel_b, p_b) = out
    assert np.array_equal(phi_a, phi_b)
    for a in range(3):
        assert np.array_equal(vel_a[a], vel_b[a]), a
    assert np.array_equal(p_a, p_b)


@pytest.mark.parametrize("precision", [cdi.FP64, cdi.FP32_MIXED], ids=["fp64", "fp32_mixed"])
def test_device_controlled_solve_is_bitwise_host_loop(precision):
    """The launch-per-kernel pressure solve runs as one CUDA graph whose V-cycle
    loop is a conditional while node, its tests taken on the device.  While the
    event profiler is on, the host drives the same loop one V-cycle at a time.
    4 steps of the 256x64x64 drop give bit-identical fields and the same V-cycle
    counts either way."""
    n = (256, 64, 64)
    out = []
    for profiled in (False, True):
        g, _, _ = _drop3d_solver(n, precision, cdi.SWEEP_AUTO, tol=1e-10)
        if profiled:
            g.profile_start("resid", 1 << 14)
        cyc = []
        for _ in range(4):
            g.step(5e-5, 1)
            cyc.append(g.last_stats()["total_cycles_call"])
        if profiled:
            _, launches = g.profile_stop()
            assert launches > 0
        out.append((g.get_fields(), cyc))
    ((phi_a, vel_a, p_a), cyc_a), ((phi_b, vel_b, p_b), cyc_b) = out
    assert cyc_a == cyc_b and min(cyc_a) > 0
    assert np.array_equal(phi_a, phi_b)
    for a in range(3):
        assert np.array_equal(vel_a[a], vel_b[a]), a
    assert np.array_equal(p_a, p_b)


def test_device_controlled_solve_zero_rhs():
    """A fluid at rest with uniform phi has f = 0 in every solve: the graph's
    first test skips the loop, p is set to zero, no V-cycle runs."""
    n = (64, 32, 32)
    h = 1.0 / 32
    g = cdi.Solver(3, n, tuple(x * h for x in n), precision=cdi.FP32_MIXED)
    g.set_fluids(1.0, 0.1, 0.05, 0.005, 1.0, h, 1.0)
    g.set_solver(1e-8, 100)
    g.set_wall(cdi.WALL_BOTH, math.radians(60), h, 0.0)
    g.set_exec(cdi.EXEC_KERNELS)
    g.set_state(np.ones(g.cell_shape))
    g.step(1e-4, 3)
    st = g.last_stats()
    assert st["total_cycles_call"] == 0 and st["resid"] == 0.0
    phi, vel, p = g.get_fields()
    assert np.all(p == 0.0) and np.all(phi == 1.0)
    for a in range(3):
        assert np.all(vel[a] == 0.0), a


@EXEC_MODES
def test_couette_full_size_512x128_parity(exec_mode):
    """The full 512x128 Couette workload in the launch configuration the bench
    times (FP64, pressure tolerance 1e-8, warm start): 3 steps, every field vs
    the oracle.  Both sides stop their V-cycles at the same 1e-8 residual, so
    the velocity bar is the solver tolerance times a safety factor of 10."""
    wl = inputs.couette_2d(512, 128, 1.0)
    g, o = pair(wl, tol=1e-8, exec_mode=exec_mode)
    g.set_solver(1e-8, 100, cdi.WARM_EXTRAP)
    g.set_state(wl.phi0)
    g.step(wl.dt, 3)
    o.step(wl.dt, 3)
    phi_g, vel_g, _ = g.get_fields()
    phi_o, vel_o, _ = o.get_state()
    assert rel(phi_g, phi_o) < 1e-11
    for a in range(2):
        assert rel(vel_g[a], vel_o[a]) < 1e-7, a


# ---------------------------------------------------------------------------
# invariants and error paths on the GPU
# ---------------------------------------------------------------------------

def test_contact_angle_of_prescribed_cap_gpu():
    nx, ny = 256, 128
    h = 1.0 / nx
    th = math.radians(60)
    R = inputs.cap_radius(0.15, th)
    phi = inputs.cap_phi_2d(nx, ny, h, R, th, 0.5, h)
    g = cdi.Solver(2, (nx, ny), (1.0, ny * h))
    g.set_fluids(1, 1, 0.1, 0.1, 1.0, h, 1.0)
    g.set_state(phi)
    o = oracle.Oracle(2, (nx, ny), (1.0, ny * h))
    o.set_fluids(1, 1, 0.1, 0.1, 1.0, h, 1.0)
    o.set_state(phi)
    tg, Lg = g.contact_angle(0)
    to, Lo = o.contact_angle(0)
    assert abs(tg - to) < 1e-12 and abs(Lg - Lo) < 1e-12
    assert abs(math.degrees(tg) - 60) < 1.5


@EXEC_MODES
def test_no_convergence_is_reported(exec_mode):
    wl = inputs.drop_2d(64, 32)
    g = cdi.from_workload(wl, tol=1e-14, max_vcycles=1)
    g.set_exec(exec_mode)
    with pytest.raises(cdi.CdiError) as e:
        g.step(wl.dt, 1)
    assert e.value.status == 4


def test_nan_input_is_rejected():
    wl = inputs.drop_2d(64, 32)
    g = cdi.from_workload(wl)
    bad = wl.phi0.copy()
    bad[3, 4] = np.nan
    with pytest.raises(cdi.CdiError) as e:
        g.set_phi(bad)
    assert e.value.status == 5


def test_adaptive_gamma_parity_both_modes():
    """gamma = 2.5 |u|_max (Sec. 5.1) with density and viscosity ratio 10:
    the persistent and per-kernel paths and the oracle agree after 50 steps."""
    nx, ny = 64, 32
    h = 1.0 / nx
    phi = inputs.add_noise(inputs.cap_phi_2d(nx, ny, h, 0.2, math.pi / 2, 0.5, h), 1e-3, 9)
    res = []
    for mode in (cdi.EXEC_PERSISTENT, cdi.EXEC_KERNELS):
        g = cdi.Solver(2, (nx, ny), (1.0, ny * h))
        g.set_fluids(1.0, 0.1, 0.05, 0.005, 1.0, h, -0.5)
        g.set_wall(cdi.WALL_BOTH, math.radians(120), h, 0.0)
        g.set_solver(1e-12, 100)
        g.set_exec(mode)
        g.set_state(phi)
        g.step(5e-5, 50)
        res.append(g.get_fields())
    o = oracle.Oracle(2, (nx, ny), (1.0, ny * h))
    o.set_fluids(1.0, 0.1, 0.05, 0.005, 1.0, h, -0.5)
    o.set_wall_slip_length(2, math.radians(120), h)
    o.set_solver(1e-12, 100)
    o.set_state(phi)
    o.step(5e-5, 50)
    phi_o, vel_o, _ = o.get_state()
    for phi_g, vel_g, _ in res:
        assert rel(phi_g, phi_o) < 1e-11
        for a in range(2):
            assert rel(vel_g[a], vel_o[a]) < 1e-10


@pytest.mark.parametrize("exec_mode", [cdi.EXEC_PERSISTENT, cdi.EXEC_KERNELS], ids=["persistent", "kernels"])
def test_extrapolated_warm_start_parity_and_fewer_cycles(exec_mode):
    """First guess by linear extrapolation in time of each RK stage's pressure:
    same solution as the oracle (whose first guess is the last solve's
    pressure) within the FP64 bar, with fewer V-cycles than the plain guess."""
    wl = inputs.couette_2d(128, 32, 1.0)
    g_prev = cdi.from_workload(wl, tol=1e-12)
    g_ext = cdi.from_workload(wl, tol=1e-12)
    g_ext.set_solver(1e-12, 100, cdi.WARM_EXTRAP)
    g_ext.set_state(wl.phi0)
    for g in (g_prev, g_ext):
        g.set_exec(exec_mode)
        g.step(wl.dt, 20)
    o = oracle.from_workload(wl, tol=1e-12)
    o.step(wl.dt, 20)
    cyc_prev = g_prev.last_stats()["total_cycles_call"]
    g_prev.step(wl.dt, 20)
    g_ext.step(wl.dt, 20)
    o.step(wl.dt, 20)
    cyc_prev = g_prev.last_stats()["total_cycles_call"]
    cyc_ext = g_ext.last_stats()["total_cycles_call"]
    phi_g, vel_g, _ = g_ext.get_fields()
    phi_o, vel_o, _ = o.get_state()
    assert rel(phi_g, phi_o) < 1e-11
    for a in range(2):
        assert rel(vel_g[a], vel_o[a]) < 1e-10
    assert cyc_ext < cyc_prev, (cyc_ext, cyc_prev)


@EXEC_MODES
def test_smoothing_counts_change_cycles_not_the_solution(exec_mode):
    """The red-black sweeps before and after each coarse-grid correction
    (cdi_set_smoothing) change only how the solve gets to its tolerance: after
    20 steps V(1,1), V(2,2) and V(3,1) all match the oracle within the FP64
    bar; more sweeps need no more V-cycles.  Counts outside [1, 4] are
    rejected."""
    wl = inputs.couette_2d(128, 32, 1.0)
    o = oracle.from_workload(wl, tol=1e-12)
    o.step(wl.dt, 20)
    phi_o, vel_o, _ = o.get_state()
    cycles = {}
    for npre, npost in ((1, 1), (2, 2), (3, 1)):
        g = cdi.from_workload(wl, tol=1e-12)
        g.set_exec(exec_mode)
        g.set_smoothing(npre, npost)
        g.step(wl.dt, 20)
        cycles[(npre, npost)] = g.last_stats()["total_cycles_call"]
        phi_g, vel_g, _ = g.get_fields()
        assert rel(phi_g, phi_o) < 1e-11
        for a in range(2):
            assert rel(vel_g[a], vel_o[a]) < 1e-10
    assert cycles[(2, 2)] <= cycles[(1, 1)], cycles
    for bad in ((0, 1), (1, 5)):
        with pytest.raises(cdi.CdiError):
            g.set_smoothing(*bad)


def test_coarse_smoothing_counts_change_cycles_not_the_solution():
    """Sweeps on the coarser separately launched levels (cdi_set_coarse_smoothing,
    launch-per-kernel path): a 64x32x32 3D drop in FP64 (level 1, 8192 cells,
    runs as separate launches; the single-CTA tail takes the levels below it)
    matches the oracle within the FP64 bar after 5 steps with the finest
    level's counts, with V(1,1) and with V(0,1) on level 1; out-of-range counts
    are rejected and (-1, -1) restores the default."""
    n = (64, 32, 32)
    h = 1.0 / 32
    L = tuple(x * h for x in n)
    phi = inputs.add_noise(inputs.cap_phi_3d(*n, h, 0.3, math.pi / 2, 1.0, 0.5, h), 1e-3, 99)
    o = oracle.Oracle(3, n, L)
    o.set_fluids(1.0, 0.1, 0.05, 0.005, 1.0, h, 1.0)
    o.set_solver(1e-12, 100)
    o.set_wall_slip_length(2, math.radians(60), h, 0.0)
    o.set_state(phi)
    o.step(5e-5, 5)
    phi_o, vel_o, _ = o.get_state()
    for coarse in ((-1, -1), (1, 1), (0, 1)):
        g = cdi.Solver(3, n, L, precision=cdi.FP64)
        g.set_fluids(1.0, 0.1, 0.05, 0.005, 1.0, h, 1.0)
        g.set_solver(1e-12, 100)
        g.set_wall(cdi.WALL_BOTH, math.radians(60), h, 0.0)
        g.set_exec(cdi.EXEC_KERNELS)
        g.set_coarse_smoothing(*coarse)
        g.set_state(phi)
        g.step(5e-5, 5)
        assert g.last_stats()["resid"] <= 1e-12
        phi_g, vel_g, _ = g.get_fields()
        assert rel(phi_g, phi_o) < 1e-11, coarse
        for a in range(3):
            assert rel(vel_g[a], vel_o[a]) < 1e-10, (coarse, a)
    for bad in ((0, 0), (1, 5), (-1, 1)):
        with pytest.raises(cdi.CdiError):
            g.set_coarse_smoothing(*bad)
    g.set_coarse_smoothing(-1, -1)
