"""The seeded synthetic inputs (paper_2412_16843_gb300/inputs.py) have the
shapes, parameters and structure their recipes state: the workloads both the
oracle and the CUDA path consume, the parameter sweep and the network's
initial parameters."""
import math

import numpy as np
import pytest

from paper_2412_16843_gb300 import inputs


def test_couette_512x128_recipe():
    wl = inputs.couette_2d(512, 128, 1.0)
    assert wl.phi0.shape == (128, 512) and wl.dim == 2
    assert wl.L == (4.0, 1.0) and wl.h == pytest.approx(1 / 128)
    assert (wl.U_lo, wl.U_hi) == (-0.1, 0.1)
    assert wl.sigma == pytest.approx(0.1 * 0.1 / 0.05)            # Ca = mu U / sigma = 0.05
    assert wl.gamma == pytest.approx(0.25) and wl.dt == 1.25e-4
    assert wl.theta_eq == pytest.approx(math.pi / 2) and wl.slip_length == pytest.approx(wl.h)
    x = (np.arange(512) + 0.5) * wl.h
    row = wl.phi0[64]
    # fluid 1 between the interfaces at x = 1 and x = 3, y-invariant
    assert row[np.argmin(abs(x - 2.0))] > 0.99 and row[0] < 0.01 and row[-1] < 0.01
    # the two cells straddling each interface sit h/2 from it: phi = (1 -/+ tanh(1/4)) / 2
    for lo, inside_right in ((127, True), (383, False)):
        a, b = row[lo], row[lo + 1]
        assert a + b == pytest.approx(1.0, abs=1e-12)
        assert (b - a if inside_right else a - b) == pytest.approx(math.tanh(0.25), abs=1e-12)
    assert np.array_equal(wl.phi0[0], wl.phi0[-1])


def test_drop_3d_noise_is_seeded_bounded_and_clamped():
    a = inputs.drop_3d(32)
    b = inputs.drop_3d(32)
    c = inputs.drop_3d(32, seed=7)
    clean = inputs.drop_3d(32, noise=0.0)
    assert a.phi0.shape == (32, 32, 32)
    assert np.array_equal(a.phi0, b.phi0) and not np.array_equal(a.phi0, c.phi0)
    assert a.phi0.min() >= 0.0 and a.phi0.max() <= 1.0
    assert np.abs(a.phi0 - clean.phi0).max() <= 1e-3 + 1e-15
    assert (a.rho1, a.rho2, a.mu1, a.mu2) == (1.0, 0.1, 0.05, 0.005)   # ratios 10 and 10


def test_drop_3d_wide_recipe():
    wl = inputs.drop_3d_wide(64)
    assert wl.n == (64, 32, 32) and wl.phi0.shape == (32, 32, 64)
    assert wl.L == (2.0, 1.0, 1.0) and wl.h == pytest.approx(2.0 / 64)
    assert wl.rho1 / wl.rho2 == pytest.approx(20.0) and wl.mu1 / wl.mu2 == pytest.approx(10.0)
    assert wl.theta_eq == pytest.approx(math.radians(45.0)) and wl.dt == 3.0e-5
    # the cap sits on the low wall at (1, 0.5): phi ~ 1 there, ~ 0 at the far corner
    assert wl.phi0[0, 16, 32] > 0.9 and wl.phi0[-1, 0, 0] < 0.1


def test_stable_dt_is_inside_every_explicit_limit():
    for wl in (inputs.drop_2d(), inputs.couette_2d(128, 32, 1.0), inputs.drop_3d(32)):
        dt = inputs.stable_dt(wl)
        h = wl.h
        visc = (0.35 if wl.dim == 2 else 0.23) * h * h * min(wl.rho1, wl.rho2) / max(wl.mu1, wl.mu2)
        cap = math.sqrt((wl.rho1 + wl.rho2) * h ** 3 / (4 * math.pi * wl.sigma))
        assert 0 < dt <= 0.4 * min(visc, cap) * (1 + 1e-12)


def test_sweep_is_seeded_and_within_its_ranges():
    a = inputs.sweep_2d(24)
    b = inputs.sweep_2d(24)
    assert [w.name for w in a] == [w.name for w in b]
    for i, w in enumerate(a):
        nx, ny = w.n
        assert nx in inputs.SWEEP_SIZES and ny == nx // 2 and w.h == pytest.approx(1 / 64)
        assert math.radians(30) <= w.theta_eq <= math.radians(150)
        assert 0.5 * w.h <= w.slip_length <= 4 * w.h
        assert 1.0 <= w.rho1 / w.rho2 <= 20.0
        assert ("drop" in w.name) == (i % 2 == 0)
        if i % 2:
            ca = w.mu1 * 0.1 / w.sigma
            assert 0.01 <= ca <= 0.1 + 1e-12 and (w.U_lo, w.U_hi) == (-0.1, 0.1)
        assert w.dt == pytest.approx(inputs.stable_dt(w))


def test_network_initial_parameters():
    v = inputs.unet_initial_params(0)
    assert v.size == 726993
    assert np.array_equal(v, inputs.unet_initial_params(0))
    o = 0
    for _, ci, co, t in inputs.UNET_LAYERS:
        w = v[o:o + t * co * ci]
        o += t * co * ci
        bias = v[o:o + co]
        o += co
        assert np.all(bias == 0.0)
        if w.size > 1000:  # He-normal: std sqrt(2 / (taps Cin)) within sampling error
            assert w.std() == pytest.approx(math.sqrt(2.0 / (t * ci)), rel=0.1)
    assert o == v.size


def test_network_pair_normalisation():
    rng = np.random.default_rng(3)
    f = rng.standard_normal((4, 5, 6))
    p = rng.standard_normal((4, 5, 6))
    phi = rng.uniform(0, 1, (4, 5, 6))
    x, t = inputs.unet_pair(f, p, phi, 1.0, 0.1, 0.5)
    assert x.shape == (4, 5, 6, 2)
    assert np.sqrt(np.mean(x[..., 0] ** 2)) == pytest.approx(1.0)
    assert x[..., 1].max() <= 1.0 and x[..., 1].min() >= 0.1 - 1e-15
    rms = np.sqrt(np.mean(f * f))
    assert np.allclose(t, p / (rms * 1.0 * 0.25))
