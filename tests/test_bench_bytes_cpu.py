"""The algorithmic byte counts behind bench.py's roofline fractions, checked
against values worked out by hand from the per-cell formula of the measurement
contract (V-cycle: four smoothing sweeps of 4 words, residual 4, restriction
1 + 2^-D, prolongation and correction 2 + 2^-D on the finest level, the
hierarchy weighing 1/(1 - 2^-D) of it)."""
import pytest

import bench


def test_vcycle_words():
    assert bench.vcycle_words(2) == pytest.approx(94 / 3)     # 23.5 / 0.75
    assert bench.vcycle_words(3) == pytest.approx(186 / 7)    # 23.25 / 0.875


def test_step_bytes_2d_fp64_three_vcycles_a_solve():
    # 4 * 5 * 3 + 4 * (3 + 5 + 3 * 94/3) = 60 + 408 = 468 words of 8 bytes
    assert bench.step_bytes(2, 1, 8, 12) == pytest.approx(3744.0)


def test_step_bytes_3d_fp32_three_vcycles_a_solve():
    # 4 * 5 * 4 + 4 * (4 + 7 + 3 * 186/7) = 124 + 2232/7 words of 4 bytes
    assert bench.step_bytes(3, 1, 4, 12) == pytest.approx(4 * (124 + 2232 / 7))


def test_step_bytes_scale_with_cells_and_vcycles():
    a = bench.step_bytes(3, 1000, 4, 20)
    b = bench.step_bytes(3, 1000, 4, 24)
    assert bench.step_bytes(3, 2000, 4, 20) == pytest.approx(2 * a)
    # four more V-cycles a step: one more in each of the four solves
    assert b - a == pytest.approx(1000 * 4 * 4 * bench.vcycle_words(3))


def test_level0_sweep_bytes():
    # 2D, one colour pass: rho N, the other colour's e N/2, own r N/2, own e written N/2, FP32
    assert bench.algorithmic_bytes("rbgs0", 2, 1000, 100, 8) == pytest.approx(2.5 * 1000 * 4)
    # 3D one-pass sweeps of a V(1,2) cycle: from zero 3 words, plain 4, the last (p updated, e not
    # written) 7
    assert bench.algorithmic_bytes("rbgs0", 3, 1000, 100, 8, 3) == pytest.approx(14 / 3 * 1000 * 4)
    assert bench.onepass_sweep_words(4) == pytest.approx((3 + 4 + 4 + 7) / 4)


def test_vcycle_words_with_the_cycles_own_sweeps():
    # V(1,2): 3 sweeps of 4 words, residual 4, restriction 1 + 1/8, prolongation 2 + 1/8 in 3D
    assert bench.vcycle_words(3, 3) == pytest.approx((12 + 4 + 1.125 + 2.125) / 0.875)
    # one fewer sweep removes 4 words on the finest level, 4 / (1 - 2^-D) over the hierarchy
    assert bench.vcycle_words(3, 4) - bench.vcycle_words(3, 3) == pytest.approx(4 / 0.875)
    assert bench.step_bytes(3, 10, 4, 20, 3) < bench.step_bytes(3, 10, 4, 20, 4)
