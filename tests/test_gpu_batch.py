"""The batched persistent sweep (one launch for many uneven instances) on
the GPU: every instance ends where stepping it alone ends, and where the FP64
oracle ends."""
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
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def small_sweep(n=6, seed=7):
    wls = [w for w in inputs.sweep_2d(64, seed=seed) if w.n[0] <= 128][:n]
    assert len(wls) == n
    return wls


@pytest.mark.parametrize("precision", [cdi.FP64, cdi.FP32_MIXED], ids=["fp64", "fp32"])
def test_batch_equals_instances_stepped_alone(precision):
    wls = small_sweep()
    alone = [cdi.from_workload(w, precision=precision, tol=1e-10) for w in wls]
    batched = [cdi.from_workload(w, precision=precision, tol=1e-10) for w in wls]
    b = cdi.Batch(batched)
    dts = np.array([w.dt for w in wls])
    b.step(dts, 5)
    tol = 1e-11 if precision == cdi.FP64 else 1e-5
    for w, s_a, s_b in zip(wls, alone, batched):
        s_a.step(w.dt, 5)
        pa, va, _ = s_a.get_fields()
        pb, vb, _ = s_b.get_fields()
        assert rel(pb, pa) < tol, w.name
        for a in range(2):
            assert rel(vb[a], va[a]) < 100 * tol, (w.name, a)
    for i in range(len(wls)):
        st = b.stats(i)
        assert st["status"] == 0 and st["total_cycles"] > 0


def test_batch_matches_oracle_fp64():
    wls = small_sweep(3, seed=11)
    batched = [cdi.from_workload(w, precision=cdi.FP64, tol=1e-12) for w in wls]
    b = cdi.Batch(batched)
    b.step(np.array([w.dt for w in wls]), 10)
    for w, s in zip(wls, batched):
        o = oracle.from_workload(w, tol=1e-12)
        o.step(w.dt, 10)
        pg, vg, _ = s.get_fields()
        po, vo, _ = o.get_state()
        assert rel(pg, po) < 1e-11, w.name
        for a in range(2):
            assert rel(vg[a], vo[a]) < 1e-9, (w.name, a)


def test_batch_autotune_picks_a_candidate():
    """The autotuner times every (CTA size, tail budget) pair that launches and
    keeps the fastest; the tail budget changes the work split between shared
    memory and global memory but not the arithmetic: a batch stepped with
    each budget ends where its instances stepped alone end."""
    wls = small_sweep(4, seed=3)
    batched = [cdi.from_workload(w, precision=cdi.FP32_MIXED, tol=1e-8) for w in wls]
    b = cdi.Batch(batched)
    best, tail, ms = b.autotune(np.array([w.dt for w in wls]), 1)
    assert best in (256, 512, 1024)
    assert tail >= 32 * 1024
    assert (ms > 0).sum() >= 6
    assert ms.min(initial=1e30, where=ms > 0) == pytest.approx(ms[ms > 0].min())
    b.step(np.array([w.dt for w in wls]), 2)


@pytest.mark.parametrize("budget", [32 * 1024, 100 * 1024])
def test_batch_tail_budget_keeps_the_arithmetic(budget):
    wls = small_sweep(4, seed=5)
    alone = [cdi.from_workload(w, precision=cdi.FP64, tol=1e-12) for w in wls]
    batched = [cdi.from_workload(w, precision=cdi.FP64, tol=1e-12) for w in wls]
    b = cdi.Batch(batched)
    b.set_tail_budget(budget)
    b.step(np.array([w.dt for w in wls]), 4)
    for w, s_a, s_b in zip(wls, alone, batched):
        s_a.step(w.dt, 4)
        assert rel(s_b.get_fields()[0], s_a.get_fields()[0]) < 1e-11, w.name


def test_timed_sweep_fp32_instances_vs_oracle():
    """A few instances of the 512-instance sweep that the bench times (FP32-mixed,
    batched, autotuned launch), 20 steps, against the FP64 oracle: the
    smallest drop and Couette instances and the largest-density-ratio one
    within 1e-5 in phi and 1e-3 relative in velocity (the FP32-level bounds
    of the 2D FP32-mixed form)."""
    wls = inputs.sweep_2d()
    pick = sorted(range(len(wls)), key=lambda i: wls[i].cells)
    drops = [i for i in pick if "drop" in wls[i].name][:2]
    couettes = [i for i in pick if "couette" in wls[i].name][:2]
    small = [i for i in pick if wls[i].cells <= 4096]
    heavy = max(small, key=lambda i: wls[i].rho1 / wls[i].rho2)
    chosen = sorted(set(drops + couettes + [heavy]))
    solvers = []
    for w in wls:
        sv = cdi.from_workload(w, precision=cdi.FP32_MIXED, tol=1e-10)
        sv.set_solver(1e-10, 100, cdi.WARM_EXTRAP)
        sv.set_smoothing(2, 2)
        solvers.append(sv)
    b = cdi.Batch(solvers)
    dts = np.array([w.dt for w in wls])
    b.autotune(dts, 1)
    for sv, w in zip(solvers, wls):  # back to the initial state after the autotuner's trial steps
        sv.set_state(w.phi0)
    b.step(dts, 20)
    for i in chosen:
        w = wls[i]
        o = oracle.from_workload(w, tol=1e-10)
        o.step(w.dt, 20)
        pg, vg, _ = solvers[i].get_fields()
        po, vo, _ = o.get_state()
        assert np.abs(pg - po).max() < 1e-5, w.name
        for a in range(2):
            assert rel(vg[a], vo[a]) < 1e-3, (w.name, a)
