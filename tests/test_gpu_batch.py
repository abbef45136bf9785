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
    wls = small_sweep(4, seed=3)
    batched = [cdi.from_workload(w, precision=cdi.FP32_MIXED, tol=1e-8) for w in wls]
    b = cdi.Batch(batched)
    best, ms = b.autotune(np.array([w.dt for w in wls]), 1)
    assert best in (256, 512, 1024)
    assert np.all(ms[ms > 0] > 0)
    b.step(np.array([w.dt for w in wls]), 2)
