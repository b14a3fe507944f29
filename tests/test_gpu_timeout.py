"""Failure detection of the FP32-mixed step: bounded device-side waits.

Each FP32 step kernel waits on a shared-memory barrier for every TMA plane
load, with an iteration limit.  cavity_test_wait_timeout shortens the limit
to a few thousand cycles and leaves one plane's load of every tile unissued
(a barrier that nothing completes), so every CTA's wait runs out: the kernel
records the timeout in the cavity's sticky flag, waits (bounded) for the
loads it did issue and returns.  No GPU fault and no hang: the context stays
usable, cavity_sync and the getters report CAVITY_ERR_TIMEOUT, and a fresh
handle afterwards still matches the oracle.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_02602_gb300 import build
    build.build()
    import paper_2006_02602_gb300 as mod
    mod.load_library()
    return mod


# the default shape (one plane in flight) and a tall tile with two in flight
@pytest.mark.parametrize("shape", ["8,32,4,3", "16,64,5,3"])
def test_wait_runs_out_and_reports_timeout(m, monkeypatch, shape):
    monkeypatch.setenv("BDC_F32_TILE", shape)
    n = (40, 20, 36)
    with m.Cavity(*n, precision=m.CAVITY_FP32_MIXED, seed=1, noise_amp=1e-3, Ra=1e4) as c:
        c.step(2)
        assert c.sync() == m.CAVITY_OK
        m.cavity_test_wait_timeout(c.h, 20000, 5)   # about 10 us per wait; plane 5 never loaded
        c.step(1)
        assert c.sync() == m.CAVITY_ERR_TIMEOUT
        with pytest.raises(m.CavityError) as e:
            c.residual
        assert e.value.code == m.CAVITY_ERR_TIMEOUT
    # the context is intact: a fresh handle steps and matches the oracle
    q = workloads.smooth_state(n, seed=2)
    o = oracle.OracleCavity(*n, dict(Ra=1e4))
    o.set_fields(q)
    o.step(20)
    with m.Cavity(*n, precision=m.CAVITY_FP32_MIXED, Ra=1e4) as c:
        c.set_fields(q)
        c.step(20)
        assert c.sync() == m.CAVITY_OK
        g, ref = c.fields(), o.fields()
        for f in range(5):
            e = np.max(np.abs(g[f] - ref[f])) / np.max(np.abs(ref[f]))
            assert e <= 1e-5, (shape, f, e)


def test_wait_hook_arguments(m):
    with m.Cavity(12, 10, 9, precision=m.CAVITY_FP32_MIXED, Ra=1e4) as c:
        for bad in ((999, -1), (4000000001, -1), (20000, -2)):
            with pytest.raises(m.CavityError) as e:
                m.cavity_test_wait_timeout(c.h, *bad)
            assert e.value.code == m.CAVITY_ERR_INVALID_ARG
        # the production limit with every load issued: steps as before
        m.cavity_test_wait_timeout(c.h, 4000000000, -1)
        c.step(3)
        assert c.sync() == m.CAVITY_OK
    with m.Cavity(12, 10, 9, Ra=1e4) as c:
        with pytest.raises(m.CavityError) as e:
            m.cavity_test_wait_timeout(c.h, 20000, 5)
        assert e.value.code == m.CAVITY_ERR_UNSUPPORTED
