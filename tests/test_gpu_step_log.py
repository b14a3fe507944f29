"""Step log (cavity_set_step_log): the device writes each step's record to
page-locked host memory in the launch that finishes the step.  The records
equal what the synchronising getters return after that step, in both forms,
for a decomposed cavity and for a batch; a ring of fewer records keeps the
latest ones; memory that is not page-locked is refused."""
import ctypes

import numpy as np
import pytest

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


def check_record(r, step, t, dt, res, nu):
    assert r["step"] == step
    assert r["t"] == t and r["dt"] == dt
    assert np.array_equal(r["res"], res)
    assert (r["nu_hot"], r["nu_cold"]) == nu
    assert r["flags"] == 0


@pytest.mark.parametrize("prec,blocks", [("fp64", (2, 2, 2)), ("fp32", (2, 2, 2)), ("fp32", (1, 1, 1))])
def test_records_equal_getters_and_ring_keeps_latest(m, prec, blocks):
    precision = m.CAVITY_FP64 if prec == "fp64" else m.CAVITY_FP32_MIXED
    cap = 7
    log = m.StepLog(cap)
    with m.Cavity(36, 30, 26, blocks=blocks, precision=precision, seed=4, noise_amp=1e-3, Ra=5e4) as c:
        m.cavity_set_step_log(c.h, log)
        for s in range(1, 11):  # one step at a time: the record against the getters
            c.step(1)
            step, t, dt = c.time
            check_record(log.array[(s - 1) % cap], s, t, dt, c.residual, c.nusselt)
        c.step(20)  # graph-replayed pairs, one synchronisation at the end
        step, t, dt = c.time
        assert step == 30
        check_record(log.array[(30 - 1) % cap], 30, t, dt, c.residual, c.nusselt)
        got = sorted(int(x) for x in log.array["step"])
        assert got == list(range(24, 31))  # the ring holds the latest `cap` steps
        ts = log.array["t"][np.argsort(log.array["step"])]
        assert np.all(np.diff(ts) > 0)
        m.cavity_set_step_log(c.h, None)
        before = log.array.copy()
        c.step(3)
        c.sync()
        assert np.array_equal(log.array, before)  # detached: nothing written
    log.close()


def test_batch_records(m):
    cavs = workloads.batch_cavities(ncav=3, nmin=12, nmax=25)
    h = m.cavity_create_batch([c["n"] for c in cavs], [m.cavity_default_params(Ra=c["Ra"], Pr=0.71) for c in cavs],
                              precision=m.CAVITY_FP32_MIXED, seeds=[c["seed"] for c in cavs], noise_amp=1e-3)
    cap = 4
    log = m.StepLog(cap * len(cavs))
    try:
        m.cavity_set_step_log(h, log, cap)
        m.cavity_step(h, 9)
        m.cavity_sync(h)
        for b in range(len(cavs)):
            st = m.cavity_batch_state(h, b)
            r = log.array[((9 - 1) % cap) * len(cavs) + b]
            check_record(r, 9, st["t"], st["dt"], st["residual"], st["nusselt"])
    finally:
        m.cavity_destroy(h)
        log.close()


def test_refuses_pageable_memory_and_bad_capacity(m):
    log = m.StepLog(2)
    with m.Cavity(12, 10, 8, seed=1, noise_amp=1e-3, Ra=1e4) as c:
        pageable = np.zeros(2 * m.STEP_RECORD.itemsize, dtype=np.uint8)
        L = m.load_library()
        assert L.cavity_set_step_log(c.h, ctypes.c_void_p(pageable.ctypes.data), 2) == m.CAVITY_ERR_INVALID_ARG
        assert L.cavity_set_step_log(c.h, ctypes.c_void_p(log.ptr), 0) == m.CAVITY_ERR_INVALID_ARG
        c.step(2)  # the handle still works, with no log
        assert c.time[0] == 2
    log.close()
