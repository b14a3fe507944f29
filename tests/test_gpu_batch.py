"""Batched form: many independent cavities of uneven sizes and Rayleigh
numbers advanced by the same launches (one descriptor table, one work list
per kernel, parallel per-cavity finalise), graph-captured, with an autotuner
over the FP32 step kernel's tile shapes.

 * every member against the FP64 oracle run alone (FP64 batch <= 1e-12,
   FP32-mixed batch <= 1e-5 relative max-norm, Nusselt <= 1e-4);
 * every member bit-identical to the same cavity in a handle of its own;
 * the autotuner restores the state and the tile shape does not change the
   fields (bit-identical to an untuned handle).
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


def relmax(a, b):
    s = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (s if s > 0 else 1.0)


SMALL = workloads.batch_cavities(ncav=6, nmin=12, nmax=33)
# degenerate members: two nodes across the x walls, two along y or z
TINY = [dict(n=(2, 9, 7), Ra=2e4, seed=21), dict(n=(5, 2, 3), Ra=5e3, seed=22), dict(n=(3, 4, 2), Ra=1e4, seed=23)]


def _params(m, cav):
    return m.cavity_default_params(Ra=cav["Ra"], Pr=0.71)


@pytest.mark.parametrize("prec,members", [("fp64", "small"), ("fp32", "small"), ("fp64", "tiny"), ("fp32", "tiny")])
def test_batch_members_match_oracle(m, prec, members):
    precision = m.CAVITY_FP64 if prec == "fp64" else m.CAVITY_FP32_MIXED
    cavs = SMALL if members == "small" else SMALL[:2] + TINY
    steps = 30
    h = m.cavity_create_batch([c["n"] for c in cavs], [_params(m, c) for c in cavs], precision=precision,
                              seeds=[c["seed"] for c in cavs], noise_amp=1e-3)
    try:
        assert m.cavity_batch_size(h) == len(cavs)
        m.cavity_step(h, steps)
        for b, cav in enumerate(cavs):
            o = oracle.OracleCavity(*cav["n"], dict(Ra=cav["Ra"], Pr=0.71), noise=1e-3, seed=cav["seed"])
            o.step(steps)
            g = m.cavity_batch_get_fields(h, b, cav["n"])
            ref = o.fields()
            tol = 1e-12 if prec == "fp64" else 1e-5
            speed = max(np.max(np.abs(ref[f])) for f in (1, 2, 3))
            for f in range(5):
                scale = speed if (prec == "fp32" and f == 2) else np.max(np.abs(ref[f]))
                e = np.max(np.abs(g[f] - ref[f])) / scale
                assert e <= tol, (b, cav, f, e)
            st = m.cavity_batch_state(h, b)
            assert st["step"] == steps
            assert st["t"] == pytest.approx(o.t, rel=1e-12 if prec == "fp64" else 1e-5)
            ntol = 1e-12 if prec == "fp64" else 1e-4
            assert abs(st["nusselt"][0] - o.nusselt[0]) <= ntol * abs(o.nusselt[0])
            assert abs(st["nusselt"][1] - o.nusselt[1]) <= ntol * abs(o.nusselt[1])
    finally:
        m.cavity_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_members_bit_identical_to_single_handles(m, prec):
    precision = m.CAVITY_FP64 if prec == "fp64" else m.CAVITY_FP32_MIXED
    steps = 25
    h = m.cavity_create_batch([c["n"] for c in SMALL], [_params(m, c) for c in SMALL], precision=precision,
                              seeds=[c["seed"] for c in SMALL], noise_amp=1e-3)
    try:
        m.cavity_step(h, steps)
        for b, cav in enumerate(SMALL):
            with m.Cavity(*cav["n"], precision=precision, seed=cav["seed"], noise_amp=1e-3, Ra=cav["Ra"],
                          Pr=0.71) as c:
                c.step(steps)
                assert np.array_equal(m.cavity_batch_get_fields(h, b, cav["n"]), c.fields()), b
                st = m.cavity_batch_state(h, b)
                assert (st["step"], st["t"], st["dt"]) == c.time
    finally:
        m.cavity_destroy(h)


def test_autotune_restores_state_and_keeps_fields(m):
    cavs = workloads.batch_cavities(ncav=8, nmin=24, nmax=64)
    sizes = [c["n"] for c in cavs]
    params = [_params(m, c) for c in cavs]
    seeds = [c["seed"] for c in cavs]
    h = m.cavity_create_batch(sizes, params, seeds=seeds, noise_amp=1e-3)
    ref = m.cavity_create_batch(sizes, params, seeds=seeds, noise_amp=1e-3)
    try:
        m.cavity_step(h, 3)
        m.cavity_step(ref, 3)
        before = [m.cavity_batch_get_fields(h, b, s) for b, s in enumerate(sizes)]
        choice = m.cavity_autotune(h, 5)
        assert choice["tile_y"] in (8, 16) and choice["kc"] in (16, 24, 32, 40, 48, 64, 96)
        assert choice["us_per_step"] > 0
        assert choice["kernel_form"] == 3
        for b, s in enumerate(sizes):
            assert np.array_equal(m.cavity_batch_get_fields(h, b, s), before[b])
            assert m.cavity_batch_state(h, b)["step"] == 3
        m.cavity_step(h, 20)
        m.cavity_step(ref, 20)
        for b, s in enumerate(sizes):
            assert np.array_equal(m.cavity_batch_get_fields(h, b, s), m.cavity_batch_get_fields(ref, b, s)), b
    finally:
        m.cavity_destroy(h)
        m.cavity_destroy(ref)


def test_fp32_tile_shapes_give_identical_fields(m, monkeypatch):
    """The tile shape (tile height, z chunk, ring depth) changes only the order
    of the residual sums, never a field; odd nx leaves a lone node in the last
    pair, and the z chunks put chunk edges next to both z walls."""
    n = (45, 38, 70)
    out = []
    for shape in ("8,16,4,3", "8,24,4,3", "8,32,4,3", "8,40,4,3", "8,64,4,3", "8,96,4,3", "8,32,5,3", "8,64,5,3",
                  "8,96,5,3", "16,32,4,3", "16,64,4,3", "16,32,5,3", "16,64,5,3"):
        monkeypatch.setenv("BDC_F32_TILE", shape)
        with m.Cavity(*n, precision=m.CAVITY_FP32_MIXED, seed=4, noise_amp=1e-3, Ra=2e5) as c:
            c.step(40)
            out.append((c.fields(), c.time))
    for f, t in out[1:]:
        assert np.array_equal(f, out[0][0])
        assert t == out[0][1]


def test_fp64_batch_with_more_tiles_than_resident_ctas(m):
    """The persistent FP64 step takes many tiles per CTA, from several cavities
    whose spectral bounds differ by orders of magnitude (Ra 1e3 .. 1e6): every
    member of the batch stays bit-equal to the same cavity stepped alone
    (fields and dt), so no state of the dt maximum leaks between cavities."""
    cavs = [dict(n=(64, 48, 56), Ra=1e6, seed=1), dict(n=(40, 64, 64), Ra=1e3, seed=2),
            dict(n=(64, 64, 40), Ra=3e4, seed=3), dict(n=(48, 40, 64), Ra=1e5, seed=4)]
    params = [m.cavity_default_params(Ra=c["Ra"], Pr=0.71) for c in cavs]
    h = m.cavity_create_batch([c["n"] for c in cavs], params, precision=m.CAVITY_FP64,
                              seeds=[c["seed"] for c in cavs], noise_amp=1e-3)
    try:
        m.cavity_step(h, 25)
        for b, c in enumerate(cavs):
            with m.Cavity(*c["n"], seed=c["seed"], noise_amp=1e-3, Ra=c["Ra"], Pr=0.71) as single:
                single.step(25)
                assert np.array_equal(m.cavity_batch_get_fields(h, b, c["n"]), single.fields()), b
                st = m.cavity_batch_state(h, b)
                assert (st["step"], st["t"], st["dt"]) == single.time, b
    finally:
        m.cavity_destroy(h)


def test_batch_rejects_mixed_precision_and_split_members(m):
    import ctypes
    L = m.load_library()
    d = (m.cavity_desc * 2)(m.cavity_desc(8, 8, 8, 1, 1, 1, 0, 0, 0.0, 0, None),
                            m.cavity_desc(8, 8, 8, 1, 1, 1, 1, 0, 0.0, 0, None))
    h = ctypes.c_void_p()
    assert L.cavity_create_batch(d, None, 2, ctypes.byref(h)) == m.CAVITY_ERR_INVALID_ARG
    d = (m.cavity_desc * 2)(m.cavity_desc(8, 8, 8, 2, 1, 1, 0, 0, 0.0, 0, None),
                            m.cavity_desc(8, 8, 8, 1, 1, 1, 0, 0, 0.0, 0, None))
    assert L.cavity_create_batch(d, None, 2, ctypes.byref(h)) == m.CAVITY_ERR_INVALID_ARG


def test_config4_batch_as_benchmarked(m):
    """Configuration 4 exactly as the benchmark runs it: all 64 cavities (n_d
    in 24..96, Ra log-uniform in [1e3, 1e6], seeds 0..63), FP32-mixed, the
    autotuner's tile shape, 1000 graph-replayed steps.  The largest, the
    smallest, the highest-Ra and the lowest-Ra members (the last two deeper
    than 64 planes: chunked z sweeps with tail tiles) against FP64 oracle runs
    of the same cavity: every field within 1e-5 of its own max-norm, both
    Nusselt numbers within 1e-4, time within 1e-5."""
    cfg = workloads.CFG4
    cavs = workloads.batch_cavities()
    sizes = [c["n"] for c in cavs]
    params = [m.cavity_default_params(Ra=c["Ra"], Pr=cfg["Pr"]) for c in cavs]
    h = m.cavity_create_batch(sizes, params, precision=m.CAVITY_FP32_MIXED, seeds=[c["seed"] for c in cavs],
                              noise_amp=cfg["noise"])
    try:
        tuned = m.cavity_autotune(h, 10)
        assert tuned["kernel_form"] == 3
        m.cavity_step(h, cfg["steps"])
        vol = [a * b * c for a, b, c in sizes]
        ra = [c["Ra"] for c in cavs]
        picks = sorted({int(np.argmax(vol)), int(np.argmin(vol)), int(np.argmax(ra)), int(np.argmin(ra))})
        assert len(picks) == 4 and sum(sizes[b][2] > 64 for b in picks) >= 2
        for b in picks:
            cav = cavs[b]
            o = oracle.OracleCavity(*cav["n"], dict(Ra=cav["Ra"], Pr=cfg["Pr"]), noise=cfg["noise"], seed=cav["seed"])
            o.step(cfg["steps"])
            g, ref = m.cavity_batch_get_fields(h, b, cav["n"]), o.fields()
            for f in range(5):
                e = relmax(g[f], ref[f])
                assert e <= 1e-5, (b, cav, oracle.FIELDS[f], e, tuned)
            st = m.cavity_batch_state(h, b)
            assert st["step"] == cfg["steps"]
            assert st["t"] == pytest.approx(o.t, rel=1e-5)
            assert abs(st["nusselt"][0] - o.nusselt[0]) <= 1e-4 * abs(o.nusselt[0]), b
            assert abs(st["nusselt"][1] - o.nusselt[1]) <= 1e-4 * abs(o.nusselt[1]), b
    finally:
        m.cavity_destroy(h)
