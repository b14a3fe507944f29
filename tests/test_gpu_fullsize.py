"""Full-size GPU checks: the 128^3 configuration as the bench runs it, and the
largest mesh of the paper (1024^3) on sampled windows.

 * 128^3, Ra 1e5, 2000 steps, FP64, 2x2x2 blocks (the bench launch
   configuration) against the FP64 oracle element by element;
 * 1x1x1, 8x1x1, 4x2x1 and 2x2x2 decompositions bit-identical after 2000 steps;
 * 1024^3 (Section 2: meshes up to 1024^3): one step from the initial state,
   compared on sampled windows that the oracle computes on its own from the
   same seeded initial condition (the state at rest has a uniform dt bound and
   keeps p = 0, so each window's new values follow from the window alone).
"""
import ctypes

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


@pytest.fixture(scope="module")
def cfg2_oracle():
    cfg = workloads.CFG2
    o = oracle.OracleCavity(*cfg["n"], dict(Ra=cfg["Ra"], Pr=cfg["Pr"]), noise=cfg["noise"], seed=cfg["seed"])
    o.step(cfg["steps"])
    return o


def _cfg2(m, blocks):
    cfg = workloads.CFG2
    c = m.Cavity(*cfg["n"], blocks=blocks, seed=cfg["seed"], noise_amp=cfg["noise"], Ra=cfg["Ra"], Pr=cfg["Pr"])
    c.step(cfg["steps"])
    return c


def test_cfg2_fp64_2x2x2_vs_oracle(m, cfg2_oracle):
    o = cfg2_oracle
    with _cfg2(m, (2, 2, 2)) as c:
        g = c.fields()
        ref = o.fields()
        for f, name in enumerate(oracle.FIELDS):
            e = relmax(g[f], ref[f])
            assert e <= 1e-12, (name, e)
        assert np.allclose(c.residual, o.residual, rtol=1e-10, atol=0)
        h, cold = c.nusselt
        assert abs(h - o.nusselt[0]) <= 1e-12 * abs(o.nusselt[0])
        assert abs(cold - o.nusselt[1]) <= 1e-12 * abs(o.nusselt[1])
        s, t, dt = c.time
        assert s == 2000 and t == pytest.approx(o.t, rel=1e-12)


def test_cfg2_fp32_mixed_2x2x2_vs_fp64_oracle(m, cfg2_oracle):
    """Configuration 2 in the FP32-mixed form: every field within 1e-5
    relative max-norm and Nusselt within 1e-4 of the FP64 oracle."""
    cfg = workloads.CFG2
    o = cfg2_oracle
    with m.Cavity(*cfg["n"], blocks=(2, 2, 2), precision=m.CAVITY_FP32_MIXED, seed=cfg["seed"],
                  noise_amp=cfg["noise"], Ra=cfg["Ra"], Pr=cfg["Pr"]) as c:
        c.step(cfg["steps"])
        g = c.fields()
        ref = o.fields()
        for f, name in enumerate(oracle.FIELDS):
            e = relmax(g[f], ref[f])
            assert e <= 1e-5, (name, e)
        h, cold = c.nusselt
        assert abs(h - o.nusselt[0]) <= 1e-4 * abs(o.nusselt[0])
        assert abs(cold - o.nusselt[1]) <= 1e-4 * abs(o.nusselt[1])


def test_cfg2_fp32_decompositions_bit_identical(m):
    cfg = workloads.CFG2
    kw = dict(precision=m.CAVITY_FP32_MIXED, seed=cfg["seed"], noise_amp=cfg["noise"], Ra=cfg["Ra"], Pr=cfg["Pr"])
    with m.Cavity(*cfg["n"], **kw) as ref:
        ref.step(cfg["steps"])
        f0 = ref.fields()
        for blocks in cfg["decomps"]:
            with m.Cavity(*cfg["n"], blocks=blocks, **kw) as c:
                c.step(cfg["steps"])
                assert np.array_equal(c.fields(), f0), blocks


def test_cfg2_decompositions_bit_identical(m):
    with _cfg2(m, (1, 1, 1)) as ref:
        f0 = ref.fields()
        t0 = ref.time
        for blocks in workloads.CFG2["decomps"]:
            with _cfg2(m, blocks) as c:
                assert np.array_equal(c.fields(), f0), blocks
                assert c.time == t0, blocks


def _oracle_window(lo, w, gn, params, seed, noise):
    """One step of the at-rest initial state on the window lo .. lo+w-1, from
    an oracle block that covers the window plus two halo layers."""
    L = oracle.lib()
    cp = oracle._cparams(params)
    nb = w + 4
    blk = oracle._Block(nb, nb, nb, lo[0] - 3, lo[1] - 3, lo[2] - 3, *gn, (ctypes.c_int * 6)(0, 0, 0, 0, 0, 0))
    q = np.zeros((5, nb + 4, nb + 4, nb + 4))
    L.orc_init(ctypes.byref(cp), ctypes.byref(blk), oracle._ptr(q), ctypes.c_uint64(seed), noise)
    dq = np.zeros((5, nb, nb, nb))
    L.orc_rates(ctypes.byref(cp), ctypes.byref(blk), oracle._ptr(q), oracle._ptr(dq))
    dt = params["cfl"] / L.orc_spectral_max(ctypes.byref(cp), ctypes.byref(blk), oracle._ptr(q))
    inner = (slice(None), slice(2, 2 + w), slice(2, 2 + w), slice(2, 2 + w))
    qi = q[:, 2:nb + 2, 2:nb + 2, 2:nb + 2][inner]
    return qi + dt * dq[inner], dt


def test_max_size_1024_sampled_windows(m):
    gn = (1024, 1024, 1024)
    params = oracle.default_params(Ra=1e5, Pr=0.71)
    seed, noise = 0, 1e-3
    w = 6
    windows = [(3, 3, 3), (100, 517, 900), (509, 509, 509), (1016, 40, 777), (250, 1016, 1016)]
    with m.Cavity(*gn, seed=seed, noise_amp=noise, Ra=1e5, Pr=0.71) as c:
        c.step(1)
        _, _, _ = c.time
        for lo in windows:
            got = m.cavity_get_fields_box(c.h, lo, (w, w, w))
            # windows touching a wall take the wall values of the GPU's walls:
            # compare them only where the oracle window is wall-free
            exp, dt = _oracle_window(lo, w, gn, params, seed, noise)
            if min(lo) <= 2 or max(lo) + w + 1 >= 1024:
                continue
            for f in range(5):
                e = np.max(np.abs(got[f] - exp[f])) / max(np.max(np.abs(exp[f])), 1e-300)
                assert e <= 1e-12 or np.max(np.abs(exp[f])) == 0.0 and np.max(np.abs(got[f])) == 0.0, (lo, f, e)
        assert c.residual[4] > 0
