"""Local time stepping (cavity_set_time_stepping(CAVITY_DT_LOCAL)): each node
advances by its own stable step dt_n = cfl / S_n (pseudo time), against the
oracle's local mode.

 * FP64: fields within 1e-12 of the oracle (ragged size, 60 steps), time and
   residuals as the oracle's; 2x2x2 and 3x2x2 blocks bit-equal to one block;
   switching back to global steps mid-run matches the oracle doing the same;
 * FP32-mixed: within the form's 1e-5 of the FP64 oracle; two tile shapes
   (8 and 16 rows) give identical fields.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


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


def local_pair(m, n, Ra, steps, precision=None, blocks=(1, 1, 1), seed=3, noise=1e-3):
    o = oracle.OracleCavity(*n, dict(Ra=Ra), noise=noise, seed=seed, local_dt=True)
    o.step(steps)
    c = m.Cavity(*n, blocks=blocks, precision=m.CAVITY_FP64 if precision is None else precision, seed=seed,
                 noise_amp=noise, Ra=Ra)
    m.cavity_set_time_stepping(c.h, m.CAVITY_DT_LOCAL)
    c.step(steps)
    return o, c


def test_fp64_local_matches_oracle(m):
    n = (27, 22, 19)
    o, c = local_pair(m, n, 3e4, 60)
    with c:
        g, ref = c.fields(), o.fields()
        for f in range(5):
            e = np.max(np.abs(g[f] - ref[f])) / np.max(np.abs(ref[f]))
            assert e <= 1e-12, (f, e)
        assert np.allclose(c.residual, o.residual, rtol=1e-10)
        steps, t, dt = c.time
        assert steps == 60 and t == pytest.approx(o.t, rel=1e-12)
        for got, want in zip(c.nusselt, o.nusselt):
            assert got == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("blocks", [(2, 2, 2), (3, 2, 2)])
def test_fp64_local_blocks_bit_identical(m, blocks):
    kw = dict(seed=5, noise_amp=1e-3, Ra=5e4)
    with m.Cavity(30, 26, 22, **kw) as ref, m.Cavity(30, 26, 22, blocks=blocks, **kw) as c:
        for h in (ref.h, c.h):
            m.cavity_set_time_stepping(h, m.CAVITY_DT_LOCAL)
        ref.step(40)
        c.step(40)
        assert np.array_equal(c.fields(), ref.fields())
        assert c.time == ref.time


def test_switch_back_to_global(m):
    n = (20, 18, 16)
    o = oracle.OracleCavity(*n, dict(Ra=2e4), noise=1e-3, seed=7, local_dt=True)
    with m.Cavity(*n, seed=7, noise_amp=1e-3, Ra=2e4) as c:
        m.cavity_set_time_stepping(c.h, m.CAVITY_DT_LOCAL)
        c.step(15)
        o.step(15)
        m.cavity_set_time_stepping(c.h, m.CAVITY_DT_GLOBAL)
        o.local_dt = False
        c.step(15)
        o.step(15)
        g, ref = c.fields(), o.fields()
        for f in range(5):
            assert np.max(np.abs(g[f] - ref[f])) <= 1e-12 * np.max(np.abs(ref[f])), f
        with pytest.raises(m.CavityError):
            m.cavity_set_time_stepping(c.h, 2)


def test_fp32_local_matches_oracle_and_shapes_agree(m, monkeypatch):
    n = (37, 21, 18)
    out = []
    for shape in ("8,64,5,3", "16,32,4,3"):
        monkeypatch.setenv("BDC_F32_TILE", shape)
        o, c = local_pair(m, n, 3e4, 40, precision=m.CAVITY_FP32_MIXED)
        with c:
            g, ref = c.fields(), o.fields()
            speed = max(np.max(np.abs(ref[f])) for f in (1, 2, 3))
            for f in range(5):
                scale = speed if f == 2 else np.max(np.abs(ref[f]))
                e = np.max(np.abs(g[f] - ref[f])) / scale
                assert e <= FP32_TOL, (shape, f, e)
            for got, want in zip(c.nusselt, o.nusselt):
                assert abs(got - want) <= 1e-4 * abs(want), (shape, c.nusselt, o.nusselt)
            out.append(g)
    assert np.array_equal(out[0], out[1])
