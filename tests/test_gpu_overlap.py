"""Interior/shell split with overlapped exchange (cavity_set_overlap): the
nodes within two layers of a cut face are stepped first, pack/unpack run on
a second stream while the rest is stepped.

 * fields and time bit-identical to the plain schedule for slabs, pencils,
   cubes and blocks only 2-3 nodes thick along a cut axis (the two faces'
   shells meet), residuals equal to rounding, Nusselt numbers identical;
 * with local time stepping as well;
 * against the FP64 oracle (1e-12);
 * FP32-mixed handles are refused; without cut faces nothing changes.
"""
import numpy as np
import pytest

import oracle

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


def run(m, n, blocks, steps, overlap, local=False, Ra=5e4):
    c = m.Cavity(*n, blocks=blocks, seed=6, noise_amp=1e-3, Ra=Ra)
    if local:
        m.cavity_set_time_stepping(c.h, m.CAVITY_DT_LOCAL)
    m.cavity_set_overlap(c.h, overlap)
    c.step(steps)
    return c


@pytest.mark.parametrize("blocks", [(2, 2, 2), (8, 1, 1), (4, 2, 1), (3, 2, 2), (12, 1, 1), (1, 1, 12)])
def test_overlap_bit_identical_to_plain(m, blocks):
    n = (40, 36, 32) if blocks != (1, 1, 12) else (30, 28, 30)
    if blocks == (12, 1, 1):
        n = (30, 28, 26)  # blocks 2-3 nodes thick in x
    with run(m, n, blocks, 30, False) as a, run(m, n, blocks, 30, True) as b:
        assert np.array_equal(a.fields(), b.fields())
        assert a.time == b.time
        assert a.nusselt == b.nusselt
        assert np.allclose(a.residual, b.residual, rtol=1e-12, atol=0.0)


def test_overlap_with_local_time_stepping(m):
    n = (34, 30, 28)
    with run(m, n, (2, 2, 2), 25, False, local=True) as a, run(m, n, (2, 2, 2), 25, True, local=True) as b:
        assert np.array_equal(a.fields(), b.fields())
        assert a.time == b.time


def test_overlap_matches_oracle(m):
    n = (26, 22, 20)
    o = oracle.OracleCavity(*n, dict(Ra=5e4), noise=1e-3, seed=6)
    o.step(25)
    with run(m, n, (2, 2, 2), 25, True) as c:
        g, ref = c.fields(), o.fields()
        for f in range(5):
            assert np.max(np.abs(g[f] - ref[f])) <= 1e-12 * np.max(np.abs(ref[f])), f
        assert c.nusselt[0] == pytest.approx(o.nusselt[0], rel=1e-12)


def test_overlap_toggle_and_refusals(m):
    n = (24, 20, 18)
    with run(m, n, (2, 1, 1), 10, True) as a, run(m, n, (2, 1, 1), 10, False) as b:
        m.cavity_set_overlap(a.h, False)
        a.step(10)
        b.step(10)
        assert np.array_equal(a.fields(), b.fields())
    with m.Cavity(*n, precision=m.CAVITY_FP32_MIXED, blocks=(2, 1, 1)) as c:
        with pytest.raises(m.CavityError):
            m.cavity_set_overlap(c.h, True)
    with run(m, n, (1, 1, 1), 5, True) as a, run(m, n, (1, 1, 1), 5, False) as b:
        assert np.array_equal(a.fields(), b.fields())
