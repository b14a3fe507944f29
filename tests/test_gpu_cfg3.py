"""Configuration 3 at full size: the 256^3 cavity at Ra 1e6 (noise 1e-4,
seed 0) advanced 5000 steps in the FP32-mixed form, against the FP64 oracle
run of the same configuration.  The oracle's state is too large to store,
so tests/golden/cfg3_oracle_samples.npz (written by make_cfg3_reference.py,
which calls only the oracle) keeps the fields on a lattice of nodes that
includes the three layers next to every wall; the comparison is element by
element on that lattice.  Tolerances: each field within 1e-5 of the
sampled field's max-norm, Nusselt numbers within 1e-4, residual norms 1e-3.
"""
import os

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cfg3_oracle_samples.npz")


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


def test_cfg3_fp32_mixed_256_5000_steps(m):
    ref = np.load(GOLDEN)
    cfg = workloads.CFG3
    assert tuple(ref["n"]) == cfg["n"] and int(ref["steps"]) == cfg["steps"]
    assert float(ref["Ra"]) == cfg["Ra"] and float(ref["noise"]) == cfg["noise"] and int(ref["seed"]) == cfg["seed"]
    with m.Cavity(*cfg["n"], precision=m.CAVITY_FP32_MIXED, seed=cfg["seed"], noise_amp=cfg["noise"], Ra=cfg["Ra"],
                  Pr=cfg["Pr"]) as c:
        # the launch configuration the bench times: the autotuner's shape
        # (it restores the state it times on)
        choice = m.cavity_autotune(c.h, 5)
        assert c.time[0] == 0
        c.step(cfg["steps"])
        f = c.fields()
        ix, iy, iz = ref["ix"], ref["iy"], ref["iz"]
        got = f[:, iz - 1][:, :, iy - 1][:, :, :, ix - 1]
        exp = ref["samples"]
        for q, name in enumerate(("p", "u", "v", "w", "T")):
            e = np.max(np.abs(got[q] - exp[q])) / np.max(np.abs(exp[q]))
            assert e <= 1e-5, (name, e)
        hot, cold = c.nusselt
        assert abs(hot - ref["nusselt"][0]) <= 1e-4 * abs(ref["nusselt"][0])
        assert abs(cold - ref["nusselt"][1]) <= 1e-4 * abs(ref["nusselt"][1])
        assert np.allclose(c.residual, ref["residual"], rtol=1e-3)
        s, t, dt = c.time
        assert s == cfg["steps"] and t == pytest.approx(float(ref["t"]), rel=1e-5), choice
