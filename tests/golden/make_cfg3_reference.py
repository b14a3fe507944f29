"""Write tests/golden/cfg3_oracle_samples.npz from the FP64 oracle.

Configuration: 256^3 cavity, Ra 1e6, Pr 0.71, initial T linear in x plus
U(-1e-4, 1e-4) noise (seed 0), 5000 explicit steps (the scheme of Section 2,
Eqs. 1-3).  The oracle's whole state is ~0.7 GB, too large to store, so the
file keeps the five fields on a lattice of sampled nodes (the three nodes
next to every wall and every 24th node in between), the five RMS residuals
of the last step, both Nusselt numbers, t and dt.  Calls nothing but
oracle/ and the input constants of workloads.py.

    OMP_NUM_THREADS=8 python tests/golden/make_cfg3_reference.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

OUT = os.path.join(HERE, "cfg3_oracle_samples.npz")


def sample_index(n: int) -> np.ndarray:
    """1-based node indices: 1, 2, 3, every 24th node, n-2, n-1, n."""
    idx = sorted(set([1, 2, 3] + list(range(12, n - 2, 24)) + [n - 2, n - 1, n]))
    return np.array(idx, dtype=np.int64)


def main():
    cfg = workloads.CFG3
    nx, ny, nz = cfg["n"]
    o = oracle.OracleCavity(nx, ny, nz, dict(Ra=cfg["Ra"], Pr=cfg["Pr"]), noise=cfg["noise"], seed=cfg["seed"])
    t0 = time.time()
    done = 0
    while done < cfg["steps"]:
        n = min(250, cfg["steps"] - done)
        o.step(n)
        done += n
        print(f"{done}/{cfg['steps']} steps, {time.time() - t0:.0f} s, res {o.residual}", flush=True)
    f = o.fields()
    ix, iy, iz = sample_index(nx), sample_index(ny), sample_index(nz)
    samples = f[:, iz - 1][:, :, iy - 1][:, :, :, ix - 1]
    np.savez_compressed(OUT, ix=ix, iy=iy, iz=iz, samples=samples, residual=o.residual,
                        nusselt=np.array(o.nusselt), t=o.t, dt=o.dt, steps=cfg["steps"],
                        n=np.array(cfg["n"]), Ra=cfg["Ra"], Pr=cfg["Pr"], noise=cfg["noise"], seed=cfg["seed"])
    print("wrote", OUT, samples.shape, f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
