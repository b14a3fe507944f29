"""Pins of the oracle's local time stepping (pseudo-time iteration with each
node at its own stable step dt_n = cfl / S_n, S_n the node's spectral bound
of Section 2).

 * from rest every node has the same S_n, so one local step is the global
   step bit for bit;
 * from a smooth random state the u, v, w, T increments of a local step are
   the global step's scaled by S_max / S_n, with S_n written out here
   independently from the wave speeds lambda_d = (|V_d| + sqrt(V_d^2 +
   4 beta^2)) / 2, beta^2 = max(|V|^2, kappa u_ref^2);
 * the conduction state (Ra = 0, T linear in x, fluid at rest) stays a fixed
   point.
"""
import math

import numpy as np
import pytest

import oracle
import workloads


def test_first_step_from_rest_equals_global_step():
    n = (13, 11, 9)
    g = oracle.OracleCavity(*n, dict(Ra=3e4), noise=1e-3, seed=2)
    l = oracle.OracleCavity(*n, dict(Ra=3e4), noise=1e-3, seed=2, local_dt=True)
    g.step(1)
    l.step(1)
    assert np.array_equal(g.fields(), l.fields())
    assert np.array_equal(g.residual, l.residual)


def spectral_by_hand(f, n, p):
    """S_n at every interior node of the fields f [5, nz, ny, nx], Section 2."""
    h = [1.0 / (m + 1) for m in n]
    V = [f[1], f[2], f[3]]
    b2 = np.maximum(V[0] ** 2 + V[1] ** 2 + V[2] ** 2, p["kappa"] * p["u_ref"] ** 2)
    s = sum(0.5 * (np.abs(V[d]) + np.sqrt(V[d] ** 2 + 4.0 * b2)) / h[d] for d in range(3))
    return s + 2.0 * max(p["Pr"], 1.0) * sum(1.0 / hd ** 2 for hd in h)


def test_increments_scale_with_local_spectral_bound():
    n = (14, 12, 10)
    Ra = 5e4
    q0 = workloads.smooth_state(n, seed=4, amp=(50.0, 300.0, 300.0, 300.0, 0.2))  # |V| above beta
    g = oracle.OracleCavity(*n, dict(Ra=Ra))
    l = oracle.OracleCavity(*n, dict(Ra=Ra), local_dt=True)
    g.set_fields(q0)
    l.set_fields(q0)
    f0 = g.fields()
    S = spectral_by_hand(f0, n, g.p)
    ratio = S.max() / S
    assert ratio.max() > 1.5  # the state is far from uniform: dt_n really varies
    g.step(1)
    l.step(1)
    dg, dl = g.fields() - f0, l.fields() - f0
    for f in (1, 2, 3, 4):  # p also carries the centre shift, which is not scaled
        big = np.abs(dg[f]) > 1e-6 * np.abs(dg[f]).max()
        assert np.allclose(dl[f][big], (ratio * dg[f])[big], rtol=1e-9, atol=0.0), f


def test_conduction_state_is_fixed_point_local():
    n = (12, 10, 9)
    o = oracle.OracleCavity(*n, dict(Ra=0.0), noise=0.0, local_dt=True)
    f0 = o.fields()
    o.step(20)
    f = o.fields()
    assert np.max(np.abs(f[1:4])) < 1e-9
    assert np.max(np.abs(f[4] - f0[4])) < 1e-12
    assert o.nusselt[0] == pytest.approx(1.0, abs=1e-10)
