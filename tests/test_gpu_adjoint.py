"""GPU discrete adjoint (checkpointed, FP64 reverse sweep) of the step.

Objective J = mean over steps 1..N of the hot-wall Nusselt number; controls
the hot-wall temperature field theta and Ra.
 * against the oracle's discrete adjoint (32^3 and a ragged small grid):
   the FP64 forward's gradient elementwise within 1e-9 of the largest
   component, Ra within 1e-9; FP32-mixed forward within 1e-4;
 * independent of the checkpoint interval;
 * through torch.autograd (the Function returns the same gradients);
 * configuration 5 at full size: 128^3, Ra 1e5, FP32-mixed forward, 500
   steps, checkpoints every 50, theta = 1 + N(0, 0.01^2); 16 seeded wall
   points and Ra against central differences with h = 1e-4 of FP64 runs.
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


def gpu_gradient(m, n, Ra, steps, ckpt, theta, precision=None, seed=3, noise=1e-3):
    precision = m.CAVITY_FP64 if precision is None else precision
    with m.Cavity(*n, precision=precision, seed=seed, noise_amp=noise, Ra=Ra, Pr=0.71) as c:
        m.cavity_set_wall_temperature(c.h, 0, theta)
        J = m.cavity_adjoint_forward(c.h, steps, ckpt)
        g, gra = m.cavity_adjoint_backward(c.h, n[1], n[2])
        return J, g, gra, c.time


@pytest.mark.parametrize("n,Ra,steps,ckpt", [((32, 32, 32), 1e5, 40, 10), ((17, 14, 11), 2e4, 23, 6), ((2, 9, 7), 1e4, 12, 5)])
def test_adjoint_matches_oracle_adjoint(m, n, Ra, steps, ckpt):
    theta = workloads.wall_temperature(n[1], n[2], seed=5)
    Jo, go, grao = oracle.nusselt_gradient(*n, dict(Ra=Ra, Pr=0.71), steps, seed=3, noise=1e-3, t_hot_wall=theta)
    J, g, gra, _ = gpu_gradient(m, n, Ra, steps, ckpt, theta)
    assert J == pytest.approx(Jo, rel=1e-12)
    assert np.max(np.abs(g - go)) <= 1e-9 * np.max(np.abs(go))
    assert gra == pytest.approx(grao, rel=1e-9)


@pytest.mark.parametrize("n,steps,ckpt", [((32, 32, 32), 40, 8), ((17, 14, 11), 23, 6), ((2, 9, 7), 12, 5)])
def test_adjoint_fp32_forward_matches_oracle(m, n, steps, ckpt):
    Ra = 1e5
    theta = workloads.wall_temperature(n[1], n[2], seed=5)
    Jo, go, grao = oracle.nusselt_gradient(*n, dict(Ra=Ra, Pr=0.71), steps, seed=3, noise=1e-3, t_hot_wall=theta)
    J, g, gra, _ = gpu_gradient(m, n, Ra, steps, ckpt, theta, precision=m.CAVITY_FP32_MIXED)
    assert J == pytest.approx(Jo, rel=1e-5)
    assert np.max(np.abs(g - go)) <= 1e-4 * np.max(np.abs(go))
    assert gra == pytest.approx(grao, rel=1e-4)


def test_adjoint_independent_of_checkpoint_interval_and_restores_state(m):
    n, Ra, steps = (24, 20, 18), 5e4, 30
    theta = workloads.wall_temperature(n[1], n[2], seed=6)
    J1, g1, r1, t1 = gpu_gradient(m, n, Ra, steps, 4, theta)
    J2, g2, r2, t2 = gpu_gradient(m, n, Ra, steps, 13, theta)
    J3, g3, r3, t3 = gpu_gradient(m, n, Ra, steps, 30, theta)
    assert J1 == J2 == J3
    assert t1 == t2 == t3 and t1[0] == steps
    for g, r in ((g2, r2), (g3, r3)):
        assert np.max(np.abs(g - g1)) <= 1e-12 * np.max(np.abs(g1))
        assert r == pytest.approx(r1, rel=1e-12)


def test_autograd_function(m):
    import torch
    from paper_2006_02602_gb300.autograd import mean_hot_wall_nusselt
    n, Ra, steps = (20, 18, 16), 3e4, 25
    theta0 = workloads.wall_temperature(n[1], n[2], seed=7)
    theta = torch.tensor(theta0.reshape(n[2], n[1]), requires_grad=True)
    ra = torch.tensor(Ra, dtype=torch.float64, requires_grad=True)
    J = mean_hot_wall_nusselt(theta, ra, n, steps, ckpt=7, seed=3, noise=1e-3)
    J.backward()
    Jr, g, gra, _ = gpu_gradient(m, n, Ra, steps, 7, theta0)
    assert float(J.detach()) == Jr
    assert np.max(np.abs(theta.grad.numpy().reshape(-1) - g)) <= 1e-12 * np.max(np.abs(g))
    assert float(ra.grad) == pytest.approx(gra, rel=1e-12)


def test_cfg5_fp32_adjoint_vs_central_differences_128(m):
    n, Ra, steps, ckpt = (128, 128, 128), 1e5, 500, 50
    rng = np.random.default_rng(2024)
    theta = workloads.wall_temperature(n[1], n[2], seed=11, base=1.0, sigma=0.01)
    J, g, gra, _ = gpu_gradient(m, n, Ra, steps, ckpt, theta, precision=m.CAVITY_FP32_MIXED, seed=0, noise=1e-3)
    J64, g64, gra64, _ = gpu_gradient(m, n, Ra, steps, ckpt, theta, seed=0, noise=1e-3)

    def J_fd(th, ra):
        with m.Cavity(*n, seed=0, noise_amp=1e-3, Ra=ra, Pr=0.71) as c:
            m.cavity_set_wall_temperature(c.h, 0, th)
            return m.cavity_adjoint_forward(c.h, steps, steps)

    h = 1e-4
    points = rng.choice(n[1] * n[2], size=16, replace=False)
    for pt in points:
        tp, tm = theta.copy(), theta.copy()
        tp[pt] += h
        tm[pt] -= h
        fd = (J_fd(tp, Ra) - J_fd(tm, Ra)) / (2 * h)
        assert g64[pt] == pytest.approx(fd, rel=1e-6), pt
        assert g[pt] == pytest.approx(fd, rel=2e-3), pt
    hr = h * Ra
    fd = (J_fd(theta, Ra + hr) - J_fd(theta, Ra - hr)) / (2 * hr)
    assert gra64 == pytest.approx(fd, rel=1e-5)
    assert gra == pytest.approx(fd, rel=2e-3)
