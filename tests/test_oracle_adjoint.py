"""Pins of the oracle's discrete adjoint against central finite differences
of the oracle's own forward run (the adjoint is the reverse of the step, the
FD quotient uses nothing but the forward), and against the linear pieces it
must reproduce exactly.

Objective: J = mean over steps 1..N of the hot-wall Nusselt number;
controls: the hot-wall temperature field and Ra.
"""
import numpy as np
import pytest

import oracle
import workloads

N_GRID = (10, 9, 8)
STEPS = 20


def J_of(theta, Ra, steps=STEPS, seed=3):
    o = oracle.OracleCavity(*N_GRID, dict(Ra=Ra, Pr=0.71), noise=1e-3, seed=seed, t_hot_wall=theta)
    J = 0.0
    for _ in range(steps):
        o.step(1)
        J += o.nusselt[0]
    return J / steps


@pytest.fixture(scope="module")
def adj():
    ny, nz = N_GRID[1], N_GRID[2]
    theta = workloads.wall_temperature(ny, nz, seed=5)
    J, g, gra = oracle.nusselt_gradient(*N_GRID, dict(Ra=2e4, Pr=0.71), STEPS, seed=3, noise=1e-3, t_hot_wall=theta)
    return theta, J, g, gra


def test_objective_matches_forward(adj):
    theta, J, g, gra = adj
    assert J == pytest.approx(J_of(theta, 2e4), rel=1e-14)


@pytest.mark.parametrize("point", [0, 17, 40, 71])
def test_wall_gradient_vs_central_differences(adj, point):
    theta, J, g, gra = adj
    h = 1e-5
    tp, tm = theta.copy(), theta.copy()
    tp[point] += h
    tm[point] -= h
    fd = (J_of(tp, 2e4) - J_of(tm, 2e4)) / (2 * h)
    assert g[point] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.max(np.abs(g)))


def test_ra_gradient_vs_central_differences(adj):
    theta, J, g, gra = adj
    Ra = 2e4
    h = 1e-5 * Ra
    fd = (J_of(theta, Ra + h) - J_of(theta, Ra - h)) / (2 * h)
    assert gra == pytest.approx(fd, rel=1e-5)


def test_one_step_gradient_is_the_direct_wall_term_plus_transport():
    """With one step from a state at rest, dJ/dtheta has the closed form of the
    Nusselt stencil: the direct term 3/(2 h dT ny nz) plus theta's transport
    into T_1 through the x-diffusion of the first step (alpha dt / h^2 each,
    times -4/(2 h dT ny nz)); nothing else moves in one step from rest."""
    nx, ny, nz = 7, 6, 5
    theta = np.ones(ny * nz)
    J, g, _ = oracle.nusselt_gradient(nx, ny, nz, dict(Ra=0.0, Pr=0.71), 1, noise=0.0, t_hot_wall=theta)
    o = oracle.OracleCavity(nx, ny, nz, dict(Ra=0.0, Pr=0.71), t_hot_wall=theta)
    dt = o.p["cfl"] / o.spectral_max()
    h = 1.0 / (nx + 1)
    c = 1.0 / (ny * nz * 2 * h)
    # T_1 gains dt * alpha * theta / h^2 (x-diffusion) minus the convective part (u = 0 at rest)
    expect = 3 * c + (-4 * c) * dt / (h * h)
    assert np.allclose(g, expect, rtol=1e-12)
