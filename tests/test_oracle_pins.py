"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test targets a plausible mistake: a dropped or mis-signed term, a wrong
spacing or index, a transposed face buffer, a wrong wall formula.
  * MMS truncation order of Eqs. 1-3 against the continuous operator (sympy);
  * closed forms of the central 4th and 1st differences of a quartic;
  * damping sign of the Eq. 1 dissipation on the odd-even (checkerboard) mode;
  * wall formulas exact on linear p and on wall-quadratic adiabatic T;
  * conduction state (Ra = 0, T = 1 - x) is a fixed point with Nu = 1;
  * centro-symmetry and y-mirror symmetry of the differentially heated cube;
  * buoyancy lifts hot fluid;
  * splitmix64 published outputs;
  * decomposition: block fields bit-identical to one block; ghost faces and
    face buffers bit-identical to brute-force reads of the global array.
"""
import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _full(nx, ny, nz):
    return np.zeros((5, nz + 4, ny + 4, nx + 4))


def _coords(nx, ny, nz):
    """Node coordinates including walls and pressure ghosts (index -1 .. n+2)."""
    xs = np.arange(-1, nx + 3) / (nx + 1)
    ys = np.arange(-1, ny + 3) / (ny + 1)
    zs = np.arange(-1, nz + 3) / (nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return X, Y, Z


# --------------------------------------------------------------------------
def test_splitmix64_published_values():
    vals = []
    with open(os.path.join(HERE, "golden", "splitmix64_seed0.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(int(line, 16))
    gamma = 0x9E3779B97F4A7C15
    got = [oracle.splitmix64((n * gamma) & 0xFFFFFFFFFFFFFFFF) for n in range(4)]
    assert got == vals


def test_init_noise_uniform_and_linear_profile():
    a = 1e-3
    o = oracle.OracleCavity(20, 18, 16, seed=3, noise=a)
    f = o.fields()
    x = np.arange(1, 21) / 21.0
    noise = f[4] - (1.0 - x)[None, None, :]
    assert np.all(np.abs(noise) <= a)
    # mean and variance of U(-a, a): 0 and a^2/3
    assert abs(noise.mean()) < 4 * a / math.sqrt(3 * noise.size)
    assert abs(noise.var() / (a * a / 3) - 1) < 0.05
    assert np.all(f[:4] == 0.0)
    # a different seed gives a different draw
    o2 = oracle.OracleCavity(20, 18, 16, seed=4, noise=a)
    assert not np.array_equal(o2.fields()[4], f[4])


# --------------------------------------------------------------------------
def _mms_case(n1, params):
    """Discrete vs continuous rates for smooth fields on a non-cubic grid."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    u = sp.sin(1.1 * x + 0.3) * sp.cos(0.7 * y + 0.2) * sp.sin(1.3 * z + 0.5)
    v = sp.cos(0.9 * x + 0.1) * sp.sin(1.2 * y + 0.4) * sp.cos(0.8 * z + 0.3)
    w = sp.sin(0.6 * x + 0.7) * sp.sin(1.0 * y + 0.2) * sp.cos(1.4 * z + 0.1)
    p = 3.0 * sp.cos(1.3 * x + 0.2) * sp.cos(0.9 * y + 0.6) * sp.sin(0.7 * z + 0.4)
    T = 0.5 + 0.3 * sp.sin(1.2 * x + 0.1) * sp.cos(1.1 * y + 0.3) * sp.cos(0.5 * z + 0.2)
    V = (u, v, w)
    X = (x, y, z)
    nu, alpha, gs = params["Pr"], 1.0, params["Ra"] * params["Pr"]
    b2f = params["kappa"] * params["u_ref"] ** 2
    beta2 = sp.Max(u * u + v * v + w * w, b2f)
    lap = lambda f: sum(sp.diff(f, s, 2) for s in X)
    adv = lambda f: sum(V[d] * sp.diff(f, X[d]) for d in range(3))
    # continuous Eqs. 1-3 (the dissipation is O(h^3) and vanishes in the limit)
    rhs = [-beta2 * sum(sp.diff(V[d], X[d]) for d in range(3))]
    for c in range(3):
        buoy = gs * (T - params["t_inf"]) if c == params["gravity_axis"] else 0
        rhs.append(-adv(V[c]) - sp.diff(p, X[c]) + nu * lap(V[c]) + buoy)
    rhs.append(-adv(T) + alpha * lap(T))
    fns = [sp.lambdify((x, y, z), e, "numpy") for e in (p, u, v, w, T)]
    rfns = [sp.lambdify((x, y, z), e, "numpy") for e in rhs]

    nx, ny, nz = 16 * n1 - 1, 20 * n1 - 1, 24 * n1 - 1
    q = _full(nx, ny, nz)
    Xg, Yg, Zg = _coords(nx, ny, nz)
    for f in range(5):
        q[f] = np.broadcast_to(fns[f](Xg, Yg, Zg), Xg.shape)
    got = oracle.rates(params, q)
    Xi, Yi, Zi = (A[2:-2, 2:-2, 2:-2] for A in (Xg, Yg, Zg))
    err = []
    for f in range(5):
        exact = np.broadcast_to(rfns[f](Xi, Yi, Zi), Xi.shape)
        err.append(np.max(np.abs(got[f] - exact)))
    return np.array(err)


def test_mms_second_order_all_fields():
    params = oracle.default_params(Ra=1e3, Pr=0.71)
    e1 = _mms_case(1, params)
    e2 = _mms_case(2, params)
    e4 = _mms_case(4, params)
    o12 = np.log2(e1 / e2)
    o24 = np.log2(e2 / e4)
    assert np.all(o24 >= 1.9), (e1, e2, e4, o12, o24)
    assert np.all(o12 >= 1.7), (e1, e2, e4, o12, o24)


def test_mms_beta_branch_uses_velocity():
    # large velocities so beta^2 = |V|^2 (not the floor) at most nodes
    params = oracle.default_params(Ra=0.0, Pr=0.71, u_ref=1.0, kappa=0.01)
    e2 = _mms_case(2, params)
    e4 = _mms_case(4, params)
    assert np.all(np.log2(e2 / e4) >= 1.9)


# --------------------------------------------------------------------------
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_quartic_pressure_closed_forms(axis):
    nx, ny, nz = 11, 9, 13
    params = oracle.default_params(Ra=1e4, Pr=0.71)
    q = _full(nx, ny, nz)
    C = _coords(nx, ny, nz)
    s = C[axis]
    a4 = 2.5
    q[0] = a4 * (s - 0.3) ** 4
    q[4] = params["t_inf"]
    r = oracle.rates(params, q)
    h = 1.0 / ((nx, ny, nz)[axis] + 1)
    beta = math.sqrt(params["kappa"]) * params["u_ref"]
    # delta^4 of a quartic = 24 a4 h^4, lambda = beta at rest
    expect_p = -24.0 * params["c4"] * beta * h ** 3 * a4
    assert np.allclose(r[0], expect_p, rtol=1e-9, atol=0)
    # central first difference of a quartic: 4 s^3 + 4 s h^2 (shifted)
    si = s[2:-2, 2:-2, 2:-2] - 0.3
    expect_v = -a4 * (4 * si ** 3 + 4 * si * h * h)
    assert np.allclose(r[1 + axis], expect_v, rtol=1e-9, atol=1e-12)
    for c in range(3):
        if c != axis:
            assert np.max(np.abs(r[1 + c])) < 1e-9
    assert np.max(np.abs(r[4])) == 0.0


def test_dissipation_damps_odd_even_mode():
    nx, ny, nz = 8, 10, 12
    params = oracle.default_params(Ra=1e4)
    q = _full(nx, ny, nz)
    K, J, I = np.meshgrid(np.arange(-1, nz + 3), np.arange(-1, ny + 3), np.arange(-1, nx + 3), indexing="ij")
    q[0] = 1e-3 * (-1.0) ** (I + J + K)
    q[4] = params["t_inf"]
    r = oracle.rates(params, q)
    p0 = q[0][2:-2, 2:-2, 2:-2]
    beta = math.sqrt(params["kappa"]) * params["u_ref"]
    inv_h = (nx + 1) + (ny + 1) + (nz + 1)
    # each 1D fourth difference of (-1)^i is 16 p0; the rate opposes p0
    assert np.all(r[0] * p0 < 0)
    assert np.allclose(r[0], -16.0 * params["c4"] * beta * inv_h * p0, rtol=1e-12)
    assert np.max(np.abs(r[1:4])) < 1e-12


# --------------------------------------------------------------------------
def test_wall_conditions_linear_pressure_and_dirichlet():
    nx, ny, nz = 9, 7, 8
    q = _full(nx, ny, nz)
    X, Y, Z = _coords(nx, ny, nz)
    lin = 0.7 + 1.3 * X - 2.1 * Y + 0.4 * Z
    q[0][2:-2, 2:-2, 2:-2] = lin[2:-2, 2:-2, 2:-2]
    q[1:4][:, 2:-2, 2:-2, 2:-2] = 1.0
    q[4][2:-2, 2:-2, 2:-2] = 0.25
    th = np.linspace(0.9, 1.1, ny * nz)
    tc = np.linspace(-0.1, 0.1, ny * nz)
    oracle.apply_bc(q, th, tc)
    P = q[0]
    # walls and ghosts on each face reproduce the linear function (face interior ranges)
    sl = slice(2, -2)
    for ax_idx in [(slice(None), sl, sl), (sl, slice(None), sl), (sl, sl, slice(None))]:
        pass
    faces = {
        "x": (P[sl, sl, [0, 1, -2, -1]], lin[sl, sl, [0, 1, -2, -1]]),
        "y": (P[sl, [0, 1, -2, -1], sl], lin[sl, [0, 1, -2, -1], sl]),
        "z": (P[[0, 1, -2, -1], sl, sl], lin[[0, 1, -2, -1], sl, sl]),
    }
    for name, (got, exp) in faces.items():
        assert np.allclose(got, exp, rtol=0, atol=1e-13), name
    # no slip on every wall (face interior ranges)
    for f in (1, 2, 3):
        assert np.all(q[f][sl, sl, [1, -2]] == 0)
        assert np.all(q[f][sl, [1, -2], sl] == 0)
        assert np.all(q[f][[1, -2], sl, sl] == 0)
    # isothermal x walls take the given wall temperatures, (j, k) order j fastest
    assert np.array_equal(q[4][2:-2, 2:-2, 1], th.reshape(nz, ny))
    assert np.array_equal(q[4][2:-2, 2:-2, -2], tc.reshape(nz, ny))


@pytest.mark.parametrize("wall", ["y0", "y1", "z0", "z1"])
def test_adiabatic_wall_exact_on_wall_quadratic(wall):
    nx, ny, nz = 6, 9, 7
    q = _full(nx, ny, nz)
    X, Y, Z = _coords(nx, ny, nz)
    s = {"y0": Y, "y1": 1 - Y, "z0": Z, "z1": 1 - Z}[wall]
    # zero normal derivative at the wall, quadratic in the wall distance
    T = 0.3 + 0.2 * X + 1.7 * s * s
    q[4][2:-2, 2:-2, 2:-2] = T[2:-2, 2:-2, 2:-2]
    oracle.apply_bc(q, np.zeros(ny * nz), np.zeros(ny * nz))
    sl = slice(2, -2)
    got = {"y0": q[4][sl, 1, sl], "y1": q[4][sl, -2, sl], "z0": q[4][1, sl, sl], "z1": q[4][-2, sl, sl]}[wall]
    exp = {"y0": T[sl, 1, sl], "y1": T[sl, -2, sl], "z0": T[1, sl, sl], "z1": T[-2, sl, sl]}[wall]
    assert np.allclose(got, exp, rtol=0, atol=1e-14)


# --------------------------------------------------------------------------
def test_conduction_state_is_fixed_point():
    nx, ny, nz = 14, 12, 10
    o = oracle.OracleCavity(nx, ny, nz, dict(Ra=0.0), noise=0.0)
    f0 = o.fields()
    assert o.nusselt[0] == pytest.approx(1.0, abs=1e-12)
    assert o.nusselt[1] == pytest.approx(1.0, abs=1e-12)
    o.step(30)
    f = o.fields()
    assert np.max(np.abs(f[1:4])) < 1e-9
    assert np.max(np.abs(f[4] - f0[4])) < 1e-12
    assert np.max(o.residual[1:]) < 1e-9
    assert o.nusselt[0] == pytest.approx(1.0, abs=1e-10)
    assert o.nusselt[1] == pytest.approx(1.0, abs=1e-10)


def test_centro_symmetry_and_y_mirror():
    o = oracle.OracleCavity(12, 10, 14, dict(Ra=1e4), noise=0.0)
    o.step(200)
    f = o.fields()
    p, u, v, w, T = f
    S = lambda a: a[::-1, ::-1, ::-1]
    scale = [np.max(np.abs(a)) for a in f]
    assert scale[1] > 1e-2 and scale[3] > 1e-2  # the flow has started
    assert np.max(np.abs(S(p) - p)) <= 1e-12 * scale[0]
    for c in (1, 2, 3):
        assert np.max(np.abs(S(f[c]) + f[c])) <= 1e-12 * scale[c]
    assert np.max(np.abs(S(T) - (1.0 - T))) <= 1e-12
    assert o.nusselt[0] == pytest.approx(o.nusselt[1], rel=1e-12)
    # mirror y -> 1 - y: v odd, every other field even
    M = lambda a: a[:, ::-1, :]
    assert np.max(np.abs(M(v) + v)) <= 1e-12 * max(scale[2], 1e-300)
    for c in (0, 1, 3, 4):
        assert np.max(np.abs(M(f[c]) - f[c])) <= 1e-12 * scale[c]


def test_buoyancy_lifts_hot_fluid():
    o = oracle.OracleCavity(16, 8, 16, dict(Ra=1e4), noise=0.0)
    o.step(100)
    w = o.fields()[3]
    mid = 8
    assert w[mid, :, 1].mean() > 0    # next to the hot wall (x = 0)
    assert w[mid, :, -2].mean() < 0   # next to the cold wall


def test_centre_pressure_gauge():
    o = oracle.OracleCavity(10, 11, 12, dict(Ra=1e4), noise=1e-3, seed=1)
    o.step(5)
    assert abs(o.centre_value()) <= 1e-14 * np.max(np.abs(o.fields()[0]))
    # the shift cancels in every rate: adding a constant to p changes no rate
    q = o.full_array().copy()
    r0 = oracle.rates(o.p, q)
    q[0] += 123.25
    r1 = oracle.rates(o.p, q)
    for f in range(5):
        assert np.max(np.abs(r1[f] - r0[f])) <= 1e-11 * max(np.max(np.abs(r0[f])), 1e-300)


def test_explicit_step_stable_at_cfl():
    # linearised one-step map about the conduction state has spectral radius <= 1
    nx, ny, nz = 4, 4, 5
    base = oracle.OracleCavity(nx, ny, nz, dict(Ra=0.0), noise=0.0)
    f0 = base.fields().copy()
    n = f0.size
    eps = 1e-7
    f_ref = oracle.OracleCavity(nx, ny, nz, dict(Ra=0.0))
    f_ref.set_fields(f0)
    f_ref.step(1)
    y0 = f_ref.fields().reshape(-1).copy()
    J = np.empty((n, n))
    for col in range(n):
        pert = f0.reshape(-1).copy()
        pert[col] += eps
        o = oracle.OracleCavity(nx, ny, nz, dict(Ra=0.0))
        o.set_fields(pert.reshape(f0.shape))
        o.step(1)
        J[:, col] = (o.fields().reshape(-1) - y0) / eps
    rho = np.max(np.abs(np.linalg.eigvals(J)))
    assert rho <= 1.0 + 1e-6


# --------------------------------------------------------------------------
DECOMPS = [(2, 2, 2), (4, 1, 1), (1, 3, 1), (1, 1, 4), (4, 2, 1), (3, 2, 2)]


@pytest.fixture(scope="module")
def global_run():
    o = oracle.OracleCavity(24, 20, 18, dict(Ra=1e5), noise=1e-3, seed=7)
    o.step(12)
    return o


@pytest.mark.parametrize("blocks", DECOMPS)
def test_blocks_bit_identical_to_single(global_run, blocks):
    o = oracle.OracleCavity(24, 20, 18, dict(Ra=1e5), blocks=blocks, noise=1e-3, seed=7)
    o.step(12)
    assert np.array_equal(o.fields(), global_run.fields())
    assert o.dt == global_run.dt
    assert np.allclose(o.residual, global_run.residual, rtol=1e-13)


@pytest.mark.parametrize("blocks", [(2, 2, 2), (3, 2, 2)])
def test_ghost_faces_match_brute_force(global_run, blocks):
    o = oracle.OracleCavity(24, 20, 18, dict(Ra=1e5), blocks=blocks, noise=1e-3, seed=7)
    o.step(12)
    G = global_run.full_array()  # G[f, K+1, J+1, I+1] by global node index
    checked = 0
    for blk in o.blocks:
        c = blk.c
        n = (c.nx, c.ny, c.nz)
        org = (c.ox, c.oy, c.oz)
        for face in range(6):
            if blk.nbr[face] < 0:
                continue
            a, hi = face // 2, face % 2
            layers_p = [n[a] + 1, n[a] + 2] if hi else [-1, 0]
            layers_v = [n[a] + 1] if hi else [0]
            for fld in range(5):
                for L in (layers_p if fld == 0 else layers_v):
                    idx = [slice(2, 2 + n[0]), slice(2, 2 + n[1]), slice(2, 2 + n[2])]
                    gidx = [slice(org[d] + 2, org[d] + 2 + n[d]) for d in range(3)]
                    idx[a] = L + 1
                    gidx[a] = org[a] + L + 1
                    mine = blk.q[fld][idx[2], idx[1], idx[0]]
                    glob = G[fld][gidx[2], gidx[1], gidx[0]]
                    assert np.array_equal(mine, glob), (blk.id, face, fld, L)
                    checked += 1
    assert checked > 0


def test_face_buffer_layout_brute_force(global_run):
    o = oracle.OracleCavity(24, 20, 18, dict(Ra=1e5), blocks=(2, 2, 2), noise=1e-3, seed=7)
    o.step(12)
    G = global_run.full_array()
    bufs = o.pack_buffers()
    assert len(bufs) == 24  # 8 blocks x 3 cut faces
    for (bid, face), buf in bufs.items():
        c = o.blocks[bid].c
        n = (c.nx, c.ny, c.nz)
        org = (c.ox, c.oy, c.oz)
        a, hi = face // 2, face % 2
        b_ax, c_ax = [d for d in range(3) if d != a]
        nb, nc = n[b_ax], n[c_ax]
        assert buf.size == 6 * nb * nc
        for ic in range(nc):
            for ib in range(nb):
                node = [0, 0, 0]
                node[b_ax] = org[b_ax] + ib + 1
                node[c_ax] = org[c_ax] + ic + 1
                for d in range(2):
                    node[a] = org[a] + (n[a] - 1 + d if hi else 1 + d)
                    assert buf[(ic * nb + ib) * 2 + d] == G[0, node[2] + 1, node[1] + 1, node[0] + 1]
                node[a] = org[a] + (n[a] if hi else 1)
                for v in range(4):
                    assert buf[2 * nb * nc + v * nb * nc + ic * nb + ib] == \
                        G[1 + v, node[2] + 1, node[1] + 1, node[0] + 1]


# --------------------------------------------------------------------------
# The stable step (Section 2: explicit Euler with the local acoustic wave
# speeds and the viscous/thermal diffusion limit) against values worked out
# by hand, not from the oracle's spectral routine.
@pytest.mark.parametrize("Pr", [0.71, 2.0])
def test_dt_at_rest_closed_form(Pr):
    # fluid at rest: beta^2 = kappa u_ref^2 everywhere and each wave speed
    # (|V_d| + sqrt(V_d^2 + 4 beta^2)) / 2 is beta itself.  Sizes 7, 9, 11
    # give 1/h = 8, 10, 12, so sum 1/h = 30 and sum 1/h^2 = 308.
    kappa, u_ref, cfl = 0.25, 6.0, 0.5           # beta = 3
    o = oracle.OracleCavity(7, 9, 11, dict(Ra=0.0, Pr=Pr, kappa=kappa, u_ref=u_ref, cfl=cfl), noise=0.0)
    diff = 2.0 * max(Pr, 1.0) * 308.0            # the larger of nu = Pr and alpha = 1
    S = 3.0 * 30.0 + diff
    assert o.spectral_max() == pytest.approx(S, rel=1e-14)
    o.step(1)
    assert o.dt == pytest.approx(cfl / S, rel=1e-14)


def test_dt_uniform_velocity_floor_branch():
    # beta^2 = kappa u_ref^2 = 900 (so 4 beta^2 = 60^2) exceeds |V|^2 = 11^2 + 25^2 = 746.
    # V = (11, -25, 0): sqrt(11^2 + 3600) = 61, sqrt(25^2 + 3600) = 65, sqrt(3600) = 60,
    # wave speeds (11 + 61)/2 = 36, (25 + 65)/2 = 45, 60/2 = 30.
    # 1/h = 8, 10, 12: 36*8 + 45*10 + 30*12 = 1098; diffusion 2 * 1 * 308 = 616.
    n = (7, 9, 11)
    o = oracle.OracleCavity(*n, dict(Ra=0.0, Pr=0.71, kappa=1.0, u_ref=30.0, cfl=0.5), noise=0.0)
    f = o.fields()
    f[1], f[2], f[3] = 11.0, -25.0, 0.0
    o.set_fields(f)
    assert o.spectral_max() == pytest.approx(1098.0 + 616.0, rel=1e-14)
    # the same wave speeds with the axes permuted: V = (0, 11, -25)
    f[1], f[2], f[3] = 0.0, 11.0, -25.0
    o.set_fields(f)
    assert o.spectral_max() == pytest.approx(30 * 8 + 36 * 10 + 45 * 12 + 616.0, rel=1e-14)


def test_dt_uniform_velocity_velocity_branch():
    # V = (0, 0, w) with w^2 above the floor: beta^2 = w^2, the transverse wave
    # speeds are sqrt(4 w^2)/2 = w and the streamwise one (w + sqrt(5) w)/2 =
    # w phi, phi the golden ratio.
    w = 40.0
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    o = oracle.OracleCavity(7, 9, 11, dict(Ra=0.0, Pr=0.71, kappa=0.01, u_ref=1.0, cfl=0.5), noise=0.0)
    f = o.fields()
    f[3] = -w
    o.set_fields(f)
    S = w * 8 + w * 10 + w * phi * 12 + 616.0
    assert o.spectral_max() == pytest.approx(S, rel=1e-14)
    o.step(1)
    assert o.dt == pytest.approx(0.5 / S, rel=1e-14)


def test_residual_is_rms_of_applied_increment():
    # Section 4.2 residual norms, read as the RMS over the N interior nodes of
    # dq/dt: after one step it must equal ||q^{n+1} - q^n||_2 / (dt sqrt(N))
    # for the fields the centre rescale does not touch (u, v, w, T), using only
    # field differences.
    import workloads
    n = (13, 11, 9)
    N = n[0] * n[1] * n[2]
    o = oracle.OracleCavity(*n, dict(Ra=1e4), noise=0.0)
    o.set_fields(workloads.smooth_state(n, seed=5))
    before = o.fields().copy()
    o.step(1)
    after = o.fields()
    for f in (1, 2, 3, 4):
        inc = after[f] - before[f]
        expect = math.sqrt(float(np.sum(inc * inc)) / N) / o.dt
        assert expect > 0
        assert o.residual[f] == pytest.approx(expect, rel=1e-8), oracle.FIELDS[f]
    # p: the increment is dt dp/dt less the centre value c of the updated p,
    # one constant over the interior; removing the mean of the increment
    # removes c, so the RMS of dp/dt bounds the RMS of the centred increment.
    incp = after[0] - before[0]
    cen = incp - incp.mean()
    assert math.sqrt(float(np.sum(cen * cen)) / N) / o.dt <= o.residual[0] * (1 + 1e-8)
