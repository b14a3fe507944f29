"""GPU (sm_103a) FP64 step against the FP64 oracle, through the C ABI.

Tolerances: fields <= 1e-12 relative max-norm per field (FP64 form), Nusselt
and dt <= 1e-12 relative, residual norms <= 1e-10 relative (sums in another
order); initial state and pack/unpack bit exact; decompositions bit exact
against the single block.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


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


def assert_fields_close(g, o, tol, what=""):
    for f, name in enumerate(oracle.FIELDS):
        e = relmax(g[f], o[f])
        assert e <= tol, f"{what} field {name}: rel max err {e:.3e} > {tol:.1e}"


def run_pair(m, n, Ra, steps, blocks=(1, 1, 1), noise=1e-3, seed=0, **kw):
    o = oracle.OracleCavity(*n, dict(Ra=Ra, **kw), noise=noise, seed=seed)
    c = m.Cavity(*n, blocks=blocks, seed=seed, noise_amp=noise, Ra=Ra, **kw)
    o.step(steps)
    c.step(steps)
    return o, c


# ---------------------------------------------------------------------------
def test_initial_state_bit_exact(m):
    n = (37, 21, 18)
    o = oracle.OracleCavity(*n, dict(Ra=1e4), noise=1e-3, seed=5)
    with m.Cavity(*n, seed=5, noise_amp=1e-3, Ra=1e4) as c:
        assert np.array_equal(c.fields(), o.fields())
        s, t, dt = c.time
        assert s == 0 and t == 0.0
        assert dt == pytest.approx(o.p["cfl"] / o.spectral_max(), rel=1e-14)
        h, cold = c.nusselt
        assert h == pytest.approx(o.nusselt[0], rel=1e-12)
        assert cold == pytest.approx(o.nusselt[1], rel=1e-12)


def test_config1_32cube_200_steps(m):
    cfg = workloads.CFG1
    o, c = run_pair(m, cfg["n"], cfg["Ra"], cfg["steps"], noise=cfg["noise"], seed=cfg["seed"], Pr=cfg["Pr"])
    with c:
        assert_fields_close(c.fields(), o.fields(), FP64_TOL, "cfg1")
        assert np.allclose(c.residual, o.residual, rtol=1e-10, atol=0)
        h, cold = c.nusselt
        assert abs(h - o.nusselt[0]) <= FP64_TOL * abs(o.nusselt[0])
        assert abs(cold - o.nusselt[1]) <= FP64_TOL * abs(o.nusselt[1])
        s, t, dt = c.time
        assert s == 200
        assert t == pytest.approx(o.t, rel=1e-13)
        assert dt == pytest.approx(o.p["cfl"] / o.spectral_max(), rel=1e-13)


@pytest.mark.parametrize("n", [(37, 21, 18), (2, 2, 2), (2, 11, 9), (3, 40, 5), (65, 9, 33)])
def test_ragged_and_degenerate_sizes(m, n):
    o, c = run_pair(m, n, 3e4, 25, noise=1e-3, seed=11)
    with c:
        assert_fields_close(c.fields(), o.fields(), FP64_TOL, f"n={n}")
        assert np.allclose(c.residual, o.residual, rtol=1e-10, atol=1e-300)
        h, cold = c.nusselt
        assert h == pytest.approx(o.nusselt[0], rel=1e-12) and cold == pytest.approx(o.nusselt[1], rel=1e-12)
        s_, t, dt = c.time
        assert s_ == 25 and t == pytest.approx(o.t, rel=1e-13)
        assert dt == pytest.approx(o.p["cfl"] / o.spectral_max(), rel=1e-13)


@pytest.mark.parametrize("gaxis", [1, 2])
def test_gravity_axis_and_params(m, gaxis):
    kw = dict(gravity_axis=gaxis, Pr=2.0, cfl=0.4, kappa=0.2, c4=0.05, t_hot=2.0, t_cold=0.5)
    o, c = run_pair(m, (20, 24, 22), 2e4, 40, noise=1e-3, seed=2, **kw)
    with c:
        assert_fields_close(c.fields(), o.fields(), FP64_TOL, f"g={gaxis}")


def test_zero_steps_is_noop(m):
    with m.Cavity(12, 10, 8, seed=1, noise_amp=1e-3, Ra=1e4) as c:
        f0 = c.fields()
        c.step(0)
        assert np.array_equal(c.fields(), f0)
        assert c.time[0] == 0


def test_conduction_state_fixed_point(m):
    with m.Cavity(24, 20, 16, noise_amp=0.0, Ra=0.0) as c:
        f0 = c.fields()
        c.step(50)
        f = c.fields()
        assert np.max(np.abs(f[1:4])) < 1e-9
        assert np.max(np.abs(f[4] - f0[4])) < 1e-12
        h, cold = c.nusselt
        assert h == pytest.approx(1.0, abs=1e-10) and cold == pytest.approx(1.0, abs=1e-10)


def test_set_fields_then_step(m):
    n = (28, 22, 19)
    q = workloads.smooth_state(n, seed=3)
    o = oracle.OracleCavity(*n, dict(Ra=5e4))
    o.set_fields(q)
    with m.Cavity(*n, Ra=5e4) as c:
        c.set_fields(q)
        assert np.array_equal(c.fields(), q)
        o.step(30)
        c.step(30)
        assert_fields_close(c.fields(), o.fields(), FP64_TOL, "set_fields")
        # partial masks: p alone and T alone round-trip, others untouched
        f = c.fields()
        c.set_fields(q[0:1], mask=m.CAVITY_FIELD_P)
        g = c.fields()
        assert np.array_equal(g[0], q[0]) and np.array_equal(g[1:], f[1:])


def test_wall_temperature_field(m):
    n = (20, 18, 16)
    th = workloads.wall_temperature(n[1], n[2], seed=4)
    o = oracle.OracleCavity(*n, dict(Ra=1e5), noise=1e-3, seed=0, t_hot_wall=th)
    with m.Cavity(*n, seed=0, noise_amp=1e-3, Ra=1e5) as c:
        m.cavity_set_wall_temperature(c.h, 0, th)
        h0, _ = c.nusselt
        assert h0 == pytest.approx(o.nusselt[0], rel=1e-12)
        o.step(40)
        c.step(40)
        assert_fields_close(c.fields(), o.fields(), FP64_TOL, "wall T")
        assert c.nusselt[0] == pytest.approx(o.nusselt[0], rel=1e-12)


# ---------------------------------------------------------------------------
# decomposition: bit exact against one block; ghosts and buffers vs brute force

DECOMPS = [(8, 1, 1), (4, 2, 1), (2, 2, 2), (1, 1, 8), (3, 2, 2)]


@pytest.fixture(scope="module")
def single_48(m):
    c = m.Cavity(48, 40, 44, seed=9, noise_amp=1e-3, Ra=1e5)
    c.step(60)
    yield c
    c.close()


@pytest.mark.parametrize("blocks", DECOMPS)
def test_blocks_bit_identical(m, single_48, blocks):
    with m.Cavity(48, 40, 44, blocks=blocks, seed=9, noise_amp=1e-3, Ra=1e5) as c:
        assert m.cavity_num_blocks(c.h) == blocks[0] * blocks[1] * blocks[2]
        c.step(60)
        assert np.array_equal(c.fields(), single_48.fields())
        assert c.time == single_48.time
        assert np.allclose(c.residual, single_48.residual, rtol=1e-13)


def test_blocks_match_oracle(m):
    n = (30, 26, 22)
    o = oracle.OracleCavity(*n, dict(Ra=1e5), blocks=(2, 2, 2), noise=1e-3, seed=3)
    with m.Cavity(*n, blocks=(2, 2, 2), seed=3, noise_amp=1e-3, Ra=1e5) as c:
        o.step(20)
        c.step(20)
        assert_fields_close(c.fields(), o.fields(), FP64_TOL, "2x2x2")


@pytest.mark.parametrize("blocks", [(2, 2, 2), (4, 2, 1), (8, 1, 1)])
def test_ghosts_and_buffers_bit_exact(m, single_48, blocks):
    """Every ghost layer equals the single-block array at the same global node,
    and every face buffer equals a brute-force read of the sending block."""
    with m.Cavity(48, 40, 44, blocks=blocks, seed=9, noise_amp=1e-3, Ra=1e5) as c:
        c.step(60)
        G = [m.cavity_get_block_array(single_48.h, 0, f)[0] for f in range(5)]
        nb_total = m.cavity_num_blocks(c.h)
        arrays = [[m.cavity_get_block_array(c.h, b, f)[0] for f in range(5)] for b in range(nb_total)]
        dims = [m.cavity_get_block_array(c.h, b, 0)[1] for b in range(nb_total)]
        ncut = 0
        for b in range(nb_total):
            nx, ny, nz, ox, oy, oz = dims[b]
            n, org = (nx, ny, nz), (ox, oy, oz)
            for face in range(6):
                a, hi = face // 2, face % 2
                coords = [b % blocks[0], (b // blocks[0]) % blocks[1], b // (blocks[0] * blocks[1])]
                nbc = coords[a] + (1 if hi else -1)
                if not (0 <= nbc < blocks[a]):
                    with pytest.raises(m.CavityError):
                        m.cavity_get_face_buffer(c.h, b, face, 1, 1)
                    continue
                ncut += 1
                # ghosts of this face (filled by the neighbour's pack + this unpack)
                layers_p = [n[a] + 1, n[a] + 2] if hi else [-1, 0]
                layers_v = [n[a] + 1] if hi else [0]
                for f in range(5):
                    for L in (layers_p if f == 0 else layers_v):
                        idx = [slice(2, 2 + n[d]) for d in range(3)]
                        gidx = [slice(org[d] + 2, org[d] + 2 + n[d]) for d in range(3)]
                        idx[a] = L + 1
                        gidx[a] = org[a] + L + 1
                        mine = arrays[b][f][idx[2], idx[1], idx[0]]
                        glob = G[f][gidx[2], gidx[1], gidx[0]]
                        assert np.array_equal(mine, glob), (b, face, f, L)
                # the face buffer this block packed, vs its own array
                bax, cax = [d for d in range(3) if d != a]
                nb, nc = n[bax], n[cax]
                buf = m.cavity_get_face_buffer(c.h, b, face, nb, nc)
                A = arrays[b]
                exp = np.empty(6 * nb * nc)
                for d in range(2):
                    idx = [slice(2, 2 + n[0]), slice(2, 2 + n[1]), slice(2, 2 + n[2])]
                    idx[a] = (n[a] - 1 + d if hi else 1 + d) + 1
                    layer = A[0][idx[2], idx[1], idx[0]]  # [c, b]: flat index ic*nb + ib
                    exp[d:2 * nb * nc:2] = layer.reshape(-1)
                for v in range(4):
                    idx = [slice(2, 2 + n[0]), slice(2, 2 + n[1]), slice(2, 2 + n[2])]
                    idx[a] = (n[a] if hi else 1) + 1
                    layer = A[1 + v][idx[2], idx[1], idx[0]]
                    exp[2 * nb * nc + v * nb * nc: 2 * nb * nc + (v + 1) * nb * nc] = layer.reshape(-1)
                assert np.array_equal(buf, exp), (b, face)
        assert ncut > 0


# ---------------------------------------------------------------------------
def test_invalid_arguments_and_nonfinite(m):
    with m.Cavity(10, 10, 10, Ra=1e4) as c:
        with pytest.raises(m.CavityError) as e:
            m.cavity_get_fields(c.h, (10, 10, 11))
        assert e.value.code == m.CAVITY_ERR_INVALID_ARG
        bad = m.cavity_default_params(Ra=1e4, gravity_axis=0)
        with pytest.raises(m.CavityError):
            m.cavity_set_params(c.h, bad)
        # beta_min^2 = kappa u_ref^2 below FP32's normal range
        for kw in (dict(kappa=1e-40, u_ref=1.0), dict(kappa=1e-10, u_ref=1e-20)):
            with pytest.raises(m.CavityError):
                m.cavity_set_params(c.h, m.cavity_default_params(Ra=1e4, **kw))
        with pytest.raises(m.CavityError):
            m.cavity_step(c.h, -1)
        # host-side injection of a non-finite value: the step flags it
        q = c.fields()
        q[1, 5, 5, 5] = np.inf
        c.set_fields(q)
        c.step(1)
        with pytest.raises(m.CavityError) as e:
            c.residual
        assert e.value.code == m.CAVITY_ERR_NONFINITE
        assert c.sync() == m.CAVITY_ERR_NONFINITE


# ---------------------------------------------------------------------------
# FP32-mixed form: u, v, w, T in FP32, p as an FP32 hi/lo pair, FP64 reductions.
# Against the FP64 oracle: fields <= 1e-5 relative max-norm, Nusselt <= 1e-4.

FP32_TOL = 1e-5
NU32_TOL = 1e-4


def run_pair32(m, n, Ra, steps, blocks=(1, 1, 1), noise=1e-3, seed=0, **kw):
    o = oracle.OracleCavity(*n, dict(Ra=Ra, **kw), noise=noise, seed=seed)
    c = m.Cavity(*n, blocks=blocks, precision=m.CAVITY_FP32_MIXED, seed=seed, noise_amp=noise, Ra=Ra, **kw)
    o.step(steps)
    c.step(steps)
    return o, c


def test_fp32_initial_state(m):
    n = (37, 21, 18)
    o = oracle.OracleCavity(*n, dict(Ra=1e4), noise=1e-3, seed=5)
    with m.Cavity(*n, precision=m.CAVITY_FP32_MIXED, seed=5, noise_amp=1e-3, Ra=1e4) as c:
        g, ref = c.fields(), o.fields()
        # T is stored as an FP32 pair: the initial values survive to ~2^-48
        assert np.max(np.abs(g[4] - ref[4])) <= 1e-14
        assert np.all(g[:4] == 0)


def test_fp32_config1_32cube_200_steps(m):
    cfg = workloads.CFG1
    o, c = run_pair32(m, cfg["n"], cfg["Ra"], cfg["steps"], noise=cfg["noise"], seed=cfg["seed"], Pr=cfg["Pr"])
    with c:
        assert_fields_close(c.fields(), o.fields(), FP32_TOL, "fp32 cfg1")
        h, cold = c.nusselt
        assert abs(h - o.nusselt[0]) <= NU32_TOL * abs(o.nusselt[0])
        assert abs(cold - o.nusselt[1]) <= NU32_TOL * abs(o.nusselt[1])
        assert np.allclose(c.residual, o.residual, rtol=1e-4)
        assert c.time[2] == pytest.approx(o.p["cfl"] / o.spectral_max(), rel=1e-5)


@pytest.mark.parametrize("n", [(37, 21, 18), (2, 2, 2), (2, 11, 9), (3, 10, 7), (65, 9, 40), (33, 17, 70)])
def test_fp32_ragged_and_degenerate_sizes(m, n):
    """Small and ragged cavities: p, u, w and T against their own max-norm; v,
    which the y-mirror symmetry of the cavity keeps near zero (only the noise
    breaks it), against the maximum speed; both Nusselt numbers (nx = 2 puts
    both x walls beside one node pair)."""
    o, c = run_pair32(m, n, 3e4, 25, noise=1e-3, seed=11)
    with c:
        g, ref = c.fields(), o.fields()
        speed = max(np.max(np.abs(ref[f])) for f in (1, 2, 3))
        for f, name in enumerate(oracle.FIELDS):
            scale = speed if f == 2 else np.max(np.abs(ref[f]))
            e = np.max(np.abs(g[f] - ref[f])) / scale
            assert e <= FP32_TOL, f"fp32 n={n} field {name}: {e:.3e}"
        h, cold = c.nusselt
        assert abs(h - o.nusselt[0]) <= NU32_TOL * abs(o.nusselt[0]), (n, h, o.nusselt)
        assert abs(cold - o.nusselt[1]) <= NU32_TOL * abs(o.nusselt[1]), (n, cold, o.nusselt)
        assert np.allclose(c.residual, o.residual, rtol=1e-3), (n, c.residual, o.residual)
        assert c.time[0] == 25 and c.time[1] == pytest.approx(o.t, rel=1e-5)


@pytest.mark.parametrize("blocks", DECOMPS)
def test_fp32_blocks_bit_identical(m, blocks):
    kw = dict(precision=m.CAVITY_FP32_MIXED, seed=9, noise_amp=1e-3, Ra=1e5)
    with m.Cavity(48, 40, 44, **kw) as ref, m.Cavity(48, 40, 44, blocks=blocks, **kw) as c:
        ref.step(60)
        c.step(60)
        assert np.array_equal(c.fields(), ref.fields())
        assert c.time == ref.time


@pytest.mark.parametrize("shape", ["8,32,4,3", "8,40,4,3", "8,32,5,3", "16,32,4,3", "8,96,5,3"])
def test_fp32_tile_shapes_ragged(m, monkeypatch, shape):
    """Each compiled tile shape (two nodes per thread): ragged sizes against
    the oracle (odd nx leaves a lone node in the last pair), and a
    decomposition with odd per-block x extents bit-equal to one block."""
    monkeypatch.setenv("BDC_F32_TILE", shape)
    for n in [(37, 21, 18), (2, 2, 2), (65, 9, 40)]:
        o, c = run_pair32(m, n, 3e4, 25, noise=1e-3, seed=11)
        with c:
            g, ref = c.fields(), o.fields()
            speed = max(np.max(np.abs(ref[f])) for f in (1, 2, 3))
            for f, name in enumerate(oracle.FIELDS):
                scale = speed if f == 2 else np.max(np.abs(ref[f]))
                e = np.max(np.abs(g[f] - ref[f])) / scale
                assert e <= FP32_TOL, f"fp32 {shape} n={n} field {name}: {e:.3e}"
            for got, want in zip(c.nusselt, o.nusselt):
                assert abs(got - want) <= NU32_TOL * abs(want), (shape, n, c.nusselt, o.nusselt)
    kw = dict(precision=m.CAVITY_FP32_MIXED, seed=9, noise_amp=1e-3, Ra=1e5)
    with m.Cavity(47, 40, 44, **kw) as ref, m.Cavity(47, 40, 44, blocks=(3, 2, 2), **kw) as c:
        ref.step(60)
        c.step(60)
        assert np.array_equal(c.fields(), ref.fields())
        assert c.time == ref.time


def test_fp32_ghosts_and_buffers_bit_exact(m):
    blocks = (2, 2, 2)
    kw = dict(precision=m.CAVITY_FP32_MIXED, seed=9, noise_amp=1e-3, Ra=1e5)
    with m.Cavity(48, 40, 44, **kw) as ref, m.Cavity(48, 40, 44, blocks=blocks, **kw) as c:
        ref.step(30)
        c.step(30)
        NA = 7  # p_hi, p_lo, u, v, w, T_hi, T_lo
        G = [m.cavity_get_block_array(ref.h, 0, f)[0] for f in range(NA)]
        for b in range(8):
            arrs = [m.cavity_get_block_array(c.h, b, f)[0] for f in range(NA)]
            nx, ny, nz, ox, oy, oz = m.cavity_get_block_array(c.h, b, 0)[1]
            n, org = (nx, ny, nz), (ox, oy, oz)
            coords = [b % 2, (b // 2) % 2, b // 4]
            for face in range(6):
                a, hi = face // 2, face % 2
                if not (0 <= coords[a] + (1 if hi else -1) < 2):
                    continue
                for f in range(NA):
                    for L in ([n[a] + 1, n[a] + 2] if hi else [-1, 0]) if f < 2 else ([n[a] + 1] if hi else [0]):
                        idx = [slice(2, 2 + n[d]) for d in range(3)]
                        gidx = [slice(org[d] + 2, org[d] + 2 + n[d]) for d in range(3)]
                        idx[a], gidx[a] = L + 1, org[a] + L + 1
                        assert np.array_equal(arrs[f][idx[2], idx[1], idx[0]], G[f][gidx[2], gidx[1], gidx[0]])
                bax, cax = [d for d in range(3) if d != a]
                nb, nc = n[bax], n[cax]
                buf = m.load_library()
                out = np.empty(9 * nb * nc)
                rc = buf.cavity_get_face_buffer(c.h, b, face, out.ctypes.data_as(m._dp), out.size)
                assert rc == 0
                exp = np.empty(9 * nb * nc)
                for pa in range(2):
                    for d in range(2):
                        idx = [slice(2, 2 + n[0]), slice(2, 2 + n[1]), slice(2, 2 + n[2])]
                        idx[a] = (n[a] - 1 + d if hi else 1 + d) + 1
                        exp[2 * pa * nb * nc + d:2 * (pa + 1) * nb * nc:2] = arrs[pa][idx[2], idx[1], idx[0]].reshape(-1)
                for v in range(5):  # u, v, w, T_hi, T_lo
                    idx = [slice(2, 2 + n[0]), slice(2, 2 + n[1]), slice(2, 2 + n[2])]
                    idx[a] = (n[a] if hi else 1) + 1
                    exp[4 * nb * nc + v * nb * nc:4 * nb * nc + (v + 1) * nb * nc] = \
                        arrs[2 + v][idx[2], idx[1], idx[0]].reshape(-1)
                assert np.array_equal(out, exp), (b, face)


@pytest.mark.parametrize("shape", ["8,16,4,3", "16,32,5,3"])
def test_fp32_exchange_straddling_tiles(m, monkeypatch, shape):
    """The step's exchange (Section 4.5 pack and unpack) with blocks of
    33 x 17 x 17, so that these tile shapes split a face's two p layers
    (n-1, n) across x tiles, y tiles and z chunks: the result equals one
    block bit for bit, and a second pack + unpack of the same state changes
    no ghost node and no buffer entry."""
    monkeypatch.setenv("BDC_F32_TILE", shape)
    L = m.load_library()
    kw = dict(precision=m.CAVITY_FP32_MIXED, seed=5, noise_amp=1e-3, Ra=2e5)
    with m.Cavity(66, 34, 34, **kw) as ref, m.Cavity(66, 34, 34, blocks=(2, 2, 2), **kw) as c:
        ref.step(40)
        c.step(40)
        assert np.array_equal(c.fields(), ref.fields())

        def snapshot():
            arrs = [[m.cavity_get_block_array(c.h, b, f)[0] for f in range(7)] for b in range(8)]
            bufs = []
            for b in range(8):
                coords = [b % 2, (b // 2) % 2, b // 4]
                n = m.cavity_get_block_array(c.h, b, 0)[1][:3]
                for face in range(6):
                    a, hi = face // 2, face % 2
                    if not (0 <= coords[a] + (1 if hi else -1) < 2):
                        continue
                    nb, nc = [n[d] for d in range(3) if d != a]
                    out = np.empty(9 * nb * nc)
                    assert L.cavity_get_face_buffer(c.h, b, face, out.ctypes.data_as(m._dp), out.size) == 0
                    bufs.append(out)
            return arrs, bufs

        arrs0, bufs0 = snapshot()
        m.cavity_exchange(c.h)
        arrs1, bufs1 = snapshot()
        for b in range(8):
            for f in range(7):
                assert np.array_equal(arrs0[b][f], arrs1[b][f]), (shape, b, f)
        assert len(bufs0) == 24
        for x, y in zip(bufs0, bufs1):
            assert np.array_equal(x, y)


def test_fp32_set_fields_wall_field_and_nonfinite(m):
    n = (28, 22, 19)
    q = workloads.smooth_state(n, seed=3)
    th = workloads.wall_temperature(n[1], n[2], seed=4)
    o = oracle.OracleCavity(*n, dict(Ra=5e4), t_hot_wall=th)
    o.set_fields(q)
    with m.Cavity(*n, precision=m.CAVITY_FP32_MIXED, Ra=5e4) as c:
        m.cavity_set_wall_temperature(c.h, 0, th)
        c.set_fields(q)
        g = c.fields()
        assert np.max(np.abs(g[0] - q[0])) <= 1e-12 * np.max(np.abs(q[0]))  # the hi/lo pair keeps p
        assert np.array_equal(g[1:4], q[1:4].astype(np.float32).astype(np.float64))
        assert np.max(np.abs(g[4] - q[4])) <= 1e-14 * np.max(np.abs(q[4]))  # and the T pair keeps T
        o.step(30)
        c.step(30)
        assert_fields_close(c.fields(), o.fields(), FP32_TOL, "fp32 set_fields")
        q2 = c.fields()
        q2[3, 4, 4, 4] = np.nan
        c.set_fields(q2)
        c.step(1)
        assert c.sync() == m.CAVITY_ERR_NONFINITE
