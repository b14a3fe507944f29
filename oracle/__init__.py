"""FP64 CPU oracle of the buoyancy-driven-cavity step (Xue & Roy, arXiv 2006.02602).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_2006_02602_gb300``)
and imports nothing from it; the per-point arithmetic lives in
``bdc_oracle.c`` (plain loops, FP64, ``-ffp-contract=off``) and this module
only orchestrates the loops over blocks in the order of one explicit step:

  a1  dt = cfl / max spectral-radius bound over the interior     (Section 2)
  a2  dq/dt from Eqs. 1-3 at every interior node                 (Eqs. 1-3, Section 3.1)
  a3  explicit Euler update, residual sums of (dq/dt)^2          (Section 2; Section 4.2 norms)
  a5  pressure rescaled at the centre                            (Section 2)
  a6  wall boundary conditions                                   (Section 2)
  a7  pack each cut face into a contiguous buffer                (Section 4.5, Listings 1-2, V3)
  a8  unpack buffers into the neighbours' ghost layers           (Section 4.5)
  a9  hot/cold wall Nusselt numbers                              (configuration text)

The multi-block form splits the cavity by the Section 3.2 rule (as even as
possible) and exchanges ghosts only through ``orc_pack`` / ``orc_unpack``;
its fields must equal the single-block run bit for bit.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bdc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libbdc_oracle.so")
_lock = threading.Lock()
_lib = None

NF = 5
FIELDS = ("p", "u", "v", "w", "T")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("Ra", ctypes.c_double), ("Pr", ctypes.c_double), ("cfl", ctypes.c_double),
                ("kappa", ctypes.c_double), ("c4", ctypes.c_double), ("u_ref", ctypes.c_double),
                ("t_inf", ctypes.c_double), ("t_hot", ctypes.c_double), ("t_cold", ctypes.c_double),
                ("gravity_axis", ctypes.c_int)]


class _Block(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("ox", ctypes.c_int), ("oy", ctypes.c_int), ("oz", ctypes.c_int),
                ("gnx", ctypes.c_int), ("gny", ctypes.c_int), ("gnz", ctypes.c_int),
                ("wall", ctypes.c_int * 6)]


_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P, B = ctypes.POINTER(_Params), ctypes.POINTER(_Block)
            L.orc_splitmix64.argtypes = [ctypes.c_uint64]
            L.orc_splitmix64.restype = ctypes.c_uint64
            L.orc_block_points.argtypes = [B]
            L.orc_block_points.restype = ctypes.c_size_t
            L.orc_init.argtypes = [P, B, _dp, ctypes.c_uint64, ctypes.c_double]
            L.orc_rates.argtypes = [P, B, _dp, _dp]
            L.orc_spectral_max.argtypes = [P, B, _dp]
            L.orc_spectral_max.restype = ctypes.c_double
            L.orc_update.argtypes = [B, _dp, _dp, ctypes.c_double, _dp]
            L.orc_update_local.argtypes = [ctypes.POINTER(_Params), B, _dp, _dp, _dp]
            L.orc_shift_pressure.argtypes = [B, _dp, ctypes.c_double]
            L.orc_bc.argtypes = [B, _dp, _dp, _dp]
            L.orc_nusselt_sums.argtypes = [P, B, _dp, _dp, _dp]
            L.orc_face_len.argtypes = [B, ctypes.c_int]
            L.orc_face_len.restype = ctypes.c_size_t
            L.orc_pack.argtypes = [B, _dp, ctypes.c_int, _dp]
            L.orc_unpack.argtypes = [B, _dp, ctypes.c_int, _dp]
            L.orc_rates_vjp.argtypes = [P, B, _dp, _dp, _dp, _dp]
            L.orc_spectral_argmax.argtypes = [P, B, _dp, ctypes.POINTER(ctypes.c_int)]
            L.orc_spectral_argmax.restype = ctypes.c_double
            L.orc_spectral_vjp.argtypes = [P, B, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           _dp, _dp]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def default_params(**kw) -> dict:
    """Nondimensional parameters (thermal scaling) with the defaults of the readings."""
    p = dict(Ra=1e4, Pr=0.71, cfl=0.5, kappa=0.1, c4=1.0 / 32.0, u_ref=None, t_inf=None,
             t_hot=1.0, t_cold=0.0, gravity_axis=2)
    p.update(kw)
    if p["u_ref"] is None:
        p["u_ref"] = max(1.0, math.sqrt(p["Ra"] * p["Pr"]))
    if p["t_inf"] is None:
        p["t_inf"] = 0.5 * (p["t_hot"] + p["t_cold"])
    return p


def _cparams(p: dict) -> _Params:
    return _Params(p["Ra"], p["Pr"], p["cfl"], p["kappa"], p["c4"], p["u_ref"], p["t_inf"],
                   p["t_hot"], p["t_cold"], int(p["gravity_axis"]))


def split_sizes(n: int, parts: int) -> list[int]:
    """Section 3.2: divide as evenly as possible (the first blocks take the remainder)."""
    base, rem = divmod(n, parts)
    return [base + (1 if r < rem else 0) for r in range(parts)]


def centre_nodes(gn: tuple[int, int, int]) -> list[tuple[int, int, int]]:
    """Global (I, J, K) of the 2^m nodes nearest the cavity centre, in (k, j, i) lexicographic order."""
    ax = []
    for n in gn:
        ax.append([(n + 1) // 2] if n % 2 == 1 else [n // 2, n // 2 + 1])
    return [(i, j, k) for k in ax[2] for j in ax[1] for i in ax[0]]


def rates(params: dict, q: np.ndarray, gn=None, origin=(0, 0, 0)) -> np.ndarray:
    """dq/dt (Eqs. 1-3) at the interior of a full array q[5, nz+4, ny+4, nx+4]."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    nz, ny, nx = (s - 4 for s in q.shape[1:])
    gn = gn or (nx, ny, nz)
    b = _Block(nx, ny, nz, *origin, *gn, (ctypes.c_int * 6)(1, 1, 1, 1, 1, 1))
    out = np.empty((NF, nz, ny, nx))
    lib().orc_rates(ctypes.byref(_cparams(params)), ctypes.byref(b), _ptr(q), _ptr(out))
    return out


def apply_bc(q: np.ndarray, t_hot_w: np.ndarray, t_cold_w: np.ndarray) -> None:
    """Apply the wall conditions in place on a single-block full array."""
    nz, ny, nx = (s - 4 for s in q.shape[1:])
    b = _Block(nx, ny, nz, 0, 0, 0, nx, ny, nz, (ctypes.c_int * 6)(1, 1, 1, 1, 1, 1))
    lib().orc_bc(ctypes.byref(b), _ptr(q), _ptr(np.ascontiguousarray(t_hot_w, dtype=np.float64)),
                 _ptr(np.ascontiguousarray(t_cold_w, dtype=np.float64)))


class _Blk:
    def __init__(self, c: _Block, bid: int, coords: tuple[int, int, int]):
        self.c = c
        self.id = bid
        self.coords = coords
        self.q = np.zeros((NF, c.nz + 4, c.ny + 4, c.nx + 4))
        self.dq = np.zeros((NF, c.nz, c.ny, c.nx))
        self.nbr = [-1] * 6


class OracleCavity:
    """One cavity, optionally split into px*py*pz blocks exchanging ghost faces."""

    def __init__(self, nx, ny, nz, params: dict | None = None, blocks=(1, 1, 1), seed: int = 0,
                 noise: float = 0.0, t_hot_wall=None, t_cold_wall=None, local_dt: bool = False):
        self.L = lib()
        self.local_dt = bool(local_dt)  # local time stepping: each node at dt_n = cfl / S_n
        self.p = default_params(**(params or {}))
        self.cp = _cparams(self.p)
        self.gn = (int(nx), int(ny), int(nz))
        self.nint = nx * ny * nz
        self.pgrid = tuple(int(v) for v in blocks)
        th = np.full(ny * nz, self.p["t_hot"]) if t_hot_wall is None else t_hot_wall
        tc = np.full(ny * nz, self.p["t_cold"]) if t_cold_wall is None else t_cold_wall
        self.t_hot_w = np.ascontiguousarray(np.asarray(th, dtype=np.float64).reshape(-1))
        self.t_cold_w = np.ascontiguousarray(np.asarray(tc, dtype=np.float64).reshape(-1))
        assert self.t_hot_w.size == ny * nz and self.t_cold_w.size == ny * nz
        sx, sy, sz = (split_sizes(n, pp) for n, pp in zip(self.gn, self.pgrid))
        ox = np.concatenate([[0], np.cumsum(sx)])
        oy = np.concatenate([[0], np.cumsum(sy)])
        oz = np.concatenate([[0], np.cumsum(sz)])
        px, py, pz = self.pgrid
        self.blocks: list[_Blk] = []
        for bz in range(pz):
            for by in range(py):
                for bx in range(px):
                    wall = (ctypes.c_int * 6)(int(bx == 0), int(bx == px - 1), int(by == 0),
                                              int(by == py - 1), int(bz == 0), int(bz == pz - 1))
                    c = _Block(sx[bx], sy[by], sz[bz], int(ox[bx]), int(oy[by]), int(oz[bz]),
                               nx, ny, nz, wall)
                    blk = _Blk(c, len(self.blocks), (bx, by, bz))
                    self.blocks.append(blk)
        for blk in self.blocks:
            bx, by, bz = blk.coords
            for face in range(6):
                a, hi = face // 2, face % 2
                cc = [bx, by, bz]
                cc[a] += 1 if hi else -1
                if 0 <= cc[a] < self.pgrid[a]:
                    blk.nbr[face] = cc[0] + px * (cc[1] + py * cc[2])
        self.dt = 0.0
        self.t = 0.0
        self.nstep = 0
        self.residual = np.zeros(NF)
        self.nusselt = (0.0, 0.0)
        for blk in self.blocks:
            self.L.orc_init(ctypes.byref(self.cp), ctypes.byref(blk.c), _ptr(blk.q),
                            ctypes.c_uint64(seed), noise)
        self._finish_state()

    # -- helpers --------------------------------------------------------
    def _locate(self, I, J, K):
        for blk in self.blocks:
            c = blk.c
            if c.ox < I <= c.ox + c.nx and c.oy < J <= c.oy + c.ny and c.oz < K <= c.oz + c.nz:
                return blk, I - c.ox, J - c.oy, K - c.oz
        raise IndexError((I, J, K))

    def _bc_and_exchange(self):
        for blk in self.blocks:
            self.L.orc_bc(ctypes.byref(blk.c), _ptr(blk.q), _ptr(self.t_hot_w), _ptr(self.t_cold_w))
        self.exchange()

    def exchange(self):
        """a7/a8: pack every cut face, then unpack into the neighbour's ghosts."""
        bufs = {}
        for blk in self.blocks:
            for face in range(6):
                if blk.nbr[face] >= 0:
                    buf = np.empty(self.L.orc_face_len(ctypes.byref(blk.c), face))
                    self.L.orc_pack(ctypes.byref(blk.c), _ptr(blk.q), face, _ptr(buf))
                    bufs[(blk.id, face)] = buf
        for (bid, face), buf in bufs.items():
            dst = self.blocks[self.blocks[bid].nbr[face]]
            self.L.orc_unpack(ctypes.byref(dst.c), _ptr(dst.q), face ^ 1, _ptr(buf))
        return bufs

    def pack_buffers(self):
        """Contiguous face buffers of the current state, keyed by (block, face)."""
        out = {}
        for blk in self.blocks:
            for face in range(6):
                if blk.nbr[face] >= 0:
                    buf = np.empty(self.L.orc_face_len(ctypes.byref(blk.c), face))
                    self.L.orc_pack(ctypes.byref(blk.c), _ptr(blk.q), face, _ptr(buf))
                    out[(blk.id, face)] = buf
        return out

    def _nusselt(self):
        sh = sc = 0.0
        for blk in self.blocks:
            h, c = ctypes.c_double(), ctypes.c_double()
            self.L.orc_nusselt_sums(ctypes.byref(self.cp), ctypes.byref(blk.c), _ptr(blk.q),
                                    ctypes.byref(h), ctypes.byref(c))
            sh += h.value
            sc += c.value
        n = self.gn[1] * self.gn[2]
        return sh / n, sc / n

    def spectral_max(self):
        return max(self.L.orc_spectral_max(ctypes.byref(self.cp), ctypes.byref(b.c), _ptr(b.q))
                   for b in self.blocks)

    def centre_value(self):
        """Mean of p over the centre nodes, summed in (k, j, i) order."""
        nodes = centre_nodes(self.gn)
        s = 0.0
        for (I, J, K) in nodes:
            blk, i, j, k = self._locate(I, J, K)
            s += blk.q[0, k + 1, j + 1, i + 1]
        return s / len(nodes)

    def _finish_state(self):
        self._bc_and_exchange()
        self.nusselt = self._nusselt()

    # -- the explicit step ------------------------------------------------
    def step(self, n: int = 1):
        cp = ctypes.byref(self.cp)
        for _ in range(int(n)):
            self.dt = self.p["cfl"] / self.spectral_max()                       # a1
            for blk in self.blocks:                                             # a2
                self.L.orc_rates(cp, ctypes.byref(blk.c), _ptr(blk.q), _ptr(blk.dq))
            tot = np.zeros(NF)
            for blk in self.blocks:                                             # a3
                s = np.zeros(NF)
                if self.local_dt:  # each node at its own stable step (pseudo time)
                    self.L.orc_update_local(cp, ctypes.byref(blk.c), _ptr(blk.q), _ptr(blk.dq), _ptr(s))
                else:
                    self.L.orc_update(ctypes.byref(blk.c), _ptr(blk.q), _ptr(blk.dq), self.dt, _ptr(s))
                tot += s
            self.residual = np.sqrt(tot / self.nint)
            c = self.centre_value()                                             # a5
            for blk in self.blocks:
                self.L.orc_shift_pressure(ctypes.byref(blk.c), _ptr(blk.q), c)
            self._bc_and_exchange()                                             # a6-a8
            self.nusselt = self._nusselt()                                      # a9
            self.t += self.dt
            self.nstep += 1
        return self

    # -- state access -----------------------------------------------------
    def fields(self) -> np.ndarray:
        """Interior fields [5, nz, ny, nx] of the whole cavity (p, u, v, w, T)."""
        nx, ny, nz = self.gn
        out = np.empty((NF, nz, ny, nx))
        for blk in self.blocks:
            c = blk.c
            out[:, c.oz:c.oz + c.nz, c.oy:c.oy + c.ny, c.ox:c.ox + c.nx] = \
                blk.q[:, 2:c.nz + 2, 2:c.ny + 2, 2:c.nx + 2]
        return out

    def set_fields(self, interior: np.ndarray):
        """Overwrite the interior fields, then re-apply walls and exchange ghosts."""
        for blk in self.blocks:
            c = blk.c
            blk.q[:, 2:c.nz + 2, 2:c.ny + 2, 2:c.nx + 2] = \
                interior[:, c.oz:c.oz + c.nz, c.oy:c.oy + c.ny, c.ox:c.ox + c.nx]
        self._finish_state()

    def full_array(self) -> np.ndarray:
        """Single-block only: the whole array including walls and pressure ghosts."""
        assert len(self.blocks) == 1
        return self.blocks[0].q


# ---------------------------------------------------------------------------
# Discrete adjoint of the explicit step (single block).  Objective: the
# hot-wall Nusselt number averaged over steps 1..N,
#     J = (1/N) sum_n Nu_hot(Q^n),
# controls: the hot-wall temperature field theta (ny*nz) and Ra.  One step
# Q^{n+1} = G(Q^n) is: dt = cfl / max_m sr(Q^n_m); Q~ = Q^n + dt R(Q^n);
# p = p~ - mean_centre(p~); walls from the new interior and theta.  Its
# adjoint, in reverse order: gauge, update (identity + dt R^T via the C
# reverse of the rates), dt through the argmax node of the spectral bound,
# then the wall values folded back onto the interior nodes they were formed
# from (and onto theta for the hot-wall temperature).

def _fold_walls(cav: "OracleCavity", qbar: np.ndarray, thetabar: np.ndarray) -> None:
    """Adjoint of the wall conditions: move wall/ghost adjoints of qbar
    (full array) onto interior nodes 1, 2 and, for the hot wall's T, onto theta."""
    c = cav.blocks[0].c
    n = (c.nx, c.ny, c.nz)
    for face in range(6):
        a, hi = face // 2, face % 2
        w = n[a] + 1 if hi else 0
        s = -1 if hi else 1

        def sl(node):  # [f, k, j, i] slices of one layer along axis a over the face interior
            idx = [slice(2, 2 + n[0]), slice(2, 2 + n[1]), slice(2, 2 + n[2])]
            idx[a] = node + 1
            return (idx[2], idx[1], idx[0])

        W, N1, N2, G = sl(w), sl(w + s), sl(w + 2 * s), sl(w - s)
        P = qbar[0]
        pw, pg = P[W].copy(), P[G].copy()
        P[N1] += 2.0 * pw + 3.0 * pg      # p_w = 2 p1 - p2, p_g = 2 p_w - p1 = 3 p1 - 2 p2
        P[N2] += -pw - 2.0 * pg
        P[W] = 0.0
        P[G] = 0.0
        T = qbar[4]
        tw = T[W].copy()
        if a == 0:
            if not hi:  # hot wall: T_w = theta(j, k), theta index (j-1) + ny (k-1)
                thetabar += tw.reshape(-1)
        else:
            T[N1] += (4.0 / 3.0) * tw        # T_w = (4 T1 - T2) / 3
            T[N2] += (-1.0 / 3.0) * tw
        T[W] = 0.0
        for f in (1, 2, 3):
            qbar[f][W] = 0.0


def nusselt_gradient(nx, ny, nz, params: dict, steps: int, seed: int = 0, noise: float = 0.0,
                     t_hot_wall=None):
    """J = mean over steps 1..N of Nu_hot, and dJ/dtheta (ny*nz), dJ/dRa by the
    discrete adjoint.  params may leave u_ref unset so that it follows Ra."""
    L = lib()
    floor_follows_ra = params.get("u_ref") is None  # u_ref = max(1, sqrt(Ra Pr))
    cav = OracleCavity(nx, ny, nz, params, noise=noise, seed=seed, t_hot_wall=t_hot_wall)
    blk = cav.blocks[0]
    cp = ctypes.byref(cav.cp)
    cb = ctypes.byref(blk.c)
    N = int(steps)
    traj, dts, argm, smaxes = [], [], [], []
    J = 0.0
    for _ in range(N):
        q = blk.q.copy()
        idx = (ctypes.c_int * 3)()
        smax = L.orc_spectral_argmax(cp, cb, _ptr(q), idx)
        traj.append(q)
        argm.append((idx[0], idx[1], idx[2]))
        smaxes.append(smax)
        cav.step(1)
        dts.append(cav.dt)
        J += cav.nusselt[0]
    J /= N
    p = cav.p
    hx = 1.0 / (nx + 1)
    coef = 1.0 / (N * ny * nz * 2.0 * hx * (p["t_hot"] - p["t_cold"]))
    xbar = np.zeros((NF, nz, ny, nx))
    thetabar = np.zeros(ny * nz)
    rabar = 0.0
    centre = centre_nodes((nx, ny, nz))
    # beta^2 floor kappa u_ref^2 = kappa max(1, Ra Pr) when u_ref follows Ra
    dfloor_dra = p["kappa"] * p["Pr"] if (floor_follows_ra and p["Ra"] * p["Pr"] > 1.0) else 0.0
    for n in range(N, 0, -1):
        # objective term of Q^n: (3 theta - 4 T_1 + T_2) / (2 h_x dT), averaged
        xbar[4][:, :, 0] += -4.0 * coef
        xbar[4][:, :, 1] += coef
        thetabar += 3.0 * coef
        q = traj[n - 1]
        # gauge: p = p~ - mean_centre(p~)
        ytil = xbar.copy()
        ssum = ytil[0].sum()
        for (I, J_, K) in centre:
            ytil[0][K - 1, J_ - 1, I - 1] -= ssum / len(centre)
        # update: X~ = X + dt R(Q)
        dt = dts[n - 1]
        R = rates(p, q)
        dtbar = float(np.sum(ytil * R))
        rbar = np.ascontiguousarray(dt * ytil)
        qbar = np.zeros_like(q)
        qbar[:, 2:-2, 2:-2, 2:-2] = ytil
        pbar = np.zeros(2)
        L.orc_rates_vjp(cp, cb, _ptr(q), _ptr(rbar), _ptr(qbar), _ptr(pbar))
        # dt = cfl / S, S = spectral bound at the argmax node
        S = smaxes[n - 1]
        sbar = -p["cfl"] * dtbar / (S * S)
        i, j, k = argm[n - 1]
        L.orc_spectral_vjp(cp, cb, _ptr(q), i, j, k, sbar, _ptr(qbar), _ptr(pbar))
        _fold_walls(cav, qbar, thetabar)
        xbar = qbar[:, 2:-2, 2:-2, 2:-2].copy()
        rabar += p["Pr"] * pbar[0] + dfloor_dra * pbar[1]
    return J, thetabar, rabar
