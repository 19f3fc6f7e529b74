"""Seeded synthetic inputs for the hygrothermal wall workloads.

This module only draws numbers: wall geometries, layer splits, material
parameters, boundary forcing descriptions and noise tables. It contains none
of the Dufort-Frankel arithmetic, so both the CUDA library binding and the
FP64 CPU oracle can be fed from it without sharing any of the method.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used in counter form: the i-th
output of the stream with key k is mix(k + (i + 1) * 0x9E3779B97F4A7C15).
Gaussian noise uses the Box-Muller transform.

Workloads (their shapes follow the paper's wall problems, Sec. 2 and Sec. 4,
with the ranges of the standard benchmark configurations):
  * ``single_wall``: one 10 cm wall, 101 nodes, dt = 60 s, one day.
  * ``wall_batch``: a batch of ragged multi-layer walls (default 4096 walls of
    50..400 nodes, dt = 600 s, one year, hourly Gaussian noise on face 0).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Physical constants used to build the inputs (not the method).
PSAT_REF = 2337.0        # Pa, saturation pressure at 20 C
LV = 2.5e6               # J/kg, latent heat of evaporation

# log10 range of the moisture storage coefficient of the batch workloads:
# cM of the paper's Table 2 walls spans 1.82e-2 .. 1.18e-1 s2/m2.
CM0_LOG10_RANGE = (math.log10(1.8e-2), math.log10(1.2e-1))

# Boundary kinds (shared numbering with the C ABI and the oracle).
BC_AMBIENT = 0           # sinusoid + optional hourly noise table
BC_ADIABATIC = 1         # no exchange through this face
BC_ROOM = 2              # face exposed to a room air node

# Column order of a boundary parameter row.
BC_FIELDS = ("hT", "hM", "q_inf", "g_inf", "T_mean", "T_amp", "P_mean",
             "P_amp", "period", "phase_T", "phase_P", "noise_dt", "period_P")
# Column order of a layer parameter row.
LAYER_FIELDS = ("kM0", "a", "cM0", "b", "kTT0", "aT", "cTT0", "bT", "chi")


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream) -> np.ndarray:
    """Key of an independent stream (vectorised over ``stream``)."""
    s = np.asarray(stream, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ _mix(s * GOLDEN + np.uint64(1)))


def uniform(key, counter) -> np.ndarray:
    """Uniform doubles in [0, 1) for (key, counter), broadcast together."""
    k = np.asarray(key, dtype=np.uint64)
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix(k + (c + np.uint64(1)) * GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal_pairs(key, counter) -> tuple[np.ndarray, np.ndarray]:
    """Box-Muller pair from the uniforms at counters 2c and 2c+1."""
    c = np.asarray(counter, dtype=np.uint64)
    u1 = 1.0 - uniform(key, c * np.uint64(2))        # (0, 1]
    u2 = uniform(key, c * np.uint64(2) + np.uint64(1))
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


@dataclasses.dataclass
class Workload:
    """A batch of 1D walls, their materials, boundaries and time grid."""
    name: str
    n_nodes: np.ndarray          # int32 [n_walls]
    thickness: np.ndarray        # float64 [n_walls], metres
    n_layers: np.ndarray         # int32 [n_walls]
    layer_first: np.ndarray      # int32 [sum n_layers], first local node of each layer
    layer_par: np.ndarray        # float64 [sum n_layers, 9] (LAYER_FIELDS)
    T_init: np.ndarray           # float64 [n_walls], K
    P_init: np.ndarray           # float64 [n_walls], Pa
    bc_kind: np.ndarray          # int32 [n_walls, 2]
    bc_par: np.ndarray           # float64 [n_walls, 2, 13] (BC_FIELDS)
    bc_room: np.ndarray          # int32 [n_walls, 2], room index for BC_ROOM faces, else -1
    noise: list                  # per face: float32 [n_walls, noise_len, 2] (T, Pv) or None
    dt: float
    t0: float
    n_steps: int
    Lv: float = LV
    Psat: float = PSAT_REF
    rooms: dict | None = None    # room description (whole-building workloads)
    vapour_frac: np.ndarray | None = None   # float64 [n_walls]: kTM = nu Lv kM inside the wall (None: 1)
    layer_law: np.ndarray | None = None     # int32 [sum n_layers]: coefficient law of each layer (None: affine)

    @property
    def n_walls(self) -> int:
        return int(self.n_nodes.shape[0])

    @property
    def total_nodes(self) -> int:
        return int(self.n_nodes.sum())

    def layer_offset(self) -> np.ndarray:
        off = np.zeros(self.n_walls + 1, dtype=np.int64)
        np.cumsum(self.n_layers, out=off[1:])
        return off

    def subset(self, walls) -> "Workload":
        """The same problem restricted to the listed walls (no rooms)."""
        walls = np.asarray(walls, dtype=np.int64)
        off = self.layer_offset()
        rows = np.concatenate([np.arange(off[w], off[w + 1]) for w in walls]) if len(walls) else np.zeros(0, np.int64)
        noise = [None if nz is None else np.ascontiguousarray(nz[walls]) for nz in self.noise]
        return dataclasses.replace(
            self, name=f"{self.name}[subset {len(walls)}]",
            n_nodes=self.n_nodes[walls].copy(), thickness=self.thickness[walls].copy(),
            n_layers=self.n_layers[walls].copy(), layer_first=self.layer_first[rows].copy(),
            layer_par=self.layer_par[rows].copy(), T_init=self.T_init[walls].copy(),
            P_init=self.P_init[walls].copy(), bc_kind=self.bc_kind[walls].copy(),
            bc_par=self.bc_par[walls].copy(), bc_room=self.bc_room[walls].copy(),
            noise=noise, rooms=None,
            vapour_frac=None if self.vapour_frac is None else self.vapour_frac[walls].copy(),
            layer_law=None if self.layer_law is None else self.layer_law[rows].copy())


def _bc_row(hT, hM, T_mean, T_amp, P_mean, P_amp, period=86400.0, phase_T=0.0,
            phase_P=0.0, noise_dt=3600.0, q_inf=0.0, g_inf=0.0, period_P=0.0) -> np.ndarray:
    return np.array([hT, hM, q_inf, g_inf, T_mean, T_amp, P_mean, P_amp, period,
                     phase_T, phase_P, noise_dt, period_P], dtype=np.float64)


def uniform_wall(N: int, L: float, layer: dict, **kw) -> Workload:
    """A single one-layer wall; ``layer`` maps LAYER_FIELDS names to values."""
    return layered_wall([N], L, [layer], **kw)


def layered_wall(counts, L: float, layers, *, T0=293.0, P0=1000.0,
                 bc0: dict | None = None, bc1: dict | None = None, dt=60.0,
                 n_steps=100, t0=0.0, Lv=LV, Psat=PSAT_REF, kinds=(BC_AMBIENT, BC_AMBIENT),
                 name="wall") -> Workload:
    """A single wall whose layer l holds ``counts[l]`` consecutive nodes."""
    N = int(sum(counts))
    first = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int32)
    par = np.array([[lay.get(k, 0.0) for k in LAYER_FIELDS] for lay in layers], dtype=np.float64)
    rows = []
    for bc in (bc0, bc1):
        bc = dict(bc or {})
        rows.append(_bc_row(bc.get("hT", 0.0), bc.get("hM", 0.0), bc.get("T_mean", T0),
                            bc.get("T_amp", 0.0), bc.get("P_mean", P0), bc.get("P_amp", 0.0),
                            bc.get("period", 86400.0), bc.get("phase_T", 0.0),
                            bc.get("phase_P", 0.0), bc.get("noise_dt", 3600.0),
                            bc.get("q_inf", 0.0), bc.get("g_inf", 0.0), bc.get("period_P", 0.0)))
    return Workload(
        name=name, n_nodes=np.array([N], np.int32), thickness=np.array([L], np.float64),
        n_layers=np.array([len(counts)], np.int32), layer_first=first, layer_par=par,
        T_init=np.array([T0]), P_init=np.array([P0]),
        bc_kind=np.array([list(kinds)], np.int32), bc_par=np.stack(rows)[None],
        bc_room=np.full((1, 2), -1, np.int32), noise=[None, None], dt=dt, t0=t0,
        n_steps=n_steps, Lv=Lv, Psat=Psat)


def concat(workloads: list[Workload], name="batch") -> Workload:
    """Stack several single- or multi-wall workloads with the same time grid."""
    w0 = workloads[0]
    noise = []
    for f in range(2):
        if all(w.noise[f] is None for w in workloads):
            noise.append(None)
            continue
        ln = max(w.noise[f].shape[1] for w in workloads if w.noise[f] is not None)
        parts = []
        for w in workloads:
            z = np.zeros((w.n_walls, ln, 2), np.float32)
            if w.noise[f] is not None:
                z[:, : w.noise[f].shape[1]] = w.noise[f]
            parts.append(z)
        noise.append(np.concatenate(parts))
    return dataclasses.replace(
        w0, name=name,
        n_nodes=np.concatenate([w.n_nodes for w in workloads]),
        thickness=np.concatenate([w.thickness for w in workloads]),
        n_layers=np.concatenate([w.n_layers for w in workloads]),
        layer_first=np.concatenate([w.layer_first for w in workloads]),
        layer_par=np.concatenate([w.layer_par for w in workloads]),
        T_init=np.concatenate([w.T_init for w in workloads]),
        P_init=np.concatenate([w.P_init for w in workloads]),
        bc_kind=np.concatenate([w.bc_kind for w in workloads]),
        bc_par=np.concatenate([w.bc_par for w in workloads]),
        bc_room=np.concatenate([w.bc_room for w in workloads]),
        noise=noise, rooms=None,
        vapour_frac=None if all(w.vapour_frac is None for w in workloads) else np.concatenate(
            [np.ones(w.n_walls) if w.vapour_frac is None else w.vapour_frac for w in workloads]),
        layer_law=None if all(w.layer_law is None for w in workloads) else np.concatenate(
            [np.zeros(len(w.layer_par), np.int32) if w.layer_law is None else w.layer_law for w in workloads]))


def single_wall(seed: int = 1) -> Workload:
    """One 10 cm wall, N = 101, dt = 60 s, 1440 steps (one day), FP64 case.

    kM = kM0 (1 + a Pv/Psat), cM = cM0 (1 + b Pv/Psat) with a, b ~ U[0, 1]
    and the phase of the vapour-pressure sinusoid ~ U[0, 2 pi). Face 0 sees
    293 + 10 sin(2 pi t/86400) K and 1200 + 400 sin(2 pi t/86400 + phi) Pa
    with hT = 25, hM = 2e-8; face 1 stays at 293 K / 1000 Pa with hT = 8,
    hM = 3e-8. Uniform initial state 293 K, 1000 Pa.
    """
    key = stream_key(seed, 0)
    u = uniform(key, np.arange(3))
    layer = dict(kM0=2e-11, a=u[0], cM0=1e-4, b=u[1], kTT0=1.5, cTT0=1.2e6)
    bc0 = dict(hT=25.0, hM=2e-8, T_mean=293.0, T_amp=10.0, P_mean=1200.0, P_amp=400.0,
               phase_P=2.0 * math.pi * u[2])
    bc1 = dict(hT=8.0, hM=3e-8, T_mean=293.0, P_mean=1000.0)
    return uniform_wall(101, 0.1, layer, bc0=bc0, bc1=bc1, dt=60.0, n_steps=1440,
                        name="single_wall: 1 wall, N=101, dt=60 s x 1440")


def _layer_split(key, N: int, n_layers: int) -> list[int]:
    """Seeded node counts per layer, each >= 3, summing to N."""
    if n_layers == 1:
        return [N]
    u = uniform(key, np.arange(100, 102))
    if n_layers == 2:
        n0 = 3 + int(u[0] * (N - 5))
        return [n0, N - n0]
    n0 = 3 + int(u[0] * (N - 8))
    n1 = 3 + int(u[1] * (N - n0 - 5))
    return [n0, n1, N - n0 - n1]


def wall_batch(seed: int = 2, n_walls: int = 4096, n_steps: int = 52560, dt: float = 600.0,
            n_min: int = 50, n_max: int = 400, noise: bool = True,
            name: str | None = None) -> Workload:
    """Batch of ragged 1..3-layer walls, per-wall seeded forcing.

    Per wall: N ~ U{n_min..n_max}, thickness ~ U[0.05, 0.4] m, layers ~ U{1,2,3}.
    Per layer: kM0 log-uniform in [1e-12, 1e-10] s, kTT ~ U[0.04, 2] W/m/K,
    cTT ~ U[1e5, 2e6] J/m3/K, a, b ~ U[0, 2], and cM0 log-uniform over the
    range of the paper's Table 2 (cM of the one-zone walls, 1.8e-2 ..
    1.2e-1 s2/m2). With cM0 = 1e-4 the nonlinear DF moisture update at these
    dt / dx (lambda up to 1e5, surface exchange far above the half-cell
    capacity) amplifies its own odd-even mode and diverges within a few
    hundred steps, so the storage coefficient is taken from the paper.
    Face 0: hT = 25, hM = 2e-8; 293 + 10 sin(2 pi t/86400 + phi_T) K and
    1200 + 400 sin(2 pi t/86400 + phi_P) Pa plus hourly Gaussian noise
    (sigma 1 K and 50 Pa, linearly interpolated). Face 1: hT = 8, hM = 3e-8,
    constant 293 K / 1000 Pa. Uniform initial state 293 K, 1000 Pa.
    """
    walls = np.arange(n_walls)
    keys = stream_key(seed, walls)
    u = uniform(keys[:, None], np.arange(8)[None, :])
    N = (n_min + np.floor(u[:, 0] * (n_max - n_min + 1))).astype(np.int32)
    L = 0.05 + 0.35 * u[:, 1]
    nl = np.minimum((1 + np.floor(u[:, 2] * 3)).astype(np.int32), N // 3)   # every layer >= 3 nodes
    phase_T = 2 * np.pi * u[:, 3]
    phase_P = 2 * np.pi * u[:, 4]
    firsts, pars = [], []
    for w in range(n_walls):
        counts = _layer_split(keys[w], int(N[w]), int(nl[w]))
        first = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int32)
        firsts.append(first)
        v = uniform(keys[w], np.arange(200, 200 + 6 * nl[w])).reshape(nl[w], 6)
        for l in range(nl[w]):
            kM0 = 10.0 ** (-12.0 + 2.0 * v[l, 0])
            kTT = 0.04 + 1.96 * v[l, 1]
            cTT = 1e5 + 1.9e6 * v[l, 2]
            a = 2.0 * v[l, 3]
            b = 2.0 * v[l, 4]
            cM0 = 10.0 ** (CM0_LOG10_RANGE[0] + (CM0_LOG10_RANGE[1] - CM0_LOG10_RANGE[0]) * v[l, 5])
            pars.append([kM0, a, cM0, b, kTT, 0.0, cTT, 0.0, 0.0])
    horizon = n_steps * dt
    noise_len = int(math.ceil(horizon / 3600.0)) + 2
    bc_par = np.zeros((n_walls, 2, len(BC_FIELDS)))
    bc_par[:, 0] = _bc_row(25.0, 2e-8, 293.0, 10.0, 1200.0, 400.0)
    bc_par[:, 0, 9] = phase_T
    bc_par[:, 0, 10] = phase_P
    bc_par[:, 1] = _bc_row(8.0, 3e-8, 293.0, 0.0, 1000.0, 0.0)
    nz0 = None
    if noise:
        nkey = stream_key(seed, walls + (1 << 32))
        z0, z1 = normal_pairs(nkey[:, None], np.arange(noise_len, dtype=np.uint64)[None, :])
        nz0 = np.stack([1.0 * z0, 50.0 * z1], axis=-1).astype(np.float32)
    return Workload(
        name=name or f"wall_batch: {n_walls} ragged walls N {n_min}-{n_max}, dt={dt:g} s x {n_steps}",
        n_nodes=N, thickness=L, n_layers=nl, layer_first=np.concatenate(firsts),
        layer_par=np.array(pars, dtype=np.float64),
        T_init=np.full(n_walls, 293.0), P_init=np.full(n_walls, 1000.0),
        bc_kind=np.zeros((n_walls, 2), np.int32), bc_par=bc_par,
        bc_room=np.full((n_walls, 2), -1, np.int32), noise=[nz0, None],
        dt=dt, t0=0.0, n_steps=n_steps)


# Column order of a room parameter row (whole-building workloads).
ROOM_FIELDS = ("volume", "ach", "Q_gain", "g_vap", "T_out_mean", "T_out_amp", "P_out_mean", "P_out_amp",
               "period", "phase_T", "phase_P", "rho_a", "cp_a", "cp_v", "Pv_ref", "scheme", "period_P",
               "g_pulse", "pulse_on", "pulse_off", "pulse_period")


def building(seed: int = 3, n_rooms: int = 64, walls_per_room: int = 6, n_steps: int = 8640,
            dt: float = 300.0, n_min: int = 80, n_max: int = 300) -> Workload:
    """Whole building: rooms of six walls each, FP64 room air balances.

    Each room is a cube of volume V ~ U[30, 200] m3 (wall area V^(2/3)) with
    ventilation ACH ~ U[0.5, 2] 1/h, internal heat gain ~ U[100, 600] W and
    vapour gain ~ U[0.05, 0.3] g/s. Walls: N ~ U{80..300}, materials as the
    batch workload; face 0 outdoors (a shared daily sinusoid, 283 +- 8 K and
    900 +- 300 Pa with seeded phases, plus hourly per-wall noise), face 1 on
    the room (hT = 8, hM = 3e-8). The room's ventilation sees the same
    outdoor sinusoid. Air: rho 1.2 kg/m3, cp 1006 / 1860 J/kg/K, Pv_ref
    1.61e5 Pa (paper Sec. 5.1). Initial state 293 K / 1000 Pa everywhere.
    dt = 300 s x 8640 (30 days).
    """
    n_walls = n_rooms * walls_per_room
    base = wall_batch(seed=seed, n_walls=n_walls, n_steps=n_steps, dt=dt, n_min=n_min, n_max=n_max,
                   name=f"building: {n_rooms} rooms x {walls_per_room} walls, dt={dt:g} s x {n_steps}")
    key = stream_key(seed, 1 << 40)
    g = uniform(key, np.arange(2))
    phase_T, phase_P = 2 * np.pi * g[0], 2 * np.pi * g[1]
    rooms = np.arange(n_rooms)
    rk = stream_key(seed, rooms + (1 << 41))
    u = uniform(rk[:, None], np.arange(4)[None, :])
    V = 30.0 + 170.0 * u[:, 0]
    par = np.zeros((n_rooms, len(ROOM_FIELDS)))
    par[:, 0] = V
    par[:, 1] = 0.5 + 1.5 * u[:, 1]
    par[:, 2] = 100.0 + 500.0 * u[:, 2]
    par[:, 3] = (0.05 + 0.25 * u[:, 3]) * 1e-3
    par[:, 4:11] = [283.0, 8.0, 900.0, 300.0, 86400.0, phase_T, phase_P]
    par[:, 11:15] = [1.2, 1006.0, 1860.0, 1.61e5]
    bc_par = base.bc_par.copy()
    bc_par[:, 0, 4:11] = [283.0, 8.0, 900.0, 300.0, 86400.0, phase_T, phase_P]
    bc_par[:, 1] = _bc_row(8.0, 3e-8, 293.0, 0.0, 1000.0, 0.0)
    bc_kind = np.zeros((n_walls, 2), np.int32)
    bc_kind[:, 1] = BC_ROOM
    bc_room = np.full((n_walls, 2), -1, np.int32)
    bc_room[:, 1] = np.repeat(rooms, walls_per_room)
    area = np.repeat(V ** (2.0 / 3.0), walls_per_room)
    return dataclasses.replace(base, bc_par=bc_par, bc_kind=bc_kind, bc_room=bc_room,
                               rooms=dict(par=par, wall_area=area, Ta0=np.full(n_rooms, 293.0),
                                          Pa0=np.full(n_rooms, 1000.0)))


@dataclasses.dataclass
class Section2D:
    """A batch of 2D wall sections on uniform grids (dx = dy = h)."""
    name: str
    h: float
    region: np.ndarray           # uint8 [G, ny, nx] material region of every node
    region_par: np.ndarray       # float64 [G, n_regions, 9] (LAYER_FIELDS)
    bc_kind: np.ndarray          # int32 [G, 4] faces 0: x = 0, 1: x = Lx, 2: y = 0, 3: y = Ly
    bc_par: np.ndarray           # float64 [G, 4, 13] (BC_FIELDS)
    noise: list                  # per face: float32 [G, noise_len, 2] or None
    T_init: np.ndarray           # float64 [G]
    P_init: np.ndarray           # float64 [G]
    dt: float
    t0: float
    n_steps: int
    Lv: float = LV
    Psat: float = PSAT_REF

    @property
    def n_grids(self) -> int:
        return int(self.region.shape[0])

    @property
    def ny(self) -> int:
        return int(self.region.shape[1])

    @property
    def nx(self) -> int:
        return int(self.region.shape[2])

    @property
    def total_nodes(self) -> int:
        return int(self.region.size)

    def subset(self, grids) -> "Section2D":
        g = np.asarray(grids, dtype=np.int64)
        return dataclasses.replace(
            self, name=f"{self.name}[subset {len(g)}]", region=self.region[g].copy(),
            region_par=self.region_par[g].copy(), bc_kind=self.bc_kind[g].copy(), bc_par=self.bc_par[g].copy(),
            noise=[None if z is None else np.ascontiguousarray(z[g]) for z in self.noise],
            T_init=self.T_init[g].copy(), P_init=self.P_init[g].copy())


def sections_2d(seed: int = 4, n_grids: int = 64, nx: int = 512, ny: int = 512, h: float = 1e-3, dt: float = 60.0,
            n_steps: int = 10000) -> Section2D:
    """Thermal-bridge corners: 2D sections with an L-shaped outer leaf and an optional inner column.

    Per grid: region 0 = base material; region 1 = the L along the two exposed faces,
    {x < a} u {y < b} with a, b ~ U[0.05, 0.25] of the section; region 2 (every other grid) = a
    rectangle inside the base. Materials per region with the batch ranges (kM0 log-U[1e-12, 1e-10],
    kTT U[0.04, 2], cTT U[1e5, 2e6], a, b U[0, 2], cM0 over Table 2's range; kTT, cTT independent of
    Pv, no cTM). Faces x = 0 and y = 0 exchange with the outdoor air (hT = 25, hM = 2e-8,
    293 + 10 sin(2 pi t/86400 + phi_T) K, 1200 + 400 sin(2 pi t/86400 + phi_P) Pa, hourly noise
    sigma 1 K / 50 Pa, the same air on both faces); faces x = L and y = L are adiabatic. Uniform
    initial state 293 K / 1000 Pa. dx = dy = 1 mm, dt = 60 s.
    """
    grids = np.arange(n_grids)
    keys = stream_key(seed, grids + (1 << 42))
    u = uniform(keys[:, None], np.arange(12)[None, :])
    region = np.zeros((n_grids, ny, nx), np.uint8)
    par = np.zeros((n_grids, 3, 9))
    yy, xx = np.mgrid[0:ny, 0:nx]
    for g in range(n_grids):
        a = int((0.05 + 0.2 * u[g, 0]) * nx)
        b = int((0.05 + 0.2 * u[g, 1]) * ny)
        r = region[g]
        r[(xx < a) | (yy < b)] = 1
        if g % 2 == 1:
            x0 = a + int(u[g, 2] * (nx - a) * 0.5)
            y0 = b + int(u[g, 3] * (ny - b) * 0.5)
            x1 = min(nx, x0 + 4 + int(u[g, 4] * nx * 0.2))
            y1 = min(ny, y0 + 4 + int(u[g, 5] * ny * 0.2))
            r[y0:y1, x0:x1] = 2
        v = uniform(keys[g], np.arange(100, 118)).reshape(3, 6)
        for k in range(3):
            par[g, k] = [10.0 ** (-12.0 + 2.0 * v[k, 0]), 2.0 * v[k, 1],
                         10.0 ** (CM0_LOG10_RANGE[0] + (CM0_LOG10_RANGE[1] - CM0_LOG10_RANGE[0]) * v[k, 2]),
                         2.0 * v[k, 3], 0.04 + 1.96 * v[k, 4], 0.0, 1e5 + 1.9e6 * v[k, 5], 0.0, 0.0]
    bc_kind = np.tile(np.array([BC_AMBIENT, BC_ADIABATIC, BC_AMBIENT, BC_ADIABATIC], np.int32), (n_grids, 1))
    bc_par = np.zeros((n_grids, 4, len(BC_FIELDS)))
    for f in (0, 2):
        bc_par[:, f] = _bc_row(25.0, 2e-8, 293.0, 10.0, 1200.0, 400.0)
        bc_par[:, f, 9] = 2 * np.pi * u[:, 6]
        bc_par[:, f, 10] = 2 * np.pi * u[:, 7]
    noise_len = int(math.ceil(n_steps * dt / 3600.0)) + 2
    nkey = stream_key(seed, grids + (1 << 43))
    z0, z1 = normal_pairs(nkey[:, None], np.arange(noise_len, dtype=np.uint64)[None, :])
    nz = np.stack([1.0 * z0, 50.0 * z1], axis=-1).astype(np.float32)
    return Section2D(name=f"sections_2d: {n_grids} sections {nx}x{ny}, h={h:g} m, dt={dt:g} s x {n_steps}",
                     h=h, region=region, region_par=par, bc_kind=bc_kind, bc_par=bc_par, noise=[nz, None, nz, None],
                     T_init=np.full(n_grids, 293.0), P_init=np.full(n_grids, 1000.0), dt=dt, t0=0.0,
                     n_steps=n_steps)


@dataclasses.dataclass
class Sensors:
    """Synthetic sensor series for the misfit loss: obs[k][w][f] = (T, Pv) at face f of wall w after step
    (k + 1) * sample_every, with the weights of the squared T and Pv mismatches."""
    obs: np.ndarray              # float32 [n_steps // sample_every, n_walls, 2, 2]
    sample_every: int
    wT: float
    wP: float


def gradient_walls(seed: int = 5, n_walls: int = 1024, n_nodes: int = 200, n_steps: int = 43200, dt: float = 60.0,
            sample_every: int = 10) -> tuple[Workload, Sensors]:
    """Gradient workload: 1024 two-layer walls of 200 nodes, 30 days at dt = 60 s, surface sensors every
    10 min.

    Per wall: thickness ~ U[0.1, 0.3] m, the interface at a node drawn in [N/4, 3N/4]; per layer kM0
    log-uniform in [1e-12, 1e-10] s, a, b ~ U[0, 2], cM0 log-uniform over Table 2's range, kTT ~ U[0.04, 2],
    cTT ~ U[1e5, 2e6] (kTT, cTT independent of Pv, no cTM). Forcing as the batch workload (face 0 outdoor
    air with hourly noise, face 1 constant indoor air). Sensors: seeded series at both faces,
    T = 293 + 4 sin(2 pi t/86400 + psi) + N(0, 0.5^2) K and Pv = 1100 + 250 sin(2 pi t/86400 + psi') +
    N(0, 30^2) Pa; weights wT = 1 K^-2, wP = 1e-4 Pa^-2.
    """
    walls = np.arange(n_walls)
    keys = stream_key(seed, walls + (1 << 44))
    u = uniform(keys[:, None], np.arange(10)[None, :])
    N = np.full(n_walls, n_nodes, np.int32)
    L = 0.1 + 0.2 * u[:, 0]
    cut = (n_nodes // 4 + np.floor(u[:, 1] * (n_nodes // 2))).astype(np.int32)
    firsts = np.stack([np.zeros(n_walls, np.int32), cut], axis=1).reshape(-1)
    pars = []
    for w in range(n_walls):
        v = uniform(keys[w], np.arange(300, 312)).reshape(2, 6)
        for l in range(2):
            pars.append([10.0 ** (-12.0 + 2.0 * v[l, 0]), 2.0 * v[l, 1],
                         10.0 ** (CM0_LOG10_RANGE[0] + (CM0_LOG10_RANGE[1] - CM0_LOG10_RANGE[0]) * v[l, 2]),
                         2.0 * v[l, 3], 0.04 + 1.96 * v[l, 4], 0.0, 1e5 + 1.9e6 * v[l, 5], 0.0, 0.0])
    noise_len = int(math.ceil(n_steps * dt / 3600.0)) + 2
    bc_par = np.zeros((n_walls, 2, len(BC_FIELDS)))
    bc_par[:, 0] = _bc_row(25.0, 2e-8, 293.0, 10.0, 1200.0, 400.0)
    bc_par[:, 0, 9] = 2 * np.pi * u[:, 2]
    bc_par[:, 0, 10] = 2 * np.pi * u[:, 3]
    bc_par[:, 1] = _bc_row(8.0, 3e-8, 293.0, 0.0, 1000.0, 0.0)
    nkey = stream_key(seed, walls + (1 << 45))
    z0, z1 = normal_pairs(nkey[:, None], np.arange(noise_len, dtype=np.uint64)[None, :])
    nz0 = np.stack([1.0 * z0, 50.0 * z1], axis=-1).astype(np.float32)
    wl = Workload(name=f"gradient_walls: {n_walls} two-layer walls N={n_nodes}, dt={dt:g} s x {n_steps}",
                  n_nodes=N, thickness=L, n_layers=np.full(n_walls, 2, np.int32), layer_first=firsts,
                  layer_par=np.array(pars, np.float64), T_init=np.full(n_walls, 293.0),
                  P_init=np.full(n_walls, 1000.0), bc_kind=np.zeros((n_walls, 2), np.int32), bc_par=bc_par,
                  bc_room=np.full((n_walls, 2), -1, np.int32), noise=[nz0, None], dt=dt, t0=0.0, n_steps=n_steps)
    K = n_steps // sample_every
    t = (np.arange(1, K + 1) * sample_every * dt)[:, None, None]
    psiT = 2 * np.pi * u[:, 4:6][None]
    psiP = 2 * np.pi * u[:, 6:8][None]
    skey = stream_key(seed, walls + (1 << 46))
    ctr = np.arange(K * 2, dtype=np.uint64).reshape(K, 1, 2)
    n0, n1 = normal_pairs(skey[None, :, None], ctr)
    T = 293.0 + 4.0 * np.sin(2 * np.pi * t / 86400.0 + psiT) + 0.5 * n0
    P = 1100.0 + 250.0 * np.sin(2 * np.pi * t / 86400.0 + psiP) + 30.0 * n1
    obs = np.stack([T, P], axis=-1).astype(np.float32)
    return wl, Sensors(obs=obs, sample_every=sample_every, wT=1.0, wP=1e-4)


# The one-zone case of Sec. 5.2 (Table 2 walls; dimensionless data of Appendix B), in SI units.
ONE_ZONE_WALLS = {  # cM, kM, cTT, kTT, cTM, kTM, hT outside, hM outside, area
    "north": (1.82e-2, 5.89e-9, 7.7e5, 0.294, 1.52e3, 1.59e-2, 5.0, 2e-7, 18.0),
    "south": (1.18e-1, 2.92e-8, 1.28e6, 0.841, 9.88e3, 2.96e-3, 25.0, 8e-7, 18.0),
    "east": (6.09e-2, 5.47e-9, 8.61e5, 0.387, 5.09e3, 1.53e-2, 12.0, 4e-7, 9.0),
    "west": (6.09e-2, 5.47e-9, 8.61e5, 0.387, 5.09e3, 1.53e-2, 12.0, 4e-7, 9.0),
}


def one_zone(N: int = 101, dt: float = 3.6, hours: float = 80.0) -> Workload:
    """The paper's one-zone building (Sec. 5.2, Table 2, Appendix B): four 10 cm walls of linear
    materials around one air zone, 80 h at dt = 3.6 s (dx = 1 mm with N = 101).

    * walls north, south (18 m2 each), east, west (9 m2 each); constant coefficients from Table 2 with
      cTM = chi cM and the cross conductivity kTM entering as the vapour fraction nu = kTM / (Lv kM)
      (Lv = 2.5e6 J/kg; Appendix B's BiTM values follow from it with Pref = Pvi and Tref = Ti);
    * face 0 outdoors with Table 2's hT, hM, face 1 on the zone with hT = 8 W/m2/K, hM = 3e-8 s/m;
    * outdoor air (Appendix B): T = Ti (1 - 0.02 sin^2(2 pi t / 24 h)) = Ti (0.99 + 0.01 sin(2 pi t / 12 h
      + pi/2)), Pv = Pvi (1 + 0.06 sin(2 pi t / 24 h)); the zone's ventilation (0.5 1/h) takes the same air;
    * zone of 54 m3, vapour load 25 g/h plus 400 g/h from 6 h to 9 h each day (its latent heat Lv g
      enters the air's heat balance, Sec. 5.1), no other gains;
    * everything starts at Ti = 20 C, Pvi = 50 % of Psat(20 C) = 1168.5 Pa.
    """
    Ti, Pvi = 293.15, 0.5 * PSAT_REF
    n_steps = int(round(hours * 3600.0 / dt))
    walls = []
    areas = []
    nu = []
    for name, (cM, kM, cTT, kTT, cTM, kTM, hT, hM, A) in ONE_ZONE_WALLS.items():
        layer = dict(kM0=kM, a=0.0, cM0=cM, b=0.0, kTT0=kTT, aT=0.0, cTT0=cTT, bT=0.0, chi=cTM / cM)
        bc0 = dict(hT=hT, hM=hM, T_mean=0.99 * Ti, T_amp=0.01 * Ti, period=43200.0, phase_T=0.5 * math.pi,
                   P_mean=Pvi, P_amp=0.06 * Pvi, period_P=86400.0, phase_P=0.0)
        bc1 = dict(hT=8.0, hM=3e-8, T_mean=Ti, P_mean=Pvi)
        walls.append(uniform_wall(N, 0.1, layer, T0=Ti, P0=Pvi, bc0=bc0, bc1=bc1, dt=dt, n_steps=n_steps,
                                  kinds=(BC_AMBIENT, BC_ROOM), name=name))
        areas.append(A)
        nu.append(kTM / (LV * kM))
    wl = concat(walls, name=f"one-zone case: 4 walls N={N}, dt={dt:g} s x {n_steps}")
    par = np.zeros((1, len(ROOM_FIELDS)))
    row = dict(volume=54.0, ach=0.5, Q_gain=0.0, g_vap=25e-3 / 3600.0, T_out_mean=0.99 * Ti, T_out_amp=0.01 * Ti,
               P_out_mean=Pvi, P_out_amp=0.06 * Pvi, period=43200.0, phase_T=0.5 * math.pi, phase_P=0.0,
               rho_a=1.2, cp_a=1006.0, cp_v=1860.0, Pv_ref=1.61e5, scheme=0.0, period_P=86400.0,
               g_pulse=400e-3 / 3600.0, pulse_on=6 * 3600.0, pulse_off=9 * 3600.0, pulse_period=86400.0)
    par[0] = [row[k] for k in ROOM_FIELDS]
    bc_room = np.full((4, 2), -1, np.int32)
    bc_room[:, 1] = 0
    return dataclasses.replace(wl, bc_room=bc_room, vapour_frac=np.array(nu),
                               rooms=dict(par=par, wall_area=np.array(areas), Ta0=np.array([Ti]),
                                          Pa0=np.array([Pvi])))


# Coefficient laws of a layer (hygro_set_layer_law): the affine laws of the layer parameters, or the load
# bearing material of Sec. 4 (Table 1) with one of three readings of its liquid-transport bracket.
LAW_AFFINE, LAW_TABLE1, LAW_TABLE1_A, LAW_TABLE1_C = 0, 1, 2, 3


def table1_walls(seed: int = 6, n_walls: int = 256, N: int = 101, L: float = 0.1, dt: float = 3.6,
                 hours: float = 120.0, law: int = LAW_TABLE1) -> Workload:
    """Walls of the load bearing material of Sec. 4 (Table 1): 10 cm slabs, N = 101 (dx = 1 mm), dt = 3.6 s
    (the paper's dx* = 1e-2, dt* = 1e-3 with a reference time of 1 h), 120 h.

    * one layer of the Table-1 law ``law`` per wall (its affine parameters are placeholders, unused);
    * initial state 20 C and 1166.7 Pa (50 % relative humidity with the library's saturation pressure);
    * face 0: hT = 25 W/m2/K, hM = 2e-7 s/m; face 1: hT = 8, hM = 3e-8 (Sec. 4);
    * the paper's boundary series exist only as figures, which are missing: each face instead sees a daily
      sinusoid with seeded phases, T = 293.15 + a_T sin(.), a_T ~ U[4, 8] K (face 1: U[1, 2]), and
      Pv = 1166.7 (1 + a_P sin(.)), a_P ~ U[0.05, 0.15] (face 1: U[0.02, 0.05]), which keeps the air below
      saturation.
    """
    Ti, Pvi = 293.15, 1166.7
    n_steps = int(round(hours * 3600.0 / dt))
    key = stream_key(seed, np.arange(n_walls))
    u = uniform(key[:, None], np.arange(8)[None, :])
    walls = []
    placeholder = dict(kM0=8.3e-10, cM0=4.0e-4, kTT0=0.2, cTT0=6.9e5)
    for w in range(n_walls):
        bc0 = dict(hT=25.0, hM=2e-7, T_mean=Ti, T_amp=4.0 + 4.0 * u[w, 0], P_mean=Pvi,
                   P_amp=Pvi * (0.05 + 0.10 * u[w, 1]), phase_T=2 * math.pi * u[w, 2], phase_P=2 * math.pi * u[w, 3])
        bc1 = dict(hT=8.0, hM=3e-8, T_mean=Ti, T_amp=1.0 + u[w, 4], P_mean=Pvi,
                   P_amp=Pvi * (0.02 + 0.03 * u[w, 5]), phase_T=2 * math.pi * u[w, 6], phase_P=2 * math.pi * u[w, 7])
        walls.append(uniform_wall(N, L, placeholder, T0=Ti, P0=Pvi, bc0=bc0, bc1=bc1, dt=dt, n_steps=n_steps))
    wl = concat(walls, name=f"Table-1 material: {n_walls} walls N={N}, dt={dt:g} s x {n_steps}")
    return dataclasses.replace(wl, layer_law=np.full(n_walls, law, np.int32))
