"""FP64 CPU oracle of the Dufort-Frankel hygrothermal wall update.

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and
by the CPU-baseline leg of the benchmark. The CUDA library never imports it.
The arithmetic lives in ``hygro_oracle.c`` (plain C, FP64, scalar loops);
this module only compiles it with gcc and marshals arrays through ctypes.

Parity pins (tests/test_oracle_*.py): the linear DF closed form [eq:dufort],
the nonlinear DF [eq:DF_NL] and the coupled form [eq:DF_eq2b] one step at a
time, the ghost-node surface update [eq:ghost_node_v0]/[eq:ghost_node_u0],
the exact series-resistance and Kirchhoff steady states, the Fourier series
of linear diffusion with Robin ends, the discrete balance identity, mirror
symmetry and uniform invariance, and a closed-form room steady state.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hygro_oracle.c")
_SRC2 = os.path.join(_HERE, "hygro_oracle2d.c")
_SRC3 = os.path.join(_HERE, "hygro_adjoint.c")
_SRC4 = os.path.join(_HERE, "hygro_comparators.c")
_HDR = os.path.join(_HERE, "hygro_oracle.h")
_HDR2 = os.path.join(_HERE, "oracle_internal.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

NLAYER_PAR = 9
NBC_PAR = 13
NROOM_PAR = 21


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available); return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in (_SRC, _SRC2, _SRC3, _SRC4, _HDR, _HDR2))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    base = [cc, "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, _SRC2, _SRC3, _SRC4, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("n_walls", C.c_int32),
        ("n_nodes", C.c_void_p), ("thickness", C.c_void_p), ("n_layers", C.c_void_p),
        ("layer_first", C.c_void_p), ("layer_par", C.c_void_p), ("bc_kind", C.c_void_p),
        ("bc_par", C.c_void_p), ("bc_room", C.c_void_p),
        ("noise", C.c_void_p * 2), ("noise_len", C.c_int32 * 2),
        ("dt", C.c_double), ("t0", C.c_double), ("Lv", C.c_double), ("Psat", C.c_double),
        ("n_rooms", C.c_int32), ("room_par", C.c_void_p), ("wall_area", C.c_void_p),
        ("vapour_frac", C.c_void_p), ("layer_law", C.c_void_p),
        ("face_emis", C.c_void_p), ("room_view", C.c_void_p), ("n_links", C.c_int32), ("link_zone", C.c_void_p),
        ("link_flow", C.c_void_p),
    ]


class _State(C.Structure):
    _fields_ = [
        ("step", C.c_int64),
        ("T_prev", C.c_void_p), ("T_cur", C.c_void_p), ("P_prev", C.c_void_p), ("P_cur", C.c_void_p),
        ("cumul", C.c_void_p), ("room", C.c_void_p),
    ]


class _Problem2D(C.Structure):
    _fields_ = [
        ("n_grids", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("h", C.c_double),
        ("region", C.c_void_p), ("n_regions", C.c_int32), ("region_par", C.c_void_p),
        ("bc_kind", C.c_void_p), ("bc_par", C.c_void_p),
        ("noise", C.c_void_p * 4), ("noise_len", C.c_int32 * 4),
        ("dt", C.c_double), ("t0", C.c_double), ("Lv", C.c_double), ("Psat", C.c_double),
    ]


class _Misfit(C.Structure):
    _fields_ = [("sample_every", C.c_int32), ("obs", C.c_void_p), ("wT", C.c_double), ("wP", C.c_double),
                ("T_init", C.c_void_p), ("P_init", C.c_void_p)]


class _State2D(C.Structure):
    _fields_ = [("step", C.c_int64), ("T_prev", C.c_void_p), ("T_cur", C.c_void_p), ("P_prev", C.c_void_p),
                ("P_cur", C.c_void_p)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.orc_run.restype = C.c_int
        lib.orc_run.argtypes = [C.POINTER(_Problem), C.POINTER(_State), C.c_int64, C.c_int32,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
        lib.orc_ambient.restype = None
        lib.orc_ambient.argtypes = [C.POINTER(_Problem), C.c_int32, C.c_int32, C.c_double,
                                    C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.orc2d_run.restype = C.c_int
        lib.orc2d_run.argtypes = [C.POINTER(_Problem2D), C.POINTER(_State2D), C.c_int64, C.c_int32]
        lib.orc_loss_adjoint.restype = C.c_int
        lib.orc_loss_adjoint.argtypes = [C.POINTER(_Problem), C.c_int64, C.POINTER(_Misfit), C.POINTER(C.c_double),
                                         C.c_void_p, C.c_int32]
        lib.orc_loss_tangent.restype = C.c_int
        lib.orc_loss_tangent.argtypes = [C.POINTER(_Problem), C.c_int64, C.POINTER(_Misfit), C.c_void_p,
                                         C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.orc_euler_start.restype = C.c_int
        lib.orc_euler_start.argtypes = [C.POINTER(_Problem), C.POINTER(_State), C.c_double, C.c_int32]
        lib.orc_coefficients.restype = None
        lib.orc_coefficients.argtypes = [C.POINTER(_Problem), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p]
        for name in ("orc_euler_implicit_run", "orc_euler_explicit_run"):
            f = getattr(lib, name)
            f.restype = C.c_int
        lib.orc_euler_implicit_run.argtypes = [C.POINTER(_Problem), C.POINTER(_State), C.c_int64, C.c_double,
                                               C.c_int32, C.c_int32, C.POINTER(C.c_int64), C.c_int32]
        lib.orc_euler_explicit_run.argtypes = [C.POINTER(_Problem), C.POINTER(_State), C.c_int64, C.c_double,
                                               C.POINTER(C.c_int64), C.c_int32]
        lib.orc_table1.restype = None
        lib.orc_table1.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_double, C.c_void_p,
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]
        _lib = lib
    return _lib


def _ptr(a) -> int | None:
    return None if a is None else a.ctypes.data


def default_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


class Oracle:
    """The oracle on one workload: holds the FP64 state between ``run`` calls.

    The state starts at the uniform initial condition [eq:HAM_ic] with level
    n-1 equal to level 0 (the scheme is stated for n >= 1; the first step
    uses u^{-1} := u^0), at step 0 (time t0).
    """

    def __init__(self, wl, n_threads: int | None = None):
        self.wl = wl
        self.n_threads = n_threads or default_threads()
        self._keep = []
        W = wl.n_walls
        self.node_off = np.zeros(W + 1, dtype=np.int64)
        np.cumsum(wl.n_nodes, out=self.node_off[1:])
        tot = int(self.node_off[-1])

        def keep(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a

        p = _Problem()
        p.n_walls = W
        p.n_nodes = _ptr(keep(wl.n_nodes, np.int32))
        p.thickness = _ptr(keep(wl.thickness, np.float64))
        p.n_layers = _ptr(keep(wl.n_layers, np.int32))
        p.layer_first = _ptr(keep(wl.layer_first, np.int32))
        p.layer_par = _ptr(keep(wl.layer_par.reshape(-1, NLAYER_PAR), np.float64))
        p.bc_kind = _ptr(keep(wl.bc_kind, np.int32))
        p.bc_par = _ptr(keep(wl.bc_par.reshape(W, 2, NBC_PAR), np.float64))
        p.bc_room = _ptr(keep(wl.bc_room, np.int32))
        for f in range(2):
            nz = wl.noise[f]
            if nz is None:
                p.noise[f] = None
                p.noise_len[f] = 0
            else:
                nz = keep(nz, np.float32)
                p.noise[f] = nz.ctypes.data
                p.noise_len[f] = nz.shape[1]
        p.dt, p.t0, p.Lv, p.Psat = wl.dt, wl.t0, wl.Lv, wl.Psat
        rooms = wl.rooms
        if rooms:
            p.n_rooms = len(rooms["par"])
            par = np.asarray(rooms["par"], np.float64)
            assert par.shape[1] == NROOM_PAR, "room rows hold ROOM_FIELDS"
            p.room_par = _ptr(keep(par, np.float64))
            p.wall_area = _ptr(keep(rooms["wall_area"], np.float64))
            # long-wave exchange among a room's surfaces, interzone airflow (both optional)
            if rooms.get("emissivity") is not None:
                p.face_emis = _ptr(keep(np.asarray(rooms["emissivity"], np.float64).reshape(W, 2), np.float64))
                p.room_view = _ptr(keep(rooms["view"], np.float64))
            links = rooms.get("links") or []
            p.n_links = len(links)
            if links:
                p.link_zone = _ptr(keep(np.array([[a, b] for a, b, _ in links], np.int32), np.int32))
                p.link_flow = _ptr(keep(np.array([g for _, _, g in links], np.float64), np.float64))
        else:
            p.n_rooms = 0
            p.room_par = None
            p.wall_area = _ptr(keep(np.zeros(max(W, 1)), np.float64))
        vf = getattr(wl, "vapour_frac", None)
        p.vapour_frac = None if vf is None else _ptr(keep(vf, np.float64))
        law = getattr(wl, "layer_law", None)
        p.layer_law = None if law is None else _ptr(keep(law, np.int32))
        self._p = p

        self.T_prev = np.repeat(np.asarray(wl.T_init, np.float64), wl.n_nodes)
        self.T_cur = self.T_prev.copy()
        self.P_prev = np.repeat(np.asarray(wl.P_init, np.float64), wl.n_nodes)
        self.P_cur = self.P_prev.copy()
        assert self.T_cur.shape[0] == tot
        self.cumul = np.zeros((W, 2, 2), np.float64)
        R = int(p.n_rooms)
        self.room = np.zeros((max(R, 1), 4), np.float64)
        if R:
            self.room[:, 0:2] = np.asarray(rooms["Ta0"], np.float64)[:, None]
            self.room[:, 2:4] = np.asarray(rooms["Pa0"], np.float64)[:, None]
        self.step = 0

    @property
    def n_rooms(self) -> int:
        return int(self._p.n_rooms)

    def set_levels(self, T_prev, T_cur, P_prev, P_cur, step: int | None = None):
        """Overwrite the two stored levels (concatenated walls)."""
        self.T_prev[:] = T_prev
        self.T_cur[:] = T_cur
        self.P_prev[:] = P_prev
        self.P_cur[:] = P_cur
        if step is not None:
            self.step = int(step)

    def run(self, n_steps: int, sample_every: int = 0, want_balance: bool = False):
        """Advance ``n_steps``; return dict(samples, room_samples, flux, balance)."""
        W, R = self.wl.n_walls, self.n_rooms
        ns = n_steps // sample_every if sample_every > 0 else 0
        samples = np.zeros((ns, W, 2, 2)) if sample_every > 0 else None
        room_samples = np.zeros((ns, R, 2)) if (sample_every > 0 and R) else None
        flux = np.zeros((W, 2, 2))
        bal = np.zeros((W, 2, 4)) if want_balance else None
        st = _State(self.step, _ptr(self.T_prev), _ptr(self.T_cur), _ptr(self.P_prev), _ptr(self.P_cur),
                    _ptr(self.cumul), _ptr(self.room))
        rc = _load().orc_run(C.byref(self._p), C.byref(st), int(n_steps), int(sample_every),
                             _ptr(samples), _ptr(room_samples), _ptr(flux), _ptr(bal), int(self.n_threads))
        if rc != 0:
            raise RuntimeError(f"oracle run failed with code {rc}")
        self.step = int(st.step)
        return dict(samples=samples, room_samples=room_samples, flux=flux if n_steps > 0 else None,
                    balance=bal)

    def _state(self):
        return _State(self.step, _ptr(self.T_prev), _ptr(self.T_cur), _ptr(self.P_prev), _ptr(self.P_cur),
                      _ptr(self.cumul), _ptr(self.room))

    def run_implicit(self, n_steps: int, eta: float, max_iter: int = 100, norm: str = "max") -> int:
        """The paper's Euler implicit scheme with fixed-point sub-iterations (Alg. 1); returns the
        sub-iterations done. norm: "max" (largest relative change) or "l2" (Euclidean norm of all)."""
        st = self._state()
        it = C.c_int64(0)
        rc = _load().orc_euler_implicit_run(C.byref(self._p), C.byref(st), int(n_steps), float(eta), int(max_iter),
                                            {"max": 0, "l2": 1}[norm], C.byref(it), int(self.n_threads))
        if rc != 0:
            raise RuntimeError(f"implicit Euler run failed with code {rc}")
        self.step = int(st.step)
        return it.value

    def run_explicit(self, n_steps: int, refine: float = 1.0) -> int:
        """The Euler explicit scheme within its stability bound; returns the substeps done."""
        st = self._state()
        ns = C.c_int64(0)
        rc = _load().orc_euler_explicit_run(C.byref(self._p), C.byref(st), int(n_steps), float(refine),
                                            C.byref(ns), int(self.n_threads))
        if rc != 0:
            raise RuntimeError(f"explicit Euler run failed with code {rc}")
        self.step = int(st.step)
        return ns.value

    def euler_start(self, refine: float = 1.0):
        """The first step by explicit Euler substeps (state at step 0): levels become (0, 1), step 1."""
        st = _State(self.step, _ptr(self.T_prev), _ptr(self.T_cur), _ptr(self.P_prev), _ptr(self.P_cur),
                    _ptr(self.cumul), _ptr(self.room))
        rc = _load().orc_euler_start(C.byref(self._p), C.byref(st), float(refine), int(self.n_threads))
        if rc != 0:
            raise RuntimeError(f"oracle Euler start failed with code {rc}")
        self.step = int(st.step)

    def wall(self, w: int, field: str = "T", level: int = 0) -> np.ndarray:
        """Nodes of wall ``w``; level 0 is the newest (n), 1 the previous (n-1)."""
        arr = {("T", 0): self.T_cur, ("T", 1): self.T_prev, ("P", 0): self.P_cur, ("P", 1): self.P_prev}[(field, level)]
        return arr[self.node_off[w]: self.node_off[w + 1]]

    def ambient(self, w: int, face: int, t: float) -> tuple[float, float]:
        T = C.c_double()
        P = C.c_double()
        _load().orc_ambient(C.byref(self._p), w, face, float(t), C.byref(T), C.byref(P))
        return T.value, P.value

    def coefficients(self, w: int, P: np.ndarray, T: np.ndarray | None = None):
        """Node (kM, cM, kTT, cTT, kTM, cTM) and face (kM_f, kTT_f, kTM_f) values at level values P (and T,
        which only the Table-1 laws use)."""
        P = np.ascontiguousarray(P, np.float64)
        T = None if T is None else np.ascontiguousarray(T, np.float64)
        N = P.shape[0]
        node = np.zeros((N, 6))
        face = np.zeros((N - 1, 3))
        _load().orc_coefficients(C.byref(self._p), int(w), _ptr(T), _ptr(P), _ptr(node), _ptr(face))
        return node, face


LAW_AFFINE, LAW_TABLE1, LAW_TABLE1_A, LAW_TABLE1_C = 0, 1, 2, 3


def table1(law: int, T: float, Pv: float, Lv: float):
    """Coefficients (kM, cM, kTT, cTT, kTM, cTM) of the Table-1 material at (T, Pv), with Ps(T) and the
    sorption isotherm f: returns (coefficients[6], Ps, f)."""
    out = np.zeros(6)
    ps = C.c_double()
    fw = C.c_double()
    _load().orc_table1(int(law), float(T), float(Pv), float(Lv), _ptr(out), C.byref(ps), C.byref(fw))
    return out, ps.value, fw.value


def _misfit(wl, obs, sample_every, wT, wP, keep):
    m = _Misfit()
    m.sample_every = int(sample_every)
    m.obs = _ptr(keep(obs, np.float64))
    m.wT, m.wP = float(wT), float(wP)
    m.T_init = _ptr(keep(wl.T_init, np.float64))
    m.P_init = _ptr(keep(wl.P_init, np.float64))
    return m


def loss_and_gradient(wl, n_steps: int, obs, sample_every: int, wT: float, wP: float, gradient: bool = True,
                      n_threads: int | None = None):
    """Sensor-misfit loss of the surface values of a fresh run of ``wl`` (uniform initial state) and its
    gradient with respect to every layer's 9 parameters [sum layers, 9], by the reverse-time adjoint.
    obs: [n_steps // sample_every, n_walls, 2 faces, 2 (T, Pv)]."""
    o = Oracle(wl, n_threads=1)
    kept = []

    def keep(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        kept.append(a)
        return a

    m = _misfit(wl, obs, sample_every, wT, wP, keep)
    loss = C.c_double()
    grad = np.zeros((len(wl.layer_par), NLAYER_PAR)) if gradient else None
    rc = _load().orc_loss_adjoint(C.byref(o._p), int(n_steps), C.byref(m), C.byref(loss), _ptr(grad),
                                  int(n_threads or default_threads()))
    if rc != 0:
        raise RuntimeError(f"oracle adjoint failed with code {rc}")
    return loss.value, grad


def loss_tangent(wl, n_steps: int, obs, sample_every: int, wT: float, wP: float, direction):
    """Loss and its derivative along ``direction`` [sum layers, 9] by forward-mode dual numbers."""
    o = Oracle(wl, n_threads=1)
    kept = []

    def keep(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        kept.append(a)
        return a

    m = _misfit(wl, obs, sample_every, wT, wP, keep)
    d = keep(direction, np.float64)
    loss = C.c_double()
    dl = C.c_double()
    rc = _load().orc_loss_tangent(C.byref(o._p), int(n_steps), C.byref(m), _ptr(d), C.byref(loss), C.byref(dl))
    if rc != 0:
        raise RuntimeError(f"oracle tangent failed with code {rc}")
    return loss.value, dl.value


class Oracle2D:
    """The oracle on a batch of 2D sections (attributes of ``sec``: n_grids, nx, ny, h, region
    [G, ny, nx] uint8, region_par [G, n_regions, 9], bc_kind [G, 4], bc_par [G, 4, 12], noise (4 faces,
    each [G, len, 2] float32 or None), dt, t0, Lv, Psat, T_init, P_init [G]). Level -1 := level 0."""

    def __init__(self, sec, n_threads: int | None = None):
        self.sec = sec
        self.n_threads = n_threads or default_threads()
        self._keep = []

        def keep(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a

        G, ny, nx = sec.region.shape
        p = _Problem2D()
        p.n_grids, p.nx, p.ny, p.h = G, nx, ny, sec.h
        p.region = _ptr(keep(sec.region, np.uint8))
        p.n_regions = sec.region_par.shape[1]
        p.region_par = _ptr(keep(sec.region_par, np.float64))
        p.bc_kind = _ptr(keep(sec.bc_kind, np.int32))
        p.bc_par = _ptr(keep(sec.bc_par, np.float64))
        for f in range(4):
            nz = sec.noise[f]
            if nz is None:
                p.noise[f] = None
                p.noise_len[f] = 0
            else:
                nz = keep(nz, np.float32)
                p.noise[f] = nz.ctypes.data
                p.noise_len[f] = nz.shape[1]
        p.dt, p.t0, p.Lv, p.Psat = sec.dt, sec.t0, sec.Lv, sec.Psat
        self._p = p
        shape = (G, ny, nx)
        self.T_cur = np.broadcast_to(np.asarray(sec.T_init, np.float64)[:, None, None], shape).copy()
        self.P_cur = np.broadcast_to(np.asarray(sec.P_init, np.float64)[:, None, None], shape).copy()
        self.T_prev = self.T_cur.copy()
        self.P_prev = self.P_cur.copy()
        self.step = 0

    def set_levels(self, T_prev, T_cur, P_prev, P_cur):
        self.T_prev[...] = T_prev
        self.T_cur[...] = T_cur
        self.P_prev[...] = P_prev
        self.P_cur[...] = P_cur

    def run(self, n_steps: int):
        st = _State2D(self.step, _ptr(self.T_prev), _ptr(self.T_cur), _ptr(self.P_prev), _ptr(self.P_cur))
        rc = _load().orc2d_run(C.byref(self._p), C.byref(st), int(n_steps), int(self.n_threads))
        if rc != 0:
            raise RuntimeError(f"2D oracle run failed with code {rc}")
        self.step = int(st.step)
