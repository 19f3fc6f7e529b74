"""Python binding of the hygro C ABI (include/hygro.h, include/hygro2d.h), argument marshalling only.

Every computation runs in ``libhygro.so`` (CUDA, sm_103a), built in tree by
``paper_1703_10119_gb300.build``. Loading fails loudly when the library is
missing: there is no CPU fallback. The functions ``hygro_*`` mirror the C
entry points one to one; :class:`Hygro` wires a
:class:`~paper_1703_10119_gb300.workloads.Workload` through them. Device
buffers may be torch CUDA tensors (PyTorch supplies device memory and
streams); host buffers are numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

HYGRO_OK = 0
HYGRO_E_INVALID = -1
HYGRO_E_NOMEM = -2
HYGRO_E_CUDA = -3
HYGRO_E_STATE = -4
HYGRO_E_NONFINITE = -5
HYGRO_E_TIMEOUT = -6
HYGRO_E_UNSUPPORTED = -7
HYGRO_FP32, HYGRO_FP64 = 0, 1
HYGRO_KERNEL_PERSISTENT, HYGRO_KERNEL_PLAIN = 0, 1
HYGRO_BC_AMBIENT, HYGRO_BC_ADIABATIC, HYGRO_BC_ROOM = 0, 1, 2
HYGRO_OPT_ROOM_SCHEME = 1
HYGRO_ROOM_DF, HYGRO_ROOM_EULER = 0, 1
HYGRO_NOALLOC_SCRATCH_BYTES = 8 << 20
STATUS_NAMES = {0: "HYGRO_OK", -1: "HYGRO_E_INVALID", -2: "HYGRO_E_NOMEM", -3: "HYGRO_E_CUDA",
                -4: "HYGRO_E_STATE", -5: "HYGRO_E_NONFINITE", -6: "HYGRO_E_TIMEOUT", -7: "HYGRO_E_UNSUPPORTED"}

# Exported entry points (names of include/hygro.h).
ABI_FUNCTIONS = ("hygro_create", "hygro_set_materials", "hygro_set_bc", "hygro_run", "hygro_sync",
                 "hygro_fluxes", "hygro_get_fields", "hygro_set_fields", "hygro_get_step", "hygro_get_state",
                 "hygro_set_state", "hygro_last_error", "hygro_destroy", "hygro_run_noalloc", "hygro_set_rooms",
                 "hygro_get_rooms", "hygro_loss_grad", "hygro_balance", "hygro_set_option",
                 "hygro_start_euler", "hygro_set_vapour_fraction", "hygro_autotune", "hygro_set_layer_law",
                 "hygro_set_radiation", "hygro_set_interzone")
HYGRO_LAW_AFFINE, HYGRO_LAW_TABLE1, HYGRO_LAW_TABLE1_A, HYGRO_LAW_TABLE1_C = 0, 1, 2, 3
# Exported entry points of the 2D sections (names of include/hygro2d.h).
ABI_FUNCTIONS_2D = ("hygro2d_create", "hygro2d_set_materials", "hygro2d_set_bc", "hygro2d_run", "hygro2d_sync",
                    "hygro2d_get_fields", "hygro2d_set_fields", "hygro2d_get_step", "hygro2d_last_error",
                    "hygro2d_destroy", "hygro2d_set_option", "hygro2d_get_option", "hygro2d_autotune")
HYGRO2D_OPT_STEPS_PER_LAUNCH = 1
HYGRO2D_OPT_GRAPH_LAUNCHES = 2
# Exported arithmetic-peak microbenchmark (include/hygro_peaks.h).
ABI_FUNCTIONS_PEAKS = ("hygro_peak_probe",)
HYGRO2D_MAX_REGIONS = 8


class hygro_desc(C.Structure):
    _fields_ = [("n_walls", C.c_int32), ("n_nodes", C.c_void_p), ("thickness", C.c_void_p),
                ("dt", C.c_double), ("t0", C.c_double), ("Lv", C.c_double), ("Psat", C.c_double),
                ("precision", C.c_int32), ("kernel", C.c_int32), ("device", C.c_int32), ("stream", C.c_void_p)]


class hygro2d_desc(C.Structure):
    _fields_ = [("n_grids", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("h", C.c_double),
                ("dt", C.c_double), ("t0", C.c_double), ("Lv", C.c_double), ("Psat", C.c_double),
                ("precision", C.c_int32), ("steps_per_launch", C.c_int32), ("device", C.c_int32),
                ("stream", C.c_void_p)]


class hygro_layer(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("kM0", "a", "cM0", "b", "kTT0", "aT", "cTT0", "bT", "chi")]


class hygro_bc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("room", C.c_int32), ("hT", C.c_double), ("hM", C.c_double),
                ("q_inf", C.c_double), ("g_inf", C.c_double), ("T_mean", C.c_double), ("T_amp", C.c_double),
                ("P_mean", C.c_double), ("P_amp", C.c_double), ("period", C.c_double), ("phase_T", C.c_double),
                ("phase_P", C.c_double), ("noise", C.c_void_p), ("noise_len", C.c_int32),
                ("noise_dt", C.c_double), ("period_P", C.c_double)]


class hygro_room(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("volume", "ach", "Q_gain", "g_vap", "T_out_mean", "T_out_amp",
                                          "P_out_mean", "P_out_amp", "period", "phase_T", "phase_P", "rho_a",
                                          "cp_a", "cp_v", "Pv_ref", "Ta0", "Pa0", "period_P", "g_pulse",
                                          "pulse_on", "pulse_off", "pulse_period")]


class HygroError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False) -> C.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise ImportError(f"hygro CUDA library not built ({path}); run paper_1703_10119_gb300.build.build()")
    L = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "hygro_create": [C.POINTER(hygro_desc), C.POINTER(P)],
        "hygro_set_materials": [P, P, P, P, P, P],
        "hygro_set_bc": [P, C.c_int32, P],
        "hygro_run": [P, C.c_int64, C.c_int32, P, C.c_size_t],
        "hygro_run_noalloc": [P, C.c_int64, C.c_int32, P, C.c_size_t],
        "hygro_sync": [P],
        "hygro_fluxes": [P, P, P],
        "hygro_get_fields": [P, C.c_int32, P, P],
        "hygro_set_fields": [P, C.c_int32, P, P],
        "hygro_balance": [P, P],
        "hygro_set_option": [P, C.c_int32, C.c_int64],
        "hygro_set_vapour_fraction": [P, P],
        "hygro_start_euler": [P],
        "hygro_get_step": [P, C.POINTER(C.c_int64)],
        "hygro_get_state": [P, P, C.POINTER(C.c_size_t)],
        "hygro_set_state": [P, P, C.c_size_t],
        "hygro_set_rooms": [P, C.c_int32, P, P],
        "hygro_get_rooms": [P, C.c_int32, P, P],
        "hygro_autotune": [P, C.c_int32, P, P],
        "hygro_set_layer_law": [P, P],
        "hygro_set_radiation": [P, P, P],
        "hygro_set_interzone": [P, C.c_int32, P, P],
        "hygro_loss_grad": [P, C.c_int64, C.c_int32, P, C.c_double, C.c_double, C.c_int32, C.POINTER(C.c_double), P],
        "hygro2d_create": [C.POINTER(hygro2d_desc), C.POINTER(P)],
        "hygro2d_set_materials": [P, C.c_int32, P, P, P, P],
        "hygro2d_set_bc": [P, C.c_int32, P],
        "hygro2d_run": [P, C.c_int64],
        "hygro2d_sync": [P],
        "hygro2d_get_fields": [P, C.c_int32, P, P],
        "hygro2d_set_fields": [P, C.c_int32, P, P],
        "hygro2d_get_step": [P, C.POINTER(C.c_int64)],
        "hygro2d_set_option": [P, C.c_int32, C.c_int64],
        "hygro2d_get_option": [P, C.c_int32, C.POINTER(C.c_int64)],
        "hygro2d_autotune": [P, C.c_int32, C.POINTER(C.c_int32), P],
        "hygro_peak_probe": [C.c_int32, C.c_int32, P, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.restype = C.c_int
        f.argtypes = args
    L.hygro_last_error.restype = C.c_char_p
    L.hygro_last_error.argtypes = [P]
    L.hygro_destroy.restype = None
    L.hygro_destroy.argtypes = [P]
    L.hygro2d_last_error.restype = C.c_char_p
    L.hygro2d_last_error.argtypes = [P]
    L.hygro2d_destroy.restype = None
    L.hygro2d_destroy.argtypes = [P]
    _lib = L
    return L


def _check(status: int, ctx) -> None:
    if status != HYGRO_OK:
        raise HygroError(status, lib().hygro_last_error(ctx).decode())


def _check2d(status: int, ctx) -> None:
    if status != HYGRO_OK:
        raise HygroError(status, lib().hygro2d_last_error(ctx).decode())


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _nbytes(a) -> int:
    if a is None:
        return 0
    if hasattr(a, "element_size"):
        return a.numel() * a.element_size()
    return a.nbytes


# ---- the C entry points, one to one ------------------------------------------

def hygro_create(desc: hygro_desc):
    out = C.c_void_p()
    _check(lib().hygro_create(C.byref(desc), C.byref(out)), None)
    return out


def hygro_set_materials(ctx, n_layers, layer_first, layers, T_init, P_init):
    _check(lib().hygro_set_materials(ctx, _ptr(n_layers), _ptr(layer_first), C.cast(layers, C.c_void_p),
                                     _ptr(T_init), _ptr(P_init)), ctx)


def hygro_set_bc(ctx, face: int, bcs):
    _check(lib().hygro_set_bc(ctx, int(face), C.cast(bcs, C.c_void_p)), ctx)


def hygro_run(ctx, n_steps: int, sample_every: int = 0, samples=None):
    _check(lib().hygro_run(ctx, int(n_steps), int(sample_every), _ptr(samples), _nbytes(samples)), ctx)


def hygro_run_noalloc(ctx, n_steps: int, sample_every: int = 0, samples=None):
    _check(lib().hygro_run_noalloc(ctx, int(n_steps), int(sample_every), _ptr(samples), _nbytes(samples)), ctx)


def hygro_sync(ctx):
    _check(lib().hygro_sync(ctx), ctx)


def hygro_start_euler(ctx):
    _check(lib().hygro_start_euler(ctx), ctx)


def hygro_fluxes(ctx, flux=None, cumulative=None):
    _check(lib().hygro_fluxes(ctx, _ptr(flux), _ptr(cumulative)), ctx)


def hygro_get_fields(ctx, level: int, T=None, P=None):
    _check(lib().hygro_get_fields(ctx, int(level), _ptr(T), _ptr(P)), ctx)


def hygro_balance(ctx, bal):
    """bal: float64 [n_walls, 2, 4] (host or device) receives S, B, D, M of the next step per wall and field."""
    _check(lib().hygro_balance(ctx, _ptr(bal)), ctx)


def hygro_set_fields(ctx, level: int, T=None, P=None):
    _check(lib().hygro_set_fields(ctx, int(level), _ptr(T), _ptr(P)), ctx)


def hygro_get_step(ctx) -> int:
    s = C.c_int64()
    _check(lib().hygro_get_step(ctx, C.byref(s)), ctx)
    return s.value


def hygro_get_state(ctx) -> bytes:
    n = C.c_size_t()
    _check(lib().hygro_get_state(ctx, None, C.byref(n)), ctx)
    buf = C.create_string_buffer(n.value)
    _check(lib().hygro_get_state(ctx, buf, C.byref(n)), ctx)
    return buf.raw


def hygro_set_state(ctx, image: bytes):
    buf = C.create_string_buffer(image, len(image))
    _check(lib().hygro_set_state(ctx, buf, len(image)), ctx)


def hygro_set_rooms(ctx, n_rooms: int, rooms, wall_area):
    _check(lib().hygro_set_rooms(ctx, int(n_rooms), C.cast(rooms, C.c_void_p) if rooms is not None else None,
                                 _ptr(wall_area)), ctx)


def hygro_set_option(ctx, option: int, value: int):
    _check(lib().hygro_set_option(ctx, int(option), int(value)), ctx)


def hygro_set_vapour_fraction(ctx, nu):
    _check(lib().hygro_set_vapour_fraction(ctx, _ptr(np.ascontiguousarray(nu, np.float64))), ctx)


def hygro_get_rooms(ctx, level: int, Ta=None, Pa=None):
    _check(lib().hygro_get_rooms(ctx, int(level), _ptr(Ta), _ptr(Pa)), ctx)


def hygro_loss_grad(ctx, n_steps: int, sample_every: int, obs, wT: float, wP: float, checkpoint_every: int = 0,
                    grad=None) -> float:
    """Misfit loss of a run from the initial state; ``grad`` ([total layers, 9] float64, host or device)
    receives its gradient. ``obs``: float32 [n_steps // sample_every, n_walls, 2, 2], host or device."""
    loss = C.c_double()
    _check(lib().hygro_loss_grad(ctx, int(n_steps), int(sample_every), _ptr(obs), float(wT), float(wP),
                                 int(checkpoint_every), C.byref(loss), _ptr(grad)), ctx)
    return loss.value


HYGRO_PEAK_FFMA, HYGRO_PEAK_FFMA2, HYGRO_PEAK_RCP, HYGRO_PEAK_DFMA = 0, 1, 2, 3


def hygro_peak_probe(kind: int, device: int = -1, stream=None, target_ms: float = 100.0):
    """One arithmetic-peak microbenchmark (include/hygro_peaks.h): (lane operations per second, ms)."""
    ops = C.c_double()
    ms = C.c_double()
    st = lib().hygro_peak_probe(int(kind), int(device), stream, float(target_ms), C.byref(ops), C.byref(ms))
    if st != HYGRO_OK:
        raise HygroError(st, f"hygro_peak_probe(kind={kind}) failed")
    return ops.value, ms.value


def hygro_set_radiation(ctx, emissivity, view):
    e = np.ascontiguousarray(emissivity, np.float64)
    v = np.ascontiguousarray(view, np.float64)
    _check(lib().hygro_set_radiation(ctx, _ptr(e), _ptr(v)), ctx)


def hygro_set_interzone(ctx, links):
    """links: [(room_i, room_j, flow kg/s), ...]."""
    z = np.ascontiguousarray([[a, b] for a, b, _ in links], np.int32).reshape(-1, 2)
    f = np.ascontiguousarray([g for _, _, g in links], np.float64)
    _check(lib().hygro_set_interzone(ctx, len(links), _ptr(z) if len(links) else None,
                                     _ptr(f) if len(links) else None), ctx)


def hygro_set_layer_law(ctx, law):
    law = np.ascontiguousarray(law, np.int32)
    _check(lib().hygro_set_layer_law(ctx, _ptr(law)), ctx)


def hygro_autotune(ctx, probe_steps: int, model=None, ms=None):
    _check(lib().hygro_autotune(ctx, int(probe_steps), _ptr(model), _ptr(ms)), ctx)


def hygro_last_error(ctx) -> str:
    return lib().hygro_last_error(ctx).decode()


def hygro_destroy(ctx):
    lib().hygro_destroy(ctx)


# ---- the 2D entry points, one to one ---------------------------------------------

def hygro2d_create(desc: hygro2d_desc):
    out = C.c_void_p()
    _check2d(lib().hygro2d_create(C.byref(desc), C.byref(out)), None)
    return out


def hygro2d_set_materials(ctx, n_regions: int, region, layers, T_init, P_init):
    _check2d(lib().hygro2d_set_materials(ctx, int(n_regions), _ptr(region), C.cast(layers, C.c_void_p),
                                         _ptr(T_init), _ptr(P_init)), ctx)


def hygro2d_set_bc(ctx, face: int, bcs):
    _check2d(lib().hygro2d_set_bc(ctx, int(face), C.cast(bcs, C.c_void_p)), ctx)


def hygro2d_run(ctx, n_steps: int):
    _check2d(lib().hygro2d_run(ctx, int(n_steps)), ctx)


def hygro2d_sync(ctx):
    _check2d(lib().hygro2d_sync(ctx), ctx)


def hygro2d_get_fields(ctx, level: int, T=None, P=None):
    _check2d(lib().hygro2d_get_fields(ctx, int(level), _ptr(T), _ptr(P)), ctx)


def hygro2d_set_fields(ctx, level: int, T=None, P=None):
    _check2d(lib().hygro2d_set_fields(ctx, int(level), _ptr(T), _ptr(P)), ctx)


def hygro2d_get_step(ctx) -> int:
    s = C.c_int64()
    _check2d(lib().hygro2d_get_step(ctx, C.byref(s)), ctx)
    return s.value


def hygro2d_set_option(ctx, option: int, value: int):
    _check2d(lib().hygro2d_set_option(ctx, int(option), int(value)), ctx)


def hygro2d_get_option(ctx, option: int) -> int:
    v = C.c_int64()
    _check2d(lib().hygro2d_get_option(ctx, int(option), C.byref(v)), ctx)
    return v.value


def hygro2d_autotune(ctx, probe_steps: int, ms_per_step=None) -> int:
    """Time each temporal blocking depth on probe_steps steps from the current state, keep the fastest."""
    k = C.c_int32()
    _check2d(lib().hygro2d_autotune(ctx, int(probe_steps), C.byref(k), _ptr(ms_per_step)), ctx)
    return k.value


def hygro2d_last_error(ctx) -> str:
    return lib().hygro2d_last_error(ctx).decode()


def hygro2d_destroy(ctx):
    lib().hygro2d_destroy(ctx)


def _bc_array(n: int, kind, par, noise):
    """hygro_bc[n] from kinds [n], rows [n, 13] (BC_FIELDS) and an optional noise table [n, len, 2] (kept
    alive by the caller)."""
    arr = (hygro_bc * n)()
    for i in range(n):
        p = par[i]
        b = arr[i]
        b.kind = int(kind[i])
        (b.hT, b.hM, b.q_inf, b.g_inf, b.T_mean, b.T_amp, b.P_mean, b.P_amp, b.period, b.phase_T,
         b.phase_P, b.noise_dt, b.period_P) = [float(x) for x in p]
        if noise is not None:
            b.noise = noise[i].ctypes.data
            b.noise_len = noise.shape[1]
    return arr


# ---- convenience wrapper over a Workload --------------------------------------

class Hygro:
    """A context holding one workload's walls on the GPU."""

    def __init__(self, wl, precision: str = "fp32", kernel: str = "persistent", device: int = 0, stream=None):
        self.wl = wl
        self.precision = {"fp32": HYGRO_FP32, "fp64": HYGRO_FP64}[precision]
        self.kernel = {"persistent": HYGRO_KERNEL_PERSISTENT, "plain": HYGRO_KERNEL_PLAIN}[kernel]
        self.dtype = np.float32 if self.precision == HYGRO_FP32 else np.float64
        self._keep = []
        n_nodes = np.ascontiguousarray(wl.n_nodes, np.int32)
        thick = np.ascontiguousarray(wl.thickness, np.float64)
        d = hygro_desc(n_walls=wl.n_walls, n_nodes=n_nodes.ctypes.data, thickness=thick.ctypes.data,
                       dt=wl.dt, t0=wl.t0, Lv=wl.Lv, Psat=wl.Psat, precision=self.precision, kernel=self.kernel,
                       device=device, stream=stream)
        self.ctx = hygro_create(d)
        try:
            self.set_materials()
            self.set_bc()
            if wl.rooms:
                self.set_rooms()
            if wl.vapour_frac is not None:
                hygro_set_vapour_fraction(self.ctx, wl.vapour_frac)
        except Exception:
            hygro_destroy(self.ctx)
            self.ctx = None
            raise

    def set_materials(self, layer_par=None):
        """Materials of the workload, or the per-layer parameters ``layer_par`` [total layers, 9] in their
        place (same layer map and initial state)."""
        wl = self.wl
        par = wl.layer_par if layer_par is None else np.asarray(layer_par, np.float64)
        lay = (hygro_layer * len(par))()
        for i, row in enumerate(par):
            lay[i] = hygro_layer(*[float(x) for x in row])
        hygro_set_materials(self.ctx, np.ascontiguousarray(wl.n_layers, np.int32),
                            np.ascontiguousarray(wl.layer_first, np.int32), lay,
                            np.ascontiguousarray(wl.T_init, np.float64), np.ascontiguousarray(wl.P_init, np.float64))
        if getattr(wl, "layer_law", None) is not None:
            hygro_set_layer_law(self.ctx, wl.layer_law)

    def set_bc(self):
        wl = self.wl
        for f in range(2):
            nz = None if wl.noise[f] is None else np.ascontiguousarray(wl.noise[f], np.float32)
            arr = _bc_array(wl.n_walls, wl.bc_kind[:, f], wl.bc_par[:, f], nz)
            for w in range(wl.n_walls):
                arr[w].room = int(wl.bc_room[w, f])
            hygro_set_bc(self.ctx, f, arr)

    def set_rooms(self):
        rm = self.wl.rooms
        par = np.asarray(rm["par"], np.float64)
        arr = (hygro_room * len(par))()
        for r in range(len(par)):
            arr[r] = hygro_room(*[float(x) for x in par[r, :15]], float(rm["Ta0"][r]), float(rm["Pa0"][r]),
                                *[float(x) for x in par[r, 16:21]])
        hygro_set_rooms(self.ctx, len(par), arr, np.ascontiguousarray(rm["wall_area"], np.float64))
        if rm.get("emissivity") is not None:
            hygro_set_radiation(self.ctx, np.asarray(rm["emissivity"], np.float64).reshape(-1, 2), rm["view"])
        if rm.get("links"):
            hygro_set_interzone(self.ctx, rm["links"])
        if par.shape[1] > 15 and np.any(par[:, 15] == 1.0):
            # the room rows' scheme slot (the oracle's layout): explicit Euler rooms
            hygro_set_option(self.ctx, HYGRO_OPT_ROOM_SCHEME, HYGRO_ROOM_EULER)

    def rooms(self, level: int = 0):
        n = len(self.wl.rooms["par"]) if self.wl.rooms else 0
        Ta = np.zeros(n)
        Pa = np.zeros(n)
        hygro_get_rooms(self.ctx, level, Ta, Pa)
        return Ta, Pa

    def run(self, n_steps: int, sample_every: int = 0, samples=None):
        """Advance; ``samples`` (numpy or torch, working dtype) receives surface values."""
        hygro_run(self.ctx, n_steps, sample_every, samples)

    def run_sampled(self, n_steps: int, sample_every: int) -> np.ndarray:
        ns = n_steps // sample_every
        out = np.zeros((ns, self.wl.n_walls, 2, 2), self.dtype)
        hygro_run(self.ctx, n_steps, sample_every, out)
        return out

    def sync(self):
        hygro_sync(self.ctx)

    def start_euler(self):
        """The first step by explicit Euler substeps (hygro_start_euler)."""
        hygro_start_euler(self.ctx)

    def loss_grad(self, n_steps: int, sample_every: int, obs, wT: float, wP: float, checkpoint_every: int = 0):
        """Misfit loss and its gradient [total layers, 9] (hygro_loss_grad)."""
        g = np.zeros((len(self.wl.layer_par), 9))
        obs = np.ascontiguousarray(obs, np.float32)
        L = hygro_loss_grad(self.ctx, n_steps, sample_every, obs, wT, wP, checkpoint_every, g)
        return L, g

    def fields(self, level: int = 0):
        n = self.wl.total_nodes
        T = np.zeros(n)
        P = np.zeros(n)
        hygro_get_fields(self.ctx, level, T, P)
        return T, P

    def set_fields(self, level: int, T, P):
        hygro_set_fields(self.ctx, level, np.ascontiguousarray(T, np.float64), np.ascontiguousarray(P, np.float64))

    def balance(self) -> np.ndarray:
        """Discrete balance (S, B, D, M) of the next step per wall and field (T, Pv), [n_walls, 2, 4]."""
        b = np.zeros((self.wl.n_walls, 2, 4))
        hygro_balance(self.ctx, b)
        return b

    def fluxes(self):
        f = np.zeros((self.wl.n_walls, 2, 2))
        c = np.zeros((self.wl.n_walls, 2, 2))
        hygro_fluxes(self.ctx, f, c)
        return f, c

    @property
    def step(self) -> int:
        return hygro_get_step(self.ctx)

    def autotune(self, probe_steps: int = 2000):
        """Refit the wall schedule's step-time model on a probe of this workload (hygro_autotune); returns
        (model a[4], b[4] in ns, probe ms with the previous and the refitted schedule)."""
        model = np.zeros(8)
        ms = np.zeros(2)
        hygro_autotune(self.ctx, probe_steps, model, ms)
        return model[:4], model[4:], ms

    def get_state(self) -> bytes:
        return hygro_get_state(self.ctx)

    def set_state(self, image: bytes):
        hygro_set_state(self.ctx, image)

    def close(self):
        if self.ctx is not None:
            hygro_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Hygro2D:
    """A context holding a batch of 2D sections (workloads.Section2D) on the GPU."""

    def __init__(self, sec, precision: str = "fp32", steps_per_launch: int = 0, device: int = 0, stream=None):
        self.sec = sec
        self.precision = {"fp32": HYGRO_FP32, "fp64": HYGRO_FP64}[precision]
        d = hygro2d_desc(n_grids=sec.n_grids, nx=sec.nx, ny=sec.ny, h=sec.h, dt=sec.dt, t0=sec.t0, Lv=sec.Lv,
                         Psat=sec.Psat, precision=self.precision, steps_per_launch=steps_per_launch, device=device,
                         stream=stream)
        self.ctx = hygro2d_create(d)
        try:
            self.set_materials()
            self.set_bc()
        except Exception:
            hygro2d_destroy(self.ctx)
            self.ctx = None
            raise

    def set_materials(self):
        sec = self.sec
        G, R = sec.region_par.shape[:2]
        lay = (hygro_layer * (G * R))()
        for i, row in enumerate(sec.region_par.reshape(G * R, -1)):
            lay[i] = hygro_layer(*[float(x) for x in row])
        hygro2d_set_materials(self.ctx, R, np.ascontiguousarray(sec.region, np.uint8), lay,
                              np.ascontiguousarray(sec.T_init, np.float64), np.ascontiguousarray(sec.P_init, np.float64))

    def set_bc(self):
        sec = self.sec
        for f in range(4):
            nz = None if sec.noise[f] is None else np.ascontiguousarray(sec.noise[f], np.float32)
            hygro2d_set_bc(self.ctx, f, _bc_array(sec.n_grids, sec.bc_kind[:, f], sec.bc_par[:, f], nz))

    def run(self, n_steps: int):
        hygro2d_run(self.ctx, n_steps)

    def set_option(self, option: int, value: int):
        hygro2d_set_option(self.ctx, option, value)

    def option(self, option: int) -> int:
        return hygro2d_get_option(self.ctx, option)

    def autotune(self, probe_steps: int = 16):
        """Pick the temporal blocking depth by timing each one (hygro2d_autotune); returns (depth, ms per
        step of depths 1..4)."""
        ms = np.zeros(4)
        k = hygro2d_autotune(self.ctx, probe_steps, ms)
        return k, ms

    def sync(self):
        hygro2d_sync(self.ctx)

    def fields(self, level: int = 0):
        shape = (self.sec.n_grids, self.sec.ny, self.sec.nx)
        T = np.zeros(shape)
        P = np.zeros(shape)
        hygro2d_get_fields(self.ctx, level, T, P)
        return T, P

    def set_fields(self, level: int, T, P):
        hygro2d_set_fields(self.ctx, level, None if T is None else np.ascontiguousarray(T, np.float64),
                           None if P is None else np.ascontiguousarray(P, np.float64))

    @property
    def step(self) -> int:
        return hygro2d_get_step(self.ctx)

    def close(self):
        if self.ctx is not None:
            hygro2d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
