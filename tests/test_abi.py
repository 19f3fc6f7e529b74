"""The C-ABI library loads and exports every entry point include/hygro.h declares;
argument validation that needs no GPU."""
import ctypes as C
import os
import re

import pytest

from paper_1703_10119_gb300 import build as hb
from paper_1703_10119_gb300 import hygro as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header=None):
    names = set()
    for h in ([header] if header else ("hygro.h", "hygro2d.h", "hygro_peaks.h")):
        src = open(os.path.join(ROOT, "include", h)).read()
        names |= set(re.findall(r"HYGRO_API\s+[\w\s\*]*?\b(hygro2?d?_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    hb.build()
    return H.lib()


def test_header_declares_the_boundary():
    names = _declared("hygro.h")
    for must in ("hygro_create", "hygro_set_materials", "hygro_set_bc", "hygro_run", "hygro_fluxes"):
        assert must in names
    assert set(names) == set(H.ABI_FUNCTIONS)
    names2d = _declared("hygro2d.h")
    assert set(names2d) == set(H.ABI_FUNCTIONS_2D)
    assert set(_declared("hygro_peaks.h")) == set(H.ABI_FUNCTIONS_PEAKS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_exports_nothing_else(lib):
    out = os.popen(f"nm -D --defined-only {hb.LIB}").read()
    exported = sorted(set(re.findall(r"\bT (hygro2?d?_\w+)", out)))
    assert exported == _declared()


def test_struct_sizes_match_header_layout():
    assert C.sizeof(H.hygro_layer) == 9 * 8
    assert C.sizeof(H.hygro_desc) == 4 + 4 + 8 + 8 + 8 * 4 + 4 * 3 + 4 + 8
    assert C.sizeof(H.hygro_bc) == 8 + 8 * 11 + 8 + 8 + 8 + 8
    assert C.sizeof(H.hygro_room) == 22 * 8


def test_struct_layout_matches_the_c_compiler(tmp_path):
    """Size and field offsets of the binding's structs against the C compiler's reading of the header."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"hygro_desc": H.hygro_desc, "hygro_layer": H.hygro_layer, "hygro_bc": H.hygro_bc,
               "hygro_room": H.hygro_room}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hygro.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for f in cls._fields_:
            assert got[(name, f[0])] == getattr(cls, f[0]).offset, (name, f[0])


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    with pytest.raises(H.HygroError) as e:
        H.hygro_create(H.hygro_desc(n_walls=0))
    assert e.value.status == H.HYGRO_E_INVALID
    import numpy as np
    n = np.array([2], np.int32)
    L = np.array([0.1])
    d = H.hygro_desc(n_walls=1, n_nodes=n.ctypes.data, thickness=L.ctypes.data, dt=1.0, Psat=2337.0)
    with pytest.raises(H.HygroError) as e:
        H.hygro_create(d)
    assert e.value.status == H.HYGRO_E_INVALID and "n_nodes" in str(e.value)
    n[0] = 600
    with pytest.raises(H.HygroError) as e:
        H.hygro_create(d)
    assert e.value.status == H.HYGRO_E_UNSUPPORTED
    n[0] = 10
    d.dt = -1.0
    with pytest.raises(H.HygroError) as e:
        H.hygro_create(d)
    assert e.value.status == H.HYGRO_E_INVALID
    assert lib.hygro_create(None, None) == H.HYGRO_E_INVALID


def test_null_context_calls_are_rejected(lib):
    assert lib.hygro_run(None, 1, 0, None, 0) == H.HYGRO_E_INVALID
    assert lib.hygro_sync(None) == H.HYGRO_E_INVALID
    lib.hygro_destroy(None)


def test_2d_desc_layout_and_rejections_before_touching_the_device(lib):
    assert C.sizeof(H.hygro2d_desc) == 3 * 4 + 4 + 5 * 8 + 3 * 4 + 4 + 8
    good = dict(n_grids=1, nx=8, ny=8, h=1e-3, dt=60.0, Psat=2337.0)
    for bad in (dict(n_grids=0), dict(nx=1), dict(ny=1), dict(h=0.0), dict(dt=-1.0), dict(Psat=0.0),
                dict(precision=2), dict(steps_per_launch=9), dict(steps_per_launch=-1)):
        d = H.hygro2d_desc(**{**good, **bad})
        with pytest.raises(H.HygroError) as e:
            H.hygro2d_create(d)
        assert e.value.status == H.HYGRO_E_INVALID, bad
    d = H.hygro2d_desc(**{**good, "precision": H.HYGRO_FP64, "steps_per_launch": 9})
    with pytest.raises(H.HygroError) as e:
        H.hygro2d_create(d)
    assert e.value.status == H.HYGRO_E_INVALID and "steps_per_launch" in str(e.value)
    assert lib.hygro2d_create(None, None) == H.HYGRO_E_INVALID
    assert lib.hygro2d_run(None, 1) == H.HYGRO_E_INVALID
    assert lib.hygro2d_sync(None) == H.HYGRO_E_INVALID
    lib.hygro2d_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built CUDA library the binding raises; there is no other code path to fall back on."""
    monkeypatch.setattr(H, "_lib", None)
    monkeypatch.setattr(H, "library_path", lambda: str(tmp_path / "absent" / "libhygro.so"))
    with pytest.raises(ImportError, match="not built"):
        H.lib()


def test_no_device_is_an_error_not_a_fallback(lib):
    """A valid description on a machine without a CUDA device gives HYGRO_E_CUDA from hygro_create: the
    library computes on the GPU only."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import numpy as np
    n = np.array([10, 12], np.int32)
    L = np.array([0.1, 0.2])
    d = H.hygro_desc(n_walls=2, n_nodes=n.ctypes.data, thickness=L.ctypes.data, dt=60.0, Psat=2337.0,
                     Lv=2.5e6)
    with pytest.raises(H.HygroError) as e:
        H.hygro_create(d)
    assert e.value.status == H.HYGRO_E_CUDA
