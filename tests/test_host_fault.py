"""CPU tests of the host-side fault injection (csrc/host_fault.h): HYGRO_FAULT=<entry point>:<n> makes the
n-th call of that C-ABI entry point fail with HYGRO_E_CUDA before it changes anything. The parser and the
call counter are checked through a g++-built shim; the library's own use of it through hygro_create, the
one entry point that reaches its checks without a GPU, in fresh processes (the variable is read once)."""
import ctypes as C
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    out = str(tmp_path_factory.mktemp("host_fault") / "libhost_logic.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                    "-I", os.path.join(ROOT, "paper_1703_10119_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host_logic_shim.cpp"), "-o", out], check=True)
    return C.CDLL(out)


def parse(lib, spec):
    name = C.create_string_buffer(64)
    n = C.c_int64(0)
    ok = lib.shim_parse_fault(None if spec is None else spec.encode(), name, C.byref(n))
    return (name.value.decode(), n.value) if ok else None


def test_parse(shim):
    assert parse(shim, "hygro_run:3") == ("hygro_run", 3)
    assert parse(shim, "hygro_set_bc:1") == ("hygro_set_bc", 1)
    assert parse(shim, "a:b:2") == ("a:b", 2)       # the count follows the last colon
    for bad in [None, "", "hygro_run", "hygro_run:", ":3", "hygro_run:0", "hygro_run:-2", "hygro_run:2x",
                "x" * 64 + ":1"]:
        assert parse(shim, bad) is None, bad


def test_only_the_nth_call_of_the_named_entry_point_fails(shim):
    names = ["hygro_run", "hygro_set_bc", "hygro_run", "hygro_run", "hygro_sync", "hygro_run"]
    arr = (C.c_char_p * len(names))(*[n.encode() for n in names])
    hits = (C.c_int32 * len(names))()
    shim.shim_fault_sequence(b"hygro_run:3", arr, len(names), hits)
    assert list(hits) == [0, 0, 0, 1, 0, 0]
    shim.shim_fault_sequence(b"hygro_sync:1", arr, len(names), hits)
    assert list(hits) == [0, 0, 0, 0, 1, 0]
    shim.shim_fault_sequence(b"hygro_run:9", arr, len(names), hits)
    assert list(hits) == [0] * len(names)
    shim.shim_fault_sequence(b"", arr, len(names), hits)
    assert list(hits) == [0] * len(names)


SCRIPT = r"""
import json
from paper_1703_10119_gb300 import hygro as H
out = []
for _ in range(3):
    try:
        H.hygro_create(H.hygro_desc(n_walls=0))
        out.append([0, ""])
    except H.HygroError as e:
        out.append([e.status, str(e)])
print(json.dumps(out))
"""


def _create_three_times(fault):
    env = dict(os.environ)
    env.pop("HYGRO_FAULT", None)
    if fault is not None:
        env["HYGRO_FAULT"] = fault
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    import json
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_library_fails_the_chosen_call_and_reports_it():
    from paper_1703_10119_gb300 import build, hygro as H

    build.build()
    plain = _create_three_times(None)
    assert [s for s, _ in plain] == [H.HYGRO_E_INVALID] * 3          # n_walls = 0 is refused every time
    faulty = _create_three_times("hygro_create:2")
    assert [s for s, _ in faulty] == [H.HYGRO_E_INVALID, H.HYGRO_E_CUDA, H.HYGRO_E_INVALID]
    assert "injected fault" in faulty[1][1] and "hygro_create" in faulty[1][1]
    other = _create_three_times("hygro_run:1")                       # another entry point: no effect here
    assert [s for s, _ in other] == [H.HYGRO_E_INVALID] * 3
