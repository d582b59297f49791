"""The autotuner's host side, without a GPU: the enable switch (and VKT_AUTOTUNE=0 in the
environment), and the JSON cache file that vktAutotuneSave writes and vktAutotuneLoad reads."""
import ctypes
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2203_10213_gb300 as m
    return m._lib


def count(lib):
    n = ctypes.c_int32()
    assert lib.vktAutotuneGetCount(ctypes.byref(n)) == 0
    return n.value


def test_enable_switch_roundtrip(lib):
    e = ctypes.c_int32()
    assert lib.vktAutotuneGetEnabled(ctypes.byref(e)) == 0
    old = e.value
    assert lib.vktAutotuneSetEnabled(0) == 0
    assert lib.vktAutotuneGetEnabled(ctypes.byref(e)) == 0 and e.value == 0
    assert lib.vktAutotuneSetEnabled(7) == 0
    assert lib.vktAutotuneGetEnabled(ctypes.byref(e)) == 0 and e.value == 1
    assert lib.vktAutotuneSetEnabled(old) == 0
    assert lib.vktAutotuneGetEnabled(None) == 1


def test_environment_switches_the_tuner_off():
    code = ("import ctypes, paper_2203_10213_gb300 as m; e = ctypes.c_int32(); "
            "m._lib.vktAutotuneGetEnabled(ctypes.byref(e)); print(e.value)")
    env = dict(os.environ, VKT_AUTOTUNE="0")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                         text=True, check=True)
    assert out.stdout.strip() == "0"
    env["VKT_AUTOTUNE"] = "1"
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                         text=True, check=True)
    assert out.stdout.strip() == "1"


def test_cache_file_roundtrip(lib, tmp_path):
    src = tmp_path / "in.json"
    entries = [
        {"key": "filter k5 dense-tc s2 d2 volume 1024x1024x512 sm152", "path": 3, "zchunk": 0, "ms": 3.25},
        {"key": "filter k3 dense s0 d2 volume 512x512x512 sm152", "path": 1, "zchunk": 32, "ms": 0.201},
        {"key": "batch n256 00ff00ff00ff00ff", "path": 1, "zchunk": 32, "ms": 1.5},
    ]
    with open(src, "w") as f:
        f.write('{"vkt_autotune": 1, "entries": [\n')
        f.write(",\n".join(json.dumps(e) for e in entries))
        f.write("\n]}\n")
    assert lib.vktAutotuneClear() == 0
    assert count(lib) == 0
    assert lib.vktAutotuneLoad(str(src).encode()) == 0
    assert count(lib) == 3
    out = tmp_path / "out.json"
    assert lib.vktAutotuneSave(str(out).encode()) == 0
    data = json.load(open(out))
    assert data["vkt_autotune"] == 1
    got = {e["key"]: e for e in data["entries"]}
    assert set(got) == {e["key"] for e in entries}
    for e in entries:
        g = got[e["key"]]
        assert (g["path"], g["zchunk"]) == (e["path"], e["zchunk"])
        assert abs(g["ms"] - e["ms"]) <= 1e-5 * e["ms"]
    # loading merges: an entry read again keeps one copy
    assert lib.vktAutotuneLoad(str(out).encode()) == 0
    assert count(lib) == 3
    assert lib.vktAutotuneClear() == 0
    assert count(lib) == 0


def test_cache_file_errors(lib, tmp_path):
    assert lib.vktAutotuneLoad(str(tmp_path / "missing.json").encode()) == 1
    assert lib.vktAutotuneSave(str(tmp_path / "no" / "dir.json").encode()) == 1
    assert lib.vktAutotuneLoad(None) == 1
    assert lib.vktAutotuneGetCount(None) == 1
