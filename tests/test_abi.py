"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/*.h declares; argument validation runs on the host."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2011_00459_gb300 import build, tds

    build.build()
    return tds.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(tds_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "tds_step" in names and "tds_create_scene" in names
    for name in names:
        assert hasattr(L, name), name


def test_binding_covers_the_header():
    from paper_2011_00459_gb300 import tds

    assert set(declared_functions()) <= set(tds.EXPORTED)


def test_invalid_descriptions_are_rejected_on_the_host(L):
    from paper_2011_00459_gb300 import tds

    nb = ctypes.c_uint64()
    assert L.tds_workspace_bytes(None, ctypes.byref(nb)) == -1
    assert b"desc" in L.tds_last_error()
    d = tds.SceneDesc()
    d.n = 0
    assert L.tds_workspace_bytes(ctypes.byref(d), ctypes.byref(nb)) == -1
    import numpy as np

    x = np.zeros(4, np.float32)
    r = np.full(4, 0.05, np.float32)
    d.n = 4
    d.x = d.y = d.z = tds._fptr(x)
    d.radius = tds._fptr(r)
    d.density, d.young, d.poisson, d.dt, d.max_iters = 2000.0, 1e9, 0.15, 1 / 60, 10
    assert L.tds_workspace_bytes(ctypes.byref(d), ctypes.byref(nb)) == 0
    assert nb.value > 0
    d.poisson = 0.7
    assert L.tds_workspace_bytes(ctypes.byref(d), ctypes.byref(nb)) == -1
    d.poisson = 0.15
    r[2] = -1.0
    assert L.tds_workspace_bytes(ctypes.byref(d), ctypes.byref(nb)) == -1
    r[2] = 0.05
    d.n_walls = 30
    assert L.tds_workspace_bytes(ctypes.byref(d), ctypes.byref(nb)) == -1
    d.n_walls = 0
    d.warm_start = 7
    assert L.tds_workspace_bytes(ctypes.byref(d), ctypes.byref(nb)) == -1


def test_null_scene_calls_fail_cleanly(L):
    assert L.tds_step(None, 1) == -1
    assert L.tds_synchronize(None) == -1
    f = (ctypes.c_float * 3)()
    assert L.tds_read_tool_force(None, f, f) == -1
    L.tds_destroy_scene(None)


def test_batch_descriptions_are_checked_on_the_host(L):
    """A batch sizes its workspace from all scenes and refuses scenes whose
    shared settings (step, material, solver) differ."""
    import numpy as np
    from paper_2011_00459_gb300 import tds
    from tests.parity_cases import packed_scene

    a, b = packed_scene(300, 1, iters=30), packed_scene(500, 2, iters=30)
    da, ka, _ = tds._make_desc(a, 0, None)
    db, kb, _ = tds._make_desc(b, 0, None)
    arr = (tds.SceneDesc * 2)(da, db)
    nb, n1, n2 = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    assert L.tds_batch_workspace_bytes(arr, 2, ctypes.byref(nb)) == 0
    assert L.tds_workspace_bytes(ctypes.byref(da), ctypes.byref(n1)) == 0
    assert L.tds_workspace_bytes(ctypes.byref(db), ctypes.byref(n2)) == 0
    assert nb.value > max(n1.value, n2.value)
    assert L.tds_batch_workspace_bytes(arr, 0, ctypes.byref(nb)) == -1
    arr[1].dt = np.float32(1 / 120)
    assert L.tds_batch_workspace_bytes(arr, 2, ctypes.byref(nb)) == -1
    assert b"share" in L.tds_last_error()
    arr[1].dt = arr[0].dt
    arr[1].mu_t = 0.9  # friction may differ per scene
    assert L.tds_batch_workspace_bytes(arr, 2, ctypes.byref(nb)) == 0
    assert L.tds_set_graph(None, 1) == -1
    assert L.tds_batch_set_tool_poses(None, None, 0) == -1
    del ka, kb


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding mirrors has the size and field offsets the C
    compiler gives the header's declaration (a C program built from
    include/tds.h prints them)."""
    import ctypes
    import shutil
    import subprocess

    from paper_2011_00459_gb300 import tds

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    pairs = {"tds_scene_desc": tds.SceneDesc, "tds_step_stats": tds.StepStats, "tds_zone": tds.Zone,
             "tds_aggregate": tds.Aggregate, "tds_grid": tds.Grid, "tds_cutter": tds.Cutter,
             "tds_launch_config": tds.LaunchConfig}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tds.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for cname, cls in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert got[(cname, field)] == getattr(cls, field).offset, (cname, field)


def test_solver_shapes_agree_everywhere():
    """The solver CTA shapes the library compiles (tds_solve.cu), the
    binding's and the tuner's lists and the header's documentation name the
    same shapes, the first being the default; every shape's staged wave keeps
    the bulk copies 16-byte aligned and fits in shared memory."""
    from paper_2011_00459_gb300 import autotune, tds

    src = open(os.path.join(ROOT, "paper_2011_00459_gb300", "csrc", "tds_solve.cu")).read()
    m = re.search(r"constexpr int kShapes\[\]\[3\] = \{(.*?)\};", src, flags=re.S)
    compiled = [tuple(int(v) for v in t) for t in re.findall(r"\{(\d+),\s*(\d+),\s*(\d+)\}", m.group(1))]
    assert [s[:2] for s in compiled] == list(tds.SHAPES)
    assert compiled == [tuple(s) for s in autotune.SHAPES]
    header = open(os.path.join(ROOT, "include", "tds.h")).read()
    doc = re.sub(r"\s+", " ", header[header.index("pgs_threads x pgs_per_thread"):][:400])
    for t, p, _ in compiled:
        assert f"{t}x{p}" in doc, (t, p)
    assert f"{compiled[0][0]}x{compiled[0][1]} (the default" in doc
    row = int(re.search(r"constexpr size_t kRowBytes = (\d+);", src).group(1))
    offs = [int(v) for v in re.findall(r"kOff[A-Za-z]+ = (\d+)", src)]
    stages = int(re.search(r"constexpr int kStages = (\d+);", src).group(1))
    for t, p, ctas in compiled:
        wave = (t - 32) * p  # the last warp stages, the others solve
        assert all(o * wave % 16 == 0 for o in offs) and row * wave % 128 == 0, (t, p)
        dyn = stages * row * wave
        assert dyn + 8192 <= 227 * 1024, (t, p)  # per CTA, beside the static shared memory
        assert ctas * (dyn + 8192) <= 228 * 1024, (t, p)  # the CTAs an SM holds
