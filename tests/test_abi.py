"""C-ABI checks that need no GPU: libhrm builds and loads, exports every
function include/hrm.h declares, and rejects bad arguments before touching
the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1105_3829_gb300 import build, hrm
    build.build()
    return hrm.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hrm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hrm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hrm_filter2d", "hrm_filter3d", "hrm_submit", "hrm_poll", "hrm_filter_batch",
                 "hrm_rank_filter2d", "hrm_server_create", "hrm_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(lib._name)
    missing = [n for n in declared_functions() if not hasattr(raw, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1105_3829_gb300 import hrm
    assert set(declared_functions()) <= set(hrm.SIGNATURES)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structures have the sizes and field offsets the C compiler
    gives the header's structs (a field added on one side only fails here)."""
    import shutil
    import subprocess
    from paper_1105_3829_gb300 import hrm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [hrm.hrm_job, hrm.hrm_request, hrm.hrm_plan, hrm.hrm_server_stats, hrm.hrm_topology_info]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hrm.h"', "int main(void) {"]
    for st in structs:
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (st.__name__, st.__name__))
        for f in st._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));'
                         % (st.__name__, f[0], st.__name__, f[0]))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                 text=True).stdout.splitlines())
    for st in structs:
        assert int(got[st.__name__]) == ctypes.sizeof(st), st.__name__
        for f in st._fields_:
            assert int(got[st.__name__ + "." + f[0]]) == getattr(st, f[0]).offset, (st.__name__, f[0])


def test_version_and_error_string(lib):
    from paper_1105_3829_gb300 import hrm
    assert hrm.hrm_version() == 110
    assert isinstance(hrm.last_error(), str)


def test_validation_without_device(lib):
    from paper_1105_3829_gb300 import hrm
    buf = ctypes.create_string_buffer(1 << 16)
    src = ctypes.addressof(buf)
    dst = src + (1 << 15)
    E = hrm.HRM_EINVAL
    assert hrm.hrm_filter2d(3, src, 64, dst, 64, 32, 8, 2, 0, 0, None) == E          # dtype
    assert hrm.hrm_filter2d(1, src, 64, dst, 64, 32, 8, 128, 0, 0, None) == E        # radius
    assert hrm.hrm_filter2d(1, src, 64, dst, 64, 32, 8, 2, 1, 0, None) == E          # border
    assert hrm.hrm_filter2d(1, src, 64, dst, 64, 32, 8, 2, 0, 2, None) == E          # flags
    assert hrm.hrm_filter2d(1, src, 16, dst, 64, 32, 8, 2, 0, 0, None) == E          # pitch
    assert hrm.hrm_filter2d(1, src, 64, src + 64, 64, 32, 8, 2, 0, 0, None) == E     # overlap
    assert hrm.hrm_filter2d(2, src + 1, 64, dst, 64, 16, 8, 2, 0, 0, None) == E      # alignment
    assert hrm.hrm_filter2d(1, 0, 0, 0, 0, 0, 5, 3, 0, 0, None) == hrm.HRM_OK        # empty
    assert hrm.hrm_filter3d(1, src, 32, 256, dst, 32, 256, 32, 8, 4, 20, 0, 0, None) == E  # radius 3D
    assert hrm.hrm_filter3d(1, src, 32, 100, dst, 32, 256, 32, 8, 4, 2, 0, 0, None) == E   # slice pitch
    assert hrm.hrm_rank_filter2d(1, src, 64, dst, 64, 32, 8, 1, 9, 0, 0, None) == E        # rank >= 9
    assert hrm.hrm_filter2d_lowprec(1, src, 64, dst, 64, 32, 8, 2, 13, None) == E          # drop bits
    assert "bits" in hrm.last_error()
    assert hrm.hrm_filter2d_video(1, src, 64, dst, 64, 32, 8, 2, None, None) == E           # no topology
    assert "topology" in hrm.last_error()


def test_plan_cache_roundtrip(lib, tmp_path):
    from paper_1105_3829_gb300 import hrm
    p = hrm.hrm_plan(128, 96, 40, 2, 2)
    hrm.set_plan(2, 2, 4096, 4096, 1, 15, p)
    path = str(tmp_path / "plans.txt")
    assert hrm.hrm_plan_save(path.encode()) == 0
    text = open(path).read()
    assert "2 2 4096 4096 1 15 0 128 96 40 2 2\n" in text
    # a line without the tree field (older files) and one with it
    open(path, "a").write("1 2 512 512 1 3 0 64 32 20 2\n1 2 512 512 1 4 1 128 32 20 2 1\n")
    assert hrm.hrm_plan_load(path.encode()) == 0
    got = hrm.get_plan(1, 2, 512, 512, 1, 3)
    assert (got.tile_width, got.strip_height, got.slot_kbytes, got.path, got.tree) == (64, 32, 20, 2, 0)
    got = hrm.get_plan(1, 2, 512, 512, 1, 4, adaptive=True)
    assert (got.tile_width, got.path, got.tree) == (128, 2, 1)
    got = hrm.get_plan(2, 2, 4096, 4096, 1, 15)
    assert (got.tile_width, got.strip_height, got.slot_kbytes, got.path, got.tree) == (128, 96, 40, 2, 2)
    for line in ("1 2 512 512 1 5 0 128 32 20 2 3\n", "1 2 512 512 1 5 0 128 32 20 2 1 7\n"):
        bad_file = tmp_path / "bad.txt"
        bad_file.write_text(line)
        assert hrm.hrm_plan_load(str(bad_file).encode()) == hrm.HRM_EINVAL
    bad = hrm.hrm_plan(100, 0, 0, 0)
    with pytest.raises(hrm.HRMError):
        hrm.set_plan(1, 2, 10, 10, 1, 3, bad)
    open(path, "a").write("garbage line\n")
    assert hrm.hrm_plan_load(path.encode()) == hrm.HRM_EINVAL


def test_batch_rejects_malformed_jobs(lib):
    from paper_1105_3829_gb300 import hrm
    jobs = (hrm.hrm_job * 1)()
    assert hrm.hrm_filter_batch(jobs, -1, None) == hrm.HRM_EINVAL
    assert hrm.hrm_filter_batch(jobs, 0, None) == hrm.HRM_OK


def test_environment_plan_cache_and_forced_path(lib, tmp_path):
    """HRM_PLAN_CACHE preloads a saved plan file; HRM_FORCE_PATH picks the
    kernel family for calls without an explicit plan (checked in fresh
    processes: both are read once per process)."""
    import subprocess
    import sys
    plans = tmp_path / "plans.txt"
    plans.write_text("# saved\n2 2 640 480 1 9 0 256 40 60 2\n")
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1105_3829_gb300 import hrm\n"
            "p = hrm.get_plan(2, 2, 640, 480, 1, 9)\n"
            "q = hrm.get_plan(2, 2, 640, 480, 1, 3)\n"
            "print(p.tile_width, p.strip_height, p.slot_kbytes, p.path, q.path)\n") % ROOT
    env = dict(os.environ, HRM_PLAN_CACHE=str(plans), HRM_FORCE_PATH="hist", CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.split() == ["256", "40", "60", "2", "2"]
    env = dict(os.environ, HRM_FORCE_PATH="sortnet", CUDA_VISIBLE_DEVICES="")
    env.pop("HRM_PLAN_CACHE", None)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.split()[3:] == ["1", "1"]


def test_server_topology_and_graph_arguments_without_device(lib):
    """Null handles and malformed arguments are refused on the host, before
    any device work (serving, frame-stream topologies, graphs, plans), and
    every refusal leaves its own message in hrm_last_error."""
    from paper_1105_3829_gb300 import hrm
    E = hrm.HRM_EINVAL
    buf = ctypes.create_string_buffer(1 << 16)
    src = ctypes.addressof(buf)

    def refused(call, code=E):
        # a different error first, so a stale message cannot pass for a fresh one
        assert hrm.hrm_filter2d(3, src, 64, src + (1 << 15), 64, 32, 8, 2, 0, 0, None) == E
        sentinel = hrm.last_error()
        assert call() == code
        msg = hrm.last_error()
        assert msg and msg != sentinel, msg
        return msg

    h = ctypes.c_void_p()
    arena = src
    refused(lambda: hrm.hrm_server_create(None, 1 << 20, 8, 0, ctypes.byref(h)))        # no arena
    refused(lambda: hrm.hrm_server_create(arena, 0, 8, 0, ctypes.byref(h)))              # empty arena
    refused(lambda: hrm.hrm_server_create(arena, 1 << 12, 0, 0, ctypes.byref(h)))        # no in-flight slots
    refused(lambda: hrm.hrm_server_create(arena, 1 << 12, 8, -1, ctypes.byref(h)))       # negative queue
    refused(lambda: hrm.hrm_server_create(arena, 1 << 12, 8, 0, None))                  # no output
    t = ctypes.c_uint64()
    refused(lambda: hrm.hrm_submit(None, None, ctypes.byref(t)))
    refused(lambda: hrm.hrm_poll(None, 1, 0))
    assert hrm.hrm_ticket_latency_us(None, 1) < 0
    refused(lambda: hrm.hrm_server_stats_get(None, None))
    assert hrm.hrm_server_destroy(None) == hrm.HRM_OK
    info = hrm.hrm_topology_info()
    refused(lambda: hrm.hrm_topology_get(None, None, ctypes.byref(info)))
    assert hrm.hrm_topology_destroy(None) == hrm.HRM_OK
    refused(lambda: hrm.hrm_topology_create(None))
    g = ctypes.c_void_p()
    jobs = (hrm.hrm_job * 1)()
    refused(lambda: hrm.hrm_batch_graph_create(jobs, 0, None, ctypes.byref(g)))
    refused(lambda: hrm.hrm_batch_graph_create(None, 1, None, ctypes.byref(g)))
    refused(lambda: hrm.hrm_batch_graph_launch(None, None))
    refused(lambda: hrm.hrm_batch_graph_status(None, None))
    refused(lambda: hrm.hrm_filter_batch_noalloc(jobs, -1, None))
    assert "64" in refused(lambda: hrm.hrm_filter_batch_noalloc((hrm.hrm_job * 65)(), 65, None))
    p = hrm.hrm_plan()
    refused(lambda: hrm.hrm_get_plan(2, 4, 64, 64, 1, 5, 0, ctypes.byref(p)))            # dims
    refused(lambda: hrm.hrm_set_plan(2, 2, 64, 64, 1, 5, 0, ctypes.byref(hrm.hrm_plan(64, 0, 0, 0))))   # tile width
    refused(lambda: hrm.hrm_set_plan(2, 2, 64, 64, 1, 5, 0, ctypes.byref(hrm.hrm_plan(0, 0, 0, 3))))    # path
    refused(lambda: hrm.hrm_set_plan(2, 2, 64, 64, 1, 5, 0, ctypes.byref(hrm.hrm_plan(0, 0, 0, 2, 3))))  # tree
