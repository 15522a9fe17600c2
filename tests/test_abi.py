"""The C-ABI library builds, loads and exports what include/rk.h declares
(CPU only: no call here reaches the GPU)."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1810_01051_gb300 import build_lib, rk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "rk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rk_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return rk.load()


def test_header_declares_binding_exports():
    assert header_functions() == sorted(rk.EXPORTS)


def test_every_declared_symbol_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build_lib.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (rk_\w+)$", out, flags=re.M))
    for name in header_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_library_is_built_for_sm103a():
    # every translation unit is compiled for sm_103a alone (a GPU test reads
    # the kernels' binary version back through rk_debug_binary_version)
    assert build_lib.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_strerror(lib):
    assert rk.strerror(rk.RK_OK) == "ok"
    assert "capacity" in rk.strerror(rk.RK_ECAPACITY)
    assert rk.strerror(99) == "unknown status"


def _build_raw(lib, pats, lens, opts=None):
    out = ctypes.c_void_p(123)
    cat = np.frombuffer(b"".join(pats) or b"\0", dtype=np.uint8).copy()
    ln = np.array(lens, dtype=np.uint32)
    rc = lib.rk_build(cat.ctypes.data, ln.ctypes.data, len(lens),
                      ctypes.byref(opts) if opts else None, ctypes.byref(out))
    return rc, out.value


def test_build_rejects_bad_patterns_before_any_cuda_call(lib):
    # empty pattern, overlong pattern, null output: RK_EINVAL, *out cleared
    assert _build_raw(lib, [b"ab", b""], [2, 0]) == (rk.RK_EINVAL, None)
    long = b"x" * (rk.RK_MAX_PATTERN_LEN + 1)
    assert _build_raw(lib, [long], [len(long)]) == (rk.RK_EINVAL, None)
    assert lib.rk_build(None, None, 3, None, None) == rk.RK_EINVAL
    for bad in (rk.BuildOpts(base_log2=61), rk.BuildOpts(filter=9), rk.BuildOpts(tile_bytes=1000),
                rk.BuildOpts(stages=1), rk.BuildOpts(warps=40)):
        assert _build_raw(lib, [b"ab"], [2], bad)[0] == rk.RK_EINVAL


def test_entry_points_reject_null_table(lib):
    assert lib.rk_scan_device(None, None, 0, None, 0, None, None) == rk.RK_EINVAL
    assert lib.rk_sort_device(None, 0, None, 0, None, None, 0, None) == rk.RK_EINVAL
    assert lib.rk_search_device(None, None, 0, None, 0, None, None, 0, None) == rk.RK_EINVAL
    cnt = ctypes.c_uint64(7)
    assert lib.rk_search(None, None, 0, None, 0, ctypes.byref(cnt)) == rk.RK_EINVAL
    assert lib.rk_table_info_get(None, None) == rk.RK_EINVAL
    assert lib.rk_workspace_bytes(None, 10) == 0
    assert lib.rk_sort_launches(None, 10, 10, None) == rk.RK_EINVAL
    assert lib.rk_scan_workspace_bytes(None, 10) == 0
    assert lib.rk_scan_launches(None, 10, 10, None) == rk.RK_EINVAL
    assert lib.rk_scan_device_ws(None, None, 0, None, 0, None, None, 0, None) == rk.RK_EINVAL
    assert lib.rk_scan_device_ws_split(None, None, 0, None, 0, None, None, 0, None, None) == rk.RK_EINVAL
    lib.rk_destroy(None)


def test_window_hashes_rejects_bad_arguments(lib):
    assert lib.rk_window_hashes_device(None, 10, 0, 8, None, None) == rk.RK_EINVAL
    assert lib.rk_window_hashes_device(None, 10, 3, 61, None, None) == rk.RK_EINVAL
    # L > n writes nothing and succeeds without touching the device
    assert lib.rk_window_hashes_device(None, 2, 3, 8, None, None) == rk.RK_OK


def test_unpack_keys():
    keys = np.array([(5 << 40) | 17, (0 << 40) | ((1 << 40) - 1)], dtype=np.uint64)
    ids, offs = rk.unpack_keys(keys)
    assert ids.tolist() == [5, 0] and offs.tolist() == [17, (1 << 40) - 1]


def test_handle_entry_points_reject_null(lib):
    # every call on a batch, table set or server checks its handle before any
    # CUDA call; the destroys ignore NULL
    n = ctypes.c_uint64(5)
    out = ctypes.c_void_p(9)
    assert lib.rk_tableset_build(0, None, None, None, None, ctypes.byref(out)) == rk.RK_EINVAL
    assert lib.rk_batch_create(None, None, ctypes.byref(out)) == rk.RK_EINVAL
    assert out.value is None  # cleared on error
    assert lib.rk_batch_set(None, 0, None, None, None, None) == rk.RK_EINVAL
    assert lib.rk_batch_run(None, None) == rk.RK_EINVAL
    assert lib.rk_batch_results(None, None, None, None) == rk.RK_EINVAL
    info = (ctypes.c_uint64 * 2)()
    assert lib.rk_batch_read(None, None, 0, None, info, None) == rk.RK_EINVAL
    assert lib.rk_batch_autotune(None, 0, 0, None, None) == rk.RK_EINVAL
    assert lib.rk_batch_info_get(None, None) == rk.RK_EINVAL
    assert lib.rk_server_create(None, None, ctypes.byref(out)) == rk.RK_EINVAL
    assert lib.rk_server_submit(None, 0, None, 0, ctypes.byref(n)) == rk.RK_EINVAL
    assert lib.rk_server_take(None, 1, 0, None, 0, ctypes.byref(n), None) == rk.RK_EINVAL
    assert lib.rk_server_stats_get(None, None) == rk.RK_EINVAL
    assert lib.rk_search_device_noalloc(None, None, 0, None, 0, None, None) == rk.RK_EINVAL
    cnt = ctypes.c_uint64(5)
    mp = ctypes.c_void_p(7)
    assert lib.rk_search_matches(None, None, 0, ctypes.byref(mp), ctypes.byref(cnt)) == rk.RK_EINVAL
    assert mp.value is None and cnt.value == 0  # cleared on error
    assert lib.rk_search_device_matches(None, None, 0, None, None, 0, ctypes.byref(cnt)) == rk.RK_EINVAL
    assert lib.rk_debug_binary_version(None) == rk.RK_EINVAL
    lib.rk_free_matches(None)
    # a null pattern pointer or a bad length is refused before any CUDA call
    a = ctypes.create_string_buffer(b"abc")
    ptrs = (ctypes.c_void_p * 2)(ctypes.addressof(a), None)
    lens = (ctypes.c_uint32 * 2)(3, 3)
    assert lib.rk_build_ptrs(ptrs, lens, 2, None, ctypes.byref(mp)) == rk.RK_EINVAL
    lens[1] = 0
    ptrs[1] = ctypes.addressof(a)
    assert lib.rk_build_ptrs(ptrs, lens, 2, None, ctypes.byref(mp)) == rk.RK_EINVAL
    # the paper's kernel checks its pattern and launch shape first
    pat = np.frombuffer(b"ACGT", dtype=np.uint8).copy()
    assert lib.rk_paper_search_device(None, 10, None, 4, None, 0, None) == rk.RK_EINVAL
    assert lib.rk_paper_search_device(None, 10, pat.ctypes.data, 0, None, 0, None) == rk.RK_EINVAL
    assert lib.rk_paper_search_device(None, 10, pat.ctypes.data, 4, None, 48, None) == rk.RK_EINVAL
    lib.rk_batch_destroy(None)
    lib.rk_tableset_destroy(None)
    lib.rk_server_destroy(None)


def test_binding_types_match_header(lib):
    # every declared function has argument types in the binding and the
    # header's return type (a uint64_t left as the ctypes default int would
    # be truncated)
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "rk.h")).read(), flags=re.S)
    decl = {m.group(2): m.group(1).strip()
            for m in re.finditer(r"\b((?:const\s+)?\w+\s*\*?)\s*(rk_\w+)\s*\(", src)}
    want = {"int": ctypes.c_int, "uint64_t": ctypes.c_uint64, "void": None,
            "const char *": ctypes.c_char_p}
    assert set(decl) == set(rk.EXPORTS)
    nparams = {}
    for m in re.finditer(r"\b(rk_\w+)\s*\(([^)]*)\)\s*;", src):
        params = m.group(2).strip()
        nparams[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    for name, ret in decl.items():
        f = getattr(lib, name)
        assert ret in want, (name, ret)
        assert f.restype == want[ret], (name, ret, f.restype)
        assert f.argtypes is not None, name
        assert len(f.argtypes) == nparams[name], (name, len(f.argtypes), nparams[name])


# ctypes mirror of each C struct: (C name, binding class)
STRUCTS = [("rk_build_opts", "BuildOpts"), ("rk_table_info", "TableInfo"), ("rk_match", "Match"),
           ("rk_batch_opts", "BatchOpts"), ("rk_batch_info", "BatchInfo"),
           ("rk_server_opts", "ServerOpts"), ("rk_request_times", "RequestTimes"),
           ("rk_server_stats", "ServerStats")]


def test_struct_layouts_match_header(tmp_path):
    # a C program compiled against include/rk.h prints every struct's size and
    # field offsets; the binding's ctypes structures must agree field by field
    import shutil
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not found")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rk.h"', "int main(void) {"]
    for cname, pyname in STRUCTS:
        cls = getattr(rk, pyname)
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-Wall", f"-I{os.path.join(ROOT, 'include')}", str(src),
                    "-o", str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out.splitlines()}
    for cname, pyname in STRUCTS:
        cls = getattr(rk, pyname)
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert got[(cname, field)] == getattr(cls, field).offset, (cname, field)


def test_binding_refuses_buffers_a_call_cannot_use(lib):
    # refused in the binding, before any CUDA call (null table handles, so a
    # check that let a buffer through would still end in RK_EINVAL, not a
    # crash; the message tells which refused): host memory where the call
    # reads device memory (a kernel would fault on it), too few bytes for what
    # the call touches, non-contiguous views
    torch = pytest.importorskip("torch")
    host_t = torch.zeros(64, dtype=torch.int64)
    info = torch.zeros(2, dtype=torch.int64)
    arr = np.zeros(64, dtype=np.uint64)
    cases = [
        (lambda: rk.rk_scan_device(0, 0, 0, host_t, 64, 0), "CUDA tensor is required"),
        (lambda: rk.rk_search_device(0, 0, 0, arr, 64, 0, 0, 0), "numpy array is host memory"),
        (lambda: rk.rk_sort_device(0, 10, 0, 0, info, 0, 0), "CUDA tensor is required"),
        (lambda: rk.rk_search(0, np.zeros(10, np.uint8), 10, arr, 65), "bytes, the call needs"),
        (lambda: rk.rk_search(0, np.zeros(20, np.uint8)[::2], 10, arr, 8), "not contiguous"),
        (lambda: rk.rk_window_hashes_device(host_t, 100, 4, 8, 0), "CUDA tensor is required"),
        (lambda: rk.rk_paper_search_device(0, 16, b"ab", arr), "numpy array is host memory"),
    ]
    for call, why in cases:
        with pytest.raises(rk.RkError) as e:
            call()
        assert e.value.code == rk.RK_EINVAL and why in str(e.value), (why, str(e.value))
    # raw addresses pass through to the library, which checks what it can
    with pytest.raises(rk.RkError) as e:
        rk.rk_scan_device(0, 0, 0, 0, 0, 0)
    assert e.value.code == rk.RK_EINVAL and "rk_scan_device" in str(e.value)


def compile_c_example(tmp_path):
    """tests/c_api_example.c compiled and linked against include/rk.h and
    librk.so, as a C user would (returns the executable's path)."""
    import shutil
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not found")
    build_lib.build()
    lib_dir = os.path.dirname(build_lib.LIB)
    exe = tmp_path / "c_api_example"
    subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", f"-I{os.path.join(ROOT, 'include')}",
                    os.path.join(ROOT, "tests", "c_api_example.c"), f"-L{lib_dir}", "-lrk",
                    f"-Wl,-rpath,{lib_dir}", "-o", str(exe)], check=True, capture_output=True,
                   text=True)
    return str(exe)


def test_c_example_builds_and_fails_cleanly_without_a_device(tmp_path):
    exe = compile_c_example(tmp_path)
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: tests/test_gpu_search.py runs the example")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    # no device: the status comes back as RK_ECUDA, nothing aborts
    assert r.returncode == 1 and "rk_build: CUDA error" in r.stderr, (r.returncode, r.stderr)
