"""Host-side checks of the C-ABI library: it builds for sm_103a, loads without a GPU and
exports every entry point include/rgs.h declares; argument validation runs before any
device work."""
import ctypes as ct
import os
import re

import pytest

from paper_2509_18497_gb300 import build, rgs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rgs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rgs_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    lib_path = build.build()
    lib = ct.CDLL(lib_path)
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(rgs.EXPORTS) == names


def test_abi_version_and_status_strings():
    L = rgs.load()
    assert rgs.rgs_abi_version() == 1
    for code in range(8):
        assert L.rgs_status_string(code).decode()
    assert rgs.rgs_launch_count() >= 0


def test_argument_validation_without_device_work():
    L = rgs.load()
    h = ct.c_void_p(None)
    # NULL surfel struct
    assert L.rgs_build_scene(None, None, None, ct.byref(h)) == 1
    assert b"NULL" in L.rgs_last_error()
    # n = 0, bad degree, NULL arrays
    for n, deg in ((0, 2), (10, 4), (10, -1)):
        sf = rgs.rgs_surfels(n, deg, *([ct.c_void_p(16)] * 9))
        assert L.rgs_build_scene(ct.byref(sf), None, None, ct.byref(h)) == 1
    sf = rgs.rgs_surfels(10, 2, *([None] * 9))
    assert L.rgs_build_scene(ct.byref(sf), None, None, ct.byref(h)) == 1
    opts = rgs.rgs_build_opts(7, 0)
    sf = rgs.rgs_surfels(10, 2, *([ct.c_void_p(16)] * 9))
    assert L.rgs_build_scene(ct.byref(sf), ct.byref(opts), None, ct.byref(h)) == 1
    assert not h.value
    # solve / adjoint / iterate on NULL handles
    assert L.rgs_solve(None, None, 1, 0, None, None, None) == 1
    assert L.rgs_adjoint(None, None, None, None, None, None) == 1
    assert L.rgs_get_iterate(None, 0, None, None) == 1
    # the center-to-center and geometry entry points on NULL handles
    assert L.rgs_trace_pairs(None, None, None, None, ct.byref(h)) == 1
    assert L.rgs_adjoint_pairs(None, None, None, None, None, None, None) == 1
    assert L.rgs_adjoint_pairs_geometry(None, None, None, None, None, None, None, None, None, None, None) == 1
    assert L.rgs_adjoint_geometry(None, None, None, None, None, None, None, None, None, None) == 1
    assert b"NULL" in L.rgs_last_error()
    L.rgs_destroy_scene(None)
    L.rgs_destroy_transport(None)


def test_service_entry_points_reject_bad_arguments_without_device_work():
    L = rgs.load()
    one = (ct.c_int32 * 1)(1)
    hs = (ct.c_void_p * 1)(None)
    # empty, oversized and NULL batches; a NULL transport inside a batch
    assert L.rgs_solve_batched(None, 1, None, one, None, None, None, None) == 1
    assert L.rgs_solve_batched(hs, 0, None, one, None, None, None, None) == 1
    assert L.rgs_solve_batched(hs, 4097, None, one, None, None, None, None) == 1
    assert L.rgs_solve_batched(hs, 1, None, None, None, None, None, None) == 1
    assert L.rgs_solve_batched(hs, 1, None, one, None, None, None, None) == 1
    assert b"NULL" in L.rgs_last_error()
    assert L.rgs_set_checkpointing(None, 2) == 1
    assert L.rgs_set_memory_budget(None, 1 << 20) == 1
    assert L.rgs_set_tensor_cores(None, 1) == 1
    assert L.rgs_set_wait_limit(None, 1000) == 1
    assert L.rgs_contraction_info(None, None, 6) == 1
    assert L.rgs_transport_info_get(None, None) == 1
    cam = (ct.c_float * 9)(0, 0, 2, 0, 0, -1, 0, 1, 0)
    assert L.rgs_render(None, p16 := ct.c_void_p(16), cam, 4, 4, 0.5, p16, None) == 1
    assert L.rgs_render_adjoint(None, p16, cam, 4, 4, 0.5, p16, None) == 1
    assert L.rgs_render(None, p16, None, 4, 4, 0.5, p16, None) == 1
    # the no-allocation norm: NULL arrays, negative and oversized lengths
    p = ct.c_void_p(16)
    assert L.rgs_residual_norm_noalloc(None, p, 1, p, None) == 1
    assert L.rgs_residual_norm_noalloc(p, p, -1, p, None) == 1
    assert L.rgs_residual_norm_noalloc(p, p, 1 << 40, p, None) == 1
    assert b"outside" in L.rgs_last_error()
    # the profiler's report wants an array when asked for entries
    assert L.rgs_profile_report(None, 4) == -1
    assert L.rgs_profile_report(None, 0) >= 0


def test_binding_checks_before_any_library_call():
    torch = pytest.importorskip("torch")
    cpu = torch.zeros(4, 3)
    with pytest.raises(TypeError, match="CUDA"):
        rgs.rgs_build_scene(cpu, cpu, cpu, torch.zeros(4, 2), torch.zeros(4), cpu, torch.zeros(4), cpu,
                            torch.zeros(4), 2)
    with pytest.raises(ValueError, match="n_bounces"):
        rgs.rgs_solve_batched([object(), object()], None, [3])
    with pytest.raises(ValueError, match="E_list"):
        rgs.rgs_solve_batched([object()], [None, None], [3])


def test_oracle_library_builds():
    from oracle import oracle as O
    assert os.path.exists(O.build())


def test_plain_c_client_compiles_links_and_runs(tmp_path):
    """include/rgs.h is a C header: a C99 client (tests/abi_c_client.c) compiles with
    -pedantic -Werror, links against librgs.so and runs the device-free entry points; the
    same header also compiles as C++."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib_dir = os.path.dirname(build.build())
    exe = str(tmp_path / "abi_c_client")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "abi_c_client.c"), "-o", exe, "-L", lib_dir, "-lrgs",
                    "-Wl,-rpath," + lib_dir], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    assert "ok" in out
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is not None:
        subprocess.run([cxx, "-std=c++11", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-x", "c++",
                        "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_c_client.c")], check=True)
