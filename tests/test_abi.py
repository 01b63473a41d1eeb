"""The C ABI library builds for sm_103a, loads without a GPU and exports every entry point
include/ivis.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", hdr)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ivis_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_all_declared_symbols():
    from paper_2609_17636_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert "ivis_cost_grad" in declared and "ivis_solve" in declared
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2609_17636_b300 import _lib
    assert sorted(_lib.EXPORTS) == _declared()


def test_missing_library_fails_loudly(tmp_path):
    from paper_2609_17636_b300 import _lib
    saved = _lib._LIB
    try:
        _lib._LIB = None
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._LIB = saved


def test_plan_rejects_bad_config_without_gpu():
    """Argument validation happens on the host before any device call."""
    from paper_2609_17636_b300 import _lib
    L = _lib.load()
    cfg = _lib.Config(64, 1, 1, 48, 1e-5, 0, 1e-9, 0, 0.0, 0.0, 1, 0, 0, 0, 0)  # nb not a power of two
    p = ctypes.c_void_p()
    st = L.ivis_plan(ctypes.byref(cfg), None, ctypes.byref(p))
    assert st == 1 and not p.value
    assert b"power of two" in L.ivis_last_error(None)


def test_rayleigh_jeans_entry_point_matches_the_oracle():
    """A host-only entry point: callable without a GPU."""
    import oracle
    from paper_2609_17636_b300 import rayleigh_jeans
    for f in (1.0e8, 1.4204058e9, 2.3e10):
        assert abs(rayleigh_jeans(f) - oracle.rayleigh_jeans_factor(f)) <= 1e-14 * oracle.rayleigh_jeans_factor(f)


GOOD = dict(n=64, nchan=1, npoint=1, nb=32, cell_rad=1e-5, precision=1, nufft_tol=1e-6,
            kernel_width=0, lambda_r=0.0, lambda_s=0.0, positivity=1, serial_pairs=0, autotune=0,
            toeplitz=0, wterm=0, grid_tile=0, grid_kernel=0)

# (overrides of a valid configuration, expected status, fragment of the error message)
BAD = [
    ({"n": 0}, 1, b">= 1"),
    ({"npoint": 0}, 1, b">= 1"),
    ({"nb": 8}, 1, b"power of two"),
    ({"nb": 4096}, 1, b"power of two"),
    ({"cell_rad": 0.0}, 1, b"cell_rad"),
    ({"cell_rad": float("inf")}, 1, b"cell_rad"),
    ({"precision": 7}, 1, b"precision"),
    ({"kernel_width": 1}, 1, b"kernel_width"),
    ({"kernel_width": 17}, 1, b"kernel_width"),
    ({"nufft_tol": 1.5}, 1, b"nufft_tol"),
    ({"lambda_r": -1.0}, 6, b"lambda"),
    ({"lambda_s": float("nan")}, 6, b"lambda"),
    ({"toeplitz": 1, "nb": 2048}, 1, b"toeplitz"),
    ({"toeplitz": 1, "serial_pairs": 1}, 1, b"exclusive"),
    ({"wterm": 1, "toeplitz": 1}, 1, b"wterm"),
    ({"wterm": 1, "nb": 2048, "cell_rad": 1e-3}, 1, b"too far"),
    ({"grid_tile": 48}, 1, b"grid_tile"),
    ({"grid_tile": 64, "precision": 0}, 1, b"grid_tile 64"),
    ({"grid_tile": 64, "nb": 16}, 1, b"grid_tile 64"),
    ({"grid_kernel": 3}, 1, b"grid_kernel"),
    ({"grid_kernel": -1}, 1, b"grid_kernel"),
]


@pytest.mark.parametrize("over,status,msg", BAD)
def test_plan_configuration_checks_run_on_the_host(over, status, msg):
    """Every configuration check of ivis_plan (include/ivis.h, ivis_config) happens before any
    device call: a bad field returns its status, no plan, and a message naming the field."""
    from paper_2609_17636_b300 import _lib
    L = _lib.load()
    cfg = _lib.Config(**{**GOOD, **over})
    p = ctypes.c_void_p()
    assert L.ivis_plan(ctypes.byref(cfg), None, ctypes.byref(p)) == status
    assert not p.value
    assert msg in L.ivis_last_error(None)


def test_entry_points_reject_null_handles_without_a_device_call():
    """A null plan or network handle is an argument error, never a crash; destroying NULL is a
    no-op."""
    from paper_2609_17636_b300 import _lib
    L = _lib.load()
    N = None
    calls = {
        "ivis_set_pointing": (N, 0, 0, 0, N), "ivis_set_pointing_grid": (N, 0, N),
        "ivis_set_vis": (N, 0, 0, 0, N, N, N), "ivis_set_sd": (N, 0, N, 1.0, 1.0),
        "ivis_prepare": (N,), "ivis_cost_grad": (N, N, N, N, N), "ivis_cost_grad_host": (N, N, N, N, N),
        "ivis_cost_grad_async": (N, N, N, N), "ivis_predict": (N, N, 0, 0, N), "ivis_sd_predict": (N, N, N),
        "ivis_solve": (N, N, 1, 10, 0.0, 0.0, N), "ivis_solve_target": (N, N, 1, 10, 0.0, 0.0, 0.0, N),
        "ivis_dirty_image": (N, N, N), "ivis_feather": (N, N, N, 1.0, 1.0, N),
        "ivis_get_nufft_params": (N, N, N, N), "ivis_profile": (N, 0),
        "ivis_stage_times": (N, N, N, 0, N), "ivis_tuning": (N, N, N, N),
        "ivis_launches_per_eval": (N, N), "ivis_get_stream": (N, N),
    }
    for name, args in calls.items():
        assert getattr(L, name)(*args) == 1, name
        assert L.ivis_last_error(None), name
    assert L.ivis_destroy(N) == 0
    unet_calls = {
        "ivis_unet_num_params": (N, N), "ivis_unet_set_params": (N, N), "ivis_unet_get_params": (N, N),
        "ivis_unet_get_grads": (N, N), "ivis_unet_forward": (N, N, N, 1, 8, 8),
        "ivis_unet_backward": (N, N, N, 1, 8, 8, N), "ivis_unet_adam_step": (N, 1e-3, 0.9, 0.999, 1e-8),
        "ivis_unet_use_tcgen05": (N, 1), "ivis_unet_warm_start": (N, N, N, 0, 8, 8, 1.0, 1.0, 1.0, N),
        "ivis_unet_planes": (N, N, 0, 64, 1.0, 1.0, N, N),
    }
    for name, args in unet_calls.items():
        assert getattr(L, name)(*args) == 1, name
    assert b"null" in L.ivis_unet_last_error(None)
    assert L.ivis_unet_destroy(N) == 0


def test_network_and_allocation_free_entry_checks_run_on_the_host():
    from paper_2609_17636_b300 import _lib
    L = _lib.load()
    u = ctypes.c_void_p()
    assert L.ivis_unet_create(12, 1, 64, None, ctypes.byref(u)) == 1 and not u.value
    assert b"multiple of 8" in L.ivis_unet_last_error(None)
    assert L.ivis_unet_create(8, 0, 64, None, ctypes.byref(u)) == 1 and not u.value
    assert L.ivis_sd_predict_noalloc(None, 16, 1, 3.0, None, None) == 1
    assert b"null" in L.ivis_last_error(None)
    # size limits are checked before any device call (the pointers are never dereferenced)
    fake = ctypes.c_void_p(256)
    assert L.ivis_sd_predict_noalloc(fake, 1025, 1, 3.0, fake, None) == 1
    assert b"too large" in L.ivis_last_error(None)
    for fwhm in (478.5, 1000.0):  # ceil(4 sigma) = 813 and 1699: past the 812 of the scratch
        assert L.ivis_sd_predict_noalloc(fake, 64, 1, fwhm, fake, None) == 1
        assert b"too wide" in L.ivis_last_error(None) and b"812" in L.ivis_last_error(None)


def test_header_is_plain_c_and_the_library_links_from_c(tmp_path):
    """include/ivis.h compiles as strict C99 (no C++ or torch types cross the boundary) and a C
    program links libivis.so and calls host-only entry points."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2609_17636_b300 import build
    lib = build.build()
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include "ivis.h"
int main(void) {
    ivis_config cfg = {0};
    ivis_plan_t plan = 0;
    cfg.n = 64; cfg.nchan = 1; cfg.npoint = 1; cfg.nb = 48; cfg.cell_rad = 1e-5;
    cfg.precision = IVIS_FP32; cfg.nufft_tol = 1e-6;
    ivis_status s = ivis_plan(&cfg, 0, &plan);
    printf("%d %d %.6e\n", (int)s, plan == 0, ivis_rayleigh_jeans(1.4204058e9));
    return ivis_destroy(plan);
}
''')
    exe = tmp_path / "use"
    libdir = os.path.dirname(lib)
    subprocess.run([gcc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", libdir, "-livis", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert out[0] == "1" and out[1] == "1"  # nb = 48 is not a power of two: IVIS_ERR_ARG, no plan
    import oracle
    assert abs(float(out[2]) - oracle.rayleigh_jeans_factor(1.4204058e9)) <= 1e-6 * float(out[2])


def _prototypes():
    """{name: [parameter declarations]} of every function include/ivis.h declares."""
    protos = {}
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", hdr)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(ivis_\w+)\s*\(([^;{]*?)\)\s*;", txt, flags=re.S):
            params = [p.strip() for p in m.group(2).split(",") if p.strip() and p.strip() != "void"]
            protos[m.group(1)] = params
    return protos


def test_binding_prototypes_match_the_header():
    """Every ctypes prototype of the binding has the header's parameter count and, per
    parameter, a matching kind: pointer, int, int64_t, float or double."""
    from paper_2609_17636_b300 import _lib
    L = _lib.load()
    protos = _prototypes()
    assert set(protos) == set(_lib.EXPORTS)
    kinds = {ctypes.c_int: "int", ctypes.c_int64: "int64_t", ctypes.c_double: "double", ctypes.c_float: "float"}
    for name, params in protos.items():
        argtypes = getattr(L, name).argtypes
        assert argtypes is not None and len(argtypes) == len(params), (name, params, argtypes)
        for decl, at in zip(params, argtypes):
            if "*" in decl:
                assert at is ctypes.c_void_p or issubclass(at, ctypes._Pointer) or at is ctypes.c_char_p, (name, decl, at)
            else:
                ctype = decl.rsplit(None, 1)[0].replace("const ", "").strip()
                if ctype in ("ivis_plan_t", "ivis_unet_t"):
                    assert at is ctypes.c_void_p, (name, decl, at)
                else:
                    assert kinds.get(at) == ctype, (name, decl, at)
