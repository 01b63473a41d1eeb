"""Source-level guarantees of the product path, checked on the CPU.

* The CUDA path and the oracle share no code: the package never imports the oracle and the
  oracle never imports the package; only the seeded generators (``synth``) serve both, and
  they hold no arithmetic of the method.
* No device code traps or asserts (a fault would take the GPU context down with it), and
  every spin on an mbarrier carries a clock bound after which the kernel records an error.
* The product path is sm_103a CUDA written here: no Triton, no torch.compile, no Hopper-only
  wgmma, and no CPU fallback in the binding.
"""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2609_17636_b300")
CSRC = os.path.join(PKG, "csrc")


def _files(top, exts):
    for dirpath, _, names in os.walk(top):
        if "__pycache__" in dirpath:
            continue
        for name in names:
            if name.endswith(exts):
                yield os.path.join(dirpath, name)


def _code(path):
    """Source text without comments (C, C++, CUDA and Python)."""
    txt = open(path).read()
    if path.endswith(".py"):
        txt = re.sub(r'"""[\s\S]*?"""', "", txt)
        return "\n".join(line.split("#", 1)[0] for line in txt.splitlines())
    txt = re.sub(r"/\*[\s\S]*?\*/", "", txt)
    return re.sub(r"//[^\n]*", "", txt)


def test_product_and_oracle_share_no_code():
    for path in _files(PKG, (".py",)):
        code = _code(path)
        assert not re.search(r"^\s*(import|from)\s+oracle\b", code, re.M), path
    for path in _files(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        assert "paper_2609_17636_b300" not in _code(path), path
    for path in _files(os.path.join(ROOT, "synth"), (".py",)):
        code = _code(path)
        assert "paper_2609_17636_b300" not in code and not re.search(r"\boracle\b", code), path


def test_device_code_neither_traps_nor_asserts():
    for path in _files(CSRC, (".cu", ".cuh")):
        code = _code(path)
        assert "__trap" not in code and not re.search(r"\btrap\s*;", code), path
        assert not re.search(r"(?<![\w.])assert\s*\(", code), path
        assert "__brkpt" not in code, path


def test_every_mbarrier_spin_is_bounded():
    spins = 0
    for path in _files(CSRC, (".cu", ".cuh")):
        code = _code(path)
        for m in re.finditer(r"while\s*\(([^)]*)\)\s*\{", code):
            body = code[m.end():m.end() + 600]
            if "mbarrier" in body and "try_wait" in body:
                spins += 1
                assert "clock64()" in body and "break" in body, (path, code[m.start():m.start() + 200])
    assert spins >= 1  # the tensor-core GEMM's completion wait is found and checked


def test_product_path_is_hand_written_sm103a_cuda():
    for path in _files(PKG, (".py",)):
        code = _code(path)
        assert not re.search(r"^\s*(import|from)\s+triton\b", code, re.M), path
        assert "torch.compile" not in code, path
    for path in _files(CSRC, (".cu", ".cuh")):
        assert "wgmma" not in _code(path), path
    kernels = "".join(_code(p) for p in _files(CSRC, (".cuh",)))
    assert "tcgen05.mma" in kernels and "tcgen05.alloc" in kernels and "tcgen05.ld" in kernels
    build = open(os.path.join(PKG, "build.py")).read()
    assert "compute_103a" in build and "sm_103a" in build


def test_binding_has_no_cpu_fallback():
    """The binding loads libivis.so or raises; it has no numpy/torch implementation of the
    method to fall back on (no FFT, no exp of the kernel, no scatter)."""
    for path in _files(PKG, (".py",)):
        if os.path.basename(path) == "build.py":
            continue
        code = _code(path)
        for pat in (r"torch\.fft", r"np\.fft", r"numpy\.fft", r"index_add", r"scatter_add", r"torch\.exp\b"):
            assert not re.search(pat, code), (path, pat)
