"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads, and
exports every entry point that include/aenet_gpu.h declares; without a GPU the
set-up call fails loudly with AENET_E_CUDA instead of falling back to the CPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(aenet_[a-z_0-9]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2107_11311_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    declared = _declared()
    assert {"aenet_setup", "aenet_compute", "aenet_md_nve", "aenet_destroy"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_setup_without_gpu_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2107_11311_gb300 import inputs
    from paper_2107_11311_gb300.aenet import AenetError, AenetGPU
    with pytest.raises(AenetError) as ei:
        AenetGPU(inputs.make_model("water"), "fp32")
    assert ei.value.code == -2


def test_setup_rejects_bad_model_before_touching_the_gpu():
    from paper_2107_11311_gb300 import inputs
    from paper_2107_11311_gb300.aenet import AenetError, AenetGPU
    m = inputs.make_model("water")
    m.widths = (50,) + tuple(m.widths[1:])  # D mismatch
    with pytest.raises(AenetError) as ei:
        AenetGPU(m, "fp32")
    assert ei.value.code == -1


def _header_constants():
    src = open(os.path.join(ROOT, "include", "aenet_gpu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"#define\s+(AENET_[A-Z0-9_]+)\s+(-?\d+)\b", src)}
    consts.update({k: int(v) for k, v in re.findall(r"\b(AENET_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)})
    return consts


def test_binding_constants_match_the_header():
    """Every status code, precision, MD flag, option and path flag the binding
    passes through the C ABI has the header's value."""
    from paper_2107_11311_gb300 import aenet
    consts = _header_constants()
    names = [n for n in dir(aenet) if n.startswith("AENET_")]
    assert len(names) >= 15
    for n in names:
        assert n in consts, f"{n} is not defined in include/aenet_gpu.h"
        assert getattr(aenet, n) == consts[n], f"{n}: binding {getattr(aenet, n)} != header {consts[n]}"
    for code, name in aenet.STATUS.items():
        assert consts[name] == code, name
    assert {name: consts[f"AENET_{name.upper()}"] for name in aenet.PRECISIONS} == aenet.PRECISIONS
