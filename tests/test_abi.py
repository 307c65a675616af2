"""The C-ABI library builds, loads and exports every entry point of include/fh.h
(no compute calls: these run without a GPU)."""
import os
import ctypes as C
import re
import subprocess

import pytest

import fh_inputs as fi
from paper_1807_02718_gb300 import build as B
from paper_1807_02718_gb300 import fh as F

HEADER = os.path.join(B.ROOT, "include", "fh.h")


def declared_entry_points():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fh_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def test_header_declares_the_path_calls():
    names = declared_entry_points()
    for must in ("fh_discretize", "fh_solve_frequencies", "fh_window_spectra", "fh_sample"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (fh_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared_entry_points() if n not in exported]
    assert not missing, missing


def test_binding_names_match_header(lib_path):
    assert sorted(F.EXPORTED) == declared_entry_points()
    lib = F.load_library(lib_path)
    for n in F.EXPORTED:
        assert hasattr(lib, n)
        assert callable(getattr(F, n))


def test_library_has_no_cpu_compute_fallback(lib_path):
    """The library links only the CUDA runtime (statically) and the C/C++ runtime."""
    out = subprocess.run(["nm", "-D", "--undefined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    assert "oracle" not in out
    assert "fho_" not in out


def test_kernels_built_for_sm103a():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_curve_struct_layout():
    c = F.make_curve(fi.random_star(__import__("numpy").random.default_rng(0)))
    assert c.kind == F.FH_CURVE_STAR and c.n_harm == 5
    # C layout: int, pad, double, int, pad, double[16], double[16], double[2]
    assert F.fh_curve.amp.offset == 24 and F.fh_curve.center.offset == 24 + 2 * 8 * 16
    assert __import__("ctypes").sizeof(F.fh_curve) == 296


def test_create_without_device_reports_cuda_error(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(F.FHError) as e:
        F.fh_create(0)
    assert e.value.status == F.FH_ECUDA


def test_timing_phases_match_header():
    """The binding's phase list (and so the fh_timings layout) is the header's enum."""
    import re
    hdr = open(HEADER).read()
    body = re.search(r"enum \{ (FH_PH_GEOMETRY = 0,[^}]*)\}", hdr).group(1)
    names = [n.strip().split("=")[0].strip() for n in body.split(",") if n.strip()]
    assert names[-1] == "FH_NUM_PHASES"
    assert [n[len("FH_PH_"):].lower() for n in names[:-1]] == F.PHASES
    assert C.sizeof(F.fh_timings) == len(F.PHASES) * 3 * 8
