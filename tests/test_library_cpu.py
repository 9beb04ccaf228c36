"""CPU-side checks of the native library: it builds for sm_103a, loads, and
exports every entry point the C header declares.  No compute call is made."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1903_07145_gb300 import build
    return build.build()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ipt.h")).read()
    return sorted(set(re.findall(r"^\s*(?:ipt_status|const char\*)\s+(ipt_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["ipt_create", "ipt_scene_upload", "ipt_views_set", "ipt_params_set", "ipt_render",
                 "ipt_backward", "ipt_loss_grad", "ipt_adam_step", "ipt_step", "ipt_trace_rays",
                 "ipt_philox"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if " T " in l)
    assert set(declared_functions()) <= exported


def test_library_built_for_sm103a_only(libpath):
    """Every kernel translation unit and the device link use one target,
    sm_103a (the GPU side checks the loaded binary's version through
    ipt_build_info)."""
    from paper_1903_07145_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_names_match_header(libpath):
    from paper_1903_07145_gb300 import _lib
    assert set(_lib.EXPORTED) == set(declared_functions())
    L = _lib.lib()
    assert L.ipt_status_string(0) == b"ok"
    assert L.ipt_status_string(1) == b"invalid argument"


def test_oracle_and_product_share_no_code():
    """The oracle is test infrastructure: nothing in the package imports it,
    and the two sources include nothing from each other."""
    pkg = os.path.join(ROOT, "paper_1903_07145_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", text, re.M), f
                assert not re.search(r"#include\s+[\"<][^\">]*oracle", text), f
    src = open(os.path.join(ROOT, "oracle", "ipt_oracle.cpp")).read()
    assert "#include \"" not in src


def test_bench_finds_the_traversal_section():
    """bench.py matches its recorded DRAM traffic to the traversal kernel's
    sources by hashing a section of the wavefront source between two marker
    comments; both markers must be present, in order."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.kernel_sources_sha256() is not None
