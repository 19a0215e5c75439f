"""The C-ABI library builds for sm_103a, loads, and exports every function that include/ifgf.h declares.

No compute call is made here (no GPU on this host): only host-side functions that touch no
device (option defaults, status strings) are called.
"""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions(header="ifgf.h"):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(ifgf_[a-z_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_2112_15198_gb300 as ifgf

    return ifgf.load(build=True)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("ifgf_plan_create", "ifgf_apply", "ifgf_plan_destroy", "ifgf_plan_query"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_host_only_helpers(lib):
    import paper_2112_15198_gb300 as ifgf

    opt = ifgf.Options()
    lib.ifgf_options_default(ctypes.byref(opt))
    assert opt.struct_size == ctypes.sizeof(ifgf.Options)
    assert tuple(opt.base_cones) == (2, 4, 8) and opt.leaf_target == 64 and opt.max_nrhs == 1
    assert abs(opt.tau - 0.5) < 1e-15
    assert lib.ifgf_status_string(0) == b"ok"
    assert lib.ifgf_status_string(1) == b"invalid argument"


def test_invalid_arguments_rejected_before_any_device_work(lib):
    import paper_2112_15198_gb300 as ifgf

    h = ctypes.c_void_p()
    o = (ctypes.c_int32 * 3)(3, 5, 5)
    # NULL points / N < 2 / negative kappa / bad levels: rejected by host-side validation
    assert lib.ifgf_plan_create(None, 10, 1.0, o, 0, None, None, ctypes.byref(h)) == 1
    assert lib.ifgf_plan_create(ctypes.c_void_p(16), 1, 1.0, o, 0, None, None, ctypes.byref(h)) == 1
    assert lib.ifgf_plan_create(ctypes.c_void_p(16), 10, -1.0, o, 0, None, None, ctypes.byref(h)) == 1
    assert lib.ifgf_plan_create(ctypes.c_void_p(16), 10, 1.0, o, 2, None, None, ctypes.byref(h)) == 1
    bad = (ctypes.c_int32 * 3)(0, 4, 4)
    assert lib.ifgf_plan_create(ctypes.c_void_p(16), 10, 1.0, bad, 0, None, None, ctypes.byref(h)) == 1
    assert b"orders" in lib.ifgf_last_error()
    # valid orders without kernels in this build: unsupported, not invalid
    for unbuilt in ((4, 4, 4), (7, 9, 9), (1, 1, 1)):
        o2 = (ctypes.c_int32 * 3)(*unbuilt)
        assert lib.ifgf_plan_create(ctypes.c_void_p(16), 10, 1.0, o2, 0, None, None, ctypes.byref(h)) == 6
        assert b"orders" in lib.ifgf_last_error()
    assert lib.ifgf_plan_destroy(None) == 0
    assert lib.ifgf_apply(None, None, 1, None, None) == 1
    assert lib.ifgf_apply_stokes(None, None, 1, None, None) == 1
    assert lib.ifgf_apply_elastic(None, None, 1, None, 1.0, 0.3, None) == 1
    assert lib.ifgf_apply_elastic(None, None, 1, None, -1.0, 0.3, None) == 1
    assert b"shear_modulus" in lib.ifgf_last_error()


def test_library_links_no_torch(lib):
    """The library's declared dependencies (readelf's NEEDED entries) hold no torch library."""
    import shutil
    import subprocess

    import paper_2112_15198_gb300 as ifgf

    tool = shutil.which("readelf")
    if tool is None:
        pytest.skip("readelf not available")
    out = subprocess.run([tool, "-d", ifgf.library_path()], capture_output=True, text=True, check=True).stdout
    needed = [ln for ln in out.splitlines() if "(NEEDED)" in ln]
    assert needed and not any("torch" in ln or "c10" in ln for ln in needed)


def test_invalid_options_rejected_before_any_device_work(lib):
    import paper_2112_15198_gb300 as ifgf

    h = ctypes.c_void_p()
    for field, value in (("cone_table", 3), ("prop_slices", -1), ("rhs_block", -1), ("max_nrhs", 0),
                         ("leaf_target", 0), ("tau", 0.0)):
        opt = ifgf.Options()
        lib.ifgf_options_default(ctypes.byref(opt))
        setattr(opt, field, value)
        st = lib.ifgf_plan_create(ctypes.c_void_p(16), 10, 1.0, None, 0, ctypes.byref(opt), None, ctypes.byref(h))
        assert st == 1, field
    opt = ifgf.Options()
    lib.ifgf_options_default(ctypes.byref(opt))
    opt.struct_size = 8
    assert lib.ifgf_plan_create(ctypes.c_void_p(16), 10, 1.0, None, 0, ctypes.byref(opt), None, ctypes.byref(h)) == 1


def test_binding_declares_every_entry_point(lib):
    """The Python binding sets argument and result types for every declared function it calls,
    so that no pointer or double is passed through ctypes' int default."""
    import paper_2112_15198_gb300 as ifgf

    src = open(ifgf.__file__).read()
    called = set(re.findall(r"\.(ifgf_[a-z_]+)\(", src))
    declared = set(_declared_functions("ifgf.h")) | set(_declared_functions("ifgf_peaks.h"))
    assert called <= declared, called - declared
    for name in called:
        assert f"lib.{name}.argtypes" in src, name


def test_header_documents_every_entry_point():
    """Each declaration in include/ifgf.h is preceded by a comment (argument meaning, layout,
    ownership, errors), and the compute entry points cite the paper's passage."""
    text = open(os.path.join(ROOT, "include", "ifgf.h")).read()
    lines = text.split("\n")
    for name in _declared_functions():
        at = re.search(r"\n(?![ /]*\*)[a-z0-9_ *]*\b" + name + r"\s*\(", text)
        assert at, name
        # walk back over the declarations grouped under one comment (and their continuation lines)
        k = text[: at.start() + 1].count("\n") - 1
        while k >= 0 and (lines[k].strip() == "" or not lines[k].rstrip().endswith("*/")):
            if lines[k].strip() == "};":  # an enum of the call's codes sits under the same comment
                while k >= 0 and not lines[k].lstrip().startswith("enum"):
                    k -= 1
            elif not (lines[k].lstrip().startswith("#define")
                      or not lines[k].lstrip().startswith(("*", "/*", "#", "typedef", "}", "{"))):
                break
            k -= 1
        assert k >= 0 and lines[k].rstrip().endswith("*/"), f"{name} has no comment block"
    for name, cite in (("ifgf_apply", "Algorithm"), ("ifgf_plan_create", "Sec."), ("ifgf_apply_stokes", "Sec. 2"),
                       ("ifgf_apply_elastic", "Sec. 2")):
        at = re.search(r"\n(?![ /]*\*)[a-z0-9_ *]*\b" + name + r"\s*\(", text).start()
        block = text[text.rindex("/*", 0, at): at]
        assert cite in block, (name, cite)


def test_batch_rejects_a_repeated_plan(lib):
    """A plan owns its buffers, so one handle may appear once per batch; the check runs on the
    host before any handle is dereferenced."""
    h = ctypes.c_void_p()
    plans = (ctypes.c_void_p * 3)(16, 32, 16)
    assert lib.ifgf_batch_create(plans, 3, ctypes.byref(h)) == 1
    assert b"repeats" in lib.ifgf_last_error()
    assert lib.ifgf_batch_create(plans, 0, ctypes.byref(h)) == 1


def test_checked_build_exports_the_same_entry_points():
    """The bounds-checked variant (-DIFGF_CHECKS) builds for sm_103a, exports every declared function
    and says it is checked; host-side validation behaves as in the ordinary build."""
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2112_15198_gb300 import _build

    chk = ctypes.CDLL(_build.build(checks=True))
    for name in _declared_functions():
        assert hasattr(chk, name), name
    chk.ifgf_checked_build.restype = ctypes.c_int32
    assert chk.ifgf_checked_build() == 1
    h = ctypes.c_void_p()
    chk.ifgf_plan_create.restype = ctypes.c_int
    assert chk.ifgf_plan_create(None, 10, ctypes.c_double(1.0), None, 0, None, None, ctypes.byref(h)) == 1
