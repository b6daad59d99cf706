"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/gbcca.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "gbcca.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    return ctypes.CDLL(os.path.join(ROOT, "paper_2106_12060_gb300", "libgbcca.so"))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("cca_plan", "cca_precondition", "cca_solve", "lda_plan", "lda_solve", "gbcca_fused_pass"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), f"{name} declared in gbcca.h but not exported"


def test_binding_covers_every_symbol():
    from paper_2106_12060_gb300 import _lib
    assert set(_declared()) == set(_lib.SIGNATURES)


def test_host_only_calls(lib):
    """Entry points that need no device: defaults, status strings, argument checks."""
    from paper_2106_12060_gb300 import _lib
    L = _lib.load()
    o = _lib.Options()
    assert L.gbcca_default_options(ctypes.byref(o)) == 0
    assert o.max_iter == 1000 and o.warm_start == 1 and o.check_every == 8
    assert o.graphs == 1 and o.time_passes == 0 and o.refine == 1
    assert L.gbcca_default_options(None) == _lib.ERR_INVALID_ARG
    assert L.gbcca_status_string(_lib.ERR_NOT_SPD) == b"matrix not positive definite"
    h = ctypes.c_void_p()
    # k > min(dx, dy) is rejected before any device work
    assert L.cca_plan(ctypes.byref(h), 100, 5, 4, 6, 2, None) == _lib.ERR_INVALID_ARG
    assert L.lda_plan(ctypes.byref(h), 100, 5, 3, 3, 2, None) == _lib.ERR_INVALID_ARG
    assert b"k" in L.gbcca_last_error()


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct of the header as laid out by the C compiler (size and
    every field offset) equals the ctypes structure of the binding."""
    import shutil
    import subprocess
    from paper_2106_12060_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gbcca.h"', "int main(void) {"]
    structs = (("gbcca_options", _lib.Options), ("gbcca_info", _lib.Info),
               ("gbcca_batch_options", _lib.BatchOptions), ("gbcca_batch_report", _lib.BatchReport),
               ("gbcca_server_options", _lib.ServerOptions), ("gbcca_request", _lib.Request),
               ("gbcca_request_times", _lib.RequestTimes))
    for cname, py in structs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs:
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_binding_rejects_host_and_mistyped_tensors():
    """The binding passes raw pointers, so a host tensor, a tensor of the wrong
    dtype or of the wrong shape is refused in Python before any call into the
    library (no device needed: the refusal comes first)."""
    import torch
    import paper_2106_12060_gb300 as gb
    A = torch.zeros(10, 4, dtype=torch.float64)
    C = torch.zeros(4, 4, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        gb.sketch_gram_noalloc(A, 0.0, C)
    with pytest.raises(ValueError, match="CUDA"):
        gb.sketch_gram_noalloc(A.float(), 0.0, C.float())
    with pytest.raises(ValueError):
        gb.sketch_gram_noalloc(A, 0.0, torch.zeros(5, 5, dtype=torch.float64))
    plan = gb.Plan(None, "cca", 10, (4, 3), 2, gb.FP32, None)
    with pytest.raises(ValueError, match="CUDA"):
        gb.cca_precondition(plan, torch.zeros(10, 4), torch.zeros(10, 3), 1e-3, 1e-3)


def test_batch_and_server_host_checks(lib):
    """Host-side argument checks of the batch and serving entry points (no
    device work): defaults, refusals of bad arguments, unknown requests."""
    from paper_2106_12060_gb300 import _lib
    L = _lib.load()
    bo = _lib.BatchOptions()
    assert L.gbcca_default_batch_options(ctypes.byref(bo)) == 0
    assert bo.clusters == 0 and bo.graphs == 1 and bo.batch_iters == 8
    h = ctypes.c_void_p()
    assert L.gbcca_batch_create(ctypes.byref(h), None, 0, None) == _lib.ERR_INVALID_ARG
    so = _lib.ServerOptions()
    assert L.gbcca_default_server_options(ctypes.byref(so)) == 0
    assert so.hbm_budget == 120 << 30 and so.max_active == 64 and so.tick_iters == 8 and so.graphs == 1
    bad = _lib.ServerOptions(hbm_budget=0, max_active=1, tick_iters=1, graphs=0)
    assert L.gbcca_server_create(ctypes.byref(h), ctypes.byref(bad)) == _lib.ERR_INVALID_ARG
    assert L.gbcca_server_create(ctypes.byref(h), ctypes.byref(so)) == 0
    rid = ctypes.c_int64()
    req = _lib.Request(kind=0, dtype=_lib.BF16, n=100, dx=8, dy=8, k=2)  # no data pointers
    assert L.gbcca_server_submit(h, ctypes.byref(req), ctypes.byref(rid)) == _lib.ERR_INVALID_ARG
    req = _lib.Request(kind=2, dtype=_lib.BF16, n=100, dx=8, dy=8, k=2, X=1, ldx=8, Y=1, ldy=8)
    assert L.gbcca_server_submit(h, ctypes.byref(req), ctypes.byref(rid)) == _lib.ERR_INVALID_ARG
    assert L.gbcca_server_state(h, 12345) == _lib.ERR_INVALID_ARG
    assert L.gbcca_server_result(h, 12345, None, None, None, None, None) == _lib.ERR_INVALID_ARG
    L.gbcca_server_destroy(h)


def test_flag_codes_map_to_statuses():
    """The device error flag values of the library (common.cuh) and their
    statuses: 4 = a bounded wait ran out -> GBCCA_ERR_TIMEOUT."""
    txt = open(os.path.join(ROOT, "paper_2106_12060_gb300", "csrc", "common.cuh")).read()
    assert "constexpr int kFlagTimeout = 4;" in txt
    body = txt[txt.index("inline int flag_status"):]
    assert "case kFlagTimeout:" in body and "return GBCCA_ERR_TIMEOUT;" in body
