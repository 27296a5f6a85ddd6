"""The C-ABI library builds, loads and exports every symbol include/flashmp.h
declares; host-only entry points behave as documented (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

from paper_2508_07193_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "flashmp.h")


@pytest.fixture(scope="module")
def so():
    path = B.build()
    return C.CDLL(path)


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fmp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("fmp_setup", "fmp_precond_apply", "fmp_curlcurl_apply", "fmp_krylov_solve", "fmp_cn_step",
              "fmp_box_solve", "fmp_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(so):
    missing = [n for n in declared() if not hasattr(so, n)]
    assert missing == []


def test_host_only_entry_points(so):
    from paper_2508_07193_b300 import flashmp as F
    F._lib = None
    L = F.lib()
    m = re.search(r"#define FMP_ABI_VERSION (\d+)", open(HEADER).read())
    assert L.fmp_abi_version() == int(m.group(1))
    assert F.status_string(F.FMP_ERR_ARG).startswith("FMP_ERR_ARG")
    assert F.status_string(12345) == "unknown fmp_status"
    o = F.default_options()
    assert (o.precision, o.krylov, o.restart, o.rtol, o.max_iters) == (0, 0, 30, 1e-8, 1000)


def test_setup_rejects_bad_arguments_before_touching_the_device(so):
    from paper_2508_07193_b300 import flashmp as F
    L = F.lib()
    h = C.c_void_p()
    g = F.Grid(8, 8, 8)
    assert L.fmp_setup(None, g, None, 0.25, None, None, None) == F.FMP_ERR_ARG
    assert L.fmp_setup(C.byref(h), F.Grid(1, 8, 8), None, 0.25, None, None, None) == F.FMP_ERR_ARG
    assert L.fmp_setup(C.byref(h), g, None, -1.0, None, None, None) == F.FMP_ERR_ARG
    sd = F.Subdomains()
    a = (C.c_int * 2)(4, 3)      # sums to 7, not 8
    sd.n_cuts[0] = 2; sd.cuts[0] = C.cast(a, C.POINTER(C.c_int)); sd.overlap = 1
    assert L.fmp_setup(C.byref(h), g, None, 0.25, C.byref(sd), None, None) == F.FMP_ERR_ARG
    b = (C.c_int * 2)(4, 4)
    sd.cuts[0] = C.cast(b, C.POINTER(C.c_int)); sd.overlap = 0   # two boxes need overlap >= 1
    assert L.fmp_setup(C.byref(h), g, None, 0.25, C.byref(sd), None, None) == F.FMP_ERR_ARG
    o = F.default_options(); o.restart = 33
    assert L.fmp_setup(C.byref(h), g, None, 0.25, None, C.byref(o), None) == F.FMP_ERR_ARG
    o = F.default_options(); o.use_learned = 3
    assert L.fmp_setup(C.byref(h), g, None, 0.25, None, C.byref(o), None) == F.FMP_ERR_ARG
    o = F.default_options(); o.precision = 9
    assert L.fmp_setup(C.byref(h), g, None, 0.25, None, C.byref(o), None) == F.FMP_ERR_ARG
    assert h.value is None
    # null context
    assert L.fmp_precond_apply(None, None, None) == F.FMP_ERR_ARG
    assert L.fmp_krylov_solve(None, None, None, None) == F.FMP_ERR_ARG
    assert L.fmp_set_streamed(None, 1) == F.FMP_ERR_ARG
    assert L.fmp_stream_check(None) == F.FMP_ERR_ARG
    L.fmp_destroy(None)


def test_orth_modes_match_the_header(so):
    """The binding's Gram-Schmidt mode names carry the values of the header's
    fmp_orth_mode; a null context is refused for every mode."""
    from paper_2508_07193_b300 import flashmp as F
    text = open(HEADER).read()
    m = re.search(r"enum fmp_orth_mode \{([^}]*)\}", text)
    vals = {k: int(v) for k, v in re.findall(r"FMP_ORTH_(\w+) = (\d+)", m.group(1))}
    assert vals == {"FLOAT64": 0, "FIXED": 1, "SPLIT": 2}
    assert F.Context.ORTH_MODES == {k.lower(): v for k, v in vals.items()}
    L = F.lib()
    for v in vals.values():
        assert L.fmp_set_orth(None, v) == F.FMP_ERR_ARG
    out = C.c_int()
    assert L.fmp_get_orth(None, C.byref(out)) == F.FMP_ERR_ARG
