"""The C ABI library loads without a GPU and exports every function include/sonotrace.h declares;
the Python binding declares exactly those symbols.  No compute calls are made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sonotrace.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:st_status|void|const char\*|int32_t)\s+(st_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_19652_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_parses():
    names = declared_functions()
    assert "st_simulate" in names and "st_scene_load" in names and len(names) >= 20


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header():
    from paper_2602_19652_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == declared_functions()


def test_host_only_calls(lib):
    """Calls that need no device: defaults, status strings, argument checks on null handles."""
    import paper_2602_19652_gb300 as st
    L = st.load()
    p = st.sim_params()
    assert p.max_bounces == 3 and abs(p.c - 343.0) < 1e-12 and p.components == 7
    assert p.los_mode == st.ST_LOS_REFERENCE == 0 and st.ST_LOS_PER_MIC == 1
    c = st.curv_params()
    assert c.samples_per_vertex == 64 and c.sample_budget == 4_000_000
    assert L.st_status_string(0) == b"ok"
    assert L.st_status_string(-4) == b"invalid mesh"
    assert L.st_destroy(None) == -1
    assert L.st_simulate(None, None, None, None, None) == -1
    assert L.st_get_receiver_masks(None, None, 0) == -1
    assert L.st_set_frequencies(None, 4, 1.0, 2.0) == -1
    assert L.st_set_stage_overlap(None, 1) == -1
