"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point that include/*.h declares; host-only plan arithmetic agrees with
the oracle.  No compute call needs a GPU here."""

import glob
import os
import re

import numpy as np
import pytest

import oracle
import paper_2506_07164_gb300 as ofg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(of_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    ofg.build()
    return ofg.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("of_create", "of_detect", "of_destroy", "of_detect_batch", "of_inspect",
                     "of_plan_levels", "of_last_error", "of_version", "of_sync", "of_test_timeout",
                     "of_time_stages", "of_autotune"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_version(lib):
    assert ofg.of_version() == 1


def test_plan_levels_match_oracle(lib):
    rng = np.random.default_rng(0)
    cases = [(1920, 1080, 8, 1.2, 1000), (640, 480, 1, 1.2, 500), (720, 540, 8, 1.2, 1000),
             (3840, 2160, 8, 1.2, 1000), (97, 61, 5, 1.5, 37)]
    for _ in range(60):
        cases.append((int(rng.integers(1, 4000)), int(rng.integers(1, 3000)), int(rng.integers(1, 17)),
                      float(rng.uniform(1.01, 3.0)), int(rng.integers(0, 8192))))
    for W, H, L, s, N in cases:
        ws, hs, q = ofg.of_plan_levels(W, H, L, s, N)
        ows, ohs, _ = oracle.level_sizes(W, H, L, s)
        oq = oracle.level_quotas(N, L, s)
        assert ws == ows.tolist() and hs == ohs.tolist() and q == oq.tolist(), (W, H, L, s, N)


def test_plan_levels_rejects_bad_arguments(lib):
    with pytest.raises(ofg.OfError):
        ofg.of_plan_levels(0, 10, 3, 1.2, 10)
    with pytest.raises(ofg.OfError):
        ofg.of_plan_levels(10, 10, 3, 1.0, 10)


def test_keypoint_record_layout():
    assert ofg.KEYPOINT_DTYPE.itemsize == 64
    assert ofg.KEYPOINT_DTYPE.fields["key"][1] == 56


def test_create_rejects_invalid_params(lib):
    # Parameter validation happens before any CUDA call.
    with pytest.raises(ofg.OfError):
        ofg.of_create(max_w=0, max_h=10)
    with pytest.raises(ofg.OfError):
        ofg.of_create(max_w=100, max_h=100, border=10, orient_radius=15)
    with pytest.raises(ofg.OfError):
        ofg.of_create(max_w=100, max_h=100, harris_block=5)


def _header_struct_fields(name):
    text = open(os.path.join(ROOT, "include", "ofast.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), text, flags=re.S).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"^(?:const\s+)?[A-Za-z_]\w*\s*\**\s*(.*)$", decl, flags=re.S)
        for part in m.group(1).split(","):
            fields.append(part.strip().lstrip("*").strip())
    return fields


@pytest.mark.parametrize("c_name,py_name", [
    ("of_params", "OfParams"), ("of_tuning", "OfTuning"), ("of_keypoint", "OfKeypoint"), ("of_frame", "OfFrame"),
    ("of_server_params", "OfServerParams"), ("of_server_result", "OfServerResult"),
    ("of_server_stats", "OfServerStats"), ("of_var_point", "OfVarPoint")])
def test_binding_structs_mirror_the_header(c_name, py_name):
    """The ctypes mirrors list the header's fields in the header's order."""
    py = [f[0] for f in getattr(ofg, py_name)._fields_]
    assert py == _header_struct_fields(c_name), c_name


def test_variant_detect_validates_before_any_device_work(lib):
    """Bad variant choices are rejected on the host (no GPU needed)."""
    for fv, hv in [(4, -1), (-1, -1), (0, 4), (0, -2), (ofg.OF_VAR_FAST_BASELINE, ofg.OF_VAR_HARRIS_SEP),
                   (ofg.OF_VAR_FAST_SM, ofg.OF_VAR_HARRIS_SEMI_SEP)]:
        with pytest.raises(ofg.OfError):
            ofg.of_variant_detect(fv, hv, 16, 64, 64, 64, 20, 19, 0.04, 16, 16, 10)
    with pytest.raises(ofg.OfError):  # border < 4
        ofg.of_variant_detect(0, -1, 16, 64, 64, 64, 20, 3, 0.04, 16, 16, 10)
