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


@pytest.mark.parametrize("bad", [dict(max_w=0), dict(max_h=-1), dict(slots=17), dict(slots=-2),
                                 dict(max_batch=257), dict(memory_budget=0), dict(levels=17),
                                 dict(n_features=8193), dict(n_features=-1)])
def test_server_create_rejects_invalid_params(lib, bad):
    # The serving loop validates its parameters before any CUDA call.
    kw = dict(max_w=1920, max_h=1080, memory_budget=1 << 30)
    kw.update(bad)
    with pytest.raises(ofg.OfError, match="invalid of_server_params"):
        ofg.of_server_create(**kw)


@pytest.mark.parametrize("bad,code", [
    (dict(img=None), ofg.OF_ERR_ARG), (dict(out_count=None), ofg.OF_ERR_ARG),
    (dict(out_kpts=None), ofg.OF_ERR_ARG), (dict(w=0), ofg.OF_ERR_ARG), (dict(pitch=1919), ofg.OF_ERR_ARG),
    (dict(w=70000, pitch=70000), ofg.OF_ERR_ARG), (dict(fast_t=0), ofg.OF_ERR_ARG),
    (dict(fast_t=256), ofg.OF_ERR_ARG), (dict(fast_t_lo=-1), ofg.OF_ERR_ARG), (dict(n_features=8193), ofg.OF_ERR_ARG),
    (dict(harris_k=0.3), ofg.OF_ERR_ARG), (dict(harris_k=0.0403), ofg.OF_ERR_ARG),
    (dict(w=3840, h=2160, pitch=3840), ofg.OF_ERR_TOO_LARGE), (dict(w=2304, h=2304, pitch=2304), ofg.OF_ERR_TOO_LARGE)])
def test_noalloc_rejects_before_any_device_work(lib, bad, code):
    # Every call here fails validation, which comes before the first CUDA call: the
    # pointers are fake (aligned, never dereferenced).  The too-large frames need far
    # more than the 16 MiB array: 2304 x 2304 holds a 5.3 MB score map and 1133^2
    # candidate slots of 12 B (15.4 MB), 3840 x 2160 about 32 MB.
    kw = dict(img=1 << 20, w=1920, h=1080, pitch=1920, fast_t=20, fast_t_lo=7, harris_k=0.04, n_features=1000,
              out_kpts=2 << 20, out_count=3 << 20)
    kw.update(bad)
    with pytest.raises(ofg.OfError) as e:
        ofg.of_detect_level_noalloc(**kw)
    assert e.value.code == code


def test_server_poll_refuses_a_keypoint_buffer_of_another_size(monkeypatch):
    # The server writes result i's keypoints at i * its own n_features: a poll sized for
    # another n_features is refused before the library is called (the handle is fake).
    monkeypatch.setitem(ofg._server_features, 0x5EED, 500)
    with pytest.raises(ValueError, match="differs"):
        ofg.of_server_poll(0x5EED, 4, 100)


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


@pytest.mark.parametrize("w,h", [(1920, 1080), (640, 480), (3840, 2160), (333, 217)])
def test_batch_bytes_is_the_documented_layout(lib, w, h):
    """of_batch_bytes (host-only) against the scratch layout of the arena,
    built here from the oracle's level sizes and quotas: per (frame, level)
    image the level (pitch rounded to 16 bytes; for level 0 the copy an
    unaligned frame needs), its score map (same pitch), 12 bytes of candidate
    key and position for each of ceil(rw/2) x ceil(rh/2) possible strict 3x3
    maxima (they are never adjacent), 12 bytes per kept keypoint of the
    level's quota, one uint32 flag word per cell and 4 int32 counters.  Every
    buffer starts on 256 bytes, so a frame costs at most 8 levels x 6 buffers
    x 255 bytes more, plus a small per-batch block."""
    levels, scale, nf, border, cell = 8, 1.2, 1000, 19, 30
    lw, lh, _ = oracle.level_sizes(w, h, levels, scale)
    quota = oracle.level_quotas(nf, levels, scale)
    frame = 0
    for l in range(levels):
        lwl, lhl = int(lw[l]), int(lh[l])
        rw, rh = lwl - 2 * border, lhl - 2 * border
        assert rw > 0 and rh > 0  # every level holds a detect region at these sizes
        pitch = -(-lwl // 16) * 16
        frame += 2 * pitch * lhl + 12 * (-(-rw // 2)) * (-(-rh // 2)) + 12 * int(quota[l])
        frame += 4 * (-(-rw // cell)) * (-(-rh // cell)) + 16
    for n in (1, 2, 5):
        got = ofg.of_batch_bytes(ofg.OfParams(), [(w, h)] * n, levels, scale, nf)
        assert 0 <= got - n * frame <= n * levels * 6 * 255 + 4096, (n, got, n * frame)
