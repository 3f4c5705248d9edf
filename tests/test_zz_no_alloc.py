"""The allocation-free single-level entry point against the regular one.

of_detect_level_noalloc serves callers that cannot call cudaMalloc (code that
runs inside a CUDA graph capture, real-time loops that must not touch the
allocator, hosts that own every device allocation).  Its scratch is a static
device array inside the library that every call reuses, so this test makes
two calls in a row on different frames and checks each against of_detect on
one level: the second call must not see anything the first one left behind.
It runs last (file name) and passes alone or after the other tests.
"""

import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2506_07164_gb300 as ofg  # noqa: E402

EXACT = ["x_l", "y_l", "level", "fast_score", "A", "B", "C", "m10", "m01", "key"]


def _same(a, b):
    """b is either of_detect's records or the oracle's (float64 x, y, response, angle)."""
    assert len(a) == len(b)
    for f in EXACT:
        np.testing.assert_array_equal(a[f], b[f], err_msg=f)
    np.testing.assert_array_equal(a["x"], b["x"].astype(np.float32))
    np.testing.assert_array_equal(a["y"], b["y"].astype(np.float32))
    np.testing.assert_allclose(a["response"].astype(np.float64), b["response"], rtol=1e-6, atol=0)
    d = (a["angle"].astype(np.float64) - b["angle"] + math.pi) % (2 * math.pi) - math.pi
    assert len(d) == 0 or np.abs(d).max() <= 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ofg.build()
    ofg.load()


def test_noalloc_matches_of_detect_on_two_calls_in_a_row():
    n = 500
    frames = [synth.scene(1280, 720, 901, background="pink"), synth.scene(640, 480, 902)]
    ref = ofg.Detector(1280, 720, max_levels=1, max_features=n, fast_t_lo=7)
    out = torch.zeros(n * 64, dtype=torch.uint8, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for img in frames:
        t = torch.from_numpy(img).cuda()
        h, w = img.shape
        expect = ref.detect(t, levels=1, fast_t=20, harris_k=0.04, n_features=n)
        assert len(expect) > 0
        ofg.of_detect_level_noalloc(t, w, h, w, 20, 7, 0.04, n, out, cnt)
        torch.cuda.synchronize()
        got = ofg.keypoints_to_numpy(out[: int(cnt.item()) * 64])
        _same(got, expect)
        _same(got, oracle.detect(img, levels=1, fast_t=20, fast_t_lo=7, n_features=n))
    ref.close()


def _noalloc(t, w, h, pitch, n, out, cnt):
    cnt.fill_(-1)
    ofg.of_detect_level_noalloc(t, w, h, pitch, 20, 7, 0.04, n, out, cnt)
    torch.cuda.synchronize()
    c = int(cnt.item())
    assert c >= 0, c
    return ofg.keypoints_to_numpy(out[: c * 64])


def test_noalloc_unaligned_frame_and_empty_detect_region():
    """A frame at a 1-byte offset with an odd pitch goes through the staging
    copy inside the static array; a frame too small for the 19-pixel border
    has no detect region and must report zero keypoints."""
    n = 300
    out = torch.zeros(n * 64, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    w, h = 701, 389
    img = synth.scene(w, h, 903, background="pink")
    host = np.zeros((h, w + 4), np.uint8)
    host[:, 1:w + 1] = img
    big = torch.from_numpy(host).cuda()
    view = big[:, 1:]  # base 1 byte past a 256-byte boundary, pitch w + 4 = 705 bytes
    assert view.data_ptr() % 16 == 1 and view.stride(0) % 16 != 0
    _same(_noalloc(view, w, h, view.stride(0), n, out, cnt),
          oracle.detect(img, levels=1, fast_t=20, fast_t_lo=7, n_features=n))
    for tw, th in [(30, 30), (38, 200), (200, 38)]:
        tiny = torch.from_numpy(synth.scene(tw, th, 904)).cuda()
        assert len(_noalloc(tiny, tw, th, tw, n, out, cnt)) == 0


def test_noalloc_keeps_working_after_a_handle_with_a_small_quota():
    """The top-N kernel's shared-memory limit is a per-device setting shared
    with every handle: creating a handle for 100 features after an
    8192-feature call must not lower it under the next such call."""
    n = 8192
    img = synth.scene(1920, 1080, 905, background="pink")
    t = torch.from_numpy(img).cuda()
    out = torch.zeros(n * 64, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    first = _noalloc(t, 1920, 1080, 1920, n, out, cnt)
    small = ofg.Detector(640, 480, max_levels=1, max_features=100)
    second = _noalloc(t, 1920, 1080, 1920, n, out, cnt)
    small.close()
    assert len(first) == n
    _same(second, first)
    _same(second, oracle.detect(img, levels=1, fast_t=20, fast_t_lo=7, n_features=n))


def test_noalloc_rejects_frames_beyond_the_static_scratch():
    big = torch.zeros((4000, 4000), dtype=torch.uint8, device="cuda")
    out = torch.zeros(64, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(ofg.OfError) as ei:
        ofg.of_detect_level_noalloc(big, 4000, 4000, 4000, 20, 0, 0.04, 1, out, cnt)
    assert ei.value.code == -2
