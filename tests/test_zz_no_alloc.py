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

import paper_2506_07164_gb300 as ofg  # noqa: E402

EXACT = ["x_l", "y_l", "level", "fast_score", "A", "B", "C", "m10", "m01", "key"]


def _same(a, b):
    assert len(a) == len(b)
    for f in EXACT:
        np.testing.assert_array_equal(a[f], b[f], err_msg=f)
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(a["y"], b["y"])
    np.testing.assert_allclose(a["response"], b["response"], rtol=1e-6, atol=0)
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
    ref.close()


def test_noalloc_rejects_frames_beyond_the_static_scratch():
    big = torch.zeros((4000, 4000), dtype=torch.uint8, device="cuda")
    out = torch.zeros(64, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(ofg.OfError) as ei:
        ofg.of_detect_level_noalloc(big, 4000, 4000, 4000, 20, 0, 0.04, 1, out, cnt)
    assert ei.value.code == -2
