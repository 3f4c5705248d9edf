"""Serving loop with continuous batching (of_server_*).

Requests of mixed resolutions -- 640x480, 1280x720, 1920x1080 and 3840x2160,
with stereo pairs -- arrive from a client thread while earlier batches are on
the GPU.  Every result must equal the CPU oracle on the same frame and
of_detect on the frame alone (bit-exact integer fields, response 1e-6
relative, angle 1e-5 rad); batches must hold several frames, and batches on
different slots must overlap in time.
"""

import math
import multiprocessing
import threading
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2506_07164_gb300 as ofg  # noqa: E402

EXACT = ["x_l", "y_l", "level", "fast_score", "A", "B", "C", "m10", "m01", "key"]
CFG = dict(levels=8, scale=1.2, fast_t=20, harris_k=0.04, n_features=500)
FULL_MIX = [(640, 480), (1280, 720), (1920, 1080), (3840, 2160), (640, 480), (1280, 720)]
SMALL_MIX = [(640, 480), (1280, 720), (1920, 1080), (640, 480), (1280, 720)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ofg.build()
    ofg.load()


def same(a, b):
    """b: of_detect's records or the oracle's (float64 x, y, response, angle)."""
    assert len(a) == len(b)
    for f in EXACT:
        np.testing.assert_array_equal(a[f], b[f], err_msg=f)
    for f in ("x", "y"):
        np.testing.assert_array_equal(a[f], b[f].astype(np.float32), err_msg=f)
    np.testing.assert_allclose(a["response"].astype(np.float64), b["response"], rtol=1e-6, atol=0)
    if len(a):
        d = (a["angle"].astype(np.float64) - b["angle"] + math.pi) % (2 * math.pi) - math.pi
        assert np.abs(d).max() <= 1e-5


def stereo_right(left: np.ndarray, disparity: int) -> np.ndarray:
    right = np.empty_like(left)
    right[:, : left.shape[1] - disparity] = left[:, disparity:]
    right[:, left.shape[1] - disparity:] = left[:, -1:]
    return right


def _pool():
    # spawn: the workers never inherit this process's CUDA context
    return ProcessPoolExecutor(max_workers=min(8, multiprocessing.cpu_count()),
                               mp_context=multiprocessing.get_context("spawn"))


def make_requests(sizes=SMALL_MIX, reps=3, pool=None):
    jobs = [(w, h, 300 + i, "pink" if i % 2 else "flat") for i, (w, h) in enumerate(sizes * reps)]
    if pool is None:
        frames = [synth.scene(w, h, seed, background=bg) for w, h, seed, bg in jobs]
    else:  # module-level functions only, so the workers import synth / oracle and nothing else
        frames = [f.result() for f in [pool.submit(synth.scene, w, h, seed, background=bg)
                                       for w, h, seed, bg in jobs]]
    reqs = []
    for i, img in enumerate(frames):
        reqs.append(img)
        if i % 4 == 1:  # a stereo pair: the right view is the left shifted by a seeded disparity
            reqs.append(stereo_right(img, 5 + i % 7))
    return reqs


def run_server(reqs, max_w=1920, max_h=1080, **params):
    srv = ofg.of_server_create(max_w=max_w, max_h=max_h, **{k: v for k, v in CFG.items()}, **params)
    results = {}
    ids = {}

    def client():
        # Bursts of 6 back-to-back requests (they queue while earlier batches
        # run), separated by short random pauses.
        rng = np.random.default_rng(0)
        for i, img in enumerate(reqs):
            ids[ofg.of_server_submit(srv, img, tag=i)] = i
            if i % 6 == 5:
                time.sleep(float(rng.exponential(0.004)))

    th = threading.Thread(target=client)
    th.start()
    deadline = time.time() + 120
    while len(results) < len(reqs) and time.time() < deadline:
        for r, kp in ofg.of_server_poll(srv, 16, CFG["n_features"], wait_ms=50):
            results[r.tag] = (r, kp)
    th.join()
    stats = ofg.of_server_stats(srv)
    ofg.of_server_destroy(srv)
    assert len(results) == len(reqs), stats
    return results, stats


def alone(reqs):
    W = max(img.shape[1] for img in reqs)
    H = max(img.shape[0] for img in reqs)
    det = ofg.Detector(W, H, max_levels=8, max_features=CFG["n_features"])
    out = [det.detect(torch.from_numpy(img).cuda(), levels=8, scale=1.2, fast_t=20, harris_k=0.04,
                      n_features=CFG["n_features"]) for img in reqs]
    det.close()
    return out


def test_mixed_stream_equals_oracle_and_alone_and_batches_overlap():
    with _pool() as pool:
        reqs = make_requests(FULL_MIX, 2, pool)
        assert {img.shape for img in reqs} == {(h, w) for w, h in FULL_MIX}
        expect = [pool.submit(oracle.detect, img, **CFG) for img in reqs]  # on the host while the GPU serves
        results, stats = run_server(reqs, max_w=3840, max_h=2160, slots=3, max_batch=4, memory_budget=3 << 30)
        ref = alone(reqs)
        expect = [f.result() for f in expect]
    for i, img in enumerate(reqs):
        r, kp = results[i]
        assert r.count >= 0 and (r.w, r.h) == (img.shape[1], img.shape[0])
        same(kp, expect[i])
        same(kp, ref[i])
    # Continuous batching: some batches carried several frames ...
    assert max(r.batch_frames for r, _ in results.values()) > 1
    assert stats["batches"] < len(reqs)
    # ... and batches on different slots were on the GPU at the same time.
    spans = sorted({(r.t_launch, r.t_done) for r, _ in results.values()})
    overlap = any(b[0] < a[1] for a, b in zip(spans, spans[1:]))
    assert overlap, spans


def test_small_budget_still_exact():
    reqs = make_requests()[:6]
    # Room for one 1080p frame per slot only: batches shrink, results do not change.
    one = ofg.of_batch_bytes(ofg.OfParams(), [(1920, 1080)], 8, 1.2, CFG["n_features"])
    budget = one + 1920 * 1080 + 8 * 500 * 64 + 4096
    results, _ = run_server(reqs, slots=1, max_batch=8, memory_budget=budget)
    ref = alone(reqs)
    for i in range(len(reqs)):
        same(results[i][1], ref[i])


def test_server_rejects_what_cannot_fit():
    with pytest.raises(ofg.OfError):
        ofg.of_server_create(max_w=1920, max_h=1080, memory_budget=1 << 20)
    srv = ofg.of_server_create(max_w=640, max_h=480, memory_budget=256 << 20, n_features=100)
    with pytest.raises(ofg.OfError):
        ofg.of_server_submit(srv, np.zeros((720, 1280), np.uint8))
    ofg.of_server_destroy(srv)
