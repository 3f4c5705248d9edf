"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer outputs (pyramid levels, score maps, cell thresholds, NMS survivors,
Harris sums and keys, moments, keypoint sets in rank order) must match
bit-exactly; the Harris response within 1e-6 relative and the angle within
1e-5 rad.  Inputs are seeded synthetic scenes (synth), sized so the oracle
finishes in seconds while spanning many tiles and ragged tails.
"""

import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_07164_gb300 as ofg  # noqa: E402

EXACT = ["x_l", "y_l", "level", "fast_score", "A", "B", "C", "m10", "m01", "key"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ofg.build()
    ofg.load()


def compare_keypoints(gpu, ora):
    assert len(gpu) == len(ora), (len(gpu), len(ora))
    if len(ora) == 0:
        return
    for f in EXACT:
        np.testing.assert_array_equal(gpu[f], ora[f], err_msg=f)
    np.testing.assert_array_equal(gpu["x"], ora["x"].astype(np.float32))
    np.testing.assert_array_equal(gpu["y"], ora["y"].astype(np.float32))
    np.testing.assert_allclose(gpu["response"].astype(np.float64), ora["response"], rtol=1e-6, atol=0)
    d = (gpu["angle"].astype(np.float64) - ora["angle"] + math.pi) % (2 * math.pi) - math.pi
    assert np.abs(d).max() <= 1e-5


def oracle_cands(img_level, border, cell, t_hi, t_lo, k=0.04):
    sm = oracle.score_map(img_level, border)
    T = oracle.cell_thresh(sm, border, cell, t_hi, t_lo)
    surv = oracle.nms(sm, border, cell, T)
    num, den = oracle.k_fraction(k)
    keys = [oracle.harris_key(*oracle.harris_sums(img_level, x, y), num, den) for x, y in surv]
    return sm, T, {(int(x), int(y), int(kk)) for (x, y), kk in zip(surv, keys)}


def gpu_cands(det, frame, level):
    raw, dims = det.inspect(ofg.OF_BUF_CAND, frame, level)
    rec = raw.view(np.dtype([("key", "i8"), ("x", "i4"), ("y", "i4")]))
    return {(int(r["x"]), int(r["y"]), int(r["key"])) for r in rec}


def clipped(sm, t_lo):
    return np.where(sm >= t_lo, sm, 0).astype(np.uint8)


def candidate_scores(sm, T, border, cell):
    """S(p) = s(p) where s(p) >= the threshold of p's cell, else 0 (detect region only)."""
    h, w = sm.shape
    tp = np.full(sm.shape, 256, np.int32)
    ys, xs = np.mgrid[border:h - border, border:w - border]
    tp[border:h - border, border:w - border] = T[(ys - border) // cell, (xs - border) // cell]
    return np.where(sm.astype(np.int32) >= tp, sm, 0).astype(np.uint8)


# ------------------------------------------------------------ config 1
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_single_level_640x480(seed):
    img = synth.scene(640, 480, seed)
    det = ofg.Detector(640, 480, max_levels=1, max_features=500)
    kp = det.detect(torch.from_numpy(img).cuda(), levels=1, fast_t=20, n_features=500)
    ora = oracle.detect(img, levels=1, fast_t=20, n_features=500)
    compare_keypoints(kp, ora)
    # Intermediates: score map (clipped at the only threshold), survivors with keys.
    sm, T, cands = oracle_cands(img, 19, 30, 20, 20)
    g_sm, _ = det.inspect(ofg.OF_BUF_SCORE)
    np.testing.assert_array_equal(g_sm.reshape(img.shape), clipped(sm, 20))
    assert gpu_cands(det, 0, 0) == cands
    det.close()


# ------------------------------------------------------------ config 2 (and the serving mix's 4K frames)
@pytest.mark.parametrize("w,h,seed", [(1920, 1080, 7), (3840, 2160, 8)])
def test_pyramid_8_levels_with_cell_fallback(w, h, seed):
    img = synth.scene(w, h, seed, background="pink")
    det = ofg.Detector(w, h, max_levels=8, max_features=1000, fast_t_lo=7)
    kp = det.detect(torch.from_numpy(img).cuda(), levels=8, scale=1.2, fast_t=20, n_features=1000)
    ora = oracle.detect(img, levels=8, scale=1.2, fast_t=20, fast_t_lo=7, n_features=1000)
    compare_keypoints(kp, ora)
    for level in range(8):
        lev = oracle.pyramid_level(img, 8, 1.2, level)
        g_lev, dims = det.inspect(ofg.OF_BUF_LEVEL, 0, level)
        np.testing.assert_array_equal(g_lev.reshape(lev.shape), lev, err_msg=f"level {level}")
        sm, T, cands = oracle_cands(lev, 19, 30, 20, 7)
        g_sm, _ = det.inspect(ofg.OF_BUF_SCORE, 0, level)
        np.testing.assert_array_equal(g_sm.reshape(lev.shape), candidate_scores(sm, T, 19, 30),
                                      err_msg=f"score {level}")
        g_T, dims = det.inspect(ofg.OF_BUF_CELLT, 0, level)
        np.testing.assert_array_equal(g_T.reshape(T.shape), T, err_msg=f"cells {level}")
        assert gpu_cands(det, 0, level) == cands, f"candidates {level}"
    det.close()


def test_unclipped_score_map_at_t1():
    """fast_t = 1 leaves every positive score in the map: s(p) = max(score, 0) everywhere."""
    det = ofg.Detector(800, 600, max_levels=1, max_features=100)
    for seed, bg in [(3, "flat"), (4, "pink")]:
        img = synth.scene(777, 555, seed, background=bg)
        det.detect(torch.from_numpy(img).cuda(), levels=1, fast_t=1, n_features=100)
        g_sm, _ = det.inspect(ofg.OF_BUF_SCORE)
        np.testing.assert_array_equal(g_sm.reshape(img.shape), oracle.score_map(img, 19))
    det.close()


@pytest.mark.parametrize("case", ["a", "b", "c", "d", "e"])
def test_fig6_pattern_images(case):
    img, centres = synth.fig6_pattern_image(case)
    det = ofg.Detector(1024, 1024, max_levels=4, max_features=1000, border=4, orient_radius=4)
    det.detect(torch.from_numpy(img).cuda(), levels=1, fast_t=1, n_features=10)
    g_sm, _ = det.inspect(ofg.OF_BUF_SCORE)
    g_sm = g_sm.reshape(img.shape)
    np.testing.assert_array_equal(g_sm, oracle.score_map(img, 4))
    exp = {"a": 40, "b": 40, "c": 40, "d": 0, "e": 0}[case]
    assert {int(g_sm[y, x]) for x, y in centres} == {exp}
    # Four-level pyramid of the same image (Fig. 7), whole keypoint sets.
    kp = det.detect(torch.from_numpy(img).cuda(), levels=4, scale=1.2, fast_t=20, n_features=1000)
    ora = oracle.detect(img, levels=4, scale=1.2, fast_t=20, n_features=1000, border=4, radius=4)
    compare_keypoints(kp, ora)
    det.close()


@pytest.mark.parametrize("n_features", [1, 16, 64, 300])
def test_top_n_with_many_equal_keys(n_features):
    """A tiled image repeats every candidate's key hundreds of times, so the
    bin of the n-th best key holds more candidates than the sort buffer: the
    exact radix select decides, and ties fall back to (y, x)."""
    patch = synth.scene(24, 20, 9)
    img = np.ascontiguousarray(np.tile(patch, (24, 20))[:480, :480])
    det = ofg.Detector(480, 480, max_levels=1, max_features=300)
    kp = det.detect(torch.from_numpy(img).cuda(), levels=1, fast_t=20, n_features=n_features)
    ora = oracle.detect(img, levels=1, fast_t=20, n_features=n_features)
    assert len(ora) == n_features and (ora["key"] == ora["key"][0]).sum() == n_features
    compare_keypoints(kp, ora)
    det.close()


@pytest.mark.parametrize("n_features", [3000, 3400, 3600, 8192])
def test_top_n_boundary_among_negative_keys(n_features):
    """At t = 1 most survivors are edge points with negative Harris keys; a
    large quota puts the n-th best key among them (8192 keeps every survivor)."""
    img = synth.scene(320, 240, 6, background="pink")
    det = ofg.Detector(320, 240, max_levels=1, max_features=8192)
    kp = det.detect(torch.from_numpy(img).cuda(), levels=1, fast_t=1, n_features=n_features)
    ora = oracle.detect(img, levels=1, fast_t=1, n_features=n_features)
    if n_features < 8192:
        assert len(ora) == n_features and ora["key"][-1] < 0
    compare_keypoints(kp, ora)
    det.close()


# ------------------------------------------------------ ragged, edges
@pytest.mark.parametrize("w,h,levels", [(333, 217, 3), (129, 77, 2), (1000, 41, 1), (41, 1000, 4),
                                        (161, 161, 5), (40, 40, 3), (38, 200, 2), (2, 3, 8)])
def test_ragged_sizes_and_unaligned_pitch(w, h, levels):
    det = ofg.Detector(1024, 1024, max_levels=8, max_features=300, fast_t_lo=9)
    img = synth.scene(w, h, 11 + w, background="pink", n_rect=max(4, w * h // 4000))
    # Unaligned: an odd pitch and an odd start offset inside a larger buffer.
    big = torch.zeros((h, w + 7), dtype=torch.uint8, device="cuda")
    big[:, 3:3 + w] = torch.from_numpy(img).cuda()
    view = big[:, 3:3 + w]
    assert view.stride(0) == w + 7
    kp = det.detect(view, levels=levels, scale=1.2, fast_t=20, n_features=300)
    ora = oracle.detect(img, levels=levels, scale=1.2, fast_t=20, fast_t_lo=9, n_features=300)
    compare_keypoints(kp, ora)
    # The aligned path gives the same.
    kp2 = det.detect(torch.from_numpy(img).cuda().contiguous(), levels=levels, scale=1.2, fast_t=20,
                     n_features=300)
    compare_keypoints(kp2, ora)
    det.close()


@pytest.mark.parametrize("n_features", [0, 1, 7, 8192])
def test_feature_counts(n_features):
    img = synth.scene(640, 480, 21, background="pink")
    det = ofg.Detector(640, 480, max_levels=8, max_features=8192, fast_t_lo=7)
    kp = det.detect(torch.from_numpy(img).cuda(), levels=8, fast_t=20, n_features=n_features)
    ora = oracle.detect(img, levels=8, fast_t=20, fast_t_lo=7, n_features=n_features)
    compare_keypoints(kp, ora)
    det.close()


def test_other_scales_k_and_borders():
    img = synth.scene(700, 500, 31, background="pink")
    det = ofg.Detector(700, 500, max_levels=6, max_features=800, min_scale=1.05, border=15,
                       cell=16, fast_t_lo=5, orient_radius=11)
    for scale, k, t in [(1.05, 0.04, 20), (1.5, 0.06, 30), (2.0, 0.05, 12), (1.2, 0.0, 20)]:
        kp = det.detect(torch.from_numpy(img).cuda(), levels=6, scale=scale, fast_t=t, harris_k=k,
                        n_features=800)
        ora = oracle.detect(img, levels=6, scale=scale, fast_t=t, fast_t_lo=5, harris_k=k,
                            n_features=800, border=15, cell=16, radius=11)
        compare_keypoints(kp, ora)
    det.close()


@pytest.mark.parametrize("border,cell", [(4, 8), (8, 33), (31, 12), (15, 16)])
def test_per_warp_fast_forms_other_borders_and_cells(border, cell):
    """The per-warp FAST kernels (form 3, and form 4 whose strips are one cell
    row high, cells up to 33 rows) on borders whose tile columns start at
    x = 0 or 16 and on ragged sizes: the oracle's keypoints, cell thresholds
    and candidate scores, in a 4-frame batch."""
    sizes = [(701, 389), (333, 217), (640, 480), (129, 77)]
    imgs = [synth.scene(w, h, 70 + i + cell, background="pink") for i, (w, h) in enumerate(sizes)]
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    radius = min(15, border)  # the centroid disc stays inside the image
    det = ofg.Detector(701, 480, max_levels=4, max_features=400, max_batch=4, fast_t_lo=6, border=border, cell=cell,
                       orient_radius=radius)
    ora = [oracle.detect(im, levels=4, scale=1.2, fast_t=21, fast_t_lo=6, n_features=400, border=border, cell=cell,
                         radius=radius) for im in imgs]
    for form in (3, 4):
        # Form 4 with the per-warp NMS kernel (it applies the thresholds), form 3 with the block kernel.
        tun = ofg.OfTuning(resize_tile_h=64, resize_tma=1, fast_blocks_per_sm=2, nms_blocks_per_sm=2,
                           stream_groups=2, fast_cell_tiles=form, nms_tile_h={3: 64, 4: 32}[form], fast_tile_h=32)
        det.set_tuning(dev, tun, levels=4, scale=1.2, fast_t=21, n_features=400)
        det.detect_batch(dev, levels=4, scale=1.2, fast_t=21, n_features=400)
        torch.cuda.synchronize()
        for f, (im, got) in enumerate(zip(imgs, det.batch_results(len(imgs), 400))):
            compare_keypoints(got, ora[f])
            lev = oracle.pyramid_level(im, 4, 1.2, 1)
            if lev.shape[0] <= 2 * border or lev.shape[1] <= 2 * border:
                continue
            sm, T, _ = oracle_cands(lev, border, cell, 21, 6)
            g_T, _ = det.inspect(ofg.OF_BUF_CELLT, f, 1)
            np.testing.assert_array_equal(g_T.reshape(T.shape), T, err_msg=f"form {form} frame {f} cells")
            g_sm, _ = det.inspect(ofg.OF_BUF_SCORE, f, 1)
            np.testing.assert_array_equal(g_sm.reshape(lev.shape), candidate_scores(sm, T, border, cell),
                                          err_msg=f"form {form} frame {f} scores")
    det.close()


def test_rebinding_new_pointers():
    """Same shape, new frame pointers every call: level-0 tensor maps are
    rewritten in place between launches and must never be read stale."""
    det = ofg.Detector(640, 480, max_levels=3, max_features=400)
    a = synth.scene(640, 480, 41)
    b = synth.scene(640, 480, 42)
    ra = oracle.detect(a, levels=3, fast_t=20, n_features=400)
    rb = oracle.detect(b, levels=3, fast_t=20, n_features=400)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    for k in range(8):
        img, t, ref = [(a, ta, ra), (b, tb, rb), (b, tb.clone(), rb), (a, ta, ra)][k % 4]
        compare_keypoints(det.detect(t, levels=3, fast_t=20, n_features=400), ref)
    det.close()
    # Batched: swap the frame order between calls.
    det = ofg.Detector(640, 480, max_levels=3, max_features=400, max_batch=2)
    for k in range(6):
        order = [(ta, ra), (tb, rb)] if k % 2 == 0 else [(tb, rb), (ta, ra)]
        det.detect_batch([t for t, _ in order], levels=3, fast_t=20, n_features=400)
        torch.cuda.synchronize()
        for got, (_, ref) in zip(det.batch_results(2, 400), order):
            compare_keypoints(got, ref)
    det.close()


# ------------------------------------------------------------- batch
def test_batch_mixed_sizes_equal_single_frames_and_oracle():
    sizes = [(720, 540), (1080, 720), (640, 480), (333, 217), (1080, 720)]
    imgs = [synth.scene(w, h, 50 + i, background="pink") for i, (w, h) in enumerate(sizes)]
    det = ofg.Detector(1440, 1080, max_levels=8, max_features=1000, max_batch=8, fast_t_lo=7)
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    det.detect_batch(dev, levels=8, fast_t=20, n_features=1000)
    torch.cuda.synchronize()
    res = det.batch_results(len(imgs), 1000)
    single = ofg.Detector(1440, 1080, max_levels=8, max_features=1000, fast_t_lo=7)
    for im, d, r in zip(imgs, dev, res):
        ora = oracle.detect(im, levels=8, fast_t=20, fast_t_lo=7, n_features=1000)
        compare_keypoints(r, ora)
        compare_keypoints(single.detect(d, levels=8, fast_t=20, n_features=1000), ora)
    det.close()
    single.close()


# ------------------------------------------------------------ errors
def test_invalid_calls_return_errors():
    det = ofg.Detector(320, 240, max_levels=4, max_features=100)
    img = torch.zeros((240, 320), dtype=torch.uint8, device="cuda")
    bad = [dict(levels=0), dict(levels=5), dict(scale=1.1), dict(fast_t=0), dict(fast_t=256),
           dict(harris_k=0.3), dict(harris_k=0.040001), dict(n_features=101)]
    for kw in bad:
        args = dict(levels=2, scale=1.2, fast_t=20, harris_k=0.04, n_features=50)
        args.update(kw)
        with pytest.raises(ofg.OfError):
            ofg.of_detect(det.h, img, 320, 240, 320, args["levels"], args["scale"], args["fast_t"],
                          args["harris_k"], args["n_features"], det.out)
    with pytest.raises(ofg.OfError):  # larger than the handle allows
        ofg.of_detect(det.h, img, 321, 240, 320, 1, 1.2, 20, 0.04, 10, det.out)
    with pytest.raises(ofg.OfError):  # pitch < w
        ofg.of_detect(det.h, img, 320, 240, 100, 1, 1.2, 20, 0.04, 10, det.out)
    # The handle still works afterwards.
    assert ofg.of_detect(det.h, img, 320, 240, 320, 2, 1.2, 20, 0.04, 50, det.out) == 0
    det.close()


# ------------------------------------------------------- failure path
def test_device_wait_timeout_is_reported_and_handle_survives():
    """A bounded device wait on a flag nothing sets expires, is reported as
    OF_ERR_TIMEOUT through of_sync, and the handle keeps working."""
    det = ofg.Detector(640, 480, max_levels=2, max_features=300)
    assert ofg.of_test_timeout(det.h, 20000) == ofg.OF_ERR_TIMEOUT
    assert ofg.of_sync(det.h) == 0  # the condition was cleared
    img = synth.scene(640, 480, 77)
    kp = det.detect(torch.from_numpy(img).cuda(), levels=2, fast_t=20, n_features=300)
    compare_keypoints(kp, oracle.detect(img, levels=2, fast_t=20, n_features=300))
    det.close()


def test_batch_then_sync_ok():
    det = ofg.Detector(640, 480, max_levels=3, max_features=200, max_batch=4)
    imgs = [torch.from_numpy(synth.scene(640, 480, 80 + i)).cuda() for i in range(4)]
    det.detect_batch(imgs, levels=3, fast_t=20, n_features=200)
    assert ofg.of_sync(det.h) == 0
    assert (det.counts[:4].cpu().numpy() > 0).all()
    det.close()


# ------------------------------------------------------------ full size
def test_full_size_batch_autotuned_matches_oracle():
    """The benchmark's workload at its full size and launch configuration:
    128 frames of 1920x1080, 8 levels at scale 1.2, t = 20 with fallback 7,
    1000 features, autotuned (forked frame groups, tall tiles).  Every
    frame's records equal those of the frame it copies (4 distinct scenes
    in 128 separate device buffers), and the 4 scenes' records equal the
    oracle's."""
    distinct = [synth.scene(1920, 1080, seed, background="pink") for seed in range(4)]
    src = [torch.from_numpy(f).cuda() for f in distinct]
    dev = [src[i % 4].clone() for i in range(128)]
    det = ofg.Detector(1920, 1080, max_levels=8, max_features=1000, max_batch=128, fast_t_lo=7)
    tun = det.autotune(dev, levels=8, fast_t=20, n_features=1000, reps=1)
    assert 1 <= tun.stream_groups <= 8
    det.detect_batch(dev, levels=8, fast_t=20, n_features=1000)
    torch.cuda.synchronize()
    res = det.batch_results(128, 1000)
    for i in range(128):
        assert np.array_equal(res[i].view(np.uint8), res[i % 4].view(np.uint8)), i
    for k in range(4):
        compare_keypoints(res[k], oracle.detect(distinct[k], levels=8, scale=1.2, fast_t=20, fast_t_lo=7,
                                                n_features=1000))
    det.close()


# ------------------------------------------------------------ autotuner
def test_autotuner_choice_is_valid_and_results_unchanged():
    sizes = [(720, 540), (1080, 720), (640, 480)]
    imgs = [synth.scene(w, h, 60 + i, background="pink") for i, (w, h) in enumerate(sizes)]
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    det = ofg.Detector(1080, 720, max_levels=8, max_features=500, max_batch=4, fast_t_lo=7)
    tun = det.autotune(dev, levels=8, fast_t=20, n_features=500, reps=2)
    assert tun.resize_tile_h in (32, 64) and tun.resize_tma in (0, 1) and 1 <= tun.stream_groups <= 3
    assert tun.fast_blocks_per_sm >= 1 and tun.nms_blocks_per_sm >= 1
    assert tun.fast_order in (0, 1) and tun.nms_order in (0, 1)
    assert tun.candidates_tried >= 2 + 2 + 2 and tun.fast_ms > 0 and tun.nms_ms > 0
    torch.cuda.synchronize()
    first = det.batch_results(len(imgs), 500)  # the tuning call's own outputs
    det.detect_batch(dev, levels=8, fast_t=20, n_features=500)  # tuned graph
    torch.cuda.synchronize()
    tuned = det.batch_results(len(imgs), 500)
    for im, a, b in zip(imgs, first, tuned):
        ora = oracle.detect(im, levels=8, fast_t=20, fast_t_lo=7, n_features=500)
        compare_keypoints(a, ora)
        compare_keypoints(b, ora)
    det.close()


# ------------------------------------------------------------ pyramid kernels
@pytest.mark.parametrize("scale", [1.05, 1.2, 1.5, 1.8, 2.0, 3.0])
def test_every_resize_kernel_matches_oracle_levels(scale):
    """Each pyramid kernel -- staged tiles of 32 or 64 rows, and the persistent
    TMA kernel (scales up to ~1.85; above that its levels use the staged
    kernel) -- gives the oracle's levels on ragged sizes, every level."""
    sizes = [(1283, 723), (640, 480), (333, 197)]
    imgs = [synth.scene(w, h, 400 + i, background="pink") for i, (w, h) in enumerate(sizes)]
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    levels = 6
    det = ofg.Detector(1283, 723, max_levels=levels, max_features=300, max_batch=3, min_scale=1.05, fast_t_lo=7)
    ora = [[oracle.pyramid_level(im, levels, scale, lv) for lv in range(levels)] for im in imgs]
    for tile_h, tma in [(32, 0), (64, 0), (64, 1)]:
        tun = ofg.OfTuning(resize_tile_h=tile_h, resize_tma=tma, fast_blocks_per_sm=1, nms_blocks_per_sm=1,
                           stream_groups=1, nms_tile_h=32, fast_tile_h=32)
        det.set_tuning(dev, tun, levels=levels, scale=scale, fast_t=20, n_features=300)
        det.detect_batch(dev, levels=levels, scale=scale, fast_t=20, n_features=300)
        torch.cuda.synchronize()
        for f in range(len(imgs)):
            for lv in range(1, levels):
                g, _ = det.inspect(ofg.OF_BUF_LEVEL, f, lv)
                np.testing.assert_array_equal(g.reshape(ora[f][lv].shape), ora[f][lv],
                                              err_msg=f"tile_h {tile_h} tma {tma} frame {f} level {lv}")
    det.close()


def test_set_tuning_rejects_out_of_range_fields():
    img = torch.from_numpy(synth.scene(320, 240, 3)).cuda()
    det = ofg.Detector(320, 240, max_levels=2, max_features=50)
    good = dict(resize_tile_h=64, resize_tma=1, fast_blocks_per_sm=1, nms_blocks_per_sm=1, stream_groups=1,
                nms_tile_h=32, fast_tile_h=32)
    for bad in (dict(resize_tile_h=48), dict(resize_tma=2), dict(fast_blocks_per_sm=0),
                dict(nms_blocks_per_sm=1000), dict(fast_order=2), dict(stream_groups=9), dict(stream_groups=0), dict(fast_cell_tiles=5),
                dict(nms_tile_h=48), dict(fast_tile_h=16)):
        with pytest.raises(ofg.OfError):
            det.set_tuning([img], ofg.OfTuning(**{**good, **bad}), levels=2, n_features=50)
    det.set_tuning([img], ofg.OfTuning(**good), levels=2, n_features=50)
    det.close()


def test_frame_groups_equal_one_group_and_oracle():
    """The forked graph (frames in 2..5 groups on as many branches) gives the same
    records as the one-group graph and the oracle, also after new pointers."""
    sizes = [(1280, 720), (640, 480), (960, 540), (333, 197), (720, 540)]
    imgs = [synth.scene(w, h, 500 + i, background="pink") for i, (w, h) in enumerate(sizes)]
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    det = ofg.Detector(1280, 720, max_levels=6, max_features=400, max_batch=5, fast_t_lo=7)
    got = {}
    for groups in (1, 2, 3, 5):
        tun = ofg.OfTuning(resize_tile_h=64, resize_tma=1, fast_blocks_per_sm=2, nms_blocks_per_sm=2,
                           stream_groups=groups, nms_tile_h={1: 64, 2: 32, 3: 128, 5: 128}[groups],
                           fast_tile_h={1: 32, 2: 64, 3: 128, 5: 256}[groups])
        det.set_tuning(dev, tun, levels=6, fast_t=20, n_features=400)
        det.detect_batch(dev, levels=6, fast_t=20, n_features=400)
        torch.cuda.synchronize()
        got[groups] = det.batch_results(len(imgs), 400)
        # New frame pointers re-encode the level-0 maps of both branches.
        dev2 = [t.clone() for t in dev]
        det.detect_batch(dev2, levels=6, fast_t=20, n_features=400)
        torch.cuda.synchronize()
        for a, b in zip(got[groups], det.batch_results(len(imgs), 400)):
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
    for i, im in enumerate(imgs):
        for k in (2, 3, 5):
            assert np.array_equal(got[1][i].view(np.uint8), got[k][i].view(np.uint8)), (i, k)
        compare_keypoints(got[5][i], oracle.detect(im, levels=6, fast_t=20, fast_t_lo=7, n_features=400))
    det.close()


@pytest.mark.parametrize("t", [1, 20])
def test_per_warp_nms_without_cell_fallback(t):
    """The per-warp NMS kernel (32-row tiles) on maps without a per-cell fallback
    (t_lo = t_hi: nothing to apply, the maps are the candidate scores) and at t = 1
    (every positive score a candidate), after FAST forms 0, 1 and 4: the oracle's
    keypoints, score maps and candidates on every level."""
    img = synth.scene(1000, 700, 31 + t, background="pink")
    dev = torch.from_numpy(img).cuda()
    det = ofg.Detector(1000, 700, max_levels=3, max_features=800)
    ora = oracle.detect(img, levels=3, scale=1.2, fast_t=t, n_features=800)
    for form in (0, 1, 4):
        tun = ofg.OfTuning(resize_tile_h=64, resize_tma=1, fast_blocks_per_sm=2, nms_blocks_per_sm=2,
                           stream_groups=1, fast_cell_tiles=form, nms_tile_h=32, fast_tile_h=32)
        det.set_tuning([dev], tun, levels=3, scale=1.2, fast_t=t, n_features=800)
        det.detect_batch([dev], levels=3, scale=1.2, fast_t=t, n_features=800)
        torch.cuda.synchronize()
        compare_keypoints(det.batch_results(1, 800)[0], ora)
        for level in range(3):
            lev = oracle.pyramid_level(img, 3, 1.2, level)
            sm, T, cands = oracle_cands(lev, 19, 30, t, t)
            g_sm, _ = det.inspect(ofg.OF_BUF_SCORE, 0, level)
            np.testing.assert_array_equal(g_sm.reshape(lev.shape), clipped(sm, t), err_msg=f"form {form} score {level}")
            assert gpu_cands(det, 0, level) == cands, f"form {form} candidates {level}"
    det.close()


@pytest.mark.parametrize("cell", [8, 13, 15, 30, 31, 40])
def test_cell_sizes_both_fast_forms(cell):
    """Both FAST forms -- the cell-tile kernel (cells of 8..30 pixels) and the
    general kernel followed by the threshold pass -- and both FAST and NMS
    tile heights give the oracle's cell thresholds, candidate scores, survivors
    and keypoints."""
    img = synth.scene(900, 700, 90 + cell, background="pink")
    dev = torch.from_numpy(img).cuda()
    det = ofg.Detector(900, 700, max_levels=3, max_features=600, fast_t_lo=6, cell=cell)
    ora = oracle.detect(img, levels=3, scale=1.2, fast_t=22, fast_t_lo=6, n_features=600, cell=cell)
    # nms_h 32: the per-warp NMS kernel, which applies the cell thresholds itself after forms 0, 3 and 4
    for form, nms_h, fast_h in ((0, 32, 32), (1, 64, 32), (0, 64, 64), (0, 128, 128), (0, 32, 256), (1, 128, 32),
                                (2, 64, 32), (3, 64, 32), (4, 64, 32), (1, 32, 32), (3, 32, 32), (4, 32, 32)):
        tun = ofg.OfTuning(resize_tile_h=64, resize_tma=1, fast_blocks_per_sm=2, nms_blocks_per_sm=2,
                           stream_groups=1, fast_cell_tiles=form, nms_tile_h=nms_h, fast_tile_h=fast_h)
        det.set_tuning([dev], tun, levels=3, scale=1.2, fast_t=22, n_features=600)
        det.detect_batch([dev], levels=3, scale=1.2, fast_t=22, n_features=600)
        torch.cuda.synchronize()
        compare_keypoints(det.batch_results(1, 600)[0], ora)
        for level in range(3):
            lev = oracle.pyramid_level(img, 3, 1.2, level)
            sm, T, cands = oracle_cands(lev, 19, cell, 22, 6)
            g_T, _ = det.inspect(ofg.OF_BUF_CELLT, 0, level)
            np.testing.assert_array_equal(g_T.reshape(T.shape), T, err_msg=f"form {form} cells {level}")
            g_sm, _ = det.inspect(ofg.OF_BUF_SCORE, 0, level)
            np.testing.assert_array_equal(g_sm.reshape(lev.shape), candidate_scores(sm, T, 19, cell),
                                          err_msg=f"form {form} score {level}")
            assert gpu_cands(det, 0, level) == cands, f"form {form} candidates {level}"
    det.close()
