"""Learned tile proposal on the GPU: kernels against the float64 oracle,
checkpoints, the all-tiles case against the plain path, and what a trained
network gains (tiles skipped at high keypoint recall) over no network."""

import numpy as np
import pytest

import synth
from oracle import tcnn as ora

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_07164_gb300 as ofg  # noqa: E402
from paper_2506_07164_gb300 import learned  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ofg.build()
    ofg.load()


def _tiles(n, seed):
    rng = np.random.default_rng(seed)
    img = synth.scene(256, 256, seed, n_rect=30, n_checker=5)
    out = np.zeros((n, 64, 64), np.uint8)
    for i in range(n):
        y, x = rng.integers(0, 192, 2)
        out[i] = img[y:y + 64, x:x + 64]
    out[0, :16, :] = 0  # a patch at the image edge (zero halo)
    return out


def test_forward_matches_oracle():
    net = learned.TileNet(3)
    rng = np.random.default_rng(0)
    ofg.of_tcnn_set_params(net.net, rng.normal(scale=0.3, size=ofg.of_tcnn_num_params()).astype(np.float32))
    tiles = _tiles(37, 1)
    z = net.logits(torch.from_numpy(tiles).cuda()).cpu().numpy()
    pq = ofg.of_tcnn_get_params(net.net, 1).astype(np.float64)  # the bf16 weights the kernels use
    zo, _ = ora.forward(tiles, pq)
    np.testing.assert_allclose(z, zo, rtol=1e-4, atol=1e-4)
    net.close()


def test_gradient_matches_oracle():
    net = learned.TileNet(4)
    tiles = _tiles(24, 2)
    labels = (np.arange(24) % 3 == 0).astype(np.float32)
    loss = ofg.of_tcnn_loss_grad(net.net, torch.from_numpy(tiles).cuda(), torch.from_numpy(labels).cuda(), 24,
                                 pos_weight=2.5)
    g = ofg.of_tcnn_get_params(net.net, 2).astype(np.float64)
    pq = ofg.of_tcnn_get_params(net.net, 1).astype(np.float64)
    lo, go = ora.loss_grad(tiles, labels, pq, pos_weight=2.5)
    assert loss == pytest.approx(lo, rel=1e-5)
    err = np.linalg.norm(g - go) / np.linalg.norm(go)
    assert err < 1e-4, err
    # Every layer's block, not only the largest one.
    for name, (a, b) in {"W1": (0, 72), "W2": (80, 1232), "W3": (1248, 3552), "wf": (3568, 3584)}.items():
        e = np.linalg.norm(g[a:b] - go[a:b]) / max(np.linalg.norm(go[a:b]), 1e-30)
        assert e < 1e-3, (name, e)
    net.close()


def test_adam_matches_oracle():
    net = learned.TileNet(5)
    tiles = torch.from_numpy(_tiles(16, 3)).cuda()
    labels = torch.from_numpy((np.arange(16) % 2).astype(np.float32)).cuda()
    p0 = ofg.of_tcnn_get_params(net.net, 0).astype(np.float64)
    m = np.zeros_like(p0)
    v = np.zeros_like(p0)
    for step in (1, 2):
        ofg.of_tcnn_loss_grad(net.net, tiles, labels, 16)
        g = ofg.of_tcnn_get_params(net.net, 2).astype(np.float64)
        ofg.of_tcnn_adam(net.net, 1e-2, weight_decay=1e-4)
        p0, m, v = ora.adam(p0, g, m, v, step, 1e-2, wd=1e-4)
        np.testing.assert_allclose(ofg.of_tcnn_get_params(net.net, 0), p0, rtol=1e-5, atol=1e-7)
    net.close()


def test_checkpoint_roundtrip_and_crc(tmp_path):
    net = learned.TileNet(6)
    tiles = torch.from_numpy(_tiles(8, 4)).cuda()
    labels = torch.ones(8, device="cuda")
    ofg.of_tcnn_loss_grad(net.net, tiles, labels, 8)
    ofg.of_tcnn_adam(net.net, 1e-3)
    path = tmp_path / "n.oftc"
    net.save(str(path))
    other = learned.TileNet(99).load(str(path))
    for which in (0, 1):
        np.testing.assert_array_equal(ofg.of_tcnn_get_params(net.net, which), ofg.of_tcnn_get_params(other.net, which))
    data = bytearray(path.read_bytes())
    data[100] ^= 1
    with pytest.raises(ofg.OfError):
        ofg.of_tcnn_load(other.net, bytes(data))
    net.close()
    other.close()


def test_all_tiles_proposed_equals_plain():
    frames = [synth.scene(w, h, 70 + i, background="pink") for i, (w, h) in enumerate([(960, 540), (640, 480)])]
    det = ofg.Detector(960, 540, max_levels=8, max_features=400, max_batch=2, fast_t_lo=7)
    net = learned.TileNet(1)
    dev = [torch.from_numpy(f).cuda() for f in frames]
    fr = [(t, t.shape[1], t.shape[0], t.stride(0)) for t in dev]
    det.detect_batch(dev, levels=8, fast_t=20, n_features=400)
    torch.cuda.synchronize()
    plain = det.batch_results(2, 400)
    st = ofg.of_detect_learned(det.h, fr, 8, 1.2, 20, 0.04, 400, net.net, 0.0, 0.0, 0, det.out, det.counts)
    assert st["proposed"] == st["tiles"] > 0
    torch.cuda.synchronize()
    lrn = det.batch_results(2, 400)
    for a, b in zip(plain, lrn):
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
    # And back to the plain path on the same handle.
    det.detect_batch(dev, levels=8, fast_t=20, n_features=400)
    torch.cuda.synchronize()
    for a, b in zip(plain, det.batch_results(2, 400)):
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
    det.close()
    net.close()


def test_labels_equal_oracle_labels():
    """Training labels come from the exact CUDA path; they must equal the tiles
    that hold the oracle's keypoints."""
    import oracle

    frames = [synth.scene(960, 540, 850 + i, background="pink") for i in range(2)]
    det = ofg.Detector(960, 540, max_levels=8, max_features=500, max_batch=2, fast_t_lo=7)
    tiles, labels = learned.label_frames(det, frames, n_features=500)
    lab = labels.cpu().numpy()
    exp = []
    for f in frames:
        kp = oracle.detect(f, levels=8, fast_t=20, fast_t_lo=7, n_features=500)
        ws, hs, _ = oracle.level_sizes(f.shape[1], f.shape[0], 8, 1.2)
        for lvl in range(8):
            rw, rh = ws[lvl] - 38, hs[lvl] - 38
            if rw <= 0 or rh <= 0:
                continue
            gx = 4 * ((ws[lvl] - 19 - 16 + 127) // 128)
            gy = (rh + 31) // 32
            e = np.zeros(gx * gy, np.float32)
            k = kp[kp["level"] == lvl]
            e[((k["y_l"] - 19) // 32) * gx + (k["x_l"] - 16) // 32] = 1
            exp.append(e)
    np.testing.assert_array_equal(lab, np.concatenate(exp))
    assert tiles.shape[0] == lab.shape[0]
    det.close()


def test_partial_proposal_same_under_every_fast_form():
    """With the committed network and threshold (about 3/4 of the tiles
    proposed), the learned path gives the same records whichever FAST form
    the plan runs: general kernel + threshold pass, cell tiles, the
    cell-aligned general kernel, the per-warp general kernel + threshold
    pass, or the per-warp cell strips -- each restricts scores and cell flags
    to the proposed tiles the same way."""
    import json

    meta = json.load(open(learned.DEFAULT_META))
    net = learned.TileNet(0).load(learned.DEFAULT_WEIGHTS)
    frames = [synth.scene(1920, 1080, 950 + i, background="pink") for i in range(2)]
    dev = [torch.from_numpy(f).cuda() for f in frames]
    fr = [(t, t.shape[1], t.shape[0], t.stride(0)) for t in dev]
    det = ofg.Detector(1920, 1080, max_levels=8, max_features=1000, max_batch=2, fast_t_lo=7)
    got = []
    # Every FAST form with the block NMS kernel, then forms 0, 1 and 4 with the
    # per-warp NMS kernel (32-row tiles), which applies the thresholds itself.
    for form, nms_h in ((0, 64), (1, 64), (2, 64), (3, 64), (4, 64), (0, 32), (1, 32), (4, 32)):
        tun = ofg.OfTuning(resize_tile_h=64, resize_tma=1, fast_blocks_per_sm=2, nms_blocks_per_sm=2,
                           stream_groups=1, fast_cell_tiles=form, nms_tile_h=nms_h, fast_tile_h=128)
        det.set_tuning(dev, tun, levels=8, fast_t=20, n_features=1000)
        st = ofg.of_detect_learned(det.h, fr, 8, 1.2, 20, 0.04, 1000, net.net, meta["threshold"],
                                   meta["min_confidence"], meta["dilate"], det.out, det.counts)
        assert 0 < st["proposed"] < st["tiles"], st
        torch.cuda.synchronize()
        got.append(det.batch_results(2, 1000))
    for k in range(1, len(got)):
        for a, b in zip(got[0], got[k]):
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), k
    det.close()
    net.close()


def test_training_skips_work_at_high_recall():
    """A short training run: the loss drops, the trained proposal skips tiles
    while keeping most keypoints, and a random proposal keeping the same
    fraction of tiles loses far more of them."""
    train = [synth.scene(960, 540, 800 + i, background="pink") for i in range(8)]
    held = [synth.scene(960, 540, 900 + i, background="pink") for i in range(2)]
    det = ofg.Detector(960, 540, max_levels=8, max_features=500, max_batch=8, fast_t_lo=7)
    tiles, labels = learned.label_frames(det, train, n_features=500)
    net = learned.TileNet(2)
    hist = learned.train(net, tiles, labels, steps=400, batch=1024)
    assert np.mean(hist[-20:]) < 0.8 * np.mean(hist[:5])
    thr = learned.choose_threshold(net, tiles, labels, 0.995)
    ev = learned.evaluate(det, net, held, thr, dilate=1, n_features=500)
    assert ev["proposed_fraction"] < 0.9, ev
    assert ev["recall"] > 0.9, ev
    rnd = learned.random_proposal_recall(det, held, ev["proposed_fraction"], n_features=500)
    assert ev["recall"] > rnd + 0.05, (ev, rnd)
    det.close()
    net.close()


def _oracle_on_tiles(img, masks, levels=8, scale=1.2, n_features=1000, border=19, cell=30, t_hi=20, t_lo=7):
    """The exact detector restricted to kept tiles, from oracle primitives:
    s(p) = 0 outside the kept 32 x 32 tiles of each level, then the cell
    thresholds, NMS, Harris keys, per-level quota and orientation as in the
    plain path.  Returns (level, x_l, y_l, key, A, B, C, m10, m01, angle)
    rows in output order."""
    import oracle

    num, den = oracle.k_fraction(0.04)
    quota = oracle.level_quotas(n_features, levels, scale)
    x0 = border & ~15
    rows = []
    for lvl in range(levels):
        lev = oracle.pyramid_level(img, levels, scale, lvl)
        h, w = lev.shape
        if w - 2 * border <= 0 or h - 2 * border <= 0:
            continue
        sm = oracle.score_map(lev, border)
        keep = np.zeros_like(sm, dtype=bool)
        gy, gx = masks[lvl].shape
        for j in range(gy):
            for i in range(gx):
                if masks[lvl][j, i]:
                    keep[border + 32 * j: border + 32 * j + 32, x0 + 32 * i: x0 + 32 * i + 32] = True
        sm = np.where(keep, sm, 0).astype(np.uint8)
        T = oracle.cell_thresh(sm, border, cell, t_hi, t_lo)
        surv = oracle.nms(sm, border, cell, T)
        if len(surv) == 0:
            continue
        sums = [oracle.harris_sums(lev, x, y) for x, y in surv]
        keys = [oracle.harris_key(a, b, c, num, den) for a, b, c in sums]
        k, xs, ys = oracle.rank_sort(keys, surv[:, 0], surv[:, 1])
        at = {(int(x), int(y)): s for (x, y), s in zip(surv, sums)}
        for i in range(min(int(quota[lvl]), len(k))):
            x, y = int(xs[i]), int(ys[i])
            m10, m01, th = oracle.orient(lev, x, y)
            rows.append((lvl, x, y, int(k[i]), *at[(x, y)], m10, m01, th))
    return rows


@pytest.mark.parametrize("tuned", [False, True])
def test_full_frame_fallback_below_min_confidence(tuned):
    """A min_confidence between the images' confidences sends some (frame,
    level) images to the full-frame fallback and leaves the others on their
    proposed tiles.  The inspected tile masks follow the network's logits
    (threshold, dilation, all ones where the image fell back); fallen-back
    images give exactly the plain path's records for that level; and every
    frame equals the oracle restricted to the kept tiles.  tuned: the cell-row
    strip FAST kernel and the per-warp NMS kernel, which zeroes the scores
    outside the proposed tiles itself (else the untuned plan's kernels)."""
    import json

    meta = json.load(open(learned.DEFAULT_META))
    thr, dil = meta["threshold"], meta["dilate"]
    net = learned.TileNet(0).load(learned.DEFAULT_WEIGHTS)
    frames = [synth.scene(1920, 1080, 960, background="pink"), synth.scene(1920, 1080, 961)]
    dev = [torch.from_numpy(f).cuda() for f in frames]
    fr = [(t, t.shape[1], t.shape[0], t.stride(0)) for t in dev]
    N, L = 1000, 8
    det = ofg.Detector(1920, 1080, max_levels=L, max_features=N, max_batch=2, fast_t_lo=7)
    if tuned:
        tun = ofg.OfTuning(resize_tile_h=64, resize_tma=1, fast_blocks_per_sm=2, nms_blocks_per_sm=2,
                           stream_groups=1, fast_cell_tiles=4, nms_tile_h=32, fast_tile_h=32)
        det.set_tuning(dev, tun, levels=L, fast_t=20, n_features=N)

    def tile_buf(what, f, lvl, dtype):
        raw, dims = det.inspect(what, f, lvl)
        return raw.view(dtype).reshape(dims[1], dims[0])

    ofg.of_detect_learned(det.h, fr, L, 1.2, 20, 0.04, N, net.net, thr, 0.0, dil, det.out, det.counts)
    logit = {(f, l): tile_buf(ofg.OF_BUF_LOGIT, f, l, np.float32) for f in range(2) for l in range(L)}
    conf = {k: float(np.mean(np.abs(2.0 / (1.0 + np.exp(-z.astype(np.float64))) - 1.0))) for k, z in logit.items()}
    c = np.sort(np.array(list(conf.values())))
    gaps = c[1:] - c[:-1]
    g = int(np.argmax(gaps))
    assert gaps[g] > 1e-3, c  # a min_confidence that no rounding difference can move across an image
    min_conf = float(0.5 * (c[g] + c[g + 1]))
    fallback = {k for k, v in conf.items() if v < min_conf}
    assert 0 < len(fallback) < 2 * L

    st = ofg.of_detect_learned(det.h, fr, L, 1.2, 20, 0.04, N, net.net, thr, min_conf, dil, det.out, det.counts)
    assert st["fallback_images"] == len(fallback), (st, sorted(conf.values()), min_conf)
    masks = {k: tile_buf(ofg.OF_BUF_PMASK, *k, np.uint8) for k in logit}
    torch.cuda.synchronize()
    got = det.batch_results(2, N)
    det.detect_batch(dev, levels=L, fast_t=20, n_features=N)
    plain = det.batch_results(2, N)

    for (f, l), m in masks.items():
        if (f, l) in fallback:
            assert m.all(), (f, l)
            a, b = got[f][got[f]["level"] == l], plain[f][plain[f]["level"] == l]
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), (f, l)
        else:
            p = 1.0 / (1.0 + np.exp(-logit[(f, l)].astype(np.float64)))
            pos = p >= thr
            if dil:
                q = np.pad(pos, 1)
                pos = np.zeros_like(pos)
                for dy in range(3):
                    for dx in range(3):
                        pos |= q[dy: dy + pos.shape[0], dx: dx + pos.shape[1]]
            sure = np.abs(p - thr) > 1e-6  # tiles whose decision no float rounding can flip
            if dil:
                s = np.pad(~sure, 1)
                near = np.zeros_like(sure)
                for dy in range(3):
                    for dx in range(3):
                        near |= s[dy: dy + sure.shape[0], dx: dx + sure.shape[1]]
                sure = ~near
            np.testing.assert_array_equal(m.astype(bool)[sure], pos[sure], err_msg=str((f, l)))
            assert not m.all() or pos.all(), (f, l)
    assert any(not masks[k].all() for k in masks)  # some images ran on their proposed tiles only

    for f in range(2):
        rows = _oracle_on_tiles(frames[f], [masks[(f, l)].astype(bool) for l in range(L)], n_features=N)
        g = got[f]
        assert len(g) == len(rows), (f, len(g), len(rows))
        ora = np.array([r[:9] for r in rows], np.int64)
        for col, name in enumerate(["level", "x_l", "y_l", "key", "A", "B", "C", "m10", "m01"]):
            np.testing.assert_array_equal(g[name].astype(np.int64), ora[:, col], err_msg=name)
        d = (g["angle"].astype(np.float64) - np.array([r[9] for r in rows]) + np.pi) % (2 * np.pi) - np.pi
        assert np.abs(d).max() <= 1e-5
    det.close()
    net.close()
