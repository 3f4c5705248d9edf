"""The paper's ablation variants (Table 2) on the GPU: every FAST variant
finds exactly the oracle's FAST points at threshold t, and every Harris
variant gives the oracle's exact Sobel sums and key at each of them."""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_07164_gb300 as ofg  # noqa: E402

COMBOS = [(f, ofg.OF_VAR_HARRIS_NONE) for f in range(4)] + \
    [(f, ofg.OF_VAR_HARRIS_BASELINE) for f in range(4)] + \
    [(ofg.OF_VAR_FAST_SM_BINARY, h) for h in (ofg.OF_VAR_HARRIS_SEP, ofg.OF_VAR_HARRIS_PARA_SEP,
                                               ofg.OF_VAR_HARRIS_SEMI_SEP)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ofg.build()
    ofg.load()


def _images():
    return [("scene 640x480", synth.scene(640, 480, 5, background="pink")),
            ("ragged 333x197", synth.scene(333, 197, 6, n_rect=40, n_checker=6)),
            ("fig6 (b) patterns", synth.fig6_pattern_image("b", size=256, reps=5)[0]),
            ("fig6 (d) patterns", synth.fig6_pattern_image("d", size=256, reps=5)[0])]


def _run(fv, hv, img, t, border, k, cap=None):
    h, w = img.shape
    pitch = (w + 15) // 16 * 16
    dev = torch.zeros((h, pitch), dtype=torch.uint8, device="cuda")
    dev[:, :w] = torch.from_numpy(img).cuda()
    cap = cap if cap is not None else w * h
    out = torch.zeros(cap * 32, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ofg.of_variant_detect(fv, hv, dev, w, h, pitch, t, border, k, out, cnt, cap)
    torch.cuda.synchronize()
    n = int(cnt.item())
    recs = out.cpu().numpy().view(ofg.VAR_POINT_DTYPE)[:min(n, cap)]
    return n, recs


@pytest.mark.parametrize("fv,hv", COMBOS)
def test_variant_matches_oracle(fv, hv):
    t, border, k = 20, 19, 0.04
    num, den = oracle.k_fraction(k)
    for name, img in _images():
        sm = oracle.score_map(img, border)
        ys, xs = np.nonzero(sm >= t)
        n, recs = _run(fv, hv, img, t, border, k)
        assert n == len(xs), (name, n, len(xs))
        got = sorted(zip(recs["y"].tolist(), recs["x"].tolist()))
        assert got == sorted(zip(ys.tolist(), xs.tolist())), name
        if hv == ofg.OF_VAR_HARRIS_NONE:
            assert not recs["key"].any() and not recs["A"].any()
            continue
        for r in recs[:: max(1, len(recs) // 400)]:  # every point of small images, a sample of large ones
            A, B, C = oracle.harris_sums(img, int(r["x"]), int(r["y"]))
            assert (int(r["A"]), int(r["B"]), int(r["C"])) == (A, B, C), (name, r)
            assert int(r["key"]) == oracle.harris_key(A, B, C, num, den)


def test_variant_other_threshold_and_border():
    img = synth.scene(400, 300, 8, background="pink")
    for t, border in [(7, 4), (35, 10)]:
        sm = oracle.score_map(img, border)
        want = int((sm >= t).sum())
        for fv, hv in COMBOS:
            n, recs = _run(fv, hv, img, t, border, 0.05)
            assert n == want, (t, border, fv, hv)
            if hv >= 0 and len(recs):
                r = recs[0]
                A, B, C = oracle.harris_sums(img, int(r["x"]), int(r["y"]))
                assert (int(r["A"]), int(r["B"]), int(r["C"])) == (A, B, C)


def test_variant_capacity_overflow_counts_all():
    img = synth.scene(320, 240, 9, background="pink")
    n_full, _ = _run(ofg.OF_VAR_FAST_SM_BINARY, ofg.OF_VAR_HARRIS_SEMI_SEP, img, 20, 19, 0.04)
    n, recs = _run(ofg.OF_VAR_FAST_SM_BINARY, ofg.OF_VAR_HARRIS_SEMI_SEP, img, 20, 19, 0.04, cap=10)
    assert n == n_full > 10 and len(recs) == 10
