"""Pins for the CPU oracle: each check ties it to something other than itself.

Brute force on tiny inputs, closed forms, the worked Fig. 6 cases, hand-worked
fixtures under tests/golden/ and independent library routines (scipy.ndimage,
Python big integers and fractions).  None of these calls the CUDA library.
"""

import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
RING = synth.RING_OFFSETS


# ----------------------------------------------------------------- helpers
def brute_arc9(mask: int) -> bool:
    """Cyclic run of >= 9 ones in a 16-bit mask, by string search on the doubled ring."""
    bits = "".join("1" if (mask >> i) & 1 else "0" for i in range(16))
    return "1" * 9 in bits + bits


def eq1_states(ring, center, t):
    """Eq. 1 literally: dark / similar / bright for each ring pixel."""
    out = []
    for v in ring:
        if v <= center - t:
            out.append("d")
        elif v >= center + t:
            out.append("b")
        else:
            out.append("s")
    return out


def brute_corner(ring, center, t) -> bool:
    st = eq1_states(ring, center, t)
    dbl = st + st
    for c in "db":
        for j in range(16):
            if all(dbl[j + k] == c for k in range(9)):
                return True
    return False


def brute_score(ring, center) -> int:
    """Largest t >= 1 at which the brute-force test passes (0 when none)."""
    best = 0
    for t in range(1, 256):
        if brute_corner(ring, center, t):
            best = t
    return best


def ring_of(img, x, y):
    return [int(img[y + dy, x + dx]) for dx, dy in RING]


# ------------------------------------------------------------- FAST pins
def test_arc9_exhaustive_all_masks():
    """Alg. 2's 9-bit window test with wraparound == brute-force arc enumeration, all 2^16 masks."""
    for m in range(1 << 16):
        assert oracle.has_arc9(m) == brute_arc9(m), hex(m)


def test_ring_masks_follow_eq1():
    rng = np.random.default_rng(1)
    for _ in range(300):
        ring = rng.integers(0, 256, 16)
        c = int(rng.integers(0, 256))
        t = int(rng.integers(1, 60))
        b, d = oracle.ring_masks(ring, c, t)
        st = eq1_states(ring, c, t)
        for i in range(16):
            assert bool((b >> i) & 1) == (st[i] == "b")
            assert bool((d >> i) & 1) == (st[i] == "d")


def test_corner_matches_eq1_brute_force():
    rng = np.random.default_rng(2)
    for _ in range(400):
        c = int(rng.integers(0, 256))
        # Mix of plain random rings and rings with a long arc planted in them.
        ring = rng.integers(0, 256, 16)
        if rng.random() < 0.6:
            j = int(rng.integers(0, 16))
            n = int(rng.integers(7, 13))
            sgn = 1 if rng.random() < 0.5 else -1
            for k in range(n):
                ring[(j + k) % 16] = np.clip(c + sgn * int(rng.integers(0, 80)), 0, 255)
        t = int(rng.integers(1, 80))
        assert oracle.is_corner(ring, c, t) == brute_corner(list(ring), c, t)


def test_score_is_largest_passing_threshold():
    """s(p) >= t  <=>  corner at t, for every t in 1..255 (brute force)."""
    rng = np.random.default_rng(3)
    for trial in range(150):
        c = int(rng.integers(0, 256))
        ring = rng.integers(0, 256, 16)
        j = int(rng.integers(0, 16))
        sgn = 1 if trial % 2 else -1
        for k in range(int(rng.integers(8, 12))):
            ring[(j + k) % 16] = np.clip(c + sgn * int(rng.integers(5, 90)), 0, 255)
        s = oracle.fast_score(ring, c)
        assert max(s, 0) == brute_score(list(ring), c)
        for t in (1, 2, 7, 20, 50, 128, 255):
            assert (s >= t) == brute_corner(list(ring), c, t)


def _golden_fig6():
    rows = []
    with open(os.path.join(GOLD, "fig6_cases.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            case, pos, corner, score = line.split()
            rows.append((case, [int(p) for p in pos.split(",")], bool(int(corner)), int(score)))
    return rows


@pytest.mark.parametrize("case,pos,corner,score", _golden_fig6())
def test_fig6_cases(case, pos, corner, score):
    assert synth.fig6_ring_states(case) == pos
    patch = synth.fig6_patch(case)
    ring = ring_of(patch, 3, 3)
    assert oracle.is_corner(ring, 100, 20) == corner
    assert max(oracle.fast_score(ring, 100), 0) == score
    # The same patch rotated to every start position and mirrored keeps its class.
    for rot in range(16):
        r2 = ring[rot:] + ring[:rot]
        assert oracle.is_corner(r2, 100, 20) == corner
        assert oracle.is_corner(r2[::-1], 100, 20) == corner


@pytest.mark.parametrize("case", ["a", "b", "c", "d", "e"])
def test_fig6_pattern_image(case):
    """Sec. 6.1: 625 copies of a Fig. 6 pattern in a 1024x1024 image; all centres share one score."""
    img, centres = synth.fig6_pattern_image(case)
    sm = oracle.score_map(img, 3)
    exp = {r[0]: r[3] for r in _golden_fig6()}[case]
    vals = {int(sm[y, x]) for x, y in centres}
    assert vals == {exp}


def test_score_map_brute_force_tiny():
    img = synth.scene(40, 32, seed=5, n_rect=12, n_checker=3)
    border = 3
    sm = oracle.score_map(img, border)
    h, w = img.shape
    for y in range(h):
        for x in range(w):
            if border <= x < w - border and border <= y < h - border:
                exp = brute_score(ring_of(img, x, y), int(img[y, x]))
            else:
                exp = 0
            assert sm[y, x] == exp, (x, y)


# --------------------------------------------------------- cells and NMS
def test_cell_thresh_block_max():
    rng = np.random.default_rng(7)
    sc = rng.integers(0, 40, (97, 131)).astype(np.uint8)
    border, cell, thi, tlo = 5, 30, 35, 9
    T = oracle.cell_thresh(sc, border, cell, thi, tlo)
    reg = sc[border:-border, border:-border].astype(np.int32)
    ph = -reg.shape[0] % cell
    pw = -reg.shape[1] % cell
    pad = np.pad(reg, ((0, ph), (0, pw)), constant_values=-1)
    blk = pad.reshape(pad.shape[0] // cell, cell, pad.shape[1] // cell, cell).max(axis=(1, 3))
    assert np.array_equal(T, np.where(blk >= thi, thi, tlo).astype(np.uint8))
    # t_lo == t_hi: every cell gets the plain threshold.
    assert (oracle.cell_thresh(sc, border, cell, 20, 20) == 20).all()


def test_nms_matches_maximum_filter():
    from scipy import ndimage

    rng = np.random.default_rng(8)
    for trial in range(6):
        sc = rng.integers(0, 30, (60, 77)).astype(np.uint8)
        sc[rng.random(sc.shape) < 0.5] = 0
        border, cell, thi, tlo = 4, 30, 25, 6
        T = oracle.cell_thresh(sc, border, cell, thi, tlo)
        got = oracle.nms(sc, border, cell, T)
        h, w = sc.shape
        S = np.zeros_like(sc, dtype=np.int32)
        for y in range(border, h - border):
            for x in range(border, w - border):
                t = T[(y - border) // cell, (x - border) // cell]
                S[y, x] = sc[y, x] if sc[y, x] >= t else 0
        fp = np.ones((3, 3), bool)
        fp[1, 1] = False
        nb = ndimage.maximum_filter(S, footprint=fp, mode="constant", cval=0)
        keep = (S > 0) & (S > nb)
        ys, xs = np.nonzero(keep)
        exp = np.stack([xs, ys], 1).astype(np.int32)
        assert np.array_equal(got, exp)


def test_nms_special_cases():
    sc = np.zeros((20, 20), np.uint8)
    sc[10, 10] = 30
    T = oracle.cell_thresh(sc, 2, 30, 20, 20)
    assert oracle.nms(sc, 2, 30, T).tolist() == [[10, 10]]
    sc[10, 11] = 30  # a two-pixel plateau suppresses both (strict comparison)
    assert oracle.nms(sc, 2, 30, T).shape[0] == 0
    sc[10, 11] = 29
    assert oracle.nms(sc, 2, 30, T).tolist() == [[10, 10]]
    sc[:] = 0
    sc[10, 10] = 15  # below the threshold of its cell: no candidate
    assert oracle.nms(sc, 2, 30, T).shape[0] == 0


# ------------------------------------------------------------ Harris pins
SOBEL_X = np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]])
SOBEL_Y = np.array([[-1, -2, -1], [0, 0, 0], [1, 2, 1]])


def test_harris_sums_match_scipy_correlation():
    from scipy import ndimage

    img = synth.scene(64, 48, seed=11, n_rect=15, n_checker=4)
    I = img.astype(np.int64)
    gx = ndimage.correlate(I, SOBEL_X, mode="constant")
    gy = ndimage.correlate(I, SOBEL_Y, mode="constant")
    box = np.ones((7, 7), np.int64)
    A = ndimage.correlate(gx * gx, box, mode="constant")
    B = ndimage.correlate(gy * gy, box, mode="constant")
    Cc = ndimage.correlate(gx * gy, box, mode="constant")
    for y in range(4, 48 - 4):
        for x in range(4, 64 - 4):
            assert oracle.harris_sums(img, x, y) == (A[y, x], B[y, x], Cc[y, x]), (x, y)


def test_harris_ramp_closed_form():
    """I = a x + b y: gx = 8a, gy = 8b everywhere, so det(M) = 0 and R = -k (A+B)^2."""
    for a, b in [(1, 0), (0, 2), (2, 3), (3, -1), (-2, -2)]:
        yy, xx = np.mgrid[0:30, 0:30]
        img = (100 + a * xx + b * yy).astype(np.uint8)
        A, B, Cc = oracle.harris_sums(img, 15, 15)
        assert (A, B, Cc) == (49 * 64 * a * a, 49 * 64 * b * b, 49 * 64 * a * b)
        num, den = oracle.k_fraction(0.04)
        key = oracle.harris_key(A, B, Cc, num, den)
        assert key == -num * (A + B) ** 2


def test_harris_step_edge():
    img = np.zeros((30, 30), np.uint8)
    img[:, 15:] = 200
    A, B, Cc = oracle.harris_sums(img, 15, 15)
    assert B == 0 and Cc == 0 and A > 0
    num, den = oracle.k_fraction(0.04)
    assert oracle.harris_key(A, B, Cc, num, den) < 0


def test_harris_key_exact_rational():
    """key / den == det - k trace^2 exactly, with k the float32 value rounded to 1e-6 (big ints)."""
    rng = np.random.default_rng(12)
    for k in [0.04, 0.05, 0.06, 0.045, 0.1, 0.0]:
        num, den = oracle.k_fraction(k)
        kq = Fraction(round(float(np.float32(k)) * 10**6), 10**6)
        assert Fraction(num, den) == kq
        for _ in range(200):
            A = int(rng.integers(0, 51_000_000))
            B = int(rng.integers(0, 51_000_000))
            Cc = int(rng.integers(-int(math.isqrt(A * B)), int(math.isqrt(A * B)) + 1))
            key = oracle.harris_key(A, B, Cc, num, den)
            exact = (A * B - Cc * Cc) - kq * (A + B) ** 2
            assert Fraction(key, den) == exact
            resp = oracle.harris_response(key, den, 7)
            f = Fraction(1, 4 * 7 * 255) ** 4
            ref = float(exact * f)
            assert resp == pytest.approx(ref, rel=1e-12, abs=1e-300)


def test_k_fraction_rejects_out_of_range():
    for k in [-0.01, 0.3, 0.040001]:
        with pytest.raises(ValueError):
            oracle.k_fraction(k)


# ------------------------------------------------------- orientation pins
def _disc(r=15):
    return [(u, v) for v in range(-r, r + 1) for u in range(-r, r + 1) if u * u + v * v <= r * r]


def test_orient_disc_closed_forms():
    disc = _disc()
    assert len(disc) == 709
    img = np.zeros((41, 41), np.uint8)
    for u, v in disc:
        img[20 + v, 20 + u] = 1
    assert oracle.orient(img, 20, 20)[:2] == (0, 0)
    # Ramp in x: m10 = sum u * (c + u) = sum u^2, m01 = sum v * (c + u) = 0.
    yy, xx = np.mgrid[0:41, 0:41]
    ramp = (50 + (xx - 20)).astype(np.uint8)
    m10, m01, th = oracle.orient(ramp, 20, 20)
    assert m10 == sum(u * u for u, v in disc) and m01 == 0 and th == 0.0


def test_orient_rotation_and_mirror():
    img = synth.scene(41, 41, seed=13, n_rect=8, n_checker=2)
    m10, m01, th = oracle.orient(img, 20, 20)
    # np.rot90 (k=1): new[r, c] = old[c, 40 - r].  A pixel at offset (u, v) moves to
    # (v, -u), so (m10, m01) -> (m01, -m10): the angle decreases by pi/2.
    r = np.ascontiguousarray(np.rot90(img))
    a, b, th2 = oracle.orient(r, 20, 20)
    assert (a, b) == (m01, -m10)
    d = (th - th2) % (2 * math.pi)
    assert d == pytest.approx(math.pi / 2, abs=1e-12)
    # Mirror in x: (u, v) -> (-u, v): m10 -> -m10, theta -> pi - theta.
    mi = np.ascontiguousarray(img[:, ::-1])
    a, b, th3 = oracle.orient(mi, 20, 20)
    assert (a, b) == (-m10, m01)
    assert ((math.pi - th) - th3) % (2 * math.pi) == pytest.approx(0.0, abs=1e-12) or \
        abs(((math.pi - th) - th3) % (2 * math.pi) - 2 * math.pi) < 1e-12


@pytest.mark.parametrize("deg", [0, 45, 90, 135, 180, -45, -90, -135, 30, 60, 120])
def test_orient_ramp_angle(deg):
    alpha = math.radians(deg)
    yy, xx = np.mgrid[0:41, 0:41].astype(np.float64)
    u, v = xx - 20, yy - 20
    img = np.clip(np.rint(128 + 3.5 * (u * math.cos(alpha) + v * math.sin(alpha))), 0, 255).astype(np.uint8)
    m10, m01, th = oracle.orient(img, 20, 20)
    err = (th - alpha + math.pi) % (2 * math.pi) - math.pi
    if deg % 45 == 0:
        assert abs(err) < 1e-12  # lattice symmetry makes these exact
    else:
        assert abs(err) < 0.02   # uint8 rounding of the ramp


# ---------------------------------------------------------- resize pins
def test_resize_golden_ramp():
    with open(os.path.join(GOLD, "resize_ramp_4to3.txt")) as f:
        rows = {l.split()[0]: [int(v) for v in l.split()[1:]] for l in f if l.strip() and not l.startswith("#")}
    src = np.array([rows["src"]] * 4, np.uint8)
    out = oracle.resize(src, 3, 3)
    assert out.tolist() == [rows["dst"]] * 3


def test_resize_constant_and_identity():
    for v in (0, 1, 128, 255):
        src = np.full((37, 53), v, np.uint8)
        assert (oracle.resize(src, 44, 31) == v).all()
    img = synth.scene(64, 40, seed=3, n_rect=10, n_checker=2)
    assert np.array_equal(oracle.resize(img, 64, 40), img)


def test_resize_within_one_of_float64_bilinear():
    img = synth.scene(97, 61, seed=4, n_rect=20, n_checker=4)
    for dw, dh in [(81, 51), (67, 42), (97, 30), (20, 61)]:
        out = oracle.resize(img, dw, dh).astype(np.float64)
        sh, sw = img.shape
        sx = np.clip((np.arange(dw) + 0.5) * (sw / dw) - 0.5, 0, sw - 1)
        sy = np.clip((np.arange(dh) + 0.5) * (sh / dh) - 0.5, 0, sh - 1)
        x0 = np.floor(sx).astype(int)
        y0 = np.floor(sy).astype(int)
        x1 = np.minimum(x0 + 1, sw - 1)
        y1 = np.minimum(y0 + 1, sh - 1)
        fx = (sx - x0)[None, :]
        fy = (sy - y0)[:, None]
        I = img.astype(np.float64)
        ref = (1 - fy) * ((1 - fx) * I[y0][:, x0] + fx * I[y0][:, x1]) + fy * ((1 - fx) * I[y1][:, x0] + fx * I[y1][:, x1])
        assert np.abs(out - ref).max() <= 1.0


# ---------------------------------------------------- sizes, quotas, rank
def test_level_sizes_1080p():
    ws, hs, sl = oracle.level_sizes(1920, 1080, 8, 1.2)
    assert ws.tolist() == [1920, 1600, 1333, 1111, 926, 772, 643, 536]
    assert hs.tolist() == [1080, 900, 750, 625, 521, 434, 362, 301]
    s = float(np.float32(1.2))
    for l in range(8):
        exact = Fraction(s) ** l
        assert ws[l] == math.floor(Fraction(1920) / exact + Fraction(1, 2))
        assert hs[l] == math.floor(Fraction(1080) / exact + Fraction(1, 2))


def test_level_quotas():
    q = oracle.level_quotas(1000, 8, 1.2)
    assert q.tolist() == [323, 224, 156, 108, 75, 52, 36, 26]
    rng = np.random.default_rng(14)
    for _ in range(50):
        N = int(rng.integers(1, 5000))
        L = int(rng.integers(1, 12))
        s = float(rng.uniform(1.05, 2.0))
        q = oracle.level_quotas(N, L, s)
        assert q.sum() == N and (q >= 0).all()
        f = 1.0 / float(np.float32(s)) ** 2
        c = (1 - f) / (1 - f ** L)
        for l in range(L - 1):
            assert q[l] <= math.floor(N * c * f ** l + 0.5) + 1e-9


def test_rank_sort_matches_python_sorted():
    rng = np.random.default_rng(15)
    n = 3000
    key = rng.integers(-50, 50, n)  # many ties
    x = rng.integers(0, 200, n)
    y = rng.integers(0, 200, n)
    k2, x2, y2 = oracle.rank_sort(key, x, y)
    exp = sorted(zip(key.tolist(), y.tolist(), x.tolist()), key=lambda t: (-t[0], t[1], t[2]))
    assert list(zip(k2.tolist(), y2.tolist(), x2.tolist())) == exp


# ------------------------------------------------------------- pipeline
def test_detect_single_level_composes_the_pinned_steps():
    img = synth.scene(160, 120, seed=21, n_rect=40, n_checker=6)
    kp, counts = oracle.detect(img, levels=1, fast_t=20, n_features=50, with_counts=True)
    sm = oracle.score_map(img, 19)
    T = oracle.cell_thresh(sm, 19, 30, 20, 20)
    surv = oracle.nms(sm, 19, 30, T)
    assert counts[0] == len(surv)
    num, den = oracle.k_fraction(0.04)
    recs = []
    for x, y in surv:
        A, B, Cc = oracle.harris_sums(img, x, y)
        recs.append((oracle.harris_key(A, B, Cc, num, den), int(y), int(x)))
    recs.sort(key=lambda t: (-t[0], t[1], t[2]))
    assert len(kp) == min(50, len(recs))
    assert [(int(k["key"]), int(k["y_l"]), int(k["x_l"])) for k in kp] == recs[:len(kp)]
    for k in kp:
        assert k["fast_score"] == sm[k["y_l"], k["x_l"]]
        m10, m01, th = oracle.orient(img, k["x_l"], k["y_l"])
        assert (k["m10"], k["m01"], k["angle"]) == (m10, m01, th)


def test_detect_degenerate_levels():
    img = synth.scene(48, 40, seed=1, n_rect=5, n_checker=1)
    # Detect region empty at border 19 (40 - 38 = 2 rows stay, 48 - 38 = 10 cols): tiny.
    kp = oracle.detect(img, levels=4, n_features=100)
    assert all(k["level"] == 0 for k in kp)
    tiny = np.zeros((30, 30), np.uint8)
    assert len(oracle.detect(tiny, levels=3, n_features=10)) == 0


# ----------------------------------------------------------------- symmetries
def test_score_map_symmetries():
    """Eq. 1 treats bright and dark alike, and the radius-3 ring of Fig. 2(a)
    is closed under quarter turns and mirrors (each maps contiguous arcs to
    contiguous arcs): the score map of the inverted, rotated or mirrored image
    is the original map, unchanged, rotated or mirrored.  A one-sided
    comparison, a wrong ring offset or an x/y swap breaks one of them."""
    ring = set(RING)
    assert {(dy, -dx) for dx, dy in RING} == ring and {(-dx, dy) for dx, dy in RING} == ring
    img = synth.scene(72, 72, 4, n_rect=25, n_checker=4)  # square: the border maps onto itself
    b = 3
    s = oracle.score_map(img, b)
    assert (s >= 20).sum() > 20
    assert np.array_equal(oracle.score_map(255 - img, b), s)
    for k in (1, 2, 3):
        assert np.array_equal(oracle.score_map(np.ascontiguousarray(np.rot90(img, k)), b), np.rot90(s, k))
    assert np.array_equal(oracle.score_map(np.ascontiguousarray(img[:, ::-1]), b), s[:, ::-1])
    assert np.array_equal(oracle.score_map(np.ascontiguousarray(img[::-1]), b), s[::-1])


def test_detect_quarter_turn_equivariance():
    """One level and one threshold (the cell fallback then has nothing to
    decide): a quarter turn of a square frame turns every keypoint with it.
    With r[i, j] = img[j, n-1-i] (numpy's rot90), the point (x, y) moves to
    (y, n-1-x), gx becomes gy and gy becomes -gx, so A and B trade places, C
    changes sign and the Harris key (det - k trace^2) is unchanged; the
    moments become (m01, -m10) and the angle turns by -90 degrees.  A
    transposed operand, a Sobel sign or a swapped record field fails it."""
    n = 160
    img = synth.scene(n, n, 9, n_rect=40, n_checker=6)
    kw = dict(levels=1, fast_t=20, fast_t_lo=20, n_features=1 << 20)
    a = oracle.detect(img, **kw)
    r = oracle.detect(np.ascontiguousarray(np.rot90(img)), **kw)
    assert len(a) == len(r) > 20

    def rec(k):
        return (int(k["x_l"]), int(k["y_l"]), int(k["fast_score"]), int(k["key"]),
                int(k["A"]), int(k["B"]), int(k["C"]), int(k["m10"]), int(k["m01"]))

    turned = {(y, n - 1 - x, s, key, B, A, -C, m01, -m10) for x, y, s, key, A, B, C, m10, m01 in map(rec, a)}
    assert turned == set(map(rec, r))
    ang_a = {(int(k["y_l"]), n - 1 - int(k["x_l"])): float(k["angle"]) for k in a}
    for k in r:
        d = float(k["angle"]) - (ang_a[(int(k["x_l"]), int(k["y_l"]))] - math.pi / 2)
        assert abs(math.remainder(d, 2 * math.pi)) < 1e-9


def test_resize_and_pyramid_commute_with_transposition():
    """Both axes follow the same sampling rule and the bilinear value is one
    exact integer expression rounded once, so resizing the transposed image
    gives the transposed result, and so does every level of the chain (sizes
    are computed per axis).  An axis sampled with the other axis' size fails
    it (swapped corner operands commute with transposition: the ramp golden
    and the float64 bilinear bound catch those)."""
    src = synth.scene(97, 61, 12, n_rect=20, n_checker=3)
    for dw, dh in ((80, 50), (41, 60), (97, 61), (150, 33)):
        assert np.array_equal(oracle.resize(np.ascontiguousarray(src.T), dh, dw), oracle.resize(src, dw, dh).T)
    img = synth.scene(333, 217, 13, n_rect=40, n_checker=5)
    for level in (1, 3, 5):
        a = oracle.pyramid_level(img, 6, 1.2, level)
        b = oracle.pyramid_level(np.ascontiguousarray(img.T), 6, 1.2, level)
        assert np.array_equal(b, a.T)
