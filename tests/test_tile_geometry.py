"""Index arithmetic of the tiled kernels, checked on the CPU.

The constants below restate the tiling of csrc/of_internal.h and the kernels
(tile sizes, TMA boxes, rows per warp).  For every level of a range of frame
sizes and pyramid scales, and for every tile kind the kernels use, the tests
check what the kernels rely on without checking it at run time:

  - every TMA box starts at an x coordinate that is a multiple of 16 bytes
    (the tiled-copy alignment rule for 8-bit data);
  - every staged row and column a thread reads lies inside the boxes loaded
    into its shared-memory buffer;
  - the tiles cover the detect region [b, w - b) x [b, h - b).
"""

import math
import os
import re

import pytest

import paper_2506_07164_gb300 as ofg

TILE_W, HALO_X, SROW = 128, 16, 160
IMG_BOX_ROWS, SCORE_BOX_ROWS = 40, 34
WARPS = 8                      # DET_THREADS / 32
CT_MAX_W, CT_RPT, CT_MAX_WARPS, CT_MAX_TILE_ROWS = 124, 5, 12, 64
AL_T, AL_RPT = 120, 15

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2506_07164_gb300", "csrc")


def source_constants(*files):
    """`constexpr int NAME = EXPR;` lines of the given sources, evaluated in
    order (integer arithmetic; names refer to earlier constants)."""
    env = {}
    pat = re.compile(r"^\s*constexpr\s+int\s+(\w+)\s*=\s*([^;]+);", re.M)
    for f in files:
        for name, expr in pat.findall(open(os.path.join(CSRC, f)).read()):
            try:
                env[name] = eval(expr.replace("/", "//"), {"__builtins__": {}}, dict(env))
            except Exception:
                pass  # an expression this restatement does not need
    return env


def test_constants_match_the_sources():
    """The tiling restated here is the tiling the kernels are built with."""
    c = source_constants("of_internal.h", "k_fast.cu", "k_nms_harris.cu")
    assert (c["TILE_W"], c["HALO_X"], c["SROW"]) == (TILE_W, HALO_X, SROW)
    assert (c["IMG_BOX_ROWS"], c["SCORE_BOX_ROWS"]) == (IMG_BOX_ROWS, SCORE_BOX_ROWS)
    assert c["DET_THREADS"] // 32 == WARPS
    assert (c["CT_MAX_W"], c["CT_RPT"], c["CT_MAX_WARPS"], c["CT_MAX_TILE_ROWS"]) == \
        (CT_MAX_W, CT_RPT, CT_MAX_WARPS, CT_MAX_TILE_ROWS)
    assert (c["AL_T"], c["AL_RPT"]) == (AL_T, AL_RPT)


SIZES = [(1920, 1080), (1280, 720), (640, 480), (3840, 2160), (720, 540), (1440, 1080), (333, 217),
         (129, 77), (1000, 41), (41, 1000), (161, 161), (1283, 723)]
SCALES = [1.05, 1.2, 2.0]


def levels(w, h, scale, n=8):
    ws, hs, _ = ofg.of_plan_levels(w, h, n, scale, 1000)
    return list(zip(ws, hs))


def det_levels(border=19):
    for (W, H) in SIZES:
        for scale in SCALES:
            for w, h in levels(W, H, scale):
                if w - 2 * border > 0 and h - 2 * border > 0:
                    yield w, h


def ceil_div(a, b):
    return -(-a // b)


@pytest.mark.parametrize("th", [32, 64, 128, 256])
def test_general_fast_tiles(th):
    """k_fast<*, TH>: 128 x TH tiles, boxes at (X0 - 16, Y0 - 4 + 40k)."""
    b = 19
    rpt = th // WARPS
    loads = ceil_div(th + 8, IMG_BOX_ROWS)
    # Staged rows a warp reads: (w * RPT + k + 1), k < RPT + 6 (row 0 = Y0 - 4).
    assert (WARPS - 1) * rpt + (rpt + 5) + 1 < loads * IMG_BOX_ROWS
    # Columns: HALO_X + 4 lane - 4 .. + 7.
    assert HALO_X - 4 >= 0 and HALO_X + 4 * 31 + 7 < SROW
    for w, h in det_levels(b):
        tile_x0 = b & ~15
        tiles_x = ceil_div(w - b - tile_x0, TILE_W)
        tiles_y = ceil_div(h - 2 * b, th)
        assert tile_x0 <= b and tile_x0 + TILE_W * tiles_x >= w - b
        assert b + th * tiles_y >= h - b
        for tx in range(tiles_x):
            assert (tile_x0 + TILE_W * tx - HALO_X) % 16 == 0


@pytest.mark.parametrize("th", [32, 64, 128])
def test_nms_tiles(th):
    """k_nms_harris<*, TH>: score boxes every 32 rows from Y0 - 1, image boxes every 40 from Y0 - 4."""
    rpt = th // WARPS
    s_rows = th + 2
    s_loads = ceil_div(s_rows - SCORE_BOX_ROWS, 32) + 1
    i_loads = ceil_div(th + 8, IMG_BOX_ROWS)
    # 3x3 test: staged score rows w * RPT + k, k < RPT + 2.
    assert (WARPS - 1) * rpt + rpt + 1 < (s_loads - 1) * 32 + SCORE_BOX_ROWS
    # Harris: image rows ly + 4 + v, ly < TH, |v| <= 4; words w0 .. w0 + 2 of each row.
    assert th - 1 + 8 < i_loads * IMG_BOX_ROWS
    for lx in range(TILE_W):
        w0 = (HALO_X + lx - 4) >> 2
        assert w0 >= 0 and 4 * (w0 + 2) + 3 < SROW
    # Score and image boxes at the tile's origin - 16: aligned (origins are multiples of 16).
    b = 19
    assert ((b & ~15) - HALO_X) % 16 == 0


def ct_cell_rows(cell):
    nw = ceil_div(cell, CT_RPT)
    return min(CT_MAX_TILE_ROWS // cell, CT_MAX_WARPS // nw)


@pytest.mark.parametrize("cell", range(8, 31))
def test_cell_tiles(cell):
    """k_fast_cells: cpt x cr whole cells; 4-pixel groups from x_lo & ~3; boxes from (gx0 - 4) & ~15."""
    b = 19
    cpt, nw, cr = CT_MAX_W // cell, ceil_div(cell, CT_RPT), ct_cell_rows(cell)
    assert cr >= 1 and nw * cr <= CT_MAX_WARPS
    tw, th = cpt * cell, cr * cell
    loads = ceil_div((cr - 1) * cell + CT_RPT * nw + 6, IMG_BOX_ROWS)
    assert loads <= 2
    # Staged rows: warp (wcr, wr) reads wcr * cell + 5 wr + k, k < 11.
    assert (cr - 1) * cell + CT_RPT * (nw - 1) + 10 < loads * IMG_BOX_ROWS
    for w, h in det_levels(b):
        ncx = ceil_div(w - 2 * b, cell)
        ftiles_x = ceil_div(ncx, cpt)
        for ftx in range(ftiles_x):
            x_lo = b + ftx * tw
            gx0 = x_lo & ~3
            box_x = (gx0 - 4) & ~15
            assert box_x % 16 == 0 and box_x >= 0
            xoff0 = gx0 - box_x
            assert xoff0 >= 4 and xoff0 + 4 * 31 + 7 < SROW  # reads xoff - 4 .. xoff + 7
            assert gx0 + 4 * 32 >= x_lo + tw                # the lanes cover the tile
        assert b + ftiles_x * tw >= w - b


@pytest.mark.parametrize("cell", [15, 30])
def test_cell_aligned_tiles(cell):
    """k_fast_aligned: 120 x 120 tiles of whole cells, 8 warps x 15 rows, four boxes from gx0 - 4."""
    b = 19
    assert AL_T % cell == 0 and cell % AL_RPT == 0 and AL_RPT * WARPS == AL_T
    loads = ceil_div(AL_T + 6, IMG_BOX_ROWS)
    assert AL_RPT * (WARPS - 1) + (AL_RPT - 1) + 6 < loads * IMG_BOX_ROWS
    for w, h in det_levels(b):
        ncx, ncy = ceil_div(w - 2 * b, cell), ceil_div(h - 2 * b, cell)
        ftiles_x, ftiles_y = ceil_div(ncx, AL_T // cell), ceil_div(ncy, AL_T // cell)
        for ftx in range(ftiles_x):
            x_lo = b + ftx * AL_T
            gx0 = x_lo & ~3
            box_x = (gx0 - 4) & ~15
            assert box_x % 16 == 0 and box_x >= 0
            xoff0 = gx0 - box_x
            assert xoff0 >= 4 and xoff0 + 4 * 31 + 7 < SROW
            assert gx0 + 4 * 32 >= x_lo + AL_T
        assert b + ftiles_x * AL_T >= w - b and b + ftiles_y * AL_T >= h - b


def test_per_warp_general_tiles():
    """k_fast_warp: one 128 x 32 detect tile per warp item, one 160 x 40 box from
    (X0 - 16, Y0 - 4); output row r (0..31) reads staged rows r + 1 .. r + 7 through a
    rotating window of FW_CHUNK = 7 slots (slot = staged row mod 7, aligned at every
    chunk start)."""
    b = 19
    chunk = source_constants("of_internal.h", "k_fast.cu")["FW_CHUNK"]
    assert chunk == 7
    for r in range(32):
        assert r + 1 >= 0 and r + 7 < IMG_BOX_ROWS
    for r0 in range(0, 32, chunk):
        assert r0 % chunk == 0  # slot (r0 + k) % 7 == k % 7 at each chunk start
    assert HALO_X - 4 >= 0 and HALO_X + 4 * 31 + 7 < SROW
    for w, h in det_levels(b):
        tile_x0 = b & ~15
        tiles_x = ceil_div(w - b - tile_x0, TILE_W)
        for tx in range(tiles_x):
            assert (tile_x0 + tx * TILE_W - HALO_X) % 16 == 0
        assert tile_x0 + tiles_x * TILE_W >= w - b


@pytest.mark.parametrize("cell", range(8, 34))
def test_cell_row_strips(cell):
    """k_fast_cstrip: one cell row of one 128-column detect tile column per warp item; one
    160 x 40 box from (X0 - 16, y0 - 4); output row r < cell reads staged rows r + 1 .. r + 7;
    the strip's cells fit the flag word.  A tile column with at most 64 (32) region columns
    left splits the lanes into 2 (4) row groups of hq = ceil(nrows / groups) rows starting
    at min(g hq, nrows - hq): every row is covered, none lies past the strip."""
    b = 19
    assert (cell - 1) + 7 < IMG_BOX_ROWS
    assert TILE_W // cell + 2 <= 32
    for nrows in range(1, cell + 1):
        for lg in (0, 1, 2):
            G = 1 << lg
            hq = -(-nrows // G)
            covered = set()
            for g in range(G):
                ro = min(g * hq, nrows - hq)
                assert 0 <= ro and ro + hq <= nrows
                covered |= set(range(ro, ro + hq))
            assert covered == set(range(nrows))
    for w, h in det_levels(b):
        tile_x0 = b & ~15
        tiles_x = ceil_div(w - b - tile_x0, TILE_W)
        ncy = ceil_div(h - 2 * b, cell)
        for tx in range(tiles_x):
            X0 = tile_x0 + tx * TILE_W
            assert (X0 - HALO_X) % 16 == 0
            useful = w - b - X0
            lg = 2 if useful <= 32 else 1 if useful <= 64 else 0
            # The lanes' columns cover the tile column's region columns.
            assert X0 + 4 * (32 >> lg) >= min(w - b, X0 + TILE_W)
            cx0 = (max(X0, b) - b) // cell
            for lane in range(32):
                x = X0 + 4 * (lane & (31 >> lg))
                for xx in range(x, x + 4):
                    if b <= xx < w - b:
                        assert 0 <= (xx - b) // cell - cx0 < 32
        assert b + ncy * cell >= h - b


@pytest.mark.parametrize("cell", range(8, 41))
def test_per_warp_nms_tiles(cell):
    """k_nms_warp: per warp one 160 x 34 score box from (X0 - 16, Y0 - 1) and one 160 x 40
    image box from (X0 - 16, Y0 - 4) on the 128 x 32 detect tiles.  The 3x3 test reads staged
    score rows 0 .. 33 at word offsets HALO_X + 4 lane and the halo words HALO_X - 4 (lane 0)
    and HALO_X + 128 (lane 31); Harris reads image rows ly .. ly + 8 and words w0 .. w0 + 2.
    A chunk of NW_CHUNK output rows reads NW_CHUNK new staged rows, which lie in at most two
    cell rows (cells of 8 or more rows); the queue holds every possible survivor; two blocks'
    buffers fit one SM's shared memory."""
    c = source_constants("of_internal.h", "k_nms_harris.cu")
    chunk, qcap, nbytes, dyn = c["NW_CHUNK"], c["NW_QCAP"], c["NW_BYTES"], c["NW_DYN"]
    assert c["S_BOX"] == SCORE_BOX_ROWS * SROW and c["I_BOX"] == IMG_BOX_ROWS * SROW
    assert 32 + 1 < SCORE_BOX_ROWS                      # staged rows 0 .. 33
    assert HALO_X - 4 >= 0 and HALO_X + TILE_W + 3 < SROW
    for ly in range(32):
        assert ly + 8 < IMG_BOX_ROWS
    for lx in range(TILE_W):
        w0 = (HALO_X + lx - 4) >> 2
        assert w0 >= 0 and 4 * (w0 + 2) + 3 < SROW
    assert qcap >= TILE_W * 32 // 4                     # strict maxima: at most one per 2 x 2 block
    assert nbytes % 128 == 0 and c["NW_SBUF"] % 128 == 0
    assert 2 * (dyn + 1024 + 8 * 16) <= 228 * 1024      # 2 blocks per SM, 1 KB reserved per block
    # New staged rows of the chunk starting at output row r0: image rows Y0 + 1 + r0 .. Y0 + r0 + chunk.
    b = 19
    for y0 in range(b, b + 4 * cell, 32):
        for r0 in range(0, 32, chunk):
            rows = range(y0 + 1 + r0, y0 + 1 + r0 + chunk)
            assert len({(y - b) // cell for y in rows}) <= 2
