"""bench.py's reference arm (the CPU oracle timed on the host) keeps the
benchmark's JSON contract: one line with the metric, value, unit, the
cpu_baseline description and an e2e entry without device copies."""

import json

import pytest

import bench


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    monkeypatch.setattr(bench.os, "cpu_count", lambda: 1)  # one frame per step, one oracle process

    class A:
        steps, warmup, gpus = 1, 0, 1

    assert bench.run_reference(A(), rank=0, world=1) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "frames/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "frames/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["frames_per_step"] == 1


def test_code_hash_ignores_comments(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    a.write_text("int f() {  // one\n    return 1;\n}\n")
    b.write_text("// header\n\nint f() {  // two\n    return 1;   \n}\n")
    assert bench.code_sha1(str(a)) == bench.code_sha1(str(b))
    b.write_text("int f() {\n    return 2;\n}\n")
    assert bench.code_sha1(str(a)) != bench.code_sha1(str(b))


def test_tuning_option_takes_the_lines_autotune_object():
    """--tuning accepts the "autotune" object a bench line printed (search
    statistics dropped) and rejects anything that is not every field as an
    integer, before any GPU work."""
    line = {"resize_tile_h": 64, "fast_blocks_per_sm": 2, "nms_blocks_per_sm": 2, "fast_order": 0,
            "nms_order": 0, "resize_tma": 1, "stream_groups": 8, "fast_cell_tiles": 4, "nms_tile_h": 32,
            "fast_tile_h": 32, "candidates_tried": 61, "resize_ms": 0.4684, "fast_ms": 3.1161, "nms_ms": 1.132}
    got = bench.parse_tuning(json.dumps(line))
    assert list(got) == list(bench.TUNING_FIELDS)
    assert all(got[k] == line[k] for k in bench.TUNING_FIELDS)
    missing = dict(line)
    del missing["stream_groups"]
    for bad in ("[64]", "not json", json.dumps(missing), json.dumps(dict(line, extra=1)),
                json.dumps(dict(line, fast_order=0.5)), json.dumps(dict(line, resize_tma=True))):
        with pytest.raises(SystemExit):
            bench.parse_tuning(bad)


def test_algorithmic_work_of_the_1080p_workload():
    """The per-frame figures the roofline fields divide by, for 1920x1080 with
    8 levels at scale 1.2: level sizes from the oracle, detect regions counted
    by masking each level with the border, and each stage's algorithmic bytes
    (pyramid: read levels 0..6, write 1..7; FAST: read every level, write its
    score map; floor: input, levels 1..7 written, every level read once, one
    64-byte record per kept keypoint)."""
    import numpy as np

    import oracle

    lw, lh, _ = oracle.level_sizes(1920, 1080, 8, 1.2)
    lw, lh = [int(v) for v in lw], [int(v) for v in lh]
    assert (lw[1], lh[1], lw[7], lh[7]) == (1600, 900, 536, 301)
    b = bench.BORDER
    px = [w * h for w, h in zip(lw, lh)]
    det = sum(int(np.ones((h, w), bool)[b:h - b, b:w - b].sum()) for w, h in zip(lw, lh))
    assert sum(px) == 6_419_321 and det == 5_905_941
    assert bench.detect_region_pixels(lw, lh) == det
    pyr, fast, nmsh, sel, orient = bench.stage_bytes(lw, lh, [10] * 8, [2] * 8)
    assert pyr == sum(px) - px[-1] + sum(px) - px[0] == 10_603_706
    assert fast == sum(px) + det == 12_325_262
    assert nmsh == det + sum(px) + 12 * 80 and sel == 12 * 80 + 12 * 16 and orient == 866 * 16
    assert bench.floor_bytes_per_frame(lw, lh, 1000) == px[0] + 2 * sum(px) - px[0] + 64_000 == 12_902_642
    # FAST's work per frame against the integer-ALU peak (152 SMs x 64 lanes x 2.07 GHz).
    assert abs(bench.FAST_OPS_PER_PX * det - 239.19e6) < 0.01e6
    assert abs(152 * bench.ALU_LANES_PER_SM_CLK * 2070e6 - 20.137e12) < 0.001e12
