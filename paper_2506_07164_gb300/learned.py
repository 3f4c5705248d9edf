"""Learned tile proposal: labelling, training and evaluation on the GPU.

The network and every step of its training run in the library's CUDA
kernels (of_tcnn_*); this module only moves tensors around:

* labels: a plain detection of each training frame marks a 32 x 32 proposal
  tile of a level positive when one of the frame's final keypoints (after
  NMS, Harris ranking and the per-level top-N) lies in it; the patches come
  from the same call's pyramid (of_extract_tiles);
* training: weighted BCE, Adam, cosine learning-rate decay;
* threshold: the largest logit threshold whose recall of positive tiles on
  the training set reaches a target;
* evaluation: the learned path (of_detect_learned) against the plain path on
  held-out frames -- keypoint recall, exact-set agreement, tiles skipped.

Command line (writes a checkpoint plus a JSON summary):
    python -m paper_2506_07164_gb300.learned train --frames 48 --out DIR
"""

from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import (Detector, of_detect_learned, of_extract_tiles, of_tcnn_adam, of_tcnn_create, of_tcnn_destroy,
               of_tcnn_forward, of_tcnn_load, of_tcnn_loss_grad, of_tcnn_save, keypoints_to_numpy)

BORDER = 19
TILE_X0 = BORDER & ~15
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "tile_proposal.oftc")
DEFAULT_META = os.path.join(HERE, "weights", "tile_proposal.json")


class TileNet:
    """Owner of an of_tcnn network."""

    def __init__(self, seed: int = 0):
        self.net = of_tcnn_create(seed)

    def close(self):
        if self.net:
            of_tcnn_destroy(self.net)
            self.net = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def save(self, path: str) -> None:
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        with open(path, "wb") as f:
            f.write(of_tcnn_save(self.net))

    def load(self, path: str) -> "TileNet":
        with open(path, "rb") as f:
            of_tcnn_load(self.net, f.read())
        return self

    def logits(self, tiles):
        import torch

        out = torch.empty(tiles.shape[0], dtype=torch.float32, device=tiles.device)
        of_tcnn_forward(self.net, tiles, tiles.shape[0], out)
        return out


def label_frames(det: Detector, frames, levels: int = 8, scale: float = 1.2, fast_t: int = 20,
                 n_features: int = 1000, neg_keep: float = 1.0, rng=None):
    """Patches and labels of every proposal tile of every level of `frames` (one
    batch of host arrays or 2-D uint8 CUDA tensors).  neg_keep < 1 keeps every
    positive tile and that fraction of the negatives (drawn with `rng`)."""
    import torch

    dev = [f if isinstance(f, torch.Tensor) else torch.from_numpy(f).cuda() for f in frames]
    det.detect_batch(dev, levels=levels, scale=scale, fast_t=fast_t, n_features=n_features)
    torch.cuda.synchronize()
    kps = det.batch_results(len(frames), n_features)
    tiles, labels = [], []
    for fi in range(len(frames)):
        for lvl in range(levels):
            n, (gx, gy) = of_extract_tiles(det.h, fi, lvl)
            if n == 0:
                continue
            t = torch.empty((n, 64, 64), dtype=torch.uint8, device="cuda")
            of_extract_tiles(det.h, fi, lvl, t, n)
            lab = np.zeros(n, np.float32)
            k = kps[fi][kps[fi]["level"] == lvl]
            px = (k["x_l"] - TILE_X0) // 32
            py = (k["y_l"] - BORDER) // 32
            lab[py * gx + px] = 1.0
            if neg_keep < 1.0:
                keep = np.nonzero((lab > 0) | (rng.random(n) < neg_keep))[0]
                t = t[torch.from_numpy(keep).cuda()]
                lab = lab[keep]
            tiles.append(t)
            labels.append(torch.from_numpy(lab).cuda())
    return torch.cat(tiles), torch.cat(labels)


def frame_variants(img, k: int):
    """Variant k (0..7) of a generated frame on the device: flips about either
    axis and intensity inversion (255 - I), each a generated frame of the same
    size and statistics; the detector labels every variant itself."""
    import torch

    t = img
    if k & 1:
        t = torch.flip(t, dims=(1,))
    if k & 2:
        t = torch.flip(t, dims=(0,))
    if k & 4:
        t = 255 - t
    return t.contiguous()


def train(net: TileNet, tiles, labels, steps: int = 1500, batch: int = 2048, lr: float = 3e-3,
          pos_weight: float = 4.0, seed: int = 0, log_every: int = 0):
    """Adam with cosine decay on random minibatches; returns the loss history."""
    import torch

    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    n = tiles.shape[0]
    hist = []
    for s in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), generator=g, device="cuda")
        tb = tiles[idx].contiguous()
        lb = labels[idx].contiguous()
        loss = of_tcnn_loss_grad(net.net, tb, lb, tb.shape[0], pos_weight)
        cur = lr * 0.5 * (1.0 + math.cos(math.pi * s / max(1, steps)))
        of_tcnn_adam(net.net, max(cur, lr * 0.02))
        hist.append(loss)
        if log_every and s % log_every == 0:
            print(f"step {s} loss {loss:.4f}", flush=True)
    return hist


def choose_threshold(net: TileNet, tiles, labels, target_recall: float = 0.995) -> float:
    """Largest sigmoid threshold keeping `target_recall` of the positive tiles."""
    import torch

    z = net.logits(tiles)
    p = torch.sigmoid(z[labels > 0.5]).sort().values.cpu().numpy()
    if len(p) == 0:
        return 0.5
    k = int(math.floor((1.0 - target_recall) * len(p)))
    return float(max(1e-4, min(p[k], 0.5)))


def _keyset(kp):
    return {(int(a), int(b), int(c)) for a, b, c in zip(kp["level"], kp["y_l"], kp["x_l"])}


def evaluate(det: Detector, net: TileNet, frames, threshold: float, min_confidence: float = 0.0,
             dilate: int = 1, levels: int = 8, scale: float = 1.2, fast_t: int = 20, n_features: int = 1000,
             chunk: int = 16):
    """Learned path vs plain path on `frames` (batches of `chunk`): recall, agreement, work skipped."""
    import torch

    inter = union = total = identical = tiles = proposed = fallback = 0
    for i in range(0, len(frames), chunk):
        part = frames[i:i + chunk]
        dev = [torch.from_numpy(f).cuda() for f in part]
        fr = [(t, t.shape[1], t.shape[0], t.stride(0)) for t in dev]
        det.detect_batch(dev, levels=levels, scale=scale, fast_t=fast_t, n_features=n_features)
        torch.cuda.synchronize()
        plain = det.batch_results(len(part), n_features)
        st = of_detect_learned(det.h, fr, levels, scale, fast_t, 0.04, n_features, net.net, threshold,
                               min_confidence, dilate, det.out, det.counts)
        torch.cuda.synchronize()
        learned = det.batch_results(len(part), n_features)
        for a, b in zip(plain, learned):
            A, B = _keyset(a), _keyset(b)
            inter += len(A & B)
            union += len(A | B)
            total += len(A)
            identical += int(len(a) == len(b) and np.array_equal(a.view(np.uint8), b.view(np.uint8)))
        tiles += st["tiles"]
        proposed += st["proposed"]
        fallback += st["fallback_images"]
    return {"recall": inter / max(1, total), "jaccard": inter / max(1, union),
            "identical_frames": identical, "frames": len(frames),
            "proposed_fraction": proposed / max(1, tiles), "tiles": tiles, "fallback_images": fallback}


def random_proposal_recall(det: Detector, frames, keep_fraction: float, seed: int = 0, levels: int = 8,
                           scale: float = 1.2, fast_t: int = 20, n_features: int = 1000, chunk: int = 16):
    """Recall of the plain keypoints when a random `keep_fraction` of tiles is kept (no network)."""
    import torch

    plain = []
    for i in range(0, len(frames), chunk):
        dev = [torch.from_numpy(f).cuda() for f in frames[i:i + chunk]]
        det.detect_batch(dev, levels=levels, scale=scale, fast_t=fast_t, n_features=n_features)
        torch.cuda.synchronize()
        plain += [k.copy() for k in det.batch_results(len(dev), n_features)]
    rng = np.random.default_rng(seed)
    hit = tot = 0
    for kp in plain:
        # A keypoint survives only if its tile is kept (independent coin per tile).
        tiles = {(int(l), int((y - BORDER) // 32), int((x - TILE_X0) // 32))
                 for l, y, x in zip(kp["level"], kp["y_l"], kp["x_l"])}
        kept = {t for t in tiles if rng.random() < keep_fraction}
        for l, y, x in zip(kp["level"], kp["y_l"], kp["x_l"]):
            tot += 1
            hit += (int(l), int((y - BORDER) // 32), int((x - TILE_X0) // 32)) in kept
    return hit / max(1, tot)


def _gen(args):
    import synth

    w, h, seed = args
    return synth.scene(w, h, seed, background="pink")


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--frames", type=int, default=48, help="generated scenes")
    t.add_argument("--variants", type=int, default=1, help="variants per scene (1..8: flips, inversion)")
    t.add_argument("--neg-keep", type=float, default=1.0, help="fraction of negative tiles kept")
    t.add_argument("--eval-frames", type=int, default=8)
    t.add_argument("--steps", type=int, default=2000)
    t.add_argument("--batch", type=int, default=2048)
    t.add_argument("--out", default=os.path.dirname(DEFAULT_WEIGHTS))
    t.add_argument("--seed", type=int, default=7)
    args = ap.parse_args()

    import multiprocessing as mp

    t0 = time.time()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        train_frames = pool.map(_gen, [(1920, 1080, 20000 + i) for i in range(args.frames)], chunksize=4)
        eval_frames = pool.map(_gen, [(1920, 1080, 30000 + i) for i in range(args.eval_frames)])
    t_gen = time.time() - t0
    import torch

    det = Detector(1920, 1080, max_levels=8, max_features=1000, max_batch=16, fast_t_lo=7)
    t0 = time.time()
    rng = np.random.default_rng(args.seed)
    tiles, labels = [], []
    n_train = 0
    for i in range(0, len(train_frames), 2):
        base = [torch.from_numpy(f).cuda() for f in train_frames[i:i + 2]]
        batch = [frame_variants(f, k) for f in base for k in range(args.variants)]
        for j in range(0, len(batch), 16):
            a, b = label_frames(det, batch[j:j + 16], neg_keep=args.neg_keep, rng=rng)
            tiles.append(a)
            labels.append(b)
        n_train += len(batch)
    tiles = torch.cat(tiles)
    labels = torch.cat(labels)
    t_label = time.time() - t0
    net = TileNet(args.seed)
    t0 = time.time()
    # Kept negatives stand for 1 / neg_keep negatives each: scale their weight back up.
    hist = train(net, tiles, labels, steps=args.steps, batch=args.batch, pos_weight=4.0 * args.neg_keep,
                 log_every=200)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    thr = choose_threshold(net, tiles, labels)
    ev = evaluate(det, net, eval_frames, thr, dilate=1)
    rnd = random_proposal_recall(det, eval_frames, ev["proposed_fraction"])
    sweep = []
    for target in (0.9, 0.95, 0.98, 0.99, 0.995, 0.999):
        t_ = choose_threshold(net, tiles, labels, target)
        for dil in (0, 1):
            e = evaluate(det, net, eval_frames, t_, dilate=dil)
            sweep.append({"tile_recall_target": target, "threshold": t_, "dilate": dil, "recall": e["recall"],
                          "jaccard": e["jaccard"], "identical_frames": e["identical_frames"],
                          "proposed_fraction": e["proposed_fraction"]})
    os.makedirs(args.out, exist_ok=True)
    wpath = os.path.join(args.out, os.path.basename(DEFAULT_WEIGHTS))
    net.save(wpath)
    meta = {"threshold": thr, "dilate": 1, "min_confidence": 0.0, "train_frames": n_train,
            "train_scenes": args.frames, "variants_per_scene": args.variants, "negative_keep": args.neg_keep,
            "train_tiles": int(tiles.shape[0]), "positive_fraction": float(labels.mean().item()),
            "steps": args.steps, "batch": args.batch, "loss_first": hist[0],
            "loss_last": float(np.mean(hist[-50:])), "generate_seconds": round(t_gen, 2),
            "label_seconds": round(t_label, 2), "train_seconds": round(t_train, 2), "eval": ev,
            "random_proposal_recall_same_keep": rnd, "sweep": sweep,
            "frames": "synthetic 1920x1080 scenes (1/f background), seeds 20000+ (train) in "
                      f"{args.variants} variants each (flips about either axis, intensity inversion), "
                      "seeds 30000+ (eval, not varied); labels from the exact path"}
    with open(os.path.join(args.out, os.path.basename(DEFAULT_META)), "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps(meta))
    det.close()
    net.close()


if __name__ == "__main__":
    main()
