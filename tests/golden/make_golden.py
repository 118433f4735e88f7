"""Writes config0_oracle.json: oracle outputs of the 1,000-sphere 64 x 64 scene.

The paper prints no worked example with numbers, so nothing here is a paper
value.  This fixture is an oracle regression record: it lets the CPU suite
notice any change of the oracle's results and lets the GPU suite compare with
stored values without rerunning the oracle.  It calls only oracle/ (and the
seeded scene generator).  Quantities and the passages they implement:
  tile lists     App. B, Step 1 (per-tile sphere lists, depth order)
  tracked hits   App. B, Step 2 (the n_track closest hits per pixel)
  image, log D   Eq. 1 (blend weights with the background term)
  gradients      App. B, "The Backward Pass" (sums under a fixed dL/dF)

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

TILES = [0, 5, 6, 9, 10, 15]


def pick_pixels(n_hits):
    """Eight pixels with at least three hits (every 7th such pixel in raster
    order) and two without any."""
    busy = [(int(u), int(v)) for v, u in np.argwhere(n_hits >= 3)]
    idle = [(int(u), int(v)) for v, u in np.argwhere(n_hits == 0)]
    return [list(p) for p in busy[::7][:8] + idle[:1] + idle[-1:]]


def golden():
    from oracle import oracle
    from paper_2004_07484_gb300 import scenes
    oracle.build()
    sc = scenes.config_scene(0)
    ref = oracle.render(sc)
    off, ids = oracle.tile_lists(sc, tile=16)
    G = scenes.grad_image(99, sc.height, sc.width, sc.n_channels)
    g = oracle.render_backward(sc, G)
    PIXELS = pick_pixels(ref.n_hits)
    return {
        "scene": "config_scene(0): 1,000 spheres, 64x64, C=3, gamma 0.1, n_track 5, seed 1000",
        "grad_image": "scenes.grad_image(99, 64, 64, 3)",
        "pixels": PIXELS,
        "image": [[float(x) for x in ref.image[v, u]] for u, v in PIXELS],
        "log_d": [float(ref.log_d[v, u]) for u, v in PIXELS],
        "tracked": [[int(x) for x in ref.tracked[v, u]] for u, v in PIXELS],
        "n_hits": [int(ref.n_hits[v, u]) for u, v in PIXELS],
        "tile_lengths": [int(off[t + 1] - off[t]) for t in range(len(off) - 1)],
        "tiles": TILES,
        "tile_lists": [[int(x) for x in ids[off[t]:off[t + 1]]] for t in TILES],
        "grad_sums": {n: float(np.sum(getattr(g, n))) for n in ("pos", "rad", "opa", "feat", "cam", "bg")},
        "grad_abs_sums": {n: float(np.sum(np.abs(getattr(g, n)))) for n in ("pos", "rad", "opa", "feat", "cam", "bg")},
        "grad_cam": [float(x) for x in g.cam],
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "config0_oracle.json"), "w") as f:
        json.dump(golden(), f, indent=1)
    print("wrote", os.path.join(HERE, "config0_oracle.json"))
