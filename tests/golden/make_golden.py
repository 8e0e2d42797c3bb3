"""Writes the regression fixtures of this folder from the FP64 oracle alone.

The paper prints no worked example of its renderer (it uses the 3DGS
rasteriser it cites, Sec. 3.2), so these fixtures are not the paper's values:
they freeze the oracle's own output on tiny inputs so that a later change of
the oracle's arithmetic shows up as a diff of a committed text file. Run from
the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import upsampler as U  # noqa: E402
from paper_2510_15352_b300 import synth  # noqa: E402

RENDER_FILE = os.path.join(HERE, "oracle_render_20000g_sh2_48x32.json")
UPSAMPLER_FILE = os.path.join(HERE, "oracle_upsampler_5x7.json")


def render_case():
    """A 20,000-Gaussian SH-degree-2 scene seen by one camera at 48x32 (f = 40),
    seed 3: every pixel's rgb, depth and T, plus the near-threshold flags."""
    scene = synth.make_scene(20_000, 2, seed=3)
    vm, it = synth.make_cameras(1, 48, 32, 40.0, (0.5, 0.5), seed=3)
    return scene, vm[0], it[0], 48, 32


def upsampler_case():
    """A 2-frame 5x7 input through the network with seed-0 weights (last layer
    non-zero): the 20x28 output."""
    rng = np.random.default_rng(5)
    rgb = rng.uniform(0, 1, size=(2, 5, 7, 3))
    params = U.init_params(0, zero_last=False)
    return params, rgb


def main():
    orc = oracle.get()
    scene, vm, it, W, H = render_case()
    r = orc.render(scene, vm, it, W, H)
    with open(RENDER_FILE, "w") as f:
        json.dump({"what": render_case.__doc__.strip(), "W": W, "H": H,
                   "rgb": np.round(r["rgb"], 12).tolist(),
                   "depth": np.round(r["depth"], 12).tolist(),
                   "T": np.round(r["T"], 12).tolist(),
                   "flags": r["flags"].tolist()}, f)
    params, rgb = upsampler_case()
    out = U.forward(params, rgb)
    with open(UPSAMPLER_FILE, "w") as f:
        json.dump({"what": upsampler_case.__doc__.strip(), "out": np.round(out, 12).tolist()}, f)


if __name__ == "__main__":
    main()
