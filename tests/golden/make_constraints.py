"""Write cfg2_constraints.json: multiple-image constraints of the 1000-potential
cluster model, produced by solving the lens equation with the FP64 oracle.

Shape of the paper's benchmark constraints (Sec. 5: 80 sources, 227 multiple
images, HST precision): here 100 sources, 20 at each distance ratio
D_ls/D_s in {0.5, 0.6, 0.7, 0.8, 0.9}; each source is drawn uniformly in a
disc around the cluster centre and kept when the brute-force search (Sec. 2.3,
Fig. 4) finds 2 to 7 images; every image then gets N(0, 0.1") noise and
sigma = 0.1".  Calls only oracle/ and the seeded input generators.

  python tests/golden/make_constraints.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2004_06352_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfg2_constraints.json")
RATIOS = (0.5, 0.6, 0.7, 0.8, 0.9)
PER_RATIO = 20
SEARCH_N = 1024
SIGMA = 0.1


def main():
    m = I.cfg2_model()
    g = I.grid(SEARCH_N)
    ag = oracle.alpha_grid(m, g)
    xs, ys, off, ratio = [], [], [0], []
    for ri, r in enumerate(RATIOS):
        got, seed = 0, 100 * ri
        while got < PER_RATIO:
            seed += 1
            sx, sy, _ = I.source_candidates(1, seed, radius=18.0, ratios=(r,))
            img, nf = oracle.find_images(m, g, r, (float(sx[0]), float(sy[0])), ag=ag, cap=64)
            if not (2 <= nf <= 7):
                continue
            noise = I.gaussian_noise(nf, 10_000 + seed, SIGMA)
            for k in range(nf):
                xs.append(float(img[k, 0] + noise[k, 0]))
                ys.append(float(img[k, 1] + noise[k, 1]))
            off.append(len(xs))
            ratio.append(r)
            got += 1
    doc = {"about": "constraints of inputs.cfg2_model(seed=2): 100 sources x 2-7 images, written by "
                    "tests/golden/make_constraints.py with the FP64 oracle (lens equation, Sec. 2.1 Eq. 1; "
                    "brute-force image search, Sec. 2.3 Fig. 4)",
           "sigma": SIGMA, "img_off": off, "x": xs, "y": ys, "dls_ds": ratio}
    with open(OUT, "w") as f:
        json.dump(doc, f)
    print(f"{len(ratio)} sources, {len(xs)} images -> {OUT}")


def load():
    """The stored constraint table as the dict the bindings take."""
    return I.load_constraints(OUT)


if __name__ == "__main__":
    main()
