"""Write the stored oracle fixtures under tests/golden/.

Calls only ``oracle`` (and the seeded input generators); no value here comes
from the CUDA path.  The paper prints no worked example, so the fixtures are
the oracle's own output on small seeded frames, kept to detect regressions in
the oracle and to give the GPU tests a stored expectation.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2010_08486_gb300 import synth  # noqa: E402

CFG1 = dict(min_sigma=1.0, max_sigma=10.0, ratio=1.6, threshold=0.1, truncate=4.0, overlap=0.5, nbins=32)


def small_frame_fixture():
    img = synth.small_blob_frame(1)
    p = oracle.OracleParams(**CFG1)
    det = oracle.detect(img.astype(np.float64), p)
    c = det.candidates.canonical()
    b = det.blobs.canonical()
    return {
        "source": "oracle.detect on synth.small_blob_frame(seed=1), 256x256; sigma ladder 1.6^i "
                  "from 1 to 10 (6 levels), truncate 4, threshold 0.1, overlap 0.5, 32 log-volume "
                  "bins (Sec. 4 and Sec. 4.1 of the paper with the readings in oracle/dog_oracle.c)",
        "params": CFG1,
        "sigmas": oracle.ladder(p).tolist(),
        "candidates": [[int(l), int(y), int(x), float(r)] for l, y, x, r in
                       zip(c.level, c.y, c.x, c.response)],
        "blobs": [[int(l), int(y), int(x), float(np.float32(s)), float(r)] for l, y, x, s, r in
                  zip(b.level, b.y, b.x, b.sigma, b.response)],
        "counts": det.counts.tolist(),
    }


def main():
    out = os.path.join(HERE, "small_frame_seed1.json")
    with open(out, "w") as f:
        json.dump(small_frame_fixture(), f, indent=1)
    print("wrote", out)


if __name__ == "__main__":
    main()
