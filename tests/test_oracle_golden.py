"""The oracle still reproduces its stored fixture (written by
tests/golden/make_golden.py, which calls only the oracle)."""
import json
import os

import numpy as np

from tests.golden.make_golden import small_frame_fixture

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_reproduces_small_frame_fixture():
    with open(os.path.join(HERE, "golden", "small_frame_seed1.json")) as f:
        want = json.load(f)
    got = small_frame_fixture()
    assert [c[:3] for c in got["candidates"]] == [c[:3] for c in want["candidates"]]
    np.testing.assert_allclose([c[3] for c in got["candidates"]], [c[3] for c in want["candidates"]],
                               rtol=1e-12, atol=0)
    assert [b[:4] for b in got["blobs"]] == [b[:4] for b in want["blobs"]]
    assert got["counts"] == want["counts"]
    assert sum(want["counts"]) == len(want["blobs"])
