"""Rendered-sphere frames on the GPU equal the CPU restatement in the oracle
bit for bit (intensity and 12-bit counts), from empty tables to the paper's
1000 x 1000 frames of 100 spheres (Sec. 5)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2010_08486_gb300 import build as libbuild
from paper_2010_08486_gb300 import dog, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


CASES = [
    # (n spheres, h, w, ss, background, gain, read noise, seed)
    (100, 1000, 1000, 4, 0.05, 2000.0, 4.0, 7),
    (0, 33, 47, 4, 0.25, 2000.0, 5.0, 1),
    (1, 64, 64, 1, 0.0, 4000.0, 0.0, 2),
    (40, 257, 130, 2, 0.1, 1000.0, 2.0, 3),
    (300, 512, 512, 8, 0.05, 3000.0, 8.0, 4),
    (5, 16, 16, 4, 2.0, 4000.0, 1.0, 5),       # saturated: every count clipped to 4095
]


@pytest.mark.parametrize("case", CASES)
def test_render_matches_cpu_restatement(case):
    n, h, w, ss, bg, gain, rn, seed = case
    table = synth.sphere_table(synth.SPHERE_SEED_BASE + seed, n=n, h=h, w=w)
    counts, inten = dog.render_spheres(torch.from_numpy(table).cuda(), h, w, ss=ss, background=bg, gain=gain,
                                       read_noise=rn, seed=seed, with_intensity=True)
    torch.cuda.synchronize()
    want_i, want_c = oracle.render_spheres(table, h, w, ss=ss, background=bg, gain=gain, read_noise=rn, seed=seed)
    got_i = inten.cpu().numpy()
    got_c = counts.cpu().numpy().view(np.uint16)
    assert np.array_equal(got_i.view(np.uint32), want_i.view(np.uint32)), \
        "intensity differs at %d pixels" % np.count_nonzero(got_i != want_i)
    assert np.array_equal(got_c, want_c), "counts differ at %d pixels" % np.count_nonzero(got_c != want_c)
