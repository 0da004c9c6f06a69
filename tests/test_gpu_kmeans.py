"""kmeans++ selection of inducing points (paper §4.1) on the GPU against the
oracle: integer D^2 weights make every sum exact, so the chosen indices agree
bit for bit."""
import numpy as np
import pytest

import fsa_inputs as fi
from oracle import fsa_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import paper_2405_14492_gb300 as F
    return F


@pytest.mark.parametrize("n,m,seed,scale,offset", [
    (5000, 100, 1, 1.0, 0.0),          # several chunks of 1024, ragged tail
    (20011, 500, 7, 1.0, 0.0),
    (1500, 1500, 3, 1.0, 0.0),         # every point chosen (the last weights are 0 but one)
    (3001, 64, 11, 2500.0, -4.0e3),    # a wide, shifted bounding box (other weight exponent)
    (1, 1, 5, 1.0, 0.0),               # a single point
])
def test_kmeanspp_matches_oracle_bit_for_bit(F, n, m, seed, scale, offset):
    locs = fi.uniform_locations(n, 31) * scale + offset
    got = F.kmeanspp(locs, m, seed)
    ref = O.kmeanspp(locs, m, seed)
    assert np.array_equal(got, ref)
    assert len(set(got.tolist())) == m


def test_kmeanspp_clustered_points_and_duplicates(F):
    rng = np.random.default_rng(8)
    locs = np.vstack([fi.uniform_locations(3000, 32), 0.5 + 1e-4 * rng.random((500, 2))])
    got = F.kmeanspp(locs, 200, 9)
    assert np.array_equal(got, O.kmeanspp(locs, 200, 9))
    dup = np.repeat(fi.uniform_locations(40, 33), 3, axis=0)     # 40 distinct locations, 120 points
    with pytest.raises(Exception):
        F.kmeanspp(dup, 41, 1)
    assert np.array_equal(F.kmeanspp(dup, 40, 1), O.kmeanspp(dup, 40, 1))
