"""The library's host LPT packer (fea_pack_lpt) equals the oracle's greedy
packing queue for queue (CPU only: a host function of the C-ABI)."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


@pytest.mark.parametrize("n,m,seed", [(0, 3, 0), (5, 9, 1), (100, 7, 2), (1000, 152, 3), (4096, 456, 4)])
def test_lpt_matches_oracle(n, m, seed):
    from paper_1805_03949_gb300 import fea
    rng = np.random.default_rng(seed)
    costs = rng.integers(1, 50, n).astype(np.float64) * rng.choice([1.0, 0.5], n)
    q, off, load = fea.fea_pack_lpt(costs, m)
    ids, off2, load2 = M.lpt(costs, m)
    np.testing.assert_array_equal(q, ids)
    np.testing.assert_array_equal(off, off2)
    np.testing.assert_allclose(load, load2, rtol=1e-15)
