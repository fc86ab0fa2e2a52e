"""The all-cores driver of the oracle (oracle/parallel.py) against the serial oracle.

The driver only splits the LED sum of Eqs. 9-11 and 18 into contiguous blocks on
worker processes and adds the blocks in block order, so three iterations must match
the serial oracle to FP64 rounding (the order of the LED sum differs); multiplexed
images are kept whole.
"""
import numpy as np
import pytest

import oracle as O
from oracle.parallel import ParallelOracle, image_blocks

from _cases import case, rel
from test_oracle_pins import _mux_problem


def test_image_blocks_partition_in_order():
    for n_img, blocks in ((49, 2), (49, 7), (5, 8), (225, 15), (1, 3)):
        r = image_blocks(n_img, blocks)
        assert r[0][0] == 0 and r[-1][1] == n_img and len(r) == min(blocks, n_img)
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        sizes = [b - a for a, b in r]
        assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)


@pytest.mark.parametrize("workers", [2, 3])
def test_parallel_oracle_matches_serial(workers):
    c = case("small32")
    I = c["I"].astype(np.float64)
    opt = O.Options()
    st = O.init_state(I, c["geo"], c["k_xy"], opt)
    ref, costs_ref = O.run(st, I, c["geo"], opt, 3)
    with ParallelOracle(c["geo"], I, workers=workers) as po:
        assert po.cores == workers + 1
        got, costs = po.run(st, opt, 3)
    assert rel(got.psi, ref.psi) < 1e-13 and rel(got.pupil, ref.pupil) < 1e-13
    assert np.allclose(costs, costs_ref, rtol=1e-13, atol=0)


def test_parallel_oracle_keeps_multiplexed_images_whole():
    geo, k_xy, I, _, _ = _mux_problem(2, 1, 61)
    opt = O.Options(alpha=0.01, beta=0.01)
    st = O.init_state(I, geo, k_xy, opt)
    ref, costs_ref = O.run(st, I, geo, opt, 2)
    with ParallelOracle(geo, I, workers=2) as po:
        got, costs = po.run(st, opt, 2)
    assert rel(got.psi, ref.psi) < 1e-13 and np.allclose(costs, costs_ref, rtol=1e-13, atol=0)
