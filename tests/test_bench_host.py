"""Host logic of bench.py that needs no GPU: the surrogate gate's per-size calibration."""

import numpy as np

import bench


def test_gate_calibration_picks_the_largest_limit_meeting_both_bounds():
    """Leaves whose K* error equals their ensemble spread (uniform on [0, 0.1]): the accepted set
    under a limit g is the spread <= ln(1 + g), whose median is about ln(1 + g) / 2 and p99 about
    ln(1 + g). With p99 <= 4 % and median <= 1.5 % the median binds: the calibrated limit is the
    largest grid value with ln(1 + g) <= 0.03 (to the grid's resolution). Sizes with no leaves,
    or whose leaves are all out of the training range, keep the smallest limit."""
    rng = np.random.default_rng(1)
    n = 20000
    sizes = np.where(np.arange(n) % 2 == 0, 8, 64)
    sd = rng.uniform(0.0, 0.1, n)
    rel = sd.copy()
    in_range = np.ones(n, dtype=bool)
    in_range[sizes == 64] = False                    # size 64: nothing in range
    gate = bench._calibrate_gate(sd, in_range, rel, sizes, p99_max=0.04, med_max=0.015)
    grid = np.geomspace(1e-3, 0.3, 60)
    g8 = gate[bench.SUR_SIZES.index(8)]
    below = grid[np.log1p(grid) <= 0.0299]
    above = grid[np.log1p(grid) >= 0.0301]
    assert below.max() <= g8 + 1e-9 and g8 < above.min()
    for s in bench.SUR_SIZES:
        if s != 8:
            assert gate[bench.SUR_SIZES.index(s)] == np.float32(grid[0])
    # the accepted leaves of size 8 meet both bounds
    acc = (sizes == 8) & (sd <= np.log1p(g8))
    assert np.percentile(rel[acc], 99) <= 0.04 and np.median(rel[acc]) <= 0.015
