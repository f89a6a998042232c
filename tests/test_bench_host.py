"""Host logic of bench.py's calibrations (no device): the FP64 iteration budget and the mixed solve's line-search
depth are chosen on a separate calibration batch, by accuracy alone."""
import numpy as np
import pytest

import bench


@pytest.mark.parametrize("acc,want", [({0: 0.969, 1: 0.969, 2: 0.969, 3: 0.969}, 0),
                                      ({0: 0.90, 1: 0.968, 2: 0.969, 3: 0.970}, 1),
                                      ({0: 0.90, 1: 0.91, 2: 0.92, 3: 0.97}, 3),
                                      ({0: 0.99, 1: 0.95, 2: 0.95, 3: 0.95}, 0)])
def test_line_search_depth_is_the_smallest_without_accuracy_loss(acc, want):
    assert bench.choose_ls_depth(acc) == want


def test_line_search_depth_slack():
    # within the slack of the deepest counts as no loss; just beyond it does not
    assert bench.choose_ls_depth({0: 0.95 - bench.LS_SLACK, 1: 0.5, 2: 0.5, 3: 0.95}) == 0
    assert bench.choose_ls_depth({0: 0.95 - 2 * bench.LS_SLACK, 1: 0.5, 2: 0.5, 3: 0.95}) == 3
