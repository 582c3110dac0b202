"""Host logic without a GPU: the two sizes a scene's next render learns from
the sweep statistics of its previous one (ar_debug_learned_prefix,
ar_debug_learned_window), against their cost model worked by hand.

The depth prefix of the first binning phase keeps each cell's first
2^-shift of its sorted events.  Its cost, in sorted entries, is the prefix's
entries, plus the full lists of the segments that stopped past the prefix
(their lengths scaled from the earlier render), plus the events of the
second phase if there is one, plus 12000 entries per restarted segment; the
shift is the cheapest of 0..6."""
import os
import shutil

import numpy as np
import pytest

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def ar():
    from paper_2503_00308_gb300 import _build, ar
    _build.build()
    return ar


def _hist(stops):
    """64-bucket weights and counts from {bucket: (summed length, segments)}."""
    w = np.zeros(64, np.uint64)
    c = np.zeros(64, np.uint32)
    for b, (length, n) in stops.items():
        w[b], c[b] = length, n
    return w, c


def test_prefix_empty_statistics_give_the_default(ar):
    assert ar.ar_debug_learned_prefix(*_hist({}), 10**6, 10**5) == 3


def test_prefix_early_stops_take_the_shortest_prefix(ar):
    # every segment stops in the first 1/64 of its cell's events: no shift
    # leaves one past its prefix, and the cost n_entries 2^-shift falls to 6
    assert ar.ar_debug_learned_prefix(*_hist({0: (10**6, 500)}), 10**6, 10**5) == 6


def test_prefix_late_stops_take_one_phase(ar):
    # every segment runs to the last bucket: any prefix re-sorts all of it and
    # pays the second phase and the restarts, so one phase (0) is cheapest
    assert ar.ar_debug_learned_prefix(*_hist({63: (10**6, 500)}), 10**6, 10**5) == 0
    # bucket 40 lies past every prefix too (64 >> 1 = 32 <= 40)
    assert ar.ar_debug_learned_prefix(*_hist({40: (10**6, 10)}), 10**6, 10**5) == 0


def test_prefix_cost_by_hand(ar):
    n_ent, n_ev = 10**6, 10**5
    # stops in bucket 20: shift 1 keeps buckets < 32, cost 5e5; shift 2 keeps
    # < 16 and pays 2.5e5 + 1e6 + 1e5 + 12000 * 10 = 1.47e6; so 1
    assert ar.ar_debug_learned_prefix(*_hist({20: (10**6, 10)}), n_ent, n_ev) == 1
    # most weight in bucket 5, one long segment in bucket 50 (weights sum to
    # tot = 1001000, scale = n_ent / tot):
    #   shift 3 (keeps < 8): 1.25e5 + 1000 scale + 1e5 + 12000 scale = 2.38e5
    #   shift 4 (keeps < 4): bucket 5 passes too: 6.25e4 + 1e6 + 1e5 + 1.2e7
    #   shifts 1, 2: 5e5 and 2.5e5 plus the same 1.13e5 as shift 3
    assert ar.ar_debug_learned_prefix(*_hist({5: (10**6, 1000), 50: (1000, 1)}), n_ent, n_ev) == 3
    # the restart term decides: 2000 short segments in bucket 12 and the rest
    # early; shift 3 (keeps < 8) restarts 2000 x 12000 = 2.4e7 entries, shift 2
    # (keeps < 16) restarts none: 2.5e5 against 1.25e5 + 2.4e7 + ...
    assert ar.ar_debug_learned_prefix(*_hist({1: (10**6, 100), 12: (2000, 2000)}), n_ent, n_ev) == 2


def test_prefix_scales_lengths_to_the_coming_render(ar):
    # the same stop pattern at ten times the entries: the choice does not move
    w, c = _hist({5: (10**6, 1000), 50: (1000, 1)})
    assert ar.ar_debug_learned_prefix(w, c, 10**7, 10**6) == ar.ar_debug_learned_prefix(w, c, 10**6, 10**5)


def test_window_by_hand(ar):
    h = np.zeros(256, np.uint32)
    assert ar.ar_debug_learned_window(h) == 512       # no statistics
    h[0] = 1000
    assert ar.ar_debug_learned_window(h) == 128       # 32 x 2 = 64, clamped up
    h[:] = 0
    h[10] = 1000
    assert ar.ar_debug_learned_window(h) == 384       # (10 + 2) x 32
    h[200] = 4                                        # 0.4 % of the segments: beyond the 99.5th percentile
    assert ar.ar_debug_learned_window(h) == 384
    h[200] = 6                                        # 0.6 %: the percentile moves there
    assert ar.ar_debug_learned_window(h) == 4096      # (200 + 2) x 32 = 6464, clamped down
    h[:] = 0
    h[255] = 7
    assert ar.ar_debug_learned_window(h) == 4096


def test_learner_arguments_refused(ar):
    with pytest.raises(ValueError):
        ar.ar_debug_learned_prefix(np.zeros(63), np.zeros(64), 1, 1)
    with pytest.raises(ValueError):
        ar.ar_debug_learned_window(np.zeros(255))
    with pytest.raises(ar.ArError) as e:
        ar.check(ar.lib().ar_debug_learned_window(None, None))
    assert e.value.code == ar.AR_EINVAL
