"""Host logic without a GPU: the pieces of ar_render_abstract_partitioned
(ar_partition_piece) are bit-identical to the oracle's partition_cells, which
states the same formula independently, and bad arguments are refused."""
import shutil
import os

import numpy as np
import pytest

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


def test_pieces_match_the_oracle(orc):
    from paper_2503_00308_gb300 import _build, ar
    _build.build()
    rng = np.random.default_rng(41)
    for trial in range(30):
        lo = rng.uniform(-0.1, 0.05, 6)
        hi = lo + rng.uniform(0.0, 0.1, 6) * (rng.uniform(size=6) < 0.8)
        parts = [int(p) if hi[k] > lo[k] else 1 for k, p in enumerate(rng.integers(1, 5, 6))]
        box = ar.make_cells(lo, hi)[0]
        olo, ohi = orc.partition_cells(lo, hi, parts)
        for i in range(olo.shape[0]):
            plo, phi = ar.ar_partition_piece(box, parts, i)
            assert np.array_equal(plo, olo[i]) and np.array_equal(phi, ohi[i]), (trial, i)


def test_piece_arguments_refused():
    from paper_2503_00308_gb300 import _build, ar
    _build.build()
    box = ar.make_cells(np.zeros(6), np.full(6, 0.01))[0]
    for parts, index in [([2, 1, 1, 1, 1, 1], 2), ([2, 1, 1, 1, 1, 1], -1), ([0, 1, 1, 1, 1, 1], 0),
                         ([4096, 4096, 2, 1, 1, 1], 0)]:
        with pytest.raises(ar.ArError) as e:
            ar.ar_partition_piece(box, parts, index)
        assert e.value.code == ar.AR_EINVAL
