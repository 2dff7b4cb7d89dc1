"""The kernels' Philox4x32-10 against the oracle's, word for word."""
import numpy as np
import pytest

import oracle
from paper_2607_03987_gb300 import pakr
from paper_2607_03987_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_philox_bit_exact(cuda_lib):
    spec = W.with_sizes(W.problem("di2"), cap=16)
    planner = pakr.Planner(spec)
    rng = np.random.Generator(np.random.Philox(1))
    ctr = rng.integers(0, 2**32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    for key in ([0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [0xA4093822, 0x299F31D0], [12345, 678]):
        got = planner.philox(ctr, key)
        want = np.array([oracle.philox4x32_10(c, key) for c in ctr[:512]], dtype=np.uint32)
        assert np.array_equal(got[:512], want)
    planner.close()
