"""The library's receiver sampler (host code behind the C ABI) against the oracle's, bit for
bit; runs without a GPU."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("nrec,nsub,seed,it", [(231, 100, 0, 0), (231, 100, 7, 3), (273, 100, 2**63 + 5, 11),
                                               (12, 12, 1, 0), (5, 1, 99, 2**40), (1000, 25, 123, 7)])
def test_sampler_matches_oracle(nrec, nsub, seed, it):
    from paper_2512_16642_gb300 import egh

    got = egh.sample_receivers(nrec, nsub, seed, it)
    assert np.array_equal(got, oracle.sample_receivers(nrec, nsub, seed, it))


def test_sampler_rejects_bad_sizes():
    from paper_2512_16642_gb300 import egh

    for nrec, nsub in ((10, 0), (10, 11), (0, 1)):
        with pytest.raises(egh.EghError):
            egh.sample_receivers(nrec, nsub, 1, 0)
