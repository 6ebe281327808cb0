"""Pin for the oracle's Philox4x32-10: the published known-answer vectors."""
from golden_io import philox_kat
from oracle import philox


def test_known_answer_vectors():
    for ctr, key, want in philox_kat():
        assert list(philox.philox4x32_10(ctr, key)) == want


def test_uniform_range_and_resolution():
    us = [philox.uniform(12345, s, n) for s in range(50) for n in range(20)]
    assert min(us) >= 0.0 and max(us) < 1.0
    assert len(set(us)) == len(us)
