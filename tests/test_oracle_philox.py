"""Pins for oracle/philox.py against numpy's independent Philox4x64-10."""
import numpy as np
import pytest

from oracle import philox


CASES = [((1, 0, 0, 0), (0, 0)), ((1, 0, 0, 0), (123, 456)), ((6, 7, 0, 0), (0, 0)),
         ((6, 7, 0, 0), (2**63 + 5, 99)), ((12345, 3, 9, 1), (7, 2**64 - 1)),
         ((2**40 + 1, 2**33, 17, 2**62), (1, 2))]


@pytest.mark.parametrize("ctr,key", CASES)
def test_scalar_matches_numpy(ctr, key):
    # numpy's random_raw() increments the counter before each block
    prev = list(ctr)
    prev[0] -= 1
    g = np.random.Philox(counter=np.array(prev, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    raw = [int(x) for x in g.random_raw(4)]
    assert philox.philox4x64_10_scalar(ctr, key) == raw


def test_vectorised_matches_scalar():
    rng = np.random.default_rng(0)
    c = rng.integers(0, 2**63, size=(4, 64), dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    k = rng.integers(0, 2**63, size=(2, 64), dtype=np.uint64)
    out = philox.philox4x64_10(c[0], c[1], c[2], c[3], k[0], k[1])
    for j in range(64):
        ref = philox.philox4x64_10_scalar([int(c[i, j]) for i in range(4)], [int(k[0, j]), int(k[1, j])])
        assert [int(o[j]) for o in out] == ref


def test_uniforms_open_interval_and_mean():
    u = philox.uniforms(np.arange(200000, dtype=np.uint64), 3, 11, 0)
    assert u.min() > 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3
    # different blocks / problems give different streams
    u2 = philox.uniforms(np.arange(1000, dtype=np.uint64), 4, 11, 0)
    u3 = philox.uniforms(np.arange(1000, dtype=np.uint64), 3, 11, 1)
    assert not np.allclose(u[:1000], u2) and not np.allclose(u[:1000], u3)


def test_uniform_formula_matches_word():
    # u = ((w0 >> 11) + 0.5) * 2^-53 for row 5, block 2, seed 9, problem 4
    w = philox.philox4x64_10_scalar((5, 2, 0, 0), (9, 4))
    expect = ((w[0] >> 11) + 0.5) / 2.0**53
    assert philox.uniforms(np.array([5], dtype=np.uint64), 2, 9, 4)[0] == expect
