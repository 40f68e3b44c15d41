"""Pins of the oracle's Philox4x32-10 generator and its normals (CPU only)."""
import os

import numpy as np
import pytest

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    got = philox.philox4x32_10(np.array(ctr, dtype=np.uint32), np.array(key, dtype=np.uint32))
    assert [int(x) for x in got] == out


def test_counter_layout_is_block_step_chain_stream():
    seed = (7 << 32) | 5
    w = philox.blocks(seed, philox.STREAM_Z, 9, [3, 4], 2)
    for ci, c in enumerate([3, 4]):
        for b in range(2):
            ref = philox.philox4x32_10(np.array([b, 9, c, philox.STREAM_Z], dtype=np.uint32),
                                       np.array([5, 7], dtype=np.uint32))
            assert np.array_equal(w[ci, b], ref)


def test_uniform_mapping_is_open_interval():
    u = philox.word_to_uniform(np.array([0, 0xFFFFFFFF], dtype=np.uint32))
    assert u[0] == 2.0 ** -33
    assert u[1] == 1.0 - 2.0 ** -33
    assert np.all((u > 0) & (u < 1))


def test_box_muller_pairs_match_definition():
    seed = 1234
    w = philox.blocks(seed, philox.STREAM_XI, 0, [0], 1)[0, 0]
    u = (w.astype(np.float64) + 0.5) * 2.0 ** -32
    n = philox.normals(seed, philox.STREAM_XI, 0, [0], 4)[0]
    rad = np.sqrt(-2 * np.log(u[0]))
    assert np.isclose(n[0], rad * np.cos(2 * np.pi * u[1]), rtol=0, atol=1e-15)
    assert np.isclose(n[1], rad * np.sin(2 * np.pi * u[1]), rtol=0, atol=1e-15)


def test_normals_moments():
    z = philox.normals(99, philox.STREAM_Z, 3, np.arange(64), 4096).ravel()
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / n)
    # fourth moment of a standard normal is 3
    assert abs(np.mean(z ** 4) - 3) < 5 * np.sqrt(96 / n)
    # adjacent draws uncorrelated
    assert abs(np.mean(z[:-1] * z[1:])) < 5 / np.sqrt(n)


def test_streams_and_steps_are_distinct():
    a = philox.normals(1, philox.STREAM_XI, 0, [0], 8)
    b = philox.normals(1, philox.STREAM_XI, 1, [0], 8)
    c = philox.normals(1, philox.STREAM_Z, 0, [0], 8)
    d = philox.normals(1, philox.STREAM_XI, 0, [1], 8)
    for x in (b, c, d):
        assert not np.allclose(a, x)
