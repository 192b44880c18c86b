"""Pins for the shared seeded input generator (no contraction arithmetic lives there)."""
import numpy as np

import tamm_synth as S


def test_philox4x32_10_known_answers():
    # Known-answer vectors published with the Random123 library (Salmon et al., SC'11).
    assert S.philox4x32_10([0, 0, 0, 0], [0, 0]) == (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)
    assert S.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)
    assert S.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0]) == (
        0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)


def test_normal_moments():
    n = 200_000
    out = np.zeros(n)
    S.fill_boxes(7, 3, 1.0, [n], False, False, [[0]], [[n]], [0], out)
    assert abs(out.mean()) < 5 * (1 / np.sqrt(n))
    assert abs(out.var() - 1.0) < 0.02
    # fourth moment of a normal is 3
    assert abs((out ** 4).mean() - 3.0) < 0.1


def test_counter_based_boxes_agree():
    dims = [6, 6, 5, 5]
    full = np.zeros(int(np.prod(dims)))
    S.fill_boxes(11, 2, 0.1, dims, True, True, [[0, 0, 0, 0]], [dims], [0], full)
    full = full.reshape(dims)
    part = np.zeros(3 * 2 * 4 * 1)
    S.fill_boxes(11, 2, 0.1, dims, True, True, [[2, 1, 1, 3]], [[3, 2, 4, 1]], [0], part)
    assert np.array_equal(part.reshape(3, 2, 4, 1), full[2:5, 1:3, 1:5, 3:4])


def test_antisymmetry_exact_and_diagonal_zero():
    dims = [7, 7, 6, 6]
    x = np.zeros(int(np.prod(dims)))
    S.fill_boxes(5, 1, 0.1, dims, True, True, [[0] * 4], [dims], [0], x)
    x = x.reshape(dims)
    assert np.array_equal(x, -x.transpose(1, 0, 2, 3))
    assert np.array_equal(x, -x.transpose(0, 1, 3, 2))
    for p in range(7):
        assert not x[p, p].any()
    # off-diagonal entries keep standard deviation sigma
    off = np.array([x[p, q, r, s] for p in range(7) for q in range(7) for r in range(6) for s in range(6)
                    if p != q and r != s])
    assert 0.08 < off.std() < 0.12
    y = np.zeros(int(np.prod(dims)))
    S.fill_boxes(5, 1, 0.1, dims, True, False, [[0] * 4], [dims], [0], y)
    y = y.reshape(dims)
    assert np.array_equal(y, -y.transpose(1, 0, 2, 3))
    assert not np.array_equal(y, -y.transpose(0, 1, 3, 2))
