"""Pins of oracle.matching: plain vs expanded distances, ties, top-k, margin."""
import numpy as np

from oracle import matching


def test_plain_and_expanded_forms_agree():
    rng = np.random.default_rng(0)
    X = rng.poisson(3.0, (20, 64)).astype(float)
    Y = rng.uniform(0, 5, (30, 64))
    d = matching.distances(X, Y)
    # brute force with explicit loops on a corner
    for i in range(3):
        for j in range(4):
            assert abs(d[i, j] - sum((X[i, p] - Y[j, p]) ** 2 for p in range(64))) < 1e-9
    np.testing.assert_allclose(matching.distances_expanded(X, Y), d, rtol=1e-12, atol=1e-9)


def test_ties_go_to_lowest_index_and_topk_order():
    rng = np.random.default_rng(1)
    Y = rng.uniform(0, 1, (10, 16))
    Y[7] = Y[3]
    Y[9] = Y[3]
    X = Y[[3, 5]] + 0.0
    res = matching.match(X, Y, k=4)
    assert res["best"][0] == 3 and res["best"][1] == 5
    assert list(res["topk"][0][:3]) == [3, 7, 9]
    assert res["d1"][0] == 0.0 and res["d2"][0] == 0.0 and res["margin"][0] == 0.0
    d = res["d"][1]
    order = res["topk"][1]
    assert np.all(np.diff(d[order]) >= 0)


def test_margin_definition():
    X = np.array([[1.0, 0.0]])
    Y = np.array([[1.0, 0.5], [0.0, 0.0], [2.0, 0.0]])
    res = matching.match(X, Y, k=2)
    # d = [0.25, 1, 1]; best 0, second 1 (tie with 2 -> lower index)
    assert res["best"][0] == 0 and list(res["topk"][0]) == [0, 1]
    assert abs(res["margin"][0] - (1.0 - 0.25) / (1.0 + 1.25)) < 1e-15
    assert abs(res["margin_alt"][0] - 0.75) < 1e-15


def test_weighted_distance_definition():
    import synth
    rng = np.random.default_rng(3)
    D = synth.beamstop_mask(8, 2.0)
    assert D.shape == (64,) and 0 < D.sum() < 64 and D[27] == 0.0      # centre pixel masked
    X = rng.uniform(0, 3, (5, 64))
    Y = rng.uniform(0, 3, (7, 64))
    d = matching.distances(X, Y, D)
    for i in range(2):
        for j in range(3):
            ref = sum(D[p] * (X[i, p] - Y[j, p]) ** 2 for p in range(64))
            assert abs(d[i, j] - ref) < 1e-10
    # equals the unweighted distance of sqrt(D)-scaled rows, and the expanded form
    s = np.sqrt(D)
    np.testing.assert_allclose(d, matching.distances(X * s, Y * s), rtol=1e-12)
    np.testing.assert_allclose(matching.distances_expanded(X, Y, D), d, rtol=1e-10, atol=1e-10)
    res = matching.match(X, Y, k=3, D=D)
    x2 = np.sum(D * X * X, 1)
    y2 = np.sum(D * Y * Y, 1)
    assert abs(res["margin"][0] - (res["d2"][0] - res["d1"][0]) / (x2[0] + y2[res["best"][0]])) < 1e-15
