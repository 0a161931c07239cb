"""Host-side logic of the M-TIP driver and the bindings, without a GPU: the
Morton renumbering of the orientation set is a permutation that keeps
neighbours close on SO(3), and the count-image binding rejects what the C
ABI cannot take."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def pkg():
    from paper_2109_05339_gb300 import build
    build.build()
    import paper_2109_05339_gb300 as p
    return p


def test_morton_order_is_a_locality_preserving_permutation(pkg):
    from paper_2109_05339_gb300.mtip import morton_order
    rng = np.random.default_rng(3)
    q = rng.standard_normal((5000, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1
    order = morton_order(q)
    np.testing.assert_array_equal(np.sort(order), np.arange(q.shape[0]))
    # 1 - |q1 . q2| grows with the rotation angle between q1 and q2
    qs = q[order]
    along = np.mean(1.0 - np.abs(np.sum(qs[1:] * qs[:-1], axis=1)))
    given = np.mean(1.0 - np.abs(np.sum(q[1:] * q[:-1], axis=1)))
    assert along < 0.2 * given


def test_counts_binding_rejects_wrong_inputs(pkg):
    import torch
    with pytest.raises(TypeError):
        pkg.counts_to_f32(torch.zeros(8, dtype=torch.float32))
    with pytest.raises(ValueError):
        pkg.counts_to_f32(torch.zeros(8, dtype=torch.int16))   # host tensor


def test_driver_binding_rejects_an_unknown_point_mode(pkg):
    with pytest.raises(ValueError):
        pkg.MTIP(17, 1.0, 256, 10, 100, cache_points="kept")


def test_lcurve_corner_matches_the_oracle(pkg):
    """The library's L-curve corner (host arithmetic behind the C ABI) picks
    the oracle's maximum-curvature point on uneven lambda grids, and its
    curvature values agree with the oracle's formula."""
    from oracle import lcurve as olc
    from paper_2109_05339_gb300.lcurve import corner
    rng = np.random.default_rng(11)
    for trial in range(20):
        n = int(rng.integers(3, 15))
        lams = np.sort(rng.uniform(-4, 2, n))
        lams = 10.0 ** np.unique(lams)
        if lams.shape[0] < 3:
            continue
        t = np.log(lams)
        res2 = np.exp(2 * (0.3 * t + 0.2 * np.tanh(t) + 0.05 * rng.standard_normal(t.shape[0])))
        reg2 = np.exp(2 * (-0.8 * t - 0.3 * np.tanh(2 * t)))
        idx, kappa = corner(lams, res2, reg2)
        assert idx == olc.corner(lams, res2, reg2)
        np.testing.assert_allclose(kappa, olc.curvature(lams, res2, reg2), rtol=1e-10, atol=1e-12)

