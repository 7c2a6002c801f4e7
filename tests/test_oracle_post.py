"""Pins of the post-processing oracle (Eqs. 8-10 and the depth reductions)."""
import numpy as np

from oracle import post


def test_coherence_bounds_and_limits():
    rng = np.random.default_rng(0)
    f = rng.standard_normal((5, 7, 9)) + 1j * rng.standard_normal((5, 7, 9))
    c = post.coherence(f)
    assert np.all(c >= 0) and np.all(c < 1)                  # 0 <= C < 1 (eps > 0)
    same = np.repeat(f[:1], 4, axis=0)                       # identical phases
    assert np.all(post.coherence(same) > 1 - 1e-5)
    cancel = np.stack([f[0], -f[0]])                         # opposite phases cancel
    assert np.all(post.coherence(cancel) < 1e-12)
    m = post.coherent_merge(same)
    np.testing.assert_allclose(m, np.abs(f[0]) * post.coherence(same), rtol=1e-12)


def test_moe_limits():
    rng = np.random.default_rng(1)
    a = rng.random((6, 5)) + 0.1
    b = rng.random((6, 5)) + 0.1
    p = post.moe_mix(a, b, beta=1.0, eps=0.0)
    q = (a / a.max()) * (b / b.max())
    np.testing.assert_allclose(p, q / q.max(), rtol=1e-12)
    np.testing.assert_allclose(post.moe_mix(a, b, beta=0.0), a / a.max(), rtol=1e-12)


def test_dda_identity_and_fixed_point():
    rng = np.random.default_rng(2)
    v = rng.random((3, 4, 10))
    np.testing.assert_allclose(post.dda(v[None]), v)          # N_w = 1
    const = np.repeat(v[None], 4, axis=0)
    np.testing.assert_allclose(post.dda(const), v)            # constant sequence
    assert list(post.dda_counts(8, 4)) == [1, 1, 2, 2, 3, 3, 4, 4]


def test_max_image():
    v = np.zeros((2, 3, 5))
    v[1, 2, 3] = 7.0
    img = post.max_image(v)
    assert img.shape == (2, 3) and img[1, 2] == 7.0 and img.sum() == 7.0


def test_dda_hand_computed_case():
    """Three frames (newest first) of four depth planes. With N_w = 3 and
    n_z = 4 the reading N(z) = min(N_w, 1 + floor(N_w z / n_z)) gives
    N = 1, 1, 2, 3, so plane 0 and 1 keep the newest frame, plane 2 averages
    the newest two and plane 3 all three (values worked out by hand)."""
    frames = np.array([[1.0, 2.0, 3.0, 4.0],
                       [10.0, 20.0, 30.0, 40.0],
                       [100.0, 200.0, 300.0, 400.0]])
    np.testing.assert_array_equal(post.dda_counts(4, 3), [1, 1, 2, 3])
    np.testing.assert_allclose(post.dda(frames), [1.0, 2.0, 16.5, 148.0], rtol=1e-15)
    # a lateral axis between frames and depth: every pixel follows the same counts
    stacked = np.stack([frames, 2 * frames], axis=1)          # [N_w][2][n_z]
    np.testing.assert_allclose(post.dda(stacked), [[1.0, 2.0, 16.5, 148.0], [2.0, 4.0, 33.0, 296.0]],
                               rtol=1e-15)
