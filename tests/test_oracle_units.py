"""Hand-worked cases for the oracle's building blocks, each one call into the
oracle: the Moller-Trumbore ray/triangle test (interior, edge, vertex, back
face, parallel, behind the origin), point and direction mirroring (the
image-source step of Section 2), the reflected cone, and the
microphone-in-beam test with its start and end planes."""
import numpy as np
import pytest

A, B, Cv = (0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0)  # unit right triangle in z = 0


@pytest.mark.parametrize("xy,hit", [((0.25, 0.25), True), ((0.5, 0.0), True), ((0.0, 0.5), True),
                                    ((0.5, 0.5), True), ((0.0, 0.0), True), ((1.0, 0.0), True),
                                    ((0.6, 0.6), False), ((-0.01, 0.5), False), ((0.5, -0.01), False),
                                    ((1.01, 0.0), False)])
def test_ray_tri_interior_edges_vertices(oracle_mod, xy, hit):
    # edges and vertices count as inside (inclusive barycentric bounds)
    t = oracle_mod.ray_tri((xy[0], xy[1], 2.0), (0, 0, -1), A, B, Cv)
    assert (t is not None) == hit
    if hit:
        assert t == pytest.approx(2.0, abs=1e-15)


def test_ray_tri_two_sided_and_signed_t(oracle_mod):
    assert oracle_mod.ray_tri((0.2, 0.2, -3.0), (0, 0, 1), A, B, Cv) == pytest.approx(3.0)  # back face
    assert oracle_mod.ray_tri((0.2, 0.2, 1.0), (0, 0, 1), A, B, Cv) == pytest.approx(-1.0)  # behind: t < 0
    # the distance along an oblique unit ray
    d = np.array([1.0, 1.0, -2.0]) / np.sqrt(6.0)
    t = oracle_mod.ray_tri((0.0, 0.0, 1.0), d, A, B, Cv)
    assert t == pytest.approx(np.sqrt(6.0) / 2.0, rel=1e-14)
    # a ray parallel to the plane (above it or in it) never hits
    assert oracle_mod.ray_tri((0.2, 0.2, 1.0), (1, 0, 0), A, B, Cv) is None
    assert oracle_mod.ray_tri((-1.0, 0.2, 0.0), (1, 0, 0), A, B, Cv) is None


def test_mirror_point_hand_cases(oracle_mod):
    assert np.allclose(oracle_mod.mirror_point((1, 2, 3), (5, 5, 0), (0, 0, 1)), (1, 2, -3))
    assert np.allclose(oracle_mod.mirror_point((1, 2, 3), (2, 0, 0), (1, 0, 0)), (3, 2, 3))
    n = np.array([1.0, 1.0, 0.0]) / np.sqrt(2.0)
    assert np.allclose(oracle_mod.mirror_point((1, 0, 0), (0, 0, 0), n), (0, -1, 0))
    assert np.allclose(oracle_mod.mirror_point((2, 0, 5), (1, 1, 0), n), (2, 0, 5))  # a point in the plane stays
    assert np.allclose(oracle_mod.mirror_dir(np.array([1.0, 0.0, -1.0]) / np.sqrt(2), (0, 0, 1)),
                       np.array([1.0, 0.0, 1.0]) / np.sqrt(2))


def test_mirror_is_an_isometry_and_an_involution(oracle_mod):
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        p, a, q = rng.normal(size=(3, 3)) * 10.0
        q = q - np.dot(q - p, n) * n  # q in the plane
        m = oracle_mod.mirror_point(a, p, n)
        assert np.allclose(oracle_mod.mirror_point(m, p, n), a, atol=1e-12)
        assert np.dot(m - p, n) == pytest.approx(-np.dot(a - p, n), abs=1e-12)
        assert np.linalg.norm(m - q) == pytest.approx(np.linalg.norm(a - q), rel=1e-12)
        d = rng.normal(size=3)
        assert np.allclose(oracle_mod.mirror_dir(oracle_mod.mirror_dir(d, n), n), d, atol=1e-12)


def _octant():
    return np.eye(3)  # edges +x, +y, +z: counter-clockwise seen from outside the first octant


def test_in_segment_cone_faces(oracle_mod):
    apex = (0.0, 0.0, 0.0)
    assert oracle_mod.in_segment(apex, _octant(), (1, 2, 3)) == (True, False)
    assert oracle_mod.in_segment(apex, _octant(), (1, 2, -0.01))[0] is False
    assert oracle_mod.in_segment(apex, _octant(), (-0.01, 2, 3))[0] is False
    # on a face: inside (inclusive) and flagged as a tie
    assert oracle_mod.in_segment(apex, _octant(), (1, 0, 3)) == (True, True)
    # the same edges in the other order describe the complementary cone's
    # faces: the octant is then outside
    assert oracle_mod.in_segment(apex, _octant()[[0, 2, 1]], (1, 2, 3))[0] is False


def test_in_segment_start_and_end_planes(oracle_mod):
    apex = (0.0, 0.0, 0.0)
    n = np.ones(3) / np.sqrt(3.0)
    start = (n, (1.0, 0.0, 0.0))   # beam side: x + y + z > 1, strictly
    end = (-n, (3.0, 0.0, 0.0))    # incident side: x + y + z <= 3, inclusive
    inside = lambda m: oracle_mod.in_segment(apex, _octant(), m, start=start, end=end)[0]
    assert inside((0.5, 0.5, 0.5))
    assert not inside((0.2, 0.2, 0.2))        # before the start plane
    assert not inside((0.0, 0.0, 1.0))        # on the start plane: outside (strict)
    assert inside((1.0, 1.0, 1.0))            # on the end plane: inside
    assert not inside((1.0, 1.0, 1.01))       # beyond the end plane
    assert inside((0.0, 0.0, 2.0))            # on two cone faces, between the planes


def test_reflected_cone_keeps_membership_and_orientation(oracle_mod):
    # a point inside the original cone, mirrored, lies inside the reflected
    # cone; the reflected edges stay counter-clockwise (the mirrored axis is
    # inside), which a dropped edge reversal would break
    rng = np.random.default_rng(5)
    dirs = np.array([[1.0, 0.1, -0.2], [0.2, 0.2, -1.0], [0.1, 1.0, -0.3]])
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    apex = np.array([3.0, -2.0, 10.0])
    assert oracle_mod.in_segment(apex, dirs, apex + dirs.sum(0))[0]  # counter-clockwise from outside
    for _ in range(10):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        p = rng.normal(size=3) * 5.0
        a2, d2 = oracle_mod.reflect_cone(apex, dirs, p, n)
        assert np.allclose(a2, oracle_mod.mirror_point(apex, p, n))
        for j in range(3):
            assert any(np.allclose(d2[k], oracle_mod.mirror_dir(dirs[j], n)) for k in range(3))
        axis2 = oracle_mod.mirror_dir(dirs.sum(0), n)
        assert oracle_mod.in_segment(a2, d2, a2 + axis2)[0]
        w = rng.dirichlet(np.ones(3), size=20)
        for m in apex + (w @ dirs) * rng.uniform(0.5, 30.0, size=(20, 1)):
            assert oracle_mod.in_segment(apex, dirs, m)[0]
            assert oracle_mod.in_segment(a2, d2, oracle_mod.mirror_point(m, p, n))[0]
