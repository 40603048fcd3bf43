"""The learning-rate rules (camera-spacing heuristic of Sec. 4.2, cosine schedule
of Supp. C): the FP64 oracle against closed forms, then the library's host
implementation (C ABI, no GPU needed) against the oracle."""
import math

import numpy as np
import pytest

from oracle import schedule as osch


# ---------------------------------------------------------------------------
# Oracle pins
# ---------------------------------------------------------------------------

def test_knn_distance_on_a_line():
    """Ten cameras 1 apart on a line, k = 3: the end cameras' three nearest are at
    1, 2, 3 (mean 2), the second ones' at 1, 1, 2 (mean 4/3), every interior one's at
    1, 1, 2 (mean 4/3): d_knn = (2 * 2 + 8 * 4/3) / 10."""
    c = np.stack([np.arange(10.0), np.zeros(10), np.zeros(10)], axis=1)
    assert osch.knn_camera_distance(c, 3) == pytest.approx((4.0 + 8 * 4.0 / 3.0) / 10.0, rel=1e-15)


def test_knn_distance_on_a_ring():
    """n cameras on a circle of radius r: the neighbours are the two at chord
    2 r sin(pi/n) and one of the two at 2 r sin(2 pi/n)."""
    n, r = 12, 2.5
    a = 2 * np.pi * np.arange(n) / n
    c = np.stack([r * np.cos(a), r * np.sin(a), np.full(n, 0.7)], axis=1)
    want = (2 * 2 * r * math.sin(math.pi / n) + 2 * r * math.sin(2 * math.pi / n)) / 3
    assert osch.knn_camera_distance(c, 3) == pytest.approx(want, rel=1e-13)


def test_knn_uses_all_cameras_when_fewer_than_k():
    c = np.array([[0.0, 0, 0], [3.0, 0, 0], [0.0, 4, 0]])  # a 3-4-5 triangle
    assert osch.knn_camera_distance(c, 3) == pytest.approx(((3 + 4) / 2 + (3 + 5) / 2 + (4 + 5) / 2) / 3, rel=1e-15)


def test_heuristic_scaling_laws():
    """Scaling the capture by s scales d_knn by s, eta_f by s^-beta and eta_sigma
    by s^gamma; at d_knn = d_ref the base rates come back."""
    rng = np.random.default_rng(3)
    c = rng.normal(size=(40, 3))
    ef, es, d = osch.lr_heuristic(c, 1.0, 2.5e-3, 5e-2)
    assert osch.lr_heuristic(c, d, 2.5e-3, 5e-2)[:2] == pytest.approx((2.5e-3, 5e-2), rel=1e-14)
    ef2, es2, d2 = osch.lr_heuristic(3.0 * c, 1.0, 2.5e-3, 5e-2)
    assert d2 == pytest.approx(3 * d, rel=1e-14)
    assert ef2 == pytest.approx(ef / 9, rel=1e-13)
    assert es2 == pytest.approx(es * 3 ** 0.6, rel=1e-13)


def test_cosine_schedule_shape():
    assert osch.cosine_factor(0, 100) == 1.0
    assert osch.cosine_factor(50, 100) == pytest.approx(0.5, abs=1e-15)
    assert osch.cosine_factor(100, 100) == 0.0
    assert osch.cosine_factor(5000, 30000, 7000) == 1.0
    assert osch.cosine_factor(7000, 30000, 7000) == 1.0
    assert osch.cosine_factor(18500, 30000, 7000) == pytest.approx(0.5, abs=1e-15)
    f = [osch.cosine_factor(t, 30000, 7000) for t in range(7000, 30001, 100)]
    assert all(b <= a for a, b in zip(f, f[1:]))


# ---------------------------------------------------------------------------
# Library (host functions of the C ABI) against the oracle
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def nb():
    from paper_2606_09794_gb300 import build as b
    b.build()
    from paper_2606_09794_gb300 import binding
    return binding


@pytest.mark.parametrize("n,k", [(2, 3), (3, 3), (8, 3), (57, 3), (200, 5), (31, 1)])
def test_library_heuristic_matches_oracle(nb, n, k):
    rng = np.random.default_rng(n * 7 + k)
    c = (rng.normal(size=(n, 3)) * rng.uniform(0.1, 10.0)).astype(np.float32)
    got = nb.nasg_lr_heuristic(c, 0.8, 1e-3, 0.05, k=k)
    ref = osch.lr_heuristic(c.astype(np.float64), 0.8, 1e-3, 0.05, k=k)
    np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_library_heuristic_rejects_bad_input(nb):
    with pytest.raises(nb.NasgError):
        nb.nasg_lr_heuristic(np.zeros((1, 3)), 1.0, 1e-3, 0.05)
    with pytest.raises(nb.NasgError):
        nb.nasg_lr_heuristic(np.zeros((4, 3)), 1.0, 1e-3, 0.05)  # all cameras at one point
    with pytest.raises(nb.NasgError):
        nb.nasg_lr_heuristic(np.eye(3), 0.0, 1e-3, 0.05)


@pytest.mark.parametrize("t0,tmax", [(0, 100), (7000, 30000), (10, 11), (5, 5)])
def test_library_cosine_matches_oracle(nb, t0, tmax):
    for t in range(max(0, t0 - 3), tmax + 3):
        assert nb.nasg_cosine_lr_factor(t, tmax, t0) == pytest.approx(osch.cosine_factor(t, tmax, t0), abs=1e-15)
