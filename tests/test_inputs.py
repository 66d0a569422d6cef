"""The seeded generators: determinism, shapes and the minimum distance."""
import numpy as np

from paper_1105_2769_gb300 import inputs


def test_uniform_min_distance_and_determinism():
    a = inputs.uniform_cube(2000, 8.0, 0.5, 5)
    b = inputs.uniform_cube(2000, 8.0, 0.5, 5)
    assert a.shape == (2000, 3)
    assert np.array_equal(a, b)
    assert a.min() >= 0.0 and a.max() <= 8.0
    assert inputs.min_pair_distance(a) >= 0.5


def test_named_small_workload():
    X = inputs.workload("exh64_n512")
    assert X.shape == (512, 3)
    assert inputs.min_pair_distance(X) >= 0.01


def test_gmm_small():
    X, st = inputs.gaussian_mixture(4096, 8, 10.0, 0.5, 3.0, 0.05, 9, return_stats=True)
    assert X.shape == (4096, 3)
    assert inputs.min_pair_distance(X) >= 0.05
    assert st["centres"].shape == (8, 3)


def test_ball_and_shell():
    B = inputs.unit_ball(1000, 0.01, 3)
    assert np.linalg.norm(B, axis=1).max() <= 1.0
    S = inputs.spherical_shell(1000, 0.9, 1.0, 0.01, 4)
    r = np.linalg.norm(S, axis=1)
    assert r.min() >= 0.9 - 1e-12 and r.max() <= 1.0 + 1e-12


def test_sample_indices():
    idx = inputs.sample_indices(100, 10, 1)
    assert len(np.unique(idx)) == 10 and idx.max() < 100
