"""The seeded input generators (host logic, no GPU): the serving stream's
Poisson arrivals and parameter ranges, Haar rotations, jitter, and the
adjoint configuration's meshes."""
import numpy as np
import pytest

import synth


def test_serve_stream_statistics():
    qs = synth.serve_stream(n_queries=4000, rate=500.0, seed=3, build_meshes=False)
    t = np.array([q.arrival_s for q in qs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential inter-arrivals, mean 1/rate: standard error of the mean is (1/rate)/sqrt(n)
    assert abs(gaps.mean() - 1 / 500.0) < 4 * (1 / 500.0) / np.sqrt(len(gaps))
    assert abs(np.median(gaps) - np.log(2) / 500.0) < 0.1 * np.log(2) / 500.0
    ns = np.array([q.n for q in qs])
    assert ns.min() == 2 and ns.max() == 48
    assert set(q.s for q in qs) == {1.0, 2.0} and set(q.R for q in qs) == {64.0, 128.0}
    again = synth.serve_stream(n_queries=50, rate=500.0, seed=3, build_meshes=False)
    assert [q.arrival_s for q in again] == [q.arrival_s for q in qs[:50]]  # seeded


def test_serve_stream_meshes_are_rotated_and_jittered():
    qs = synth.serve_stream(n_queries=6, rate=500.0, seed=5)
    for q in qs:
        assert q.tris.shape == (20 * q.n * q.n, 3)
        r = np.linalg.norm(q.verts, axis=1)
        h = synth.mean_edge_length(q.verts, q.tris)
        assert np.abs(r - 1.0).max() < 10e-3 * h  # jitter sigma = 1e-3 h
        assert np.abs(r - 1.0).max() > 0.0


@pytest.mark.parametrize("seed", [0, 1, 12345])
def test_haar_rotation_is_a_proper_rotation(seed):
    Q = synth.haar_rotation(seed)
    assert np.allclose(Q @ Q.T, np.eye(3), atol=1e-14)
    assert np.linalg.det(Q) == pytest.approx(1.0, abs=1e-14)
    assert not np.allclose(Q, synth.haar_rotation(seed + 1))


def test_haar_rotations_are_uniform_in_the_mean():
    # E[Q] = 0 for the Haar measure on SO(3)
    Qs = np.array([synth.haar_rotation(s) for s in range(3000)])
    assert np.abs(Qs.mean(axis=0)).max() < 0.05


def test_jitter_is_seeded_and_of_the_stated_size():
    v, _ = synth.icosphere(8)
    a = synth.jitter_isotropic(v, 0.01, 4)
    b = synth.jitter_isotropic(v, 0.01, 4)
    c = synth.jitter_isotropic(v, 0.01, 5)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    d = (a - v).ravel()
    assert abs(d.std() - 0.01) < 0.1 * 0.01 and abs(d.mean()) < 0.1 * 0.01
    r = synth.jitter_radial(v, 1e-4, 7)
    ratio = np.linalg.norm(r, axis=1) / np.linalg.norm(v, axis=1)
    assert np.allclose(np.cross(r, v), 0.0, atol=1e-12)  # radial only
    assert abs((ratio - 1).std() - 1e-4) < 0.1 * 1e-4


def test_adjoint_meshes():
    v0, t0 = synth.adjoint_mesh(16, 0)
    v1, t1 = synth.adjoint_mesh(16, 1)
    vu, tu = synth.icosphere(16)
    assert t0.shape == (5120, 3) and np.array_equal(t0, t1) and np.array_equal(t0, tu)
    assert not np.array_equal(v0, v1)
    assert abs((v0 - vu).std() - synth.ADJOINT_SIGMA) < 0.1 * synth.ADJOINT_SIGMA
