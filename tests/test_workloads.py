"""Input generators of the learned-model workload (no method arithmetic): the
stream-function face velocities are discretely divergence-free and normalised, the
cell-centre velocity is the mean of each cell's faces, the bumps are periodic."""
import numpy as np

from workloads import gen


def test_stream_function_faces_divergence_free_and_normalised():
    rng = np.random.default_rng(3)
    ax, ay = gen.stream_function_faces(64, rng)
    div = (ax.astype(np.float64) - np.roll(ax, 1, axis=0)) + (ay.astype(np.float64) - np.roll(ay, 1, axis=1))
    assert np.abs(div).max() < 1e-5
    assert abs(max(np.abs(ax).max(), np.abs(ay).max()) - 1.0) < 1e-6
    v = gen.cell_velocity(ax, ay).reshape(64, 64, 2)
    assert np.allclose(v[3, 5, 0], 0.5 * (ax[3, 5] + ax[2, 5]))
    assert np.allclose(v[3, 5, 1], 0.5 * (ay[3, 5] + ay[3, 4]))


def test_periodic_bumps_wrap_around():
    u = gen.periodic_bumps_2d(64, np.random.default_rng(4))
    # a field of periodic bumps is smooth across the boundary: the jump between the
    # last and first rows is like any other neighbour difference
    d_inner = np.abs(np.diff(u, axis=0)).max()
    d_wrap = np.abs(u[0] - u[-1]).max()
    assert d_wrap <= 1.5 * d_inner
    X = gen.cell_centers_2d(4)
    assert np.allclose(X[:4, 1], [0.125, 0.375, 0.625, 0.875]) and np.allclose(X[::4, 0], X[:4, 1])
