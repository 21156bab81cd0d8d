"""The droplet tracker used by the workload tests (host-side, no GPU)."""
import numpy as np

from harness import droplet_centroids


def _tanh_drops(shape, drops, xi=4.0):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz) + .5, np.arange(ny) + .5, np.arange(nx) + .5, indexing="ij")
    phi = np.zeros(shape)
    for cx, cy, cz, R in drops:
        dx = x - cx
        dx -= nx * np.round(dx / nx)
        dy = y - cy
        dy -= ny * np.round(dy / ny)
        r = np.sqrt(dx ** 2 + dy ** 2 + (z - cz) ** 2)
        phi = np.maximum(phi, 0.5 * (1 + np.tanh(2 * (R - r) / xi)))
    return phi


def test_centroids_of_separate_and_wrapped_droplets():
    """Two droplets, one straddling the periodic x face: both centres are
    recovered (sorted by x) to a small fraction of a cell."""
    drops = [(20.3, 17.6, 14.2, 6.0), (1.4, 30.5, 20.0, 7.0)]   # second one wraps in x
    phi = _tanh_drops((40, 48, 64), drops)
    c = droplet_centroids(phi)
    assert c.shape == (2, 3)
    want = np.array(sorted([[d[0], d[1], d[2]] for d in drops]))
    assert np.abs(c - want).max() < 0.05, (c, want)


def test_single_droplet_without_periodic_axes():
    phi = _tanh_drops((30, 30, 30), [(15.2, 14.7, 16.1, 5.0)])
    c = droplet_centroids(phi, periodic_xy=False)
    assert np.abs(c[0] - [15.2, 14.7, 16.1]).max() < 0.05
