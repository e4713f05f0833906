"""Seeded input generators: the meshes they draw are valid triangulations of their rectangle
(positive areas, every interior edge shared by exactly two triangles, boundary edges on the
boundary), and the same seed gives the same workload."""
import numpy as np
import pytest

from paper_2307_14302_gb300 import workloads as W


def _check_mesh(m, lx, ly):
    P = m.xy[m.tri]
    area = 0.5 * ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                  - (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1]))
    assert (area > 0).all()
    assert abs(area.sum() - lx * ly) <= 1e-9 * lx * ly
    e = np.sort(np.concatenate([m.tri[:, [0, 1]], m.tri[:, [1, 2]], m.tri[:, [2, 0]]]), axis=1)
    _, counts = np.unique(e, axis=0, return_counts=True)
    assert counts.max() == 2
    assert (counts == 1).sum() == len(m.bedge)
    mid = 0.5 * (m.xy[m.bedge[:, 0]] + m.xy[m.bedge[:, 1]])
    tol = 1e-6 * max(lx, ly)
    on = (mid[:, 0] < tol) | (mid[:, 0] > lx - tol) | (mid[:, 1] < tol) | (mid[:, 1] > ly - tol)
    assert on.all()


@pytest.mark.parametrize("n", [500, 5000])
def test_jittered_grid_mesh_is_a_triangulation(n):
    m = W.jittered_grid_mesh(40_000.0, 30_000.0, n, seed=1)
    _check_mesh(m, 40_000.0, 30_000.0)
    assert abs(m.n_tri - n) < 0.1 * n


def test_graded_strip_mesh_is_graded_and_valid():
    lx, ly = 400_000.0, 300_000.0
    m = W.graded_strip_mesh(lx, ly, 0.78 * lx, 1000.0, 50_000.0, 20_000, seed=3)
    _check_mesh(m, lx, ly)
    assert abs(m.n_tri - 20_000) < 0.05 * 20_000
    c = m.xy[m.tri].mean(axis=1)
    P = m.xy[m.tri]
    L = np.linalg.norm(P[:, 1] - P[:, 0], axis=1)
    near = np.abs(c[:, 0] - 0.78 * lx) < 5_000.0
    far = np.abs(c[:, 0] - 0.78 * lx) > 150_000.0
    assert np.median(L[near]) < 2_000.0 < 20_000.0 < np.median(L[far])


def test_workloads_are_reproducible():
    a = W.graded_c3(n_tri=5000)
    b = W.graded_c3(n_tri=5000)
    assert np.array_equal(a.mesh.xy, b.mesh.xy) and np.array_equal(a.hb, b.hb)
    c = W.ensemble_c4(n_scen=3, lo=1000, hi=3000)
    d = W.ensemble_c4(n_scen=3, lo=1000, hi=3000)
    assert all(np.array_equal(x.manning, y.manning) for x, y in zip(c, d))
    h = W.hurricane_c5(n_tri=4000)
    assert 0.2 < np.mean(W.element_mean(h.mesh, h.hb) < h.h0) < 0.4
    assert h.rain_grid.mm_per_h.max() <= 100.0 and h.rain_grid.mm_per_h.min() >= 0.0
