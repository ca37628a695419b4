"""Input generators: meshes, hierarchy, colourings, manufactured solutions."""
import numpy as np
import pytest

from workloads import unit_square, unit_square_hierarchy, curl_bubble_2d, polynomial_2d
from workloads.manufactured import lattice_barycentric_2d, lattice_points_2d
from oracle.quadrature import triangle_points


def cross2(a, b):
    return a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]


def test_unit_square_counts_and_orientation():
    m = unit_square(5)
    assert m.n_cells == 50 and m.n_vertices == 36
    X = m.coords[m.cells]
    det = cross2(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])
    assert np.allclose(det, 1 / 25)          # all counter-clockwise, area 1/(2N²)


@pytest.mark.parametrize("kw", [{}, {"jitter": 0.3, "seed": 4}])
def test_hierarchy_parents_and_colouring(kw):
    ms = unit_square_hierarchy(2, 4, **kw)
    for l in range(1, len(ms)):
        f, c = ms[l], ms[l - 1]
        assert np.bincount(f.parent, minlength=c.n_cells).tolist() == [4] * c.n_cells
        cen = f.coords[f.cells].mean(1)
        P = c.coords[c.cells[f.parent]]
        T = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]], -1)
        lam = np.linalg.solve(T, (cen - P[:, 0])[..., None])[..., 0]
        assert (lam > 1e-12).all() and (lam.sum(1) < 1 - 1e-12).all()
        area_f = 0.5 * np.abs(cross2(f.coords[f.cells[:, 1]] - f.coords[f.cells[:, 0]],
                                     f.coords[f.cells[:, 2]] - f.coords[f.cells[:, 0]]))
        assert abs(area_f.sum() - 1.0) < 1e-13
    for m in ms:
        if m.vertex_colour is not None:
            for cell in m.cells:
                assert len(set(m.vertex_colour[cell].tolist())) == 3


def test_lattice_points():
    lam = lattice_barycentric_2d(3)
    assert lam.shape == (10, 3) and np.allclose(lam.sum(1), 1)
    m = unit_square(1)
    X = lattice_points_2d(m.coords, m.cells, 2)
    assert np.allclose(X[0, 0], m.coords[m.cells[0, 0]])
    assert np.allclose(X[0, 2], m.coords[m.cells[0, 1]])
    assert np.allclose(X[0, 5], m.coords[m.cells[0, 2]])


@pytest.mark.parametrize("sol", [curl_bubble_2d(), polynomial_2d()])
def test_manufactured_derivatives(sol):
    x = np.random.default_rng(0).uniform(0.05, 0.95, (20, 2))
    h = 1e-5
    G = sol.grad_u(x)
    for j in range(2):
        e = np.zeros(2)
        e[j] = h
        assert np.abs((sol.u(x + e) - sol.u(x - e)) / (2 * h) - G[:, :, j]).max() < 1e-6
        gp = (sol.p(x + e) - sol.p(x - e)) / (2 * h)
        assert np.abs(gp - sol.grad_p(x)[:, j]).max() < 1e-6
    hh = 1e-4
    lap = sum((sol.u(x + e) - 2 * sol.u(x) + sol.u(x - e)) / hh ** 2
              for e in (np.array([hh, 0]), np.array([0, hh])))
    assert np.abs(lap - sol.lap_u(x)).max() < 1e-4 * np.abs(lap).max()
    assert np.abs(G[:, 0, 0] + G[:, 1, 1]).max() < 1e-12
    # zero boundary values and mean-free pressure
    s = np.linspace(0, 1, 7)
    for bx in (np.stack([s, 0 * s], 1), np.stack([s, 0 * s + 1], 1),
               np.stack([0 * s, s], 1), np.stack([0 * s + 1, s], 1)):
        assert np.abs(sol.u(bx)).max() < 1e-12
    m = unit_square(8)
    tot = 0.0
    for c in m.cells:
        xq, wq = triangle_points(m.coords[c], 8)
        tot += wq @ sol.p(xq)
    assert abs(tot) < 1e-12
