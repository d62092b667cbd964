"""Pins of the near-zone search oracle (Sec. 3.2, closest point on the patch
surface) against closed forms: the Lagrange basis on Clenshaw-Curtis nodes
and its derivative reproduce polynomials of degree <= q; on a cylinder wall
the closest point is the radial projection and the distance |R - rho|; on a
cubed sphere the closest point is a x/|x| (up to the patches' interpolation
error); targets beyond d_eps have no patch."""
import numpy as np
import pytest

from oracle import nearzone as NZ
from synth import geometry as G

Q = 10


def test_lagrange_basis_reproduces_polynomials():
    rng = np.random.default_rng(4)
    c = rng.normal(size=Q + 1)
    p = np.polynomial.Polynomial(c)
    t = rng.uniform(-1, 1, 40)
    L, D = NZ.lagrange(Q, t)
    x = np.cos(np.pi * np.arange(Q + 1) / Q)
    np.testing.assert_allclose(L @ p(x), p(t), atol=1e-12 * np.abs(c).sum())
    np.testing.assert_allclose(D @ p(x), p.deriv()(t), atol=1e-10 * np.abs(c).sum())
    Ln, _ = NZ.lagrange(Q, x)
    np.testing.assert_allclose(Ln, np.eye(Q + 1), atol=1e-14)


@pytest.fixture(scope="module")
def wall():
    Rw, Lw, nth, nz = 6.0, 8.0, 6, 2
    cp, cn, cw, ch = G.cylinder_wall_patches(Rw, Lw, nth, nz, Q)
    return Rw, Lw, cp, nth * nz


def test_cylinder_wall_closest_points(wall):
    Rw, Lw, cp, npatch = wall
    rng = np.random.default_rng(5)
    th = rng.uniform(0, 2 * np.pi, 12)
    rho = Rw - rng.uniform(0.05, 0.9, 12)
    z = rng.uniform(1.0, Lw - 1.0, 12)
    x = np.stack([rho * np.cos(th), rho * np.sin(th), z], axis=1)
    patch, uv, y, n, dist = NZ.near_patch_search(cp, npatch, Q, x, 1.0)
    assert (patch >= 0).all()
    yref = np.stack([Rw * np.cos(th), Rw * np.sin(th), z], axis=1)
    np.testing.assert_allclose(dist, Rw - rho, atol=1e-7)
    np.testing.assert_allclose(y, yref, atol=1e-7)
    np.testing.assert_allclose(n, np.stack([np.cos(th), np.sin(th), 0 * th], axis=1), atol=1e-6)
    # beyond the near zone: no patch
    far = np.array([[0.0, 0.0, 4.0], [0.5 * Rw, 0.0, 3.0]])
    p2, *_ = NZ.near_patch_search(cp, npatch, Q, far, 1.0)
    assert (p2 == -1).all()


def test_cubed_sphere_closest_points():
    a = 1.5
    cp, cn, cw, ch = G.cubed_sphere_patches(a, Q, 1)
    rng = np.random.default_rng(6)
    d = rng.normal(size=(8, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    rho = a + rng.uniform(-0.3, 0.3, 8)
    x = d * rho[:, None]
    patch, uv, y, n, dist = NZ.near_patch_search(cp, 6, Q, x, 0.5)
    assert (patch >= 0).all()
    np.testing.assert_allclose(dist, np.abs(rho - a), atol=2e-4)
    np.testing.assert_allclose(y, a * d, atol=2e-4)
    np.testing.assert_allclose(n, d, atol=2e-4)


def test_planar_patch_with_curved_parameters():
    """A patch of the plane z = 0 whose (u, v) map is a quadratic warp (the
    interpolant reproduces it exactly): the closest point of x is its orthogonal
    projection, the distance |x_z| and the normal +-e_z, whatever the map."""
    n1 = Q + 1
    t = np.cos(np.pi * np.arange(n1) / Q)
    U, V = np.meshgrid(t, t, indexing="ij")
    X = U + 0.15 * V ** 2 - 0.1 * U * V
    Y = V + 0.2 * U ** 2
    nodes = np.stack([X, Y, np.zeros_like(X)], axis=-1).reshape(-1, 3)
    rng = np.random.default_rng(11)
    for _ in range(8):
        u0, v0 = rng.uniform(-0.7, 0.7, 2)
        p = np.array([u0 + 0.15 * v0 ** 2 - 0.1 * u0 * v0, v0 + 0.2 * u0 ** 2, 0.0])
        h = rng.uniform(-0.5, 0.5)
        x = p + np.array([0.0, 0.0, h])
        d, u, v, y = NZ.closest_on_patch(nodes, Q, x)
        assert abs(d - abs(h)) <= 1e-9 and np.abs(y - p).max() <= 1e-7, (d, h, y, p)
        assert abs(u - u0) <= 1e-6 and abs(v - v0) <= 1e-6
        _, Pu, Pv = NZ.patch_eval(nodes, Q, u, v)
        nrm = np.cross(Pu[0], Pv[0])
        nrm /= np.linalg.norm(nrm)
        np.testing.assert_allclose(np.abs(nrm), [0.0, 0.0, 1.0], atol=1e-12)
