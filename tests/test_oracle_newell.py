"""Pins for the oracle's Newell demag tensor (Sec. II, Eq. 2; tensor of
ref. [24]) against facts fixed by magnetostatics, not by the oracle itself:
self trace 1, the cube's 1/3, zero trace between disjoint cells, parity,
the point-dipole far field, brute-force quadrature of the defining double
volume integral, and the published closed-form demag factor of a
rectangular prism (Aharoni 1998) for the cell-averaged block sum."""
import itertools

import numpy as np
import pytest

import oracle as O


def aharoni_Dz(a, b, c):
    """Demag factor along z of the prism |x|<=a, |y|<=b, |z|<=c
    (A. Aharoni, J. Appl. Phys. 83, 3432 (1998), Eq. 1)."""
    r = np.sqrt(a * a + b * b + c * c)
    rab, rbc, rac = np.sqrt(a * a + b * b), np.sqrt(b * b + c * c), np.sqrt(a * a + c * c)
    s = ((b * b - c * c) / (2 * b * c) * np.log((r - a) / (r + a))
         + (a * a - c * c) / (2 * a * c) * np.log((r - b) / (r + b))
         + b / (2 * c) * np.log((rab + a) / (rab - a))
         + a / (2 * c) * np.log((rab + b) / (rab - b))
         + c / (2 * a) * np.log((rbc - b) / (rbc + b))
         + c / (2 * b) * np.log((rac - a) / (rac + a))
         + 2 * np.arctan(a * b / (c * r))
         + (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
         + (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
         + c / (a * b) * (rac + rbc)
         - (rab ** 3 + rbc ** 3 + rac ** 3) / (3 * a * b * c))
    return s / np.pi


def aharoni_all(a, b, c):
    return np.array([aharoni_Dz(b, c, a), aharoni_Dz(c, a, b), aharoni_Dz(a, b, c)])


def test_aharoni_formula_itself():
    # the closed form must give 1/3 for a cube and sum to 1 for any prism
    assert aharoni_Dz(1.0, 1.0, 1.0) == pytest.approx(1 / 3, abs=1e-14)
    for abc in [(1, 2, 3), (5, 5, 0.5), (0.3, 7, 2), (128, 64, 2)]:
        assert aharoni_all(*abc).sum() == pytest.approx(1.0, abs=1e-12)
    # thin film limit: D_z -> 1
    assert aharoni_Dz(1000.0, 1000.0, 0.01) > 0.999


@pytest.mark.parametrize("d", [(1, 1, 1), (2.5e-9, 2.5e-9, 1e-9), (4e-9, 4e-9, 4e-9),
                               (1, 2, 3), (5, 0.5, 2)])
def test_self_trace_is_one(d):
    e = O.newell_entry(0, 0, 0, *d)
    assert e[:3].sum() == pytest.approx(1.0, abs=1e-15)
    assert np.all(np.abs(e[3:]) < 1e-15)  # self tensor is diagonal


def test_cube_self_factor_one_third():
    e = O.newell_entry(0, 0, 0, 3e-9, 3e-9, 3e-9)
    assert np.allclose(e[:3], 1 / 3, atol=1e-15, rtol=0)


@pytest.mark.parametrize("d", [(1, 1, 1), (2.5, 2.5, 1), (1, 2, 3)])
def test_self_factor_matches_single_cell_prism(d):
    e = O.newell_entry(0, 0, 0, *d)
    ref = aharoni_all(d[0] / 2, d[1] / 2, d[2] / 2)
    assert np.allclose(e[:3], ref, atol=1e-13, rtol=0)


def test_trace_vanishes_between_disjoint_cells():
    rng = np.random.default_rng(1)
    for _ in range(30):
        X, Y, Z = rng.integers(-12, 13, size=3)
        if X == Y == Z == 0:
            continue
        d = rng.uniform(0.5, 3.0, size=3)
        e = O.newell_entry(X, Y, Z, *d)
        scale = np.abs(e[:3]).max()
        assert abs(e[:3].sum()) <= 1e-12 * max(scale, 1e-300) + 1e-30


def test_parity():
    d = (1.0, 1.7, 0.6)
    for X, Y, Z in [(3, 2, 1), (1, 4, 2), (5, 1, 3), (2, 0, 1), (0, 3, 2)]:
        base = O.newell_entry(X, Y, Z, *d)
        for sx, sy, sz in itertools.product([1, -1], repeat=3):
            e = O.newell_entry(sx * X, sy * Y, sz * Z, *d)
            expect = base * np.array([1, 1, 1, sx * sy, sx * sz, sy * sz])
            assert np.allclose(e, expect, rtol=1e-13, atol=1e-18)


def dipole(R, V):
    r = np.linalg.norm(R)
    T = -(V / (4 * np.pi)) * (3 * np.outer(R, R) / r ** 5 - np.eye(3) / r ** 3)
    return np.array([T[0, 0], T[1, 1], T[2, 2], T[0, 1], T[0, 2], T[1, 2]])


def test_far_field_tends_to_point_dipole():
    d = np.array([1.0, 1.3, 0.7])
    direction = np.array([3.0, 2.0, 1.0])
    prev = None
    for k in [4, 8, 16, 32]:
        X, Y, Z = (direction * k).astype(int)
        e = O.newell_entry(X, Y, Z, *d)
        R = np.array([X, Y, Z]) * d
        ref = dipole(R, d.prod())
        rel = np.abs(e - ref).max() / np.abs(ref).max()
        if prev is not None:
            # relative deviation falls as (cell/R)^2: a factor ~4 per doubling
            assert rel < prev / 3.0
        prev = rel
    assert prev < 1e-4


def quadrature_tensor(R, d, ng=20):
    """Brute force of N_ab(R) = -(1/(4 pi V)) int_target int_source
    d_a d_b (1/|x - x'|), reduced to one 3D integral over u = x - x' with the
    triangular overlap weight, Gauss-Legendre on each half interval."""
    gx, gw = np.polynomial.legendre.leggauss(ng)
    nodes, weights = [], []
    for c in range(3):
        pts, wts = [], []
        for lo, hi in [(R[c] - d[c], R[c]), (R[c], R[c] + d[c])]:
            pts.append(0.5 * (hi - lo) * gx + 0.5 * (hi + lo))
            wts.append(0.5 * (hi - lo) * gw)
        p = np.concatenate(pts)
        w = np.concatenate(wts) * (d[c] - np.abs(p - R[c]))
        nodes.append(p)
        weights.append(w)
    ux, uy, uz = np.meshgrid(*nodes, indexing="ij")
    W = np.einsum("i,j,k->ijk", *weights)
    u = [ux, uy, uz]
    r2 = ux * ux + uy * uy + uz * uz
    r5 = r2 ** 2.5
    V = d.prod()
    out = []
    for a, b in [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]:
        f = (3 * u[a] * u[b] - (a == b) * r2) / r5
        out.append(-(W * f).sum() / (4 * np.pi * V))
    return np.array(out)


@pytest.mark.parametrize("off", [(2, 0, 0), (0, 2, 1), (2, 1, 1), (3, -2, 2), (-2, 3, 0), (4, 1, -3)])
def test_matches_bruteforce_quadrature(off):
    d = np.array([1.0, 1.4, 0.8])
    e = O.newell_entry(*off, *d)
    q = quadrature_tensor(np.array(off) * d, d)
    scale = np.abs(q).max()
    assert np.allclose(e, q, atol=1e-10 * scale, rtol=0)


@pytest.mark.parametrize("n,d", [((4, 3, 2), (1.0, 1.0, 1.0)),
                                 ((8, 4, 1), (2.5, 2.5, 1.0)),
                                 ((5, 5, 3), (1.0, 2.0, 0.5)),
                                 ((16, 8, 2), (4.0, 4.0, 4.0))])
def test_block_average_equals_prism_factor(n, d):
    """Newell's tensor is the cell-averaged field of a uniformly magnetised
    cell, so the block average of sum_r N(r - r0) is the prism's factor."""
    nx, ny, nz = n
    N6 = O.newell_octant(nx, ny, nz, *d)
    tot = np.zeros(3)
    for Z in range(-(nz - 1), nz):
        for Y in range(-(ny - 1), ny):
            for X in range(-(nx - 1), nx):
                w = (nx - abs(X)) * (ny - abs(Y)) * (nz - abs(Z))
                tot += w * N6[:3, abs(Z), abs(Y), abs(X)]
    tot /= nx * ny * nz
    ref = aharoni_all(nx * d[0] / 2, ny * d[1] / 2, nz * d[2] / 2)
    assert np.allclose(tot, ref, atol=2e-13, rtol=0)
    assert tot.sum() == pytest.approx(1.0, abs=1e-13)


def test_octant_matches_entries():
    N6 = O.newell_octant(5, 3, 2, 1.0, 2.0, 3.0)
    for (X, Y, Z) in [(0, 0, 0), (4, 2, 1), (2, 1, 0)]:
        assert np.array_equal(N6[:, Z, Y, X], O.newell_entry(X, Y, Z, 1.0, 2.0, 3.0))
