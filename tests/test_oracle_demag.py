"""Pins for the oracle's demag field, Eq. 2: the literal O(N^2) sum against
the zero-padded FFT convolution, the single-cell self field, and the
uniformly magnetised block against the published prism factor."""
import numpy as np
import pytest

import oracle as O
from test_oracle_newell import aharoni_all


def rand_m(shape, seed):
    rng = np.random.default_rng(seed)
    m = rng.normal(size=(3,) + shape)
    return m / np.linalg.norm(m, axis=0)


@pytest.mark.parametrize("n,d", [((1, 1, 1), (1, 1, 1)), ((2, 1, 1), (1, 1, 1)),
                                 ((3, 5, 2), (1.0, 1.5, 0.7)), ((8, 4, 1), (4e-9, 4e-9, 4e-9)),
                                 ((6, 6, 3), (2.5e-9, 2.5e-9, 1e-9)), ((16, 8, 2), (1, 1, 1))])
def test_direct_sum_equals_fft_convolution(n, d):
    nx, ny, nz = n
    N6 = O.newell_octant(nx, ny, nz, *d)
    m = rand_m((nz, ny, nx), seed=nx * 100 + ny * 10 + nz)
    Ms = 8e5
    Hd = O.demag_direct(N6, Ms, m)
    Hf = O.demag_fft(N6, Ms, m)
    scale = np.abs(Hd).max()
    assert np.abs(Hd - Hf).max() <= 1e-13 * scale


def test_single_cell_is_self_field():
    d = (2.0, 1.0, 0.5)
    N6 = O.newell_octant(1, 1, 1, *d)
    m = np.array([0.6, -0.48, 0.64]).reshape(3, 1, 1, 1)
    H = O.demag_direct(N6, 1e6, m)
    D = aharoni_all(d[0] / 2, d[1] / 2, d[2] / 2)
    assert np.allclose(H.ravel(), -1e6 * D * m.ravel(), rtol=1e-13, atol=0)
    assert np.allclose(O.demag_fft(N6, 1e6, m).ravel(), H.ravel(), rtol=1e-13, atol=1e-9)


@pytest.mark.parametrize("n,d", [((8, 8, 2), (4e-9, 4e-9, 4e-9)), ((12, 6, 3), (2.5e-9, 2.5e-9, 1e-9))])
def test_uniform_block_mean_field_is_prism_factor(n, d):
    nx, ny, nz = n
    N6 = O.newell_octant(nx, ny, nz, *d)
    mdir = np.array([0.3, -0.5, 0.81])
    mdir /= np.linalg.norm(mdir)
    m = np.broadcast_to(mdir.reshape(3, 1, 1, 1), (3, nz, ny, nx)).copy()
    Ms = 8e5
    H = O.demag_fft(N6, Ms, m)
    mean = H.reshape(3, -1).mean(axis=1)
    D = aharoni_all(nx * d[0] / 2, ny * d[1] / 2, nz * d[2] / 2)
    assert np.allclose(mean, -Ms * D * mdir, rtol=0, atol=1e-10 * Ms)


def test_linearity_and_superposition():
    nx, ny, nz = 5, 4, 2
    N6 = O.newell_octant(nx, ny, nz, 1.0, 1.0, 1.0)
    a = rand_m((nz, ny, nx), 3)
    b = rand_m((nz, ny, nx), 4)
    Ha = O.demag_fft(N6, 1.0, a)
    Hb = O.demag_fft(N6, 1.0, b)
    Hab = O.demag_fft(N6, 1.0, 2.0 * a - 0.5 * b)
    assert np.allclose(Hab, 2.0 * Ha - 0.5 * Hb, atol=1e-14, rtol=0)


def test_impulse_response_is_tensor_column():
    # M = Ms e_y in cell (1, 2, 0) only: H(r0) = -Ms N(r0 - r) e_y
    nx, ny, nz = 4, 5, 2
    d = (1.0, 1.2, 0.9)
    N6 = O.newell_octant(nx, ny, nz, *d)
    m = np.zeros((3, nz, ny, nx))
    m[1, 0, 2, 1] = 1.0
    H = O.demag_direct(N6, 2.0, m)
    for (x0, y0, z0) in [(0, 0, 0), (3, 4, 1), (1, 2, 0), (2, 1, 1)]:
        e = O.newell_entry(x0 - 1, y0 - 2, z0 - 0, *d)
        tol = 1e-14 * 2.0 * np.abs(e).max()
        assert H[0, z0, y0, x0] == pytest.approx(-2.0 * e[3], rel=1e-14, abs=tol)
        assert H[1, z0, y0, x0] == pytest.approx(-2.0 * e[1], rel=1e-14, abs=tol)
        assert H[2, z0, y0, x0] == pytest.approx(-2.0 * e[5], rel=1e-14, abs=tol)
