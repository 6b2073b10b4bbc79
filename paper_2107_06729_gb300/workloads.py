"""Seeded synthetic workloads: problem descriptions and initial magnetisation
generators.  This module holds inputs only (no part of the method's
arithmetic) and is the one module that both the CUDA path's tests/bench and
the CPU oracle's tests consume.

All randomness comes from ``numpy.random.Generator(PCG64(seed))``.
Magnetisation arrays are unit vectors in SoA layout ``[3, nz, ny, nx]``.
Fields are in A/m; a field given in mT is converted with H = B / mu0.

The paper's own workloads (muMAG standard problem 4, the 3.2 um x 1.6 um x
20 nm Py slab in an S-state, the checkerboard particle array; Sec. III) are
not reproduced: their initial states and geometries are not fully specified.
The films below stand in for them, with the paper's Ni80Fe20 material
(Ms = 800 kA/m, A = 13 pJ/m, alpha = 0.02) and comparable cell sizes.
"""
import numpy as np

MU0 = 4e-7 * np.pi
GAMMA = 2.211e5  # m/(A s)


def mT(b):
    """Field in A/m for a flux density given in mT."""
    return np.asarray(b, dtype=np.float64) * 1e-3 / MU0


def _normalise(m):
    return m / np.linalg.norm(m, axis=0, keepdims=True)


def m_uniform_noise(n, direction=(1.0, 1.0, 1.0), noise=0.05, seed=0):
    """Uniform direction plus U(-noise, noise) per component, renormalised."""
    nx, ny, nz = n
    rng = np.random.default_rng(np.random.PCG64(seed))
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    m = d.reshape(3, 1, 1, 1) + rng.uniform(-noise, noise, size=(3, nz, ny, nx))
    return _normalise(m)


def m_random(n, seed=0):
    """Independent uniformly random directions on the unit sphere."""
    nx, ny, nz = n
    rng = np.random.default_rng(np.random.PCG64(seed))
    return _normalise(rng.normal(size=(3, nz, ny, nx)))


def checkerboard_mask(n, p):
    """[1, nz, ny, nx] array: 1 on the cells of p x p squares of a
    checkerboard (the square holding cell (0, 0) occupied), 0 elsewhere --
    a particle array in vacuum (cells with m = 0 hold no material)."""
    nx, ny, nz = n
    x = np.arange(nx) // p
    y = np.arange(ny) // p
    occ = ((x.reshape(1, nx) + y.reshape(ny, 1)) % 2 == 0).astype(np.float64)
    return np.broadcast_to(occ, (nz, ny, nx)).reshape(1, nz, ny, nx).copy()


def m_vortex(n, d, core_radius=10e-9, noise=0.05, seed=0):
    """In-plane curl (-y, x)/r around the film centre, out-of-plane core
    m_z = exp(-r^2 / core_radius^2), plus U(-noise, noise), renormalised."""
    nx, ny, nz = n
    rng = np.random.default_rng(np.random.PCG64(seed))
    x = (np.arange(nx) + 0.5 - nx / 2) * d[0]
    y = (np.arange(ny) + 0.5 - ny / 2) * d[1]
    X, Y = np.meshgrid(x, y, indexing="xy")
    r = np.sqrt(X * X + Y * Y) + 1e-30
    mz = np.exp(-(r * r) / core_radius ** 2)
    inpl = np.sqrt(np.clip(1 - mz * mz, 0, 1))
    m = np.stack([-Y / r * inpl, X / r * inpl, mz])[:, None, :, :].repeat(nz, axis=1)
    m = m + rng.uniform(-noise, noise, size=m.shape)
    return _normalise(m)


def m_smooth(n, seed=0):
    """Smooth, low-wavenumber pattern used for convergence studies."""
    nx, ny, nz = n
    rng = np.random.default_rng(np.random.PCG64(seed))
    ph = rng.uniform(0, 2 * np.pi, size=3)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) + 0.5) / max(nz, 1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    m = np.stack([1.0 + 0.4 * np.sin(np.pi * X + ph[0]),
                  0.6 * np.cos(np.pi * Y + ph[1]),
                  0.3 * np.sin(np.pi * (X + Y + Z) + ph[2])])
    return _normalise(m)


def film_config1(seed=0):
    """Thin film 64 x 32 x 1 cells of 4 nm, fixed-step RK4 h = 0.1 ps, full
    demag at all sub-steps, FP64; 2000 steps = 0.2 ns."""
    n = (64, 32, 1)
    d = (4e-9, 4e-9, 4e-9)
    return {
        "name": "film_64x32x1_rk4_fp64",
        "mesh": {"n": n, "d": d},
        "material": {"Ms": 8e5, "A": 1.3e-11, "K": 0.0, "ku": (1.0, 0.0, 0.0),
                     "alpha": 0.02, "gamma": GAMMA},
        "field": {"H0": tuple(mT((-24.6, 4.3, 0.0))), "pulse": (0.0, 0.0, 0.0),
                  "t_on": 0.0, "t_off": 0.0},
        "integrator": {"method": "RK4", "extrap_order": -1, "adaptive": False, "h": 1e-13},
        "precision": "fp64",
        "t_end": 2000 * 1e-13,
        "m0": m_uniform_noise(n, seed=seed),
    }


def film_config2(seed=0):
    """Film 256 x 128 x 4 cells of 2.5 x 2.5 x 1 nm, uniaxial K along x,
    Dormand-Prince 5(4) at e_max = 1e-5, demag exact at stage 1 only and
    4th-order extrapolation, FP32 fields, 20 mT pulse along y on [0, 200 ps)."""
    n = (256, 128, 4)
    d = (2.5e-9, 2.5e-9, 1e-9)
    return {
        "name": "film_256x128x4_dp54_p4_fp32",
        "mesh": {"n": n, "d": d},
        "material": {"Ms": 8e5, "A": 1.3e-11, "K": 5e4, "ku": (1.0, 0.0, 0.0),
                     "alpha": 0.01, "gamma": GAMMA},
        "field": {"H0": (0.0, 0.0, 0.0), "pulse": tuple(mT((0.0, 20.0, 0.0))),
                  "t_on": 0.0, "t_off": 200e-12},
        "integrator": {"method": "RKDP54", "extrap_order": 4, "adaptive": True, "h": 1e-13,
                       "tol": 1e-5, "hmin": 1e-15, "hmax": 3e-12, "cmin": 0.01, "cmax": 2.0},
        "precision": "fp32",
        "t_end": 1e-9,
        "m0": m_random(n, seed=seed),
    }


def film_large3d(seed=0):
    """512 x 512 x 16 cells of 2 nm (4.2M cells), vortex plus noise."""
    n = (512, 512, 16)
    d = (2e-9, 2e-9, 2e-9)
    return {
        "name": "box_512x512x16_rk23_p2_fp32",
        "mesh": {"n": n, "d": d},
        "material": {"Ms": 8e5, "A": 1.3e-11, "K": 0.0, "ku": (1.0, 0.0, 0.0),
                     "alpha": 0.02, "gamma": GAMMA},
        "field": {"H0": (0.0, 0.0, 0.0), "pulse": (0.0, 0.0, 0.0), "t_on": 0.0, "t_off": 0.0},
        "integrator": {"method": "RK23", "extrap_order": 2, "adaptive": True, "h": 1e-13,
                       "tol": 1e-5, "hmin": 1e-15, "hmax": 3e-12, "cmin": 0.01, "cmax": 2.0},
        "precision": "fp32",
        "t_end": 1e-10,
        "m0_fn": lambda: m_vortex(n, d, seed=seed),
    }


def ensemble_config3(seed=0, n_samples=64):
    """Batched ensemble of independent films of uneven sizes: side lengths
    drawn from {32, 64, 128, 256} per axis, 1 or 2 layers, 4 nm cells; per
    sample Ms ~ U[4e5, 1.2e6] A/m, alpha ~ U[0.005, 0.1], and a static
    in-plane field of magnitude ~ U[0, 50] mT at a uniform random angle;
    A = 13 pJ/m, no anisotropy.  Initial m: a random in-plane direction plus
    U(-0.05, 0.05) noise, renormalised.  RKF45 at e_max = 1e-5 with
    4th-order extrapolation, FP32 fields.  Returns a list of sample dicts in
    the format of the single-film configurations."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    sides = (32, 64, 128, 256)
    out = []
    for i in range(n_samples):
        nx = int(rng.choice(sides))
        ny = int(rng.choice(sides))
        nz = int(rng.integers(1, 3))
        Ms = float(rng.uniform(4e5, 1.2e6))
        alpha = float(rng.uniform(0.005, 0.1))
        b = float(rng.uniform(0.0, 50.0))
        phi = float(rng.uniform(0.0, 2 * np.pi))
        psi = float(rng.uniform(0.0, 2 * np.pi))
        m_seed = int(rng.integers(0, 2 ** 31))
        n = (nx, ny, nz)
        out.append({
            "name": "film_%dx%dx%d_rkf45_p4_fp32" % n,
            "mesh": {"n": n, "d": (4e-9, 4e-9, 4e-9)},
            "material": {"Ms": Ms, "A": 1.3e-11, "K": 0.0, "ku": (1.0, 0.0, 0.0),
                         "alpha": alpha, "gamma": GAMMA},
            "field": {"H0": tuple(mT((b * np.cos(phi), b * np.sin(phi), 0.0))),
                      "pulse": (0.0, 0.0, 0.0), "t_on": 0.0, "t_off": 0.0},
            "integrator": {"method": "RKF45", "extrap_order": 4, "adaptive": True, "h": 1e-13,
                           "tol": 1e-5, "hmin": 1e-15, "hmax": 3e-12, "cmin": 0.01, "cmax": 2.0},
            "precision": "fp32",
            "m0": m_uniform_noise(n, direction=(np.cos(psi), np.sin(psi), 0.0), seed=m_seed),
        })
    return out


# layer widths (cin, cout) of the learned residual net, in parameter order
RNET_LAYERS = ((6, 32), (32, 32), (32, 32), (32, 3))


def rnet_params(seed=0, out_scale=0.1):
    """Seeded initial parameters of the residual net, flat float32 in the
    library's layout (per layer W[27][cout][cin], then b[cout]): He-uniform
    weights U(-sqrt(6/fan_in), +sqrt(6/fan_in)), fan_in = 27 cin, the last
    layer's scaled by out_scale, small uniform biases."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    parts = []
    for li, (ci, co) in enumerate(RNET_LAYERS):
        lim = np.sqrt(6.0 / (27 * ci)) * (out_scale if li == len(RNET_LAYERS) - 1 else 1.0)
        parts.append(rng.uniform(-lim, lim, size=27 * co * ci))
        parts.append(rng.uniform(-0.01, 0.01, size=co))
    return np.concatenate(parts).astype(np.float32)
