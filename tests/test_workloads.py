"""The seeded input generators: unit vectors, the stated sizes and ranges,
and reproducibility (the same seed gives the same inputs)."""
import numpy as np

from paper_2107_06729_gb300 import workloads as W
from paper_2107_06729_gb300 import experiments as E


def _unit(m):
    return np.abs(np.linalg.norm(m, axis=0) - 1).max() < 1e-12


def test_ensemble_workload_ranges_and_reproducibility():
    a = W.ensemble_config3(seed=0)
    b = W.ensemble_config3(seed=0)
    assert len(a) == 64
    for s, t in zip(a, b):
        nx, ny, nz = s["mesh"]["n"]
        assert nx in (32, 64, 128, 256) and ny in (32, 64, 128, 256) and nz in (1, 2)
        assert s["mesh"]["d"] == (4e-9, 4e-9, 4e-9)
        assert 4e5 <= s["material"]["Ms"] <= 1.2e6 and 0.005 <= s["material"]["alpha"] <= 0.1
        H = np.array(s["field"]["H0"])
        assert H[2] == 0 and np.linalg.norm(H) <= W.mT(50.0) * (1 + 1e-12)
        assert s["integrator"]["method"] == "RKF45" and s["integrator"]["extrap_order"] == 4
        assert s["m0"].shape == (3, nz, ny, nx) and _unit(s["m0"])
        assert np.array_equal(s["m0"], t["m0"])
    assert len({s["mesh"]["n"] for s in a}) > 10  # uneven sizes
    assert not np.array_equal(a[0]["m0"], W.ensemble_config3(seed=1)[0]["m0"]) or \
        a[0]["mesh"] != W.ensemble_config3(seed=1)[0]["mesh"]


def test_slab_stand_in():
    c = E.slab_config()
    assert c["mesh"]["n"] == (512, 256, 4) and c["mesh"]["d"] == (5e-9, 5e-9, 5e-9)
    m = c["m0"]
    assert _unit(m)
    # S-like: the two ends tilt to opposite sides of +x
    assert m[1, :, :, :8].mean() > 0.3 and m[1, :, :, -8:].mean() < -0.3
    assert m[0].mean() > 0.9
    assert c["field"]["H0"] == (-20e3, 1e3, 0.0)


def test_rnet_params_are_seeded_and_within_the_he_bounds():
    a, b, c = W.rnet_params(3), W.rnet_params(3), W.rnet_params(4)
    assert a.dtype == np.float32 and a.size == 63171
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    off = 0
    for li, (ci, co) in enumerate(W.RNET_LAYERS):
        lim = np.sqrt(6.0 / (27 * ci)) * (0.1 if li == len(W.RNET_LAYERS) - 1 else 1.0)
        w = a[off:off + 27 * co * ci]
        off += 27 * co * ci
        bias = a[off:off + co]
        off += co
        assert np.abs(w).max() <= lim and np.abs(w).max() > 0.9 * lim
        assert np.abs(bias).max() <= 0.01
    assert off == a.size
