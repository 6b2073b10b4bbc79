"""GPU parity of the exact demag evaluation (Eq. 2) on the FFT code paths that
the full-size workloads run, element by element against the CPU oracle.

The FFT kernels are instantiated per transform length, and several code
paths exist only at some lengths: the radix-16 butterfly of the 1024-point
FP32 warp transforms, the CTA-wide stages of FP64 transforms longer than
256 points, the pipelined split passes of large meshes and the tensor-copy
x-inverse pass.  Each case below names the instances it reaches.

* Dense random magnetisation against ``O.demag_fft`` on every mesh whose
  oracle tensor takes seconds: the 256 x 128 x 4 film itself (the bench's
  workload, both precisions) and meshes with one axis of 512 cells (padded
  length 1024) on each axis, with and without the forced split passes.
* The 512 x 512 x 16 box (padded 1024 x 1024 x 32), whose full oracle tensor
  would take many minutes: a sparse magnetisation of a few point moments,
  so that each sampled output cell is an exact short sum that the oracle
  evaluates entry by entry, H(r) = -Ms sum_j N(r - r_j) m_j.  A point moment
  excites every spatial frequency, so a wrong twiddle, index or pruning
  decision in any stage shows up in the samples.

Tolerances (max-norm relative to max|H|): 1e-12 in FP64, 1e-5 in FP32.
"""
import functools
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as O
from paper_2107_06729_gb300 import workloads as W
from gpu_util import gpu_context, gpu_demag, rel_max, torch_cuda

pytestmark = pytest.mark.gpu

MAT = {"Ms": 8e5, "alpha": 0.0, "gamma": W.GAMMA}
TOL = {"fp64": 1e-12, "fp32": 1e-5}


@functools.lru_cache(maxsize=None)
def _tensor(n, d):
    return O.newell_octant(*n, *d)


def _dense_case(n, d, prec, seed):
    m = W.m_random(n, seed=seed)
    ref = O.demag_fft(_tensor(n, d), MAT["Ms"], m)
    got = gpu_demag({"n": n, "d": d}, MAT, m, prec)
    return rel_max(got, ref)


FILM = ((256, 128, 4), (2.5e-9, 2.5e-9, 1e-9))


@pytest.mark.parametrize("env", [{}, {"MMX_AUTOTUNE": "0"}, {"MMX_NO_TMA": "1"}, {"MMX_NO_R4": "1"}])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_film_256x128x4_matches_oracle(prec, env, monkeypatch):
    """The bench's film: FP32 runs the four-step k_xf4h<float,8>, k_yz<float,256>
    and the tensor-copy four-step k_xi_t<float,512,true> (plain k_xi<float,512>
    with MMX_NO_TMA; the Stockham k_xf<float,512> and k_xi_t<float,512> with
    MMX_NO_R4); FP64 runs the CTA-wide 512-point x transforms and k_yz<double,256>."""
    if prec == "fp64" and (env.get("MMX_NO_TMA") or env.get("MMX_NO_R4")):
        pytest.skip("FP64 has neither the tensor-copy nor the four-step passes")
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    n, d = FILM
    assert _dense_case(n, d, prec, seed=21) < TOL[prec]


# (mesh, environment, what it reaches)
LONG_CASES = [
    # x padded to 1024: FP32 warp transform with the radix-16 stage (k_xf / k_xi(_t) <float,1024>);
    # FP64 CTA-wide stages (k_xf / k_xi <double,1024>)
    (((512, 8, 2), (2e-9, 2e-9, 2e-9)), {}),
    (((512, 8, 2), (2e-9, 2e-9, 2e-9)), {"MMX_NO_TMA": "1"}),
    # x padded to 512 in FP64: CTA-wide stages at the next length down
    (((256, 8, 2), (2e-9, 3e-9, 1e-9)), {}),
    # y padded to 1024: fused k_yz<float,1024> (radix-16) / split k_yf, k_yi <double,1024> (CTA-wide)
    (((8, 512, 2), (2e-9, 2e-9, 2e-9)), {}),
    # y padded to 512 in FP64: fused k_yz<double,512> with CTA-wide stages
    (((8, 256, 2), (1e-9, 2e-9, 3e-9)), {}),
    # split passes, forced: four-step k_xf4 / k_xi_t<float,1024,true>, k_yf_p / k_yi_p <float,64>
    (((512, 32, 2), (2e-9, 2e-9, 2e-9)), {"MMX_FORCE_SPLIT": "1"}),
    # ... and the Stockham k_xf_p<float,1024>, k_xi_t<float,1024> instead
    (((512, 32, 2), (2e-9, 2e-9, 2e-9)), {"MMX_FORCE_SPLIT": "1", "MMX_NO_R4": "1"}),
    # split passes, forced: four-step k_yf4 / k_yi4, k_zm_r<float,4>
    (((32, 512, 2), (2e-9, 2e-9, 2e-9)), {"MMX_FORCE_SPLIT": "1"}),
    # ... and the Stockham k_yf_p / k_yi_p <float,1024> instead
    (((32, 512, 2), (2e-9, 2e-9, 2e-9)), {"MMX_FORCE_SPLIT": "1", "MMX_NO_R4": "1"}),
    # the box's z length: k_zm_r<float,32> / k_zm<double,32> behind the split passes
    (((32, 32, 16), (2e-9, 2e-9, 2e-9)), {"MMX_FORCE_SPLIT": "1"}),
]


@pytest.mark.parametrize("case,env", LONG_CASES, ids=lambda v: str(v))
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_long_transforms_match_oracle(case, env, prec, monkeypatch):
    n, d = case
    if prec == "fp64" and (env.get("MMX_NO_TMA") or env.get("MMX_NO_R4")):
        pytest.skip("FP64 has neither the tensor-copy nor the four-step passes")
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    assert _dense_case(n, d, prec, seed=sum(n) + 5) < TOL[prec]


BOX = ((512, 512, 16), (2e-9, 2e-9, 2e-9))


def _sparse_moments(n, k, seed):
    """k point moments of random direction at random cells (distinct), plus
    one at each corner of the mesh so that the longest offsets occur."""
    nx, ny, nz = n
    rng = np.random.default_rng(np.random.PCG64(seed))
    cells = {(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx - 1, 0, 0), (0, ny - 1, nz - 1)}
    while len(cells) < k:
        cells.add((int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))))
    cells = sorted(cells)
    dirs = rng.normal(size=(len(cells), 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    return cells, dirs


def _sample_points(n, cells, count, seed):
    """The moment cells, their face neighbours, and random cells."""
    nx, ny, nz = n
    rng = np.random.default_rng(np.random.PCG64(seed + 1))
    pts = set()
    for (x, y, z) in cells:
        pts.add((x, y, z))
        for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            if 0 <= x + dx < nx and 0 <= y + dy < ny and 0 <= z + dz < nz:
                pts.add((x + dx, y + dy, z + dz))
    while len(pts) < count:
        pts.add((int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))))
    return sorted(pts)


def _oracle_samples(d, Ms, cells, dirs, pts):
    """H at each sampled cell from the oracle's Newell entries at the signed
    offsets r - r_j (the oracle's ctypes calls release the GIL)."""
    def one(p):
        h = np.zeros(3)
        for (c, mj) in zip(cells, dirs):
            e = O.newell_entry(p[0] - c[0], p[1] - c[1], p[2] - c[2], *d)
            T = np.array([[e[0], e[3], e[4]], [e[3], e[1], e[5]], [e[4], e[5], e[2]]])
            h -= Ms * (T @ mj)
        return h
    with ThreadPoolExecutor(max_workers=16) as ex:
        return np.array(list(ex.map(one, pts)))


@functools.lru_cache(maxsize=None)
def _box_reference():
    n, d = BOX
    cells, dirs = _sparse_moments(n, 16, seed=3)
    pts = _sample_points(n, cells, 320, seed=3)
    return cells, dirs, pts, _oracle_samples(d, MAT["Ms"], cells, dirs, pts)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_box_512x512x16_sampled_point_moments_match_oracle(prec):
    """Full-size 512 x 512 x 16 evaluation in the configuration the bench
    times (FP32: k_xf_p, k_yf_p, k_zm_r<float,32>, k_yi_p at 1024 points and
    the tensor-copy k_xi_t<float,1024>; FP64: the CTA-wide split passes),
    sampled at 320 cells against the oracle's exact sums."""
    torch = torch_cuda()
    n, d = BOX
    cells, dirs, pts, ref = _box_reference()
    m = np.zeros((3, n[2], n[1], n[0]))
    for (x, y, z), mj in zip(cells, dirs):
        m[:, z, y, x] = mj
    dt = torch.float64 if prec == "fp64" else torch.float32
    ctx = gpu_context({"n": n, "d": d}, MAT, {}, {"method": "RK4", "h": 1e-13}, prec)
    try:
        if prec == "fp32":
            p = ctx.plan()
            assert p["yz_pass"] == 1 and p["kernels_per_demag"] == 5
        m_t = torch.from_numpy(m).to("cuda", dt)
        H_t = torch.empty_like(m_t)
        ctx.demag(m_t, H_t)
        torch.cuda.synchronize()
        idx = torch.tensor([(z * n[1] + y) * n[0] + x for (x, y, z) in pts], device="cuda")
        got = H_t.reshape(3, -1)[:, idx].double().cpu().numpy().T
    finally:
        ctx.close()
    assert rel_max(got, ref) < TOL[prec]
