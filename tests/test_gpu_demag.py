"""GPU parity of the exact demag evaluation (Eq. 2) against the CPU oracle.

Tolerances (max-norm, relative to max|H|): 1e-12 in FP64 and 1e-5 in FP32
per evaluation.  Shapes span several FFT radix stages, the unpadded axes
(ny = 1, nz = 1), the packed kx = 0 / kx = nx column and ragged row counts
for the x passes."""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2107_06729_gb300 import workloads as W
from gpu_util import gpu_demag, rel_max

pytestmark = pytest.mark.gpu

SHAPES = [((2, 1, 1), (1e-9, 1e-9, 1e-9)), ((4, 2, 1), (2e-9, 1e-9, 3e-9)), ((8, 4, 2), (4e-9, 4e-9, 4e-9)),
          ((16, 8, 4), (2.5e-9, 2.5e-9, 1e-9)), ((64, 32, 1), (4e-9, 4e-9, 4e-9)), ((32, 16, 4), (2e-9, 3e-9, 1e-9)),
          ((8, 8, 8), (1e-9, 1e-9, 1e-9)), ((4, 2, 16), (3e-9, 2e-9, 1e-9)), ((128, 2, 2), (2e-9, 2e-9, 2e-9)),
          ((2, 64, 1), (1e-9, 1e-9, 1e-9))]
MAT = {"Ms": 8e5, "alpha": 0.0, "gamma": W.GAMMA}


@pytest.mark.parametrize("n,d", SHAPES)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_demag_matches_oracle(n, d, prec, tol):
    m = W.m_random(n, seed=sum(n))
    N6 = O.newell_octant(*n, *d)
    ref = O.demag_fft(N6, MAT["Ms"], m)
    got = gpu_demag({"n": n, "d": d}, MAT, m, prec)
    assert rel_max(got, ref) < tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_impulse_response_is_tensor(prec, tol):
    """M = Ms e_b in one corner cell: H(r0) = -Ms N(r0) e_b over the mesh."""
    n, d = (16, 8, 4), (2e-9, 3e-9, 1.5e-9)
    N6 = O.newell_octant(*n, *d)
    for b in range(3):
        m = np.zeros((3, n[2], n[1], n[0]))
        m[b, 0, 0, 0] = 1.0
        got = gpu_demag({"n": n, "d": d}, MAT, m, prec)
        comp = {0: (0, 3, 4), 1: (3, 1, 5), 2: (4, 5, 2)}[b]
        expect = np.stack([-MAT["Ms"] * N6[c] for c in comp])
        assert np.abs(got - expect).max() < tol * MAT["Ms"] * np.abs(N6).max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 2e-6)])
def test_uniform_film_full_size_prism_factor(prec, tol):
    """At the 256 x 128 x 4 film size: the mean demag field of a uniformly
    magnetised film equals -Ms D m with D the published prism factor."""
    from test_oracle_newell import aharoni_all
    n, d = (256, 128, 4), (2.5e-9, 2.5e-9, 1e-9)
    mdir = np.array([0.48, 0.6, 0.64])
    m = np.broadcast_to(mdir.reshape(3, 1, 1, 1), (3, n[2], n[1], n[0])).copy()
    got = gpu_demag({"n": n, "d": d}, MAT, m, prec)
    D = aharoni_all(n[0] * d[0] / 2, n[1] * d[1] / 2, n[2] * d[2] / 2)
    mean = got.reshape(3, -1).mean(axis=1)
    assert np.allclose(mean, -MAT["Ms"] * D * mdir, rtol=0, atol=tol * MAT["Ms"])


def test_linearity_fp64():
    n, d = (32, 16, 2), (2e-9, 2e-9, 2e-9)
    a, b = W.m_random(n, seed=1), W.m_random(n, seed=2)
    Ha = gpu_demag({"n": n, "d": d}, MAT, a, "fp64")
    Hb = gpu_demag({"n": n, "d": d}, MAT, b, "fp64")
    Hab = gpu_demag({"n": n, "d": d}, MAT, 0.3 * a - 1.7 * b, "fp64")
    assert rel_max(Hab, 0.3 * Ha - 1.7 * Hb) < 1e-13


SPLIT_SHAPES = [((8, 4, 2), (1e-9, 2e-9, 1e-9)), ((16, 8, 4), (2.5e-9, 2.5e-9, 1e-9)),
                ((32, 16, 4), (2e-9, 3e-9, 1e-9)), ((4, 2, 16), (3e-9, 2e-9, 1e-9)),
                ((2, 64, 1), (1e-9, 1e-9, 1e-9)), ((16, 32, 8), (2e-9, 2e-9, 2e-9))]


@pytest.mark.parametrize("n,d", SPLIT_SHAPES)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_split_yz_path_matches_oracle(n, d, prec, tol, monkeypatch):
    """The three-kernel y / z path used for large meshes, forced on small ones."""
    monkeypatch.setenv("MMX_FORCE_SPLIT", "1")
    m = W.m_random(n, seed=sum(n) + 7)
    N6 = O.newell_octant(*n, *d)
    ref = O.demag_fft(N6, MAT["Ms"], m)
    got = gpu_demag({"n": n, "d": d}, MAT, m, prec)
    assert rel_max(got, ref) < tol


@functools.lru_cache(maxsize=None)
def _large_case():
    n, d = (16, 64, 32), (2e-9, 2e-9, 2e-9)
    m = W.m_vortex(n, d, seed=1)
    N6 = O.newell_octant(*n, *d)
    return n, d, m, O.demag_fft(N6, MAT["Ms"], m)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_large_column_uses_split_path_and_matches_oracle(prec, tol):
    """16 x 64 x 32: the padded y-z column (128 x 64 x 3 complex words)
    exceeds one CTA's shared-memory budget, so the split path runs without
    being forced."""
    n, d, m, ref = _large_case()
    got = gpu_demag({"n": n, "d": d}, MAT, m, prec)
    assert rel_max(got, ref) < tol


def test_live_contexts_of_one_length_keep_their_shared_memory():
    """Two live FP32 contexts whose fused y-z pass has the same transform
    length (Py = 128) but different shared-memory needs (110 KB for nz = 16,
    55 KB for nz = 8): creating the smaller one after the larger must not
    lower the kernel's limit under the larger one."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import gpu_context
    d = (2e-9, 2e-9, 2e-9)
    big = gpu_context({"n": (8, 64, 16), "d": d}, MAT, {}, {"method": "RK4", "h": 1e-13}, "fp32")
    small = gpu_context({"n": (8, 64, 8), "d": d}, MAT, {}, {"method": "RK4", "h": 1e-13}, "fp32")
    try:
        for ctx, n in ((big, (8, 64, 16)), (small, (8, 64, 8)), (big, (8, 64, 16))):
            m = W.m_random(n, seed=5)
            ref = O.demag_fft(O.newell_octant(*n, *d), MAT["Ms"], m)
            m_t = torch.from_numpy(m).to("cuda", torch.float32)
            H_t = torch.empty_like(m_t)
            ctx.demag(m_t, H_t)
            torch.cuda.synchronize()
            assert rel_max(H_t.double().cpu().numpy(), ref) < 1e-5
    finally:
        big.close()
        small.close()


# more shapes of the split passes, forced (FP32): y lengths 128-512, z lengths 4-32
SPLIT_SHAPES = [((16, 64, 4), (2e-9, 2e-9, 1e-9)), ((4, 64, 2), (1e-9, 3e-9, 2e-9)),
                ((8, 128, 16), (2e-9, 2e-9, 2e-9)), ((2, 256, 8), (1e-9, 1e-9, 1e-9)),
                ((32, 64, 8), (3e-9, 2e-9, 1e-9))]


def _launches_of_one_demag(n, d, m, prec):
    torch = pytest.importorskip("torch")
    from gpu_util import gpu_context
    ctx = gpu_context({"n": n, "d": d}, MAT, {}, {"method": "RK4", "h": 1e-13}, prec)
    try:
        dt = torch.float64 if prec == "fp64" else torch.float32
        m_t = torch.from_numpy(np.ascontiguousarray(m)).to("cuda", dt)
        H_t = torch.empty_like(m_t)
        before = ctx.stats()["kernel_launches"]
        ctx.demag(m_t, H_t)
        torch.cuda.synchronize()
        return H_t.double().cpu().numpy(), ctx.stats()["kernel_launches"] - before
    finally:
        ctx.close()


@pytest.mark.parametrize("n,d", SPLIT_SHAPES)
def test_forced_split_passes_match_oracle_fp32(n, d, monkeypatch):
    """XF, YF, ZM, YI, XI (five launches) on meshes small enough for the oracle."""
    monkeypatch.setenv("MMX_FORCE_SPLIT", "1")
    m = W.m_random(n, seed=sum(n) + 11)
    ref = O.demag_fft(O.newell_octant(*n, *d), MAT["Ms"], m)
    got, launches = _launches_of_one_demag(n, d, m, "fp32")
    assert launches == 5
    assert rel_max(got, ref) < 1e-5


def test_large_column_fp32_split_path_matches_oracle():
    """16 x 128 x 16: the y-z column (256 x 32 x 3 complex words, 221 KB)
    does not fit one CTA, so the split passes run it (five launches)."""
    n, d = (16, 128, 16), (2e-9, 2e-9, 2e-9)
    m = W.m_vortex(n, d, seed=2)
    ref = O.demag_fft(O.newell_octant(*n, *d), MAT["Ms"], m)
    got, launches = _launches_of_one_demag(n, d, m, "fp32")
    assert launches == 5 and rel_max(got, ref) < 1e-5
    got, launches = _launches_of_one_demag(n, d, m, "fp64")
    assert launches == 5 and rel_max(got, ref) < 1e-12


@pytest.mark.parametrize("env", [{"MMX_AUTOTUNE": "0"}, {"MMX_NO_TMA": "1"}, {"MMX_TROWS": "2"},
                                 {"MMX_TROWS": "4"}, {"MMX_TROWS": "8"}, {"MMX_TROWS": "16"}])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_each_pass_configuration_matches_oracle(env, prec, tol, monkeypatch):
    """Every configuration the autotuner chooses from, forced one at a time:
    x rows per CTA 2..16, XI with or without TMA tile copies."""
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    for n, d in (((32, 16, 4), (2e-9, 3e-9, 1e-9)), ((64, 32, 1), (4e-9, 4e-9, 4e-9))):
        m = W.m_random(n, seed=sum(n) + 3)
        ref = O.demag_fft(O.newell_octant(*n, *d), MAT["Ms"], m)
        got = gpu_demag({"n": n, "d": d}, MAT, m, prec)
        assert rel_max(got, ref) < tol


def test_autotuned_plan_is_reported():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import gpu_context
    ctx = gpu_context({"n": (64, 32, 2), "d": (4e-9,) * 3}, MAT, {}, {"method": "RK4", "h": 1e-13}, "fp32")
    try:
        p = ctx.plan()
        assert p["tuned"] == 1 and p["demag_us"] > 0
        assert p["yz_pass"] == 0 and p["kernels_per_demag"] == 3 and p["x_rows"] in (2, 4, 8, 16)
    finally:
        ctx.close()
    big = gpu_context({"n": (16, 128, 16), "d": (2e-9,) * 3}, MAT, {}, {"method": "RK4", "h": 1e-13}, "fp32")
    try:
        p = big.plan()
        assert p["yz_pass"] == 1 and p["kernels_per_demag"] == 5
    finally:
        big.close()


def test_bounded_tma_wait_runs_out_and_is_reported(monkeypatch):
    """Failure path of the TMA passes, without a GPU fault: with the test
    switch MMX_TEST_STALL_TMA the XI tile copies announce 16 bytes more than
    they bring, so every mbarrier wait runs out after its 20 ms limit; the
    kernel sets the context's fault word and returns, the host reports
    MMX_ERR_CUDA, and the CUDA context stays usable."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2107_06729_gb300 as pkg
    from gpu_util import gpu_context
    n, d = (64, 32, 2), (4e-9, 4e-9, 4e-9)
    monkeypatch.setenv("MMX_AUTOTUNE", "0")
    monkeypatch.setenv("MMX_TEST_STALL_TMA", "1")
    ctx = gpu_context({"n": n, "d": d}, MAT, {}, {"method": "RK4", "h": 1e-13}, "fp32")
    try:
        assert ctx.plan()["xi_tma"] == 1
        m = torch.from_numpy(W.m_random(n, seed=9)).to("cuda", torch.float32)
        H = torch.empty_like(m)
        ctx.demag(m, H)
        with pytest.raises(pkg.MMXError) as ei:
            ctx.stats()
        assert ei.value.code == pkg.MMX_ERR_CUDA and "bounded device wait" in str(ei.value)
        x = torch.ones(4, device="cuda")
        assert float((2 * x).sum()) == 8.0
    finally:
        ctx.close()
    monkeypatch.delenv("MMX_TEST_STALL_TMA")
    m = W.m_random(n, seed=9)
    ref = O.demag_fft(O.newell_octant(*n, *d), MAT["Ms"], m)
    assert rel_max(gpu_demag({"n": n, "d": d}, MAT, m, "fp32"), ref) < 1e-5


def test_bounded_wait_fault_stops_an_integration(monkeypatch):
    """The controller ends a run as soon as any kernel of the attempt has set
    the context's fault word (the demag passes' and the learned residual's
    tensor copies and tensor-core waits all report there): with the stall
    switch of the TMA x-inverse pass, mmx_run returns MMX_ERR_CUDA after its
    first attempt instead of integrating on with stale fields."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2107_06729_gb300 as pkg
    from gpu_util import gpu_context
    n, d = (64, 32, 2), (4e-9, 4e-9, 4e-9)
    monkeypatch.setenv("MMX_AUTOTUNE", "0")
    monkeypatch.setenv("MMX_TEST_STALL_TMA", "1")
    integ = {"method": "RKDP54", "extrap_order": 4, "adaptive": True, "h": 1e-13, "tol": 1e-5}
    mat = dict(MAT, A=1.3e-11, alpha=0.02)
    ctx = gpu_context({"n": n, "d": d}, mat, {}, integ, "fp32")
    try:
        assert ctx.plan()["xi_tma"] == 1
        ctx.set_m(torch.from_numpy(W.m_random(n, seed=4)).to("cuda", torch.float32))
        with pytest.raises(pkg.MMXError) as ei:
            ctx.run(1e-12)
        assert ei.value.code == pkg.MMX_ERR_CUDA and "bounded device wait" in str(ei.value)
        x = torch.ones(4, device="cuda")
        assert float((2 * x).sum()) == 8.0
    finally:
        ctx.close()
