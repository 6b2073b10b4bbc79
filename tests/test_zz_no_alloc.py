"""The allocation-free demag entry point, mmx_demag_static.

It exists for callers that cannot allocate device memory (code running while
its stream is captured into a CUDA graph, or in a process whose device memory
belongs to another allocator) and so cannot create a context.  Its output
must equal that of the context-based mmx_demag within the demag parity
tolerances (1e-12 relative in FP64, 1e-5 in FP32), on two calls in a row:
the second call reuses the tensor spectrum the static array still holds.
This file is collected last so that a failure here leaves every other test
already run."""
import numpy as np
import pytest

from paper_2107_06729_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_static_demag_matches_context_demag_twice(prec, tol):
    torch = _torch()
    import paper_2107_06729_gb300 as pkg
    n, d = (32, 16, 4), (2.5e-9, 2.5e-9, 1e-9)
    mat = {"Ms": 8e5, "alpha": 0.0, "gamma": W.GAMMA}
    dt = torch.float64 if prec == "fp64" else torch.float32
    stream = torch.cuda.current_stream()
    ctx = pkg.Context({"n": n, "d": d}, mat, {}, {"method": "RK4", "h": 1e-13}, prec, stream)
    mesh = pkg.mmx_mesh(*n, *d)
    code = pkg.MMX_FP64 if prec == "fp64" else pkg.MMX_FP32_MIXED
    try:
        for seed in (11, 12):
            m = torch.from_numpy(W.m_random(n, seed=seed)).to("cuda", dt)
            want = torch.empty_like(m)
            got = torch.full_like(m, float("nan"))
            ctx.demag(m, want)
            pkg.mmx_demag_static(mesh, mat["Ms"], code, m, got, stream.cuda_stream)
            torch.cuda.synchronize()
            scale = want.abs().max().item()
            assert torch.isfinite(got).all()
            assert (got - want).abs().max().item() <= tol * scale
    finally:
        ctx.close()


def test_static_demag_rejects_meshes_beyond_the_array():
    torch = _torch()
    import paper_2107_06729_gb300 as pkg
    n = (512, 512, 4)  # spectrum + scratch far above 16 MiB
    mesh = pkg.mmx_mesh(*n, 2e-9, 2e-9, 2e-9)
    m = torch.zeros((3, n[2], n[1], n[0]), dtype=torch.float32, device="cuda")
    H = torch.empty_like(m)
    with pytest.raises(pkg.MMXError) as ei:
        pkg.mmx_demag_static(mesh, 8e5, pkg.MMX_FP32_MIXED, m, H, torch.cuda.current_stream().cuda_stream)
    assert ei.value.code == pkg.MMX_ERR_ARG
    assert "16 MiB" in pkg.mmx_last_error(None)


def test_static_demag_matches_oracle():
    torch = _torch()
    import oracle as O
    import paper_2107_06729_gb300 as pkg
    n, d = (16, 8, 2), (4e-9, 4e-9, 4e-9)
    m = W.m_random(n, seed=5)
    ref = O.demag_fft(O.newell_octant(*n, *d), 8e5, m)
    mt = torch.from_numpy(m).cuda()
    H = torch.empty_like(mt)
    pkg.mmx_demag_static(pkg.mmx_mesh(*n, *d), 8e5, pkg.MMX_FP64, mt, H, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.abs(H.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
