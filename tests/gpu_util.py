"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
the oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle as O


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_context(mesh, mat, fld, integ, precision):
    torch = torch_cuda()
    import paper_2107_06729_gb300 as pkg
    return pkg.Context(mesh, mat, fld, integ, precision, torch.cuda.current_stream())


def gpu_demag(mesh, mat, m, precision):
    torch = torch_cuda()
    dt = torch.float64 if precision == "fp64" else torch.float32
    ctx = gpu_context(mesh, mat, {}, {"method": "RK4", "h": 1e-13}, precision)
    try:
        m_t = torch.from_numpy(np.ascontiguousarray(m)).to("cuda", dt)
        H_t = torch.empty_like(m_t)
        ctx.demag(m_t, H_t)
        torch.cuda.synchronize()
        return H_t.double().cpu().numpy()
    finally:
        ctx.close()


def gpu_run(mesh, mat, fld, integ, m0, t_end, precision="fp64", chunks=1):
    torch = torch_cuda()
    dt = torch.float64 if precision == "fp64" else torch.float32
    ctx = gpu_context(mesh, mat, fld, integ, precision)
    try:
        m_t = torch.from_numpy(np.ascontiguousarray(m0)).to("cuda", dt)
        ctx.set_m(m_t)
        for k in range(1, chunks + 1):
            ctx.run(t_end * k / chunks)
        out = torch.empty_like(m_t)
        ctx.get_m(out)
        return out.double().cpu().numpy(), ctx.stats()
    finally:
        ctx.close()


def oracle_run(mesh, mat, fld, integ, m0, t_end, N6=None):
    sim = O.Simulation(mesh, mat, fld, integ, m0, N6=N6)
    sim.run(t_end)
    out = sim.m(), sim.stats()
    sim.close()
    return out


def rel_max(a, b):
    return np.abs(a - b).max() / np.abs(b).max()
