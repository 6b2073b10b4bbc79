"""Batched ensembles (mmx_batch_*): members of uneven size, method, order
and precision advanced by one graph launch give, member by member, exactly
what their own mmx_run gives (same kernels, same per-member controller, so
the comparison is bitwise); an FP64 member matches the CPU oracle step for
step; idle members stay untouched; a failing member does not stop the rest."""
import numpy as np
import pytest

from paper_2107_06729_gb300 import workloads as W
from gpu_util import oracle_run, torch_cuda

pytestmark = pytest.mark.gpu

FLD = {"H0": tuple(W.mT((-24.6, 4.3, 0.0))), "pulse": tuple(W.mT((0.0, 20.0, 0.0))),
       "t_on": 1e-12, "t_off": 3e-12}


def _mat(Ms, alpha):
    return {"Ms": Ms, "A": 1.3e-11, "K": 2e4, "ku": (1.0, 0.0, 0.0), "alpha": alpha, "gamma": W.GAMMA}


def _adaptive(method, p):
    return {"method": method, "extrap_order": p, "adaptive": True, "h": 1e-13, "tol": 1e-5}


# uneven members: mesh, material, integrator, precision, t_end
MEMBERS = [
    ((32, 32, 1), _mat(8e5, 0.02), _adaptive("RKF45", 4), "fp32", 6e-12),
    ((64, 32, 2), _mat(1.1e6, 0.05), _adaptive("RKF45", 4), "fp32", 4e-12),
    ((16, 128, 1), _mat(5e5, 0.01), _adaptive("RKDP54", 4), "fp32", 5e-12),
    ((128, 64, 2), _mat(9e5, 0.08), _adaptive("RK23", 2), "fp32", 3e-12),
    ((16, 8, 2), _mat(8e5, 0.02), _adaptive("RKF45", 4), "fp64", 5e-12),
    ((32, 16, 1), _mat(7e5, 0.03), {"method": "RK4", "extrap_order": -1, "adaptive": False, "h": 1e-13}, "fp64",
     2e-12),
    ((8, 8, 4), _mat(8e5, 0.02), _adaptive("RKDP54", -1), "fp32", 4e-12),
]


def _m0(i, n):
    return W.m_uniform_noise(n, seed=100 + i, noise=0.2)


def _contexts(torch, members):
    import paper_2107_06729_gb300 as pkg
    out = []
    for i, (n, mat, integ, prec, _) in enumerate(members):
        ctx = pkg.Context({"n": n, "d": (4e-9, 4e-9, 4e-9)}, mat, FLD, integ, prec, torch.cuda.current_stream())
        dt = torch.float64 if prec == "fp64" else torch.float32
        ctx.set_m(torch.from_numpy(_m0(i, n)).to("cuda", dt))
        out.append(ctx)
    return out


def _state(torch, ctx):
    out = torch.empty(ctx.shape, dtype=getattr(torch, ctx.dtype_name), device="cuda")
    ctx.get_m(out)
    return out.cpu().numpy(), ctx.stats()


def _close(ctxs):
    for c in ctxs:
        c.close()


COUNTERS = ("t", "h", "accepted", "rejected", "exact_evals", "extrap_evals", "forced_accepts", "attempts")


def test_batch_equals_member_runs_bitwise():
    torch = torch_cuda()
    import paper_2107_06729_gb300 as pkg
    solo = _contexts(torch, MEMBERS)
    batch_ctx = _contexts(torch, MEMBERS)
    try:
        for ctx, mem in zip(solo, MEMBERS):
            ctx.run(mem[4])
        b = pkg.Batch(batch_ctx, torch.cuda.current_stream())
        rc, status = b.run([mem[4] for mem in MEMBERS])
        assert rc == 0 and status == [0] * len(MEMBERS)
        for i, (cs, cb) in enumerate(zip(solo, batch_ctx)):
            ms, ss = _state(torch, cs)
            mb, sb = _state(torch, cb)
            assert np.array_equal(ms, mb), i
            for k in COUNTERS:
                assert ss[k] == sb[k], (i, k)
            assert sb["t"] == MEMBERS[i][4]
        b.close()
    finally:
        _close(solo + batch_ctx)


def test_repeated_batch_runs_continue_like_chunked_member_runs():
    """Two launches of the same (cached) batch graph to t1 then t2, with a
    different end time per member, against each member's own two runs."""
    torch = torch_cuda()
    import paper_2107_06729_gb300 as pkg
    mems = MEMBERS[:4]
    solo = _contexts(torch, mems)
    batch_ctx = _contexts(torch, mems)
    try:
        b = pkg.Batch(batch_ctx)
        for frac in (0.4, 1.0):
            t = [frac * mem[4] for mem in mems]
            for ctx, te in zip(solo, t):
                ctx.run(te)
            b.run(t)
        for cs, cb in zip(solo, batch_ctx):
            ms, ss = _state(torch, cs)
            mb, sb = _state(torch, cb)
            assert np.array_equal(ms, mb)
            assert ss["accepted"] == sb["accepted"] and ss["rejected"] == sb["rejected"]
        b.close()
    finally:
        _close(solo + batch_ctx)


def test_fp64_member_matches_oracle_step_for_step():
    torch = torch_cuda()
    import paper_2107_06729_gb300 as pkg
    ctxs = _contexts(torch, MEMBERS)
    try:
        b = pkg.Batch(ctxs)
        b.run([mem[4] for mem in MEMBERS])
        i = 4
        n, mat, integ, _, t_end = MEMBERS[i]
        got, gs = _state(torch, ctxs[i])
        ref, rs = oracle_run({"n": n, "d": (4e-9, 4e-9, 4e-9)}, mat, FLD, integ, _m0(i, n), t_end)
        assert gs["accepted"] == rs["accepted"] and gs["rejected"] == rs["rejected"]
        assert gs["exact_evals"] == rs["exact_evals"] and gs["extrap_evals"] == rs["extrap_evals"]
        assert np.abs(got - ref).max() < 1e-10
        b.close()
    finally:
        _close(ctxs)


def test_idle_member_is_untouched_and_reports_ok():
    torch = torch_cuda()
    import paper_2107_06729_gb300 as pkg
    mems = MEMBERS[:3]
    ctxs = _contexts(torch, mems)
    try:
        ctxs[1].run(2e-12)
        before_m, before_s = _state(torch, ctxs[1])
        b = pkg.Batch(ctxs)
        rc, status = b.run([3e-12, 1e-12, 3e-12])  # member 1 is already past 1 ps
        assert rc == 0 and status == [0, 0, 0]
        after_m, after_s = _state(torch, ctxs[1])
        assert np.array_equal(before_m, after_m)
        for k in COUNTERS:
            assert before_s[k] == after_s[k]
        assert ctxs[0].stats()["t"] == 3e-12 and ctxs[2].stats()["t"] == 3e-12
        b.close()
    finally:
        _close(ctxs)


def test_failing_member_is_reported_and_others_finish():
    torch = torch_cuda()
    import paper_2107_06729_gb300 as pkg
    mems = MEMBERS[:3]
    ctxs = _contexts(torch, mems)
    try:
        n = mems[1][0]
        m = _m0(1, n)
        m[0, 0, 1, 2] = np.nan  # planted on the host before upload
        ctxs[1].set_m(torch.from_numpy(m).to("cuda", torch.float32))
        b = pkg.Batch(ctxs)
        rc, status = pkg.mmx_batch_run(b.handle, [2e-12] * 3)
        assert rc == pkg.MMX_ERR_NONFINITE
        assert status == [0, pkg.MMX_ERR_NONFINITE, 0]
        assert "non-finite" in pkg.mmx_last_error(ctxs[1].handle)
        assert ctxs[0].stats()["t"] == 2e-12 and ctxs[2].stats()["t"] == 2e-12
        with pytest.raises(pkg.MMXError):
            b.run(3e-12)
        b.close()
    finally:
        _close(ctxs)


def test_duplicate_member_is_rejected():
    torch = torch_cuda()
    import paper_2107_06729_gb300 as pkg
    ctxs = _contexts(torch, MEMBERS[:1])
    try:
        with pytest.raises(pkg.MMXError) as ei:
            pkg.mmx_batch_create([ctxs[0].handle, ctxs[0].handle])
        assert ei.value.code == pkg.MMX_ERR_ARG
    finally:
        _close(ctxs)


def test_ensemble_workload_member_sample_matches_solo_runs():
    """The 64-film ensemble workload: a spread of 8 of its members (small to
    largest) run as one batch for 2 ps equal their own runs bitwise."""
    torch = torch_cuda()
    import paper_2107_06729_gb300 as pkg
    ens = W.ensemble_config3(seed=0)
    order = sorted(range(len(ens)), key=lambda i: np.prod(ens[i]["mesh"]["n"]))
    pick = [order[k] for k in np.linspace(0, len(ens) - 1, 8).astype(int)]

    def make(i):
        s = ens[i]
        ctx = pkg.Context(s["mesh"], s["material"], s["field"], s["integrator"], "fp32")
        ctx.set_m(torch.from_numpy(s["m0"]).to("cuda", torch.float32))
        return ctx

    solo = [make(i) for i in pick]
    bat = [make(i) for i in pick]
    try:
        for c in solo:
            c.run(2e-12)
        b = pkg.Batch(bat)
        b.run(2e-12)
        for cs, cb in zip(solo, bat):
            ms, ss = _state(torch, cs)
            mb, sb = _state(torch, cb)
            assert np.array_equal(ms, mb)
            assert ss["accepted"] == sb["accepted"]
        b.close()
    finally:
        _close(solo + bat)
