"""GPU parity of the learned residual net (include/mmx_residual.h) against
the FP64 oracle (oracle/residual.py) on the same seeded inputs: the packed
BF16 input bit for bit, every layer's output within one BF16 rounding of
the exact value computed from the GPU's own layer input (the BF16 rounding
of the hidden outputs is a quantisation decision, so each layer is checked
from the same rounded input), the output within FP32 accumulation error,
the gradients and the Adam update of a training step, the training pairs
built from the exact demag, and the gain of the trained correction over
extrapolation alone on held-out states of a trajectory."""
import numpy as np
import pytest

import oracle as O
from oracle import residual as R
from paper_2107_06729_gb300 import workloads as W
from gpu_util import gpu_context, oracle_run, torch_cuda

pytestmark = pytest.mark.gpu

MAT = {"Ms": 8e5, "A": 1.3e-11, "K": 0.0, "ku": (1.0, 0.0, 0.0), "alpha": 0.02, "gamma": W.GAMMA}


def _input(n, seed):
    """x = (m, G_ext/Ms): a noisy uniform state and a field of demag scale."""
    nx, ny, nz = n
    rng = np.random.default_rng(np.random.PCG64(seed))
    m = W.m_uniform_noise(n, seed=seed, noise=0.3)
    g = rng.normal(0.0, 0.3, size=(3, nz, ny, nx))
    return np.concatenate([m, g]).astype(np.float32)


def _to_cf(a_cl, n, ch):
    nx, ny, nz = n
    return np.ascontiguousarray(a_cl[:, :ch].T.reshape(ch, nz, ny, nx)).astype(np.float64)


def _ulp_bf16(v):
    a = np.abs(v)
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    return np.where(a > 0, 2.0 ** (e - 7), 0.0)


def _net(torch, cells, params):
    import paper_2107_06729_gb300 as pkg
    return pkg.RNet(cells, params, torch.cuda.current_stream())


@pytest.mark.parametrize("n", [(40, 12, 3), (8, 8, 1), (64, 32, 4), (5, 3, 2), (1, 1, 1), (61, 9, 2)])
def test_forward_layer_by_layer_matches_oracle(n):
    """Every tcgen05 layer kernel, from meshes smaller than one tile to
    several tiles with ragged edges."""
    torch = torch_cuda()
    nx, ny, nz = n
    cells = nx * ny * nz
    params = W.rnet_params(seed=1, out_scale=1.0)
    x = _input(n, seed=2)
    net = _net(torch, cells, params)
    try:
        r = net.forward(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        acts = [net.activation(l, cells) for l in range(4)]
        r_gpu = r.cpu().numpy().astype(np.float64)
        assert np.array_equal(net.activation(4, cells), r.cpu().numpy().reshape(3, -1))
    finally:
        net.close()
    # packed input: the BF16 rounding of x, bit for bit, padding zero
    assert np.array_equal(_to_cf(acts[0], n, 6), R.bf16_round(x))
    assert not acts[0][:, 6:].any()
    layers = R.unpack(params.astype(np.float64))
    for l in range(4):
        ci, co, relu = R.LAYERS[l]
        A = _to_cf(acts[l], n, ci)
        Wq = R.bf16_round(layers[l][0])
        b = layers[l][1].astype(np.float32).astype(np.float64)
        exact = R.conv3d(A, Wq, b)
        mag = R.conv3d(np.abs(A), np.abs(Wq), np.abs(b))
        if relu:
            want = np.maximum(exact, 0.0)
            got = _to_cf(acts[l + 1], n, co)
            bound = _ulp_bf16(want) + 1e-5 * mag + 1e-30
            assert np.all(np.abs(got - want) <= bound), (l, np.abs(got - want).max())
        else:
            assert np.all(np.abs(r_gpu - exact) <= 1e-5 * mag + 1e-30), np.abs(r_gpu - exact).max()
    # the whole net against the oracle's own quantised forward (BF16 roundings
    # taken independently may differ by one unit and propagate)
    ref = R.forward(x.astype(np.float64), params.astype(np.float64))[-1]
    assert np.abs(r_gpu - ref).max() <= 3e-2 * np.abs(ref).max()


@pytest.mark.parametrize("n", [(24, 8, 2), (33, 5, 3)])
def test_train_step_gradient_and_adam_update_match_oracle(n):
    """The whole backward on the tensor cores: input gradients with the
    output gradient rounded to BF16 where it enters (the oracle's
    quantize_grad), weight gradients with the output gradient as a BF16 pair
    hi + lo (about 16 bits: the oracle's unrounded weight gradient within
    FP32-level error).  The last layer's output gradient is the same on both
    sides, so its weight gradient is held to 2e-5; the others inherit the
    input gradients' BF16 decisions."""
    torch = torch_cuda()
    nx, ny, nz = n
    cells = nx * ny * nz
    params = W.rnet_params(seed=3, out_scale=1.0)
    x = _input(n, seed=4)
    rng = np.random.default_rng(5)
    target = rng.normal(0.0, 0.5, size=(3, nz, ny, nx)).astype(np.float32)
    lr = 1e-3
    net = _net(torch, cells, params)
    try:
        loss = net.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(target).cuda(), lr)
        acts = [net.activation(l, cells) for l in range(4)]
        r = net.activation(4, cells).astype(np.float64).reshape(3, nz, ny, nx)
        g_gpu = net.grads().astype(np.float64)
        p1 = net.params().astype(np.float64)
    finally:
        net.close()
    assert loss == pytest.approx(R.loss(r, target), rel=1e-6)
    oacts = [_to_cf(acts[l], n, R.LAYERS[l][0]) for l in range(4)] + [r]
    g_ref = R.backward(oacts, params.astype(np.float64), target.astype(np.float64), quantize_grad=True)
    # FP32 accumulation; with BF16 gradients also the rare rounding decided
    # differently by the FP32 and FP64 sides (one unit, 2^-8, of one entry)
    off = 0
    for li, (ci, co, _) in enumerate(R.LAYERS):
        k = 27 * co * ci + co
        tol = 2e-5 if li == len(R.LAYERS) - 1 else 2e-3
        gl, rl = g_gpu[off:off + k], g_ref[off:off + k]
        assert np.abs(gl - rl).max() <= tol * np.abs(rl).max(), (ci, co, np.abs(gl - rl).max(), np.abs(rl).max())
        off += k
    # the update: Adam's first step from zero moments with the GPU's gradient
    want, _, _ = R.adam(params.astype(np.float64), g_gpu, np.zeros_like(g_gpu), np.zeros_like(g_gpu), 1, lr)
    assert np.abs(p1 - want).max() <= 1e-3 * lr + 1e-7


def test_training_fits_a_teacher_net():
    """Targets from a second (unquantised) net: 150 Adam steps cut the loss
    at least fourfold."""
    torch = torch_cuda()
    n = (32, 16, 2)
    nx, ny, nz = n
    x = _input(n, seed=6)
    teacher = W.rnet_params(seed=7, out_scale=1.0).astype(np.float64)
    target = R.forward(x.astype(np.float64), teacher, quantize=False)[-1].astype(np.float32)
    net = _net(torch, nx * ny * nz, W.rnet_params(seed=8))
    try:
        xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(target).cuda()
        losses = [net.train_step(xd, td, 2e-3) for _ in range(150)]
    finally:
        net.close()
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.25 * losses[0], (losses[0], losses[-1])


def _nonself_oracle(N6, Ms, m, N00):
    return O.demag_fft(N6, Ms, m) + Ms * N00.reshape(3, 1, 1, 1) * m


@pytest.mark.parametrize("prec,p", [("fp64", 2), ("fp64", 4), ("fp32", 3)])
def test_residual_sample_matches_oracle(prec, p):
    torch = torch_cuda()
    n, d = (16, 8, 2), (4e-9, 4e-9, 4e-9)
    nx, ny, nz = n
    dt = torch.float64 if prec == "fp64" else torch.float32
    ctx = gpu_context({"n": n, "d": d}, MAT, {}, {"method": "RK4", "h": 1e-13}, prec)
    nodes = [W.m_uniform_noise(n, seed=20 + j, noise=0.2) for j in range(p + 1)]
    m = W.m_uniform_noise(n, seed=40, noise=0.2)
    t_nodes = np.array([0.0, 0.9e-13, 2.1e-13, 2.9e-13, 4.2e-13, 5.0e-13][:p + 1])
    t = t_nodes[-1] + 1.1e-13
    try:
        md = torch.from_numpy(np.stack(nodes)).to("cuda", dt).contiguous()
        mt = torch.from_numpy(m).to("cuda", dt)
        x = torch.empty((6, nz, ny, nx), dtype=torch.float32, device="cuda")
        tg = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
        import paper_2107_06729_gb300 as pkg
        pkg.mmx_residual_sample(ctx.handle, p, md, t_nodes, mt, t, x, tg)
        torch.cuda.synchronize()
        xg, tgg = x.cpu().numpy().astype(np.float64), tg.cpu().numpy().astype(np.float64)
        # a misaligned node array is refused on the host
        bad = torch.empty(md.numel() + 1, dtype=dt, device="cuda")[1:]
        with pytest.raises(pkg.MMXError) as ei:
            pkg.mmx_residual_sample(ctx.handle, p, bad, t_nodes, mt, t, x, tg)
        assert ei.value.code == pkg.MMX_ERR_ARG
    finally:
        ctx.close()
    N6 = O.newell_octant(*n, *d)
    N00 = O.newell_entry(0, 0, 0, *d)[:3]
    Gs = [_nonself_oracle(N6, MAT["Ms"], mj, N00) for mj in nodes]
    x_ref, t_ref = R.residual_sample(Gs, t_nodes, _nonself_oracle(N6, MAT["Ms"], m, N00), m, t, MAT["Ms"],
                                     O.lagrange_weights)
    w = O.lagrange_weights(t_nodes - t_nodes[-1], t - t_nodes[-1])
    scale = np.abs(x_ref[3:]).max() * np.abs(w).sum()
    # the pair is stored in FP32: its rounding (2^-24 relative) comes on top
    # of the context precision's demag and sum errors
    tol = 1e-11 if prec == "fp64" else 1e-5
    f32 = 2.0 ** -24
    assert np.all(np.abs(xg[:3] - x_ref[:3]) <= f32 * np.abs(x_ref[:3]))
    assert np.abs(xg[3:] - x_ref[3:]).max() <= tol * scale + f32 * np.abs(x_ref[3:]).max()
    assert np.abs(tgg - t_ref).max() <= tol * scale + f32 * np.abs(t_ref).max()


def test_learned_correction_gain_over_extrapolation_alone():
    """States of an RKDP54 trajectory (FP64, 64 x 32 x 2 film, 20 mT pulse):
    pairs at the next step's start from p = 2 extrapolation of the last
    three; train on the first 70 %, measure on the last 30 %.  The gain is
    rms(G - G_ext) / rms(G - G_ext - Ms r)."""
    torch = torch_cuda()
    import paper_2107_06729_gb300 as pkg
    n, d = (64, 32, 2), (4e-9, 4e-9, 4e-9)
    nx, ny, nz = n
    fld = {"H0": tuple(W.mT((-24.6, 4.3, 0.0))), "pulse": tuple(W.mT((0.0, 20.0, 0.0))), "t_on": 0.0,
           "t_off": 1e-9}
    integ = {"method": "RKDP54", "extrap_order": 4, "adaptive": True, "h": 1e-13, "tol": 1e-5}
    ctx = gpu_context({"n": n, "d": d}, MAT, fld, integ, "fp64")
    p = 2
    try:
        m = torch.from_numpy(W.m_uniform_noise(n, seed=9, noise=0.3)).cuda()
        ctx.set_m(m)
        ts, ms = [0.0], [m.clone()]
        for _ in range(160):
            ctx.step(1)
            cur = torch.empty_like(m)
            ctx.get_m(cur)
            ts.append(ctx.stats()["t"])
            ms.append(cur)
        X, T = [], []
        for i in range(p, len(ms) - 1):
            nodes = torch.stack(ms[i - p:i + 1]).contiguous()
            x = torch.empty((6, nz, ny, nx), dtype=torch.float32, device="cuda")
            tg = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
            pkg.mmx_residual_sample(ctx.handle, p, nodes, ts[i - p:i + 1], ms[i + 1], ts[i + 1], x, tg)
            X.append(x)
            T.append(tg)
    finally:
        ctx.close()
    ntrain = int(0.7 * len(X))
    # scale the target so that the net's outputs are of order one
    s = float(torch.stack(T[:ntrain]).std())
    net = pkg.RNet(nx * ny * nz, W.rnet_params(seed=10), torch.cuda.current_stream())
    try:
        rng = np.random.default_rng(11)
        for it in range(1500):
            j = int(rng.integers(0, ntrain))
            net.train_step(X[j], T[j] / s, 1e-3 if it < 1000 else 3e-4)

        def gain(idx):
            num = den = 0.0
            for j in idx:
                r = net.forward(X[j]) * s
                den += float((T[j].double() ** 2).sum())
                num += float(((T[j] - r).double() ** 2).sum())
            return (den / num) ** 0.5

        g_train, g_test = gain(range(ntrain)), gain(range(ntrain, len(X)))
    finally:
        net.close()
    print("residual-net gain: train %.3f held-out %.3f (%d/%d pairs)" % (g_train, g_test, ntrain, len(X) - ntrain))
    assert np.isfinite(g_train) and np.isfinite(g_test)
    # measured on a GB300: 9.0 on the training pairs, 2.2 held out
    assert g_train > 2.0 and g_test > 1.3


def _film_run(torch, ctx, blob, t_end):
    """From the saved start state (time, step, history, counters) to t_end."""
    ctx.load_state(blob)
    ctx.run(t_end)
    out = torch.empty(ctx.shape, dtype=torch.float32, device="cuda")
    ctx.get_m(out)
    return out.double().cpu().numpy(), ctx.stats()


def test_residual_in_the_stage_loop():
    """mmx_set_residual: a zero net reproduces the plain extrapolated run
    (G_ext + Ms * 0 is G_ext, summed the same way), a small random net
    changes it slightly, detaching restores the plain run; invalid
    attachments are refused."""
    torch = torch_cuda()
    import paper_2107_06729_gb300 as pkg
    n = (32, 16, 2)
    nx, ny, nz = n
    mesh = {"n": n, "d": (4e-9, 4e-9, 4e-9)}
    fld = {"H0": tuple(W.mT((-24.6, 4.3, 0.0))), "pulse": tuple(W.mT((0.0, 20.0, 0.0))), "t_on": 1e-12,
           "t_off": 3e-12}
    integ = {"method": "RKDP54", "extrap_order": 4, "adaptive": True, "h": 1e-13, "tol": 1e-5}
    m0 = W.m_uniform_noise(n, seed=5, noise=0.2)
    ctx = gpu_context(mesh, MAT, fld, integ, "fp32")
    zero = pkg.RNet(nx * ny * nz, np.zeros(pkg.MMX_RNET_PARAMS, dtype=np.float32), torch.cuda.current_stream())
    small = pkg.RNet(nx * ny * nz, W.rnet_params(seed=6, out_scale=1e-3), torch.cuda.current_stream())
    try:
        ctx.set_m(torch.from_numpy(m0).to("cuda", torch.float32))
        blob = ctx.save_state()
        ref, rs = _film_run(torch, ctx, blob, 5e-12)
        ctx.set_residual(zero)
        got, gs = _film_run(torch, ctx, blob, 5e-12)
        if rs["rejected"] == 0:
            # no rejection, so no exact-demag fallback: the same attempts
            assert gs["accepted"] == rs["accepted"] and gs["rejected"] == 0
            assert gs["extrap_evals"] == rs["extrap_evals"] and gs["exact_evals"] == rs["exact_evals"]
            assert np.abs(got - ref).max() <= 1e-6
        else:
            # a rejected attempt is retried with exact demag at every stage
            assert ctx.residual_stats()["fallbacks"] >= 1
            assert np.abs(got - ref).max() <= 1e-4
        ctx.set_residual(small)
        per, ps = _film_run(torch, ctx, blob, 5e-12)
        d = np.abs(per - ref).max()
        assert np.all(np.isfinite(per)) and 0 < d < 1e-2, d
        ctx.set_residual(None)
        back, bs = _film_run(torch, ctx, blob, 5e-12)
        assert np.array_equal(back, ref) and bs["accepted"] == rs["accepted"]
        # refused: FP64 context, no extrapolation, a net for fewer cells
        c64 = gpu_context(mesh, MAT, fld, integ, "fp64")
        cfull = gpu_context(mesh, MAT, fld, dict(integ, extrap_order=-1), "fp32")
        tiny = pkg.RNet(8, None, torch.cuda.current_stream())
        try:
            for c, net in ((c64, zero), (cfull, zero), (ctx, tiny)):
                with pytest.raises(pkg.MMXError) as ei:
                    c.set_residual(net)
                assert ei.value.code == pkg.MMX_ERR_ARG
        finally:
            tiny.close()
            c64.close()
            cfull.close()
    finally:
        ctx.close()
        zero.close()
        small.close()


def test_net_refuses_invalid_calls_before_launching():
    torch = torch_cuda()
    import paper_2107_06729_gb300 as pkg
    net = pkg.RNet(64, W.rnet_params(0), torch.cuda.current_stream())
    try:
        x = torch.zeros((6, 2, 8, 8), dtype=torch.float32, device="cuda")  # 128 cells > 64
        with pytest.raises(pkg.MMXError) as ei:
            net.forward(x)
        assert ei.value.code == pkg.MMX_ERR_ARG and "out of range" in str(ei.value)
        x = torch.zeros((6, 1, 8, 8), dtype=torch.float32, device="cuda")
        t = torch.zeros((3, 1, 8, 8), dtype=torch.float32, device="cuda")
        with pytest.raises(pkg.MMXError) as ei:
            net.train_step(x, t, 0.0)
        assert ei.value.code == pkg.MMX_ERR_ARG
        net.forward(x)
        with pytest.raises(pkg.MMXError) as ei:
            pkg.mmx_rnet_get_activation(net.handle, 1, np.empty((64, 16), dtype=np.uint16))  # wrong size
        assert ei.value.code == pkg.MMX_ERR_ARG
        assert net.activation(1, 64).shape == (64, 32)
    finally:
        net.close()


# The tensor-core kernels are persistent: a CTA takes tile after tile, with
# the halo barrier's and the MMA barrier's parity alternating and the next
# tile's copies issued while the current one finishes.  The cases above fit
# one tile per CTA; these cap the grid (MMX_RNET_GRID_CAP) so that every CTA
# runs many tiles, and check the size the bench times.
def test_multi_tile_ctas_forward_and_gradient(monkeypatch):
    monkeypatch.setenv("MMX_RNET_GRID_CAP", "3")
    test_forward_layer_by_layer_matches_oracle((64, 32, 4))
    test_train_step_gradient_and_adam_update_match_oracle((33, 5, 3))
    monkeypatch.setenv("MMX_RNET_GRID_CAP", "1")
    test_train_step_gradient_and_adam_update_match_oracle((24, 8, 2))


def test_forward_at_the_timed_size_layer_by_layer(monkeypatch):
    """The 128 x 128 x 4 film the bench times, in its launch configuration
    (tcgen05 layers, persistent grid): every layer within one BF16 unit of
    the exact convolution of the GPU's own layer input, the output within
    FP32 accumulation error."""
    torch = torch_cuda()
    n = (128, 128, 4)
    nx, ny, nz = n
    cells = nx * ny * nz
    params = W.rnet_params(seed=0)
    x = _input(n, seed=0)
    net = _net(torch, cells, params)
    try:
        r = net.forward(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        acts = [net.activation(l, cells) for l in range(4)]
        r_gpu = r.cpu().numpy().astype(np.float64)
    finally:
        net.close()
    assert np.array_equal(_to_cf(acts[0], n, 6), R.bf16_round(x))
    layers = R.unpack(params.astype(np.float64))
    for l in range(4):
        ci, co, relu = R.LAYERS[l]
        A = _to_cf(acts[l], n, ci)
        Wq = R.bf16_round(layers[l][0])
        b = layers[l][1].astype(np.float32).astype(np.float64)
        exact = R.conv3d(A, Wq, b)
        mag = R.conv3d(np.abs(A), np.abs(Wq), np.abs(b))
        if relu:
            want = np.maximum(exact, 0.0)
            got = _to_cf(acts[l + 1], n, co)
            assert np.all(np.abs(got - want) <= _ulp_bf16(want) + 1e-5 * mag + 1e-30), l
        else:
            assert np.all(np.abs(r_gpu - exact) <= 1e-5 * mag + 1e-30)


def _fallback_film():
    n = (32, 16, 2)
    mesh = {"n": n, "d": (4e-9, 4e-9, 4e-9)}
    fld = {"H0": tuple(W.mT((-24.6, 4.3, 0.0))), "pulse": tuple(W.mT((0.0, 20.0, 0.0))), "t_on": 1e-12,
           "t_off": 3e-12}
    integ = {"method": "RKDP54", "extrap_order": 4, "adaptive": True, "h": 1e-13, "tol": 1e-5}
    return n, mesh, fld, integ, W.m_uniform_noise(n, seed=5, noise=0.2)


@pytest.mark.parametrize("check_every", [0, 1])
def test_exact_demag_fallback_replaces_a_failing_net(check_every):
    """A net whose correction is far off.  Without a periodic check, every
    attempt that uses it fails the error estimate and is retried with exact
    demag at every stage.  With a check after every accepted step (tolerance
    1e-2), the first check (due right after the priming steps) finds the net
    beyond tolerance and every later attempt runs with exact demag.  Either
    way the run ends finite and as accurate as an exact-demag integration:
    within 1e-3 of the FP64 oracle with full demag after 5 ps (two valid
    DP54 integrations at e_max 1e-5 differ by up to a few 1e-4 here); the
    counters show which fallback acted."""
    torch = torch_cuda()
    import paper_2107_06729_gb300 as pkg
    n, mesh, fld, integ, m0 = _fallback_film()
    ctx = gpu_context(mesh, MAT, fld, integ, "fp32")
    bad = pkg.RNet(int(np.prod(n)), W.rnet_params(seed=7, out_scale=50.0), torch.cuda.current_stream())
    try:
        ctx.set_residual(bad)
        ctx.set_residual_check(check_every, 1e-2)
        ctx.set_m(torch.from_numpy(m0).to("cuda", torch.float32))
        ctx.run(5e-12)
        out = torch.empty(ctx.shape, dtype=torch.float32, device="cuda")
        ctx.get_m(out)
        got = out.double().cpu().numpy()
        st = ctx.residual_stats()
        assert np.all(np.isfinite(got))
        if check_every == 0:
            assert st["fallbacks"] >= 1 and st["checks"] == 0 and st["net_ok"] == 1
            assert ctx.stats()["rejected"] >= st["fallbacks"]
        else:
            assert st["checks"] >= 1 and st["check_fails"] == st["checks"] and st["net_ok"] == 0
        ref, _ = oracle_run(mesh, MAT, fld, dict(integ, extrap_order=-1), m0, 5e-12)
        assert np.abs(got - ref).max() < 1e-3
    finally:
        ctx.close()
        bad.close()


def test_periodic_check_keeps_a_good_net():
    """A zero net (its correction is G_ext itself) under a periodic check
    every third accepted step at tolerance 5e-2: every check passes (the
    extrapolation's own error is far smaller), the net stays in use, and the
    run stays within 1e-4 of the plain extrapolated run (the checked
    attempts themselves run with exact demag)."""
    torch = torch_cuda()
    import paper_2107_06729_gb300 as pkg
    n, mesh, fld, integ, m0 = _fallback_film()
    ctx = gpu_context(mesh, MAT, fld, integ, "fp32")
    zero = pkg.RNet(int(np.prod(n)), np.zeros(pkg.MMX_RNET_PARAMS, dtype=np.float32), torch.cuda.current_stream())
    try:
        ctx.set_m(torch.from_numpy(m0).to("cuda", torch.float32))
        blob = ctx.save_state()
        ref, _ = _film_run(torch, ctx, blob, 5e-12)
        ctx.set_residual(zero)
        ctx.set_residual_check(3, 5e-2)
        got, gs = _film_run(torch, ctx, blob, 5e-12)
        st = ctx.residual_stats()
        assert st["checks"] >= 2 and st["check_fails"] == 0 and st["net_ok"] == 1
        assert np.abs(got - ref).max() <= 1e-4
    finally:
        ctx.close()
        zero.close()


def test_trained_net_error_and_speed_against_plain_extrapolation():
    """The learned residual in the integrator's own terms: a net trained on
    RK4 sub-step snapshots (the config-5 recipe of bench.residual_config5 at
    32 x 32 x 2) is attached to DP54 p = 4 (FP32, exact-demag fallback on)
    and compared with plain extrapolation at each e_max: Eq. 7 error against
    an FP64 full-demag run, and simulated ns/s.  The net must learn (loss
    falls, held-out gain > 1) and keep the run within the fallback's bound of
    the plain run's error; the speed at equal error is reported (the net's
    forward costs several exact demag evaluations of this mesh)."""
    import os
    import sys
    torch = torch_cuda()
    import paper_2107_06729_gb300 as pkg
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    res = bench.residual_config5(pkg, torch, torch.device("cuda", 0), n=(32, 32, 2), n_samples=480, epochs=2, lr=1e-3,
                                 tols=(1e-5, 3e-5), horizon_ps=5.0, seed=3)
    print("config-5 recipe at 32x32x2:", res["gain_held_out"], res["at_equal_error"], res["sweep"])
    assert res["samples"] == 480
    first, last = res["loss_first_last"]
    assert np.isfinite(first) and last < first
    assert res["gain_held_out"] > 1.0
    for plain, withnet in zip(res["sweep"]["extrapolated"], res["sweep"]["extrapolated_plus_net"]):
        assert plain["tol"] == withnet["tol"]
        assert np.isfinite(plain["eps"]) and np.isfinite(withnet["eps"])
        assert plain["ns_per_s"] > 0 and withnet["ns_per_s"] > 0
        # accepted steps all passed the same error test as the plain run's
        assert withnet["eps"] <= 3.0 * plain["eps"] + 1e-6
    eq = res["at_equal_error"]
    assert eq["net_ns_per_s"] > 0 and eq["plain_ns_per_s"] > 0
