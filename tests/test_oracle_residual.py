"""Pins for the oracle of the learned residual net (oracle/residual.py):
BF16 rounding against torch's conversion and hand values, the convolution
against scipy.ndimage.correlate and the single-cell case, the backward pass
against central finite differences, Adam's first step against its closed
form, and the training pair against an exactly extrapolated field."""
import numpy as np
import pytest

import oracle as O
from oracle import residual as R
from paper_2107_06729_gb300 import workloads as W


def test_param_count_and_layout_match_the_generator():
    p = W.rnet_params(0)
    assert p.size == R.param_count() == 63171
    layers = R.unpack(p)
    assert [w.shape for w, _ in layers] == [(27, 32, 6), (27, 32, 32), (27, 32, 32), (27, 3, 32)]


def test_bf16_round_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-30, 30, 20000)).astype(np.float32)
    # exact ties: 8 random bits of mantissa followed by a 1 and zeros
    ties = (np.float32(1.0) + rng.integers(0, 256, 2000).astype(np.float32) / 128 + np.float32(2.0 ** -8))
    x = np.concatenate([x, ties.astype(np.float32), -ties.astype(np.float32), [0.0, -0.0, 1e-40, -3e-39]])
    x = x.astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(R.bf16_round(x), want)
    assert R.bf16_round(1 + 2.0 ** -8) == 1.0                        # tie -> even (down)
    assert R.bf16_round(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6          # tie -> even (up)
    assert R.bf16_round(1 + 2.0 ** -8 + 2.0 ** -20) == 1 + 2.0 ** -7  # above the tie


def test_conv3d_matches_scipy_correlate():
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(2)
    ci, co = 3, 2
    A = rng.standard_normal((ci, 3, 4, 5))
    Wt = rng.standard_normal((27, co, ci))
    b = rng.standard_normal(co)
    got = R.conv3d(A, Wt, b)
    for o in range(co):
        want = b[o] + sum(nd.correlate(A[c], Wt[:, o, c].reshape(3, 3, 3), mode="constant", cval=0.0)
                          for c in range(ci))
        assert np.abs(got[o] - want).max() < 1e-12


def test_conv3d_single_cell_is_the_centre_tap():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((4, 1, 1, 1))
    Wt = rng.standard_normal((27, 5, 4))
    b = rng.standard_normal(5)
    got = R.conv3d(A, Wt, b)[:, 0, 0, 0]
    assert np.allclose(got, Wt[13] @ A[:, 0, 0, 0] + b, rtol=0, atol=1e-13)
    assert R.TAPS[13] == (0, 0, 0)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(4)
    shape = (2, 3, 4)
    p = W.rnet_params(5, out_scale=1.0).astype(np.float64)
    x = rng.standard_normal((6,) + shape)
    target = rng.standard_normal((3,) + shape) * 0.1
    acts = R.forward(x, p, quantize=False)
    g = R.backward(acts, p, target, quantize=False)
    # indices from every layer's weights and biases
    offs, idx = 0, []
    for ci, co, _ in R.LAYERS:
        nW = 27 * co * ci
        idx += list(rng.integers(offs, offs + nW, 8)) + list(rng.integers(offs + nW, offs + nW + co, 2))
        offs += nW + co
    eps = 1e-6
    gmax = np.abs(g).max()
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (R.loss(R.forward(x, pp, False)[-1], target) - R.loss(R.forward(x, pm, False)[-1], target)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * gmax + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(6)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr = 1e-3
    p1, m1, v1 = R.adam(p, g, np.zeros(50), np.zeros(50), 1, lr)
    assert np.allclose(m1, 0.1 * g, rtol=1e-15, atol=0)
    assert np.allclose(v1, 0.001 * g * g, rtol=1e-13, atol=0)
    # bias-corrected moments are g and g^2: the step is lr g / (|g| + eps)
    assert np.allclose(p1, p - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_residual_sample_is_zero_for_an_exactly_extrapolated_field(p):
    """A non-self field polynomial of degree p in time is extrapolated
    exactly by Eq. 6 with p+1 nodes: the target vanishes and the input's
    field channels equal G(t)/Ms."""
    rng = np.random.default_rng(7 + p)
    shape = (3, 2, 4, 8)
    coef = [rng.standard_normal(shape) * 1e5 for _ in range(p + 1)]
    Ms = 8e5

    def G(t):
        return sum(c * (t * 1e12) ** k for k, c in enumerate(coef))

    t_nodes = np.cumsum(rng.uniform(0.5e-13, 2e-13, p + 1))
    t = t_nodes[-1] + 0.7e-13
    m = W.m_uniform_noise(shape[1:][::-1], seed=1)
    x, target = R.residual_sample([G(ti) for ti in t_nodes], t_nodes, G(t), m, t, Ms, O.lagrange_weights)
    assert x.shape == (6,) + shape[1:] and target.shape == shape
    scale = np.abs(G(t)).max() / Ms
    assert np.abs(target).max() < 1e-9 * scale
    assert np.array_equal(x[:3], m)
    assert np.abs(x[3:] - G(t) / Ms).max() < 1e-9 * scale


def test_backward_gradient_rounding_only_enters_the_input_gradient():
    """quantize_grad rounds the output gradient where it enters the
    input-gradient convolution: the last layer's gradient is unchanged, the
    earlier ones move by a few BF16 units at most."""
    rng = np.random.default_rng(12)
    shape = (2, 3, 4)
    p = W.rnet_params(13, out_scale=1.0).astype(np.float64)
    x = rng.standard_normal((6,) + shape)
    target = rng.standard_normal((3,) + shape) * 0.1
    acts = R.forward(x, p)
    g0 = R.backward(acts, p, target)
    g1 = R.backward(acts, p, target, quantize_grad=True)
    n3 = 27 * 3 * 32 + 3
    assert np.array_equal(g0[-n3:], g1[-n3:])
    assert not np.array_equal(g0[:-n3], g1[:-n3])
    assert np.abs(g1 - g0).max() <= 2 ** -6 * np.abs(g0).max()
