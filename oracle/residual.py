"""CPU FP64 oracle of the learned residual correction of the extrapolated
demag field.  TEST INFRASTRUCTURE ONLY: only tests/,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import it.

The paper has no learned component: its method stops at the polynomial
extrapolation of the non-self demag field (Sec. II, Eq. 6).  The residual
net is this project's extension of that step, defined here and only here
for the parity tests:

* input  x  = (m, G_ext / Ms), 6 channels on the mesh [6, nz, ny, nx]: the
  stage magnetisation and the extrapolated non-self field of Eq. 6;
* output r  = (G - G_ext) / Ms, 3 channels: the extrapolation's error, so
  that G_ext + Ms r is the corrected non-self field;
* four 3x3x3 cross-correlation layers with zero padding ("same" size),
  6 -> 32 -> 32 -> 32 -> 3 channels, a bias per output channel, ReLU after
  the first three;
* BF16 quantisation points (round to nearest, ties to even, of the FP32
  value): the input x, every weight, and the output of each hidden layer
  after its ReLU; accumulation is exact (FP64) here, the last layer's
  output is not rounded;
* training loss: the mean over cells and the 3 channels of (r - target)^2;
  gradients treat the BF16 roundings as the identity (straight-through) and
  use the rounded weights and stored activations; with the tensor-core
  backward the output gradient of each layer is rounded to BF16 where it
  enters the input-gradient convolution (``quantize_grad``); Adam (Kingma and Ba,
  2015: beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected moments) updates
  the FP32 master parameters.

Parameter layout (flat vector): for each layer, W[27][cout][cin] then
b[cout]; tap t = (tz*3 + ty)*3 + tx reads the input at (z+tz-1, y+ty-1,
x+tx-1).

Pins (tests/test_oracle_residual.py): ``bf16_round`` against torch's
bfloat16 conversion and hand values; ``conv3d`` against
scipy.ndimage.correlate and the single-cell case; ``backward`` against
central finite differences of ``loss`` (unquantised); ``adam``'s first step
against its closed form; ``residual_sample`` against the case where the
extrapolation is exact (a field linear in time extrapolated with p >= 1).
"""
import numpy as np

LAYERS = ((6, 32, True), (32, 32, True), (32, 32, True), (32, 3, False))  # (cin, cout, relu)
TAPS = tuple((tz - 1, ty - 1, tx - 1) for tz in range(3) for ty in range(3) for tx in range(3))


def param_count():
    return sum(27 * co * ci + co for ci, co, _ in LAYERS)


def unpack(params):
    """Flat parameter vector -> [(W [27, cout, cin], b [cout]), ...] (views)."""
    params = np.asarray(params, dtype=np.float64)
    out, o = [], 0
    for ci, co, _ in LAYERS:
        W = params[o:o + 27 * co * ci].reshape(27, co, ci)
        o += 27 * co * ci
        b = params[o:o + co]
        o += co
        out.append((W, b))
    assert o == params.size
    return out


def bf16_round(x):
    """x (values exactly representable in FP32, or first rounded to FP32)
    rounded to the nearest BF16 value, ties to even; returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


def shift(A, dz, dy, dx):
    """B[..., z, y, x] = A[..., z+dz, y+dy, x+dx], zero where that is
    outside the mesh."""
    B = np.zeros_like(A)
    nz, ny, nx = A.shape[-3:]

    def rng(d, n):
        return slice(max(0, -d), min(n, n - d)), slice(max(0, d), min(n, n + d))

    (oz, iz), (oy, iy), (ox, ix) = rng(dz, nz), rng(dy, ny), rng(dx, nx)
    B[..., oz, oy, ox] = A[..., iz, iy, ix]
    return B


def conv3d(A, W, b):
    """out[o] = b[o] + sum_t sum_c W[t, o, c] A[c] shifted by tap t."""
    co = W.shape[1]
    out = np.broadcast_to(np.asarray(b, dtype=np.float64).reshape(co, 1, 1, 1), (co,) + A.shape[1:]).copy()
    for t, (dz, dy, dx) in enumerate(TAPS):
        out += np.einsum("oc,czyx->ozyx", W[t], shift(A, dz, dy, dx))
    return out


def forward(x, params, quantize=True):
    """Returns [a0, a1, a2, a3, r]: the (rounded) input of every layer and
    the output r [3, nz, ny, nx]."""
    q = bf16_round if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    a = q(x)
    acts = [a]
    layers = unpack(params)
    for (W, b), (_, _, relu) in zip(layers, LAYERS):
        z = conv3d(a, q(W), b)
        if relu:
            a = q(np.maximum(z, 0.0))
            acts.append(a)
        else:
            acts.append(z)
    return acts


def loss(r, target):
    return float(np.mean((np.asarray(r, dtype=np.float64) - target) ** 2))


def backward(acts, params, target, quantize=True, quantize_grad=False):
    """Gradient of ``loss(acts[-1], target)`` with respect to the flat
    parameters, given the activations of ``forward``.  With quantize_grad,
    the output gradient of each layer l > 0 is rounded to BF16 where it
    enters the input-gradient convolution (the tensor-core backward); the
    weight gradient uses it unrounded."""
    q = bf16_round if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    qg = bf16_round if quantize_grad else (lambda v: v)
    layers = unpack(params)
    r = acts[-1]
    dz = 2.0 * (r - target) / r.size
    grads = [None] * len(LAYERS)
    for l in range(len(LAYERS) - 1, -1, -1):
        A = acts[l]
        Wq = q(layers[l][0])
        dW = np.zeros_like(Wq)
        for t, (tz, ty, tx) in enumerate(TAPS):
            dW[t] = np.einsum("ozyx,czyx->oc", dz, shift(A, tz, ty, tx))
        db = dz.sum(axis=(1, 2, 3))
        grads[l] = (dW, db)
        if l > 0:
            dA = np.zeros_like(A)
            dzq = qg(dz)
            for t, (tz, ty, tx) in enumerate(TAPS):
                dA += np.einsum("oc,ozyx->czyx", Wq[t], shift(dzq, -tz, -ty, -tx))
            dz = dA * (A > 0)
    return np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])


def adam(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns (params, m, v)."""
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


def residual_sample(G_nodes, t_nodes, G_exact, m, t, Ms, lagrange_weights):
    """Training pair of the net at time t: x = (m, G_ext/Ms) and target
    (G_exact - G_ext)/Ms, where G_ext = sum_i L_i(t) G_i is Eq. 6's
    extrapolation of the non-self fields G_nodes[i] at times t_nodes[i]
    (weights from ``lagrange_weights(tau_nodes, tau)`` on tau = t - t0,
    t0 = t_nodes[-1])."""
    t0 = t_nodes[-1]
    w = lagrange_weights(np.asarray(t_nodes, dtype=np.float64) - t0, t - t0)
    G_ext = sum(wi * Gi for wi, Gi in zip(w, G_nodes))
    x = np.concatenate([np.asarray(m, dtype=np.float64), G_ext / Ms], axis=0)
    return x, (G_exact - G_ext) / Ms
