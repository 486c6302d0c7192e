"""Per-element tolerances of the surrogate MLP's GPU arithmetic against the
FP64 oracle (oracle/mlp.py).

Both sides round to bfloat16 at the same storage points (inputs, weights,
hidden activations, output gradient, backward gradients); the GPU differs
only by its FP32 arithmetic between them: tensor-core accumulation, the bias
add, GELU / GELU' with erff and expf, the backward epilogue's product.  Those
FP32 errors are propagated as per-element standard deviations, layer by
layer:

* a dot product of n terms: n * u * sum |terms| (u = 2^-24, with a factor 2
  for accumulation that is not round-to-nearest), plus the input deviations
  weighted by the other operand;
* GELU and GELU': their derivatives times the input deviation, plus a few
  FP32 ulps of evaluation;
* a bf16 storage point: the two sides store the same number unless their
  pre-rounding values straddle a rounding boundary, which happens with
  probability about 0.8 sigma / ulp and then costs one bf16 ulp, so the
  variance after it is sigma^2 + sigma * ulp.

An element passes when |gpu - oracle| <= 6 sigma (plus 1e-12 of the tensor's
largest magnitude).  A wrong element (a wrong GEMM tile, a swapped operand,
a dropped bias) lies far outside (checked on the CPU in test_oracle_mlp.py).
"""
import numpy as np

from oracle import mlp as ref

U32 = 2.0 ** -24        # FP32 unit roundoff
K_SIGMA = 6.0
L_DGELU = 0.80          # max |GELU''| = 2 phi(0)


def _acc(n, terms_abs):
    """FP32 accumulation error of an n-term sum whose |terms| sum to terms_abs."""
    return 2.0 * n * U32 * terms_abs


def _ulp_bf16(v):
    """Spacing of bf16 numbers at |v| (8 significant bits)."""
    m = np.maximum(np.abs(v), 2.0 ** -126)
    return 2.0 ** (np.floor(np.log2(m)) - 7)


def _store(sig, v):
    """Deviation after both sides round v (deviation sig) to bf16."""
    return np.sqrt(sig * sig + sig * _ulp_bf16(v))


def setup(B=600, n_in=12, width=256, depth=3, n_out=2, seed=0):
    rng = np.random.default_rng(seed)
    params = ref.init_params(n_in, width, depth, n_out, seed=seed)
    for W, b in params:
        b += 0.05 * rng.standard_normal(b.shape)
    x = rng.standard_normal((B, n_in)).astype(np.float32)
    t = rng.standard_normal((B, n_out)).astype(np.float32)
    return params, x, t


def forward_sigma(p16, cache, y):
    """Deviations of the stored activations (sa[l], layer inputs), the FP32
    pre-activations (sz[l]) and the output y."""
    sa = [np.zeros_like(cache[0][0])]
    sz = []
    for li, (W, b) in enumerate(p16):
        a, z = cache[li]
        s = np.sqrt((sa[li] ** 2) @ (W ** 2) + _acc(W.shape[0], np.abs(a) @ np.abs(W)) ** 2 + (U32 * np.abs(z)) ** 2)
        sz.append(s)
        if li < len(p16) - 1:
            v = ref.gelu(z)
            sv = np.sqrt((ref.gelu_grad(z) * s) ** 2 + (8 * U32 * (np.abs(v) + U32 * np.abs(z))) ** 2)
            sa.append(_store(sv, v))
    return sa, sz, np.sqrt(sz[-1] ** 2 + (U32 * np.abs(y)) ** 2)


def backward_sigma(p16, cache, sa, sz, s_dy, g_out):
    """Deviations of every weight and bias gradient: [(sW, sb)] per layer.
    s_dy is the deviation of the stored output gradient g_out (bf16)."""
    nl = len(p16)
    out = [None] * nl
    g, sg = g_out, s_dy
    for li in range(nl - 1, -1, -1):
        W, _ = p16[li]
        a, _ = cache[li]
        B = a.shape[0]
        sw = np.sqrt((sa[li] ** 2).T @ (g ** 2) + (a ** 2).T @ (sg ** 2) + (sa[li] ** 2).T @ (sg ** 2)
                     + _acc(B, np.abs(a).T @ np.abs(g)) ** 2)
        sb = np.sqrt((sg ** 2).sum(0) + _acc(B, np.abs(g).sum(0)) ** 2)
        out[li] = (sw, sb)
        if li > 0:
            zp = cache[li - 1][1]
            h = g @ W.T
            sh = np.sqrt((sg ** 2) @ (W ** 2).T + _acc(W.shape[1], np.abs(g) @ np.abs(W).T) ** 2)
            s = ref.gelu_grad(zp)
            ss = L_DGELU * sz[li - 1] + 16 * U32 * (1.0 + np.abs(zp))
            v = h * s
            sv = np.sqrt((sh * s) ** 2 + (h * ss) ** 2 + (2 * U32 * v) ** 2)
            g = ref.bf16(v)
            sg = _store(sv, v)
    return out


def output_grad_sigma(sy, dy):
    """Deviation of the stored output gradient bf16(2 (y - t) / (B n_out)):
    y's deviation, two FP32 products (the scale rounded to FP32), then bf16."""
    s = np.sqrt((2.0 * sy / dy.size) ** 2 + (4 * U32 * dy) ** 2)
    return _store(s, dy)


def outside(got, want, sigma):
    """Mask of elements whose deviation exceeds K_SIGMA sigma."""
    err = np.abs(np.asarray(got, np.float64) - want)
    return err > K_SIGMA * sigma + 1e-12 * (np.abs(want).max() + 1e-30)


def assert_within(got, want, sigma, what):
    bad = outside(got, want, sigma)
    err = np.abs(np.asarray(got, np.float64) - want)
    ratio = err / (K_SIGMA * sigma + 1e-300)
    assert not bad.any(), (f"{what}: {int(bad.sum())} of {bad.size} elements beyond {K_SIGMA:g} sigma; worst "
                           f"|err| {err.max():.3g}, worst err/bound {ratio.max():.3g}")
