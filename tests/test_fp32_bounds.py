"""The error bound behind the heatbath's FP32 pre-decision, checked on the CPU.

The CUDA kernel decides most of Creutz's accept tests u1^2 <= 1 - b0^2 in FP32 and takes
an FP32 decision only when |u1^2 - (1 - b0^2)| > 2^-11, claiming the FP32 error of
1 - b0^2 = t (2 - t), t = -log1p(-u0 span) / alpha, stays below 2.2e-4 while
u0 span <= 1 - 2^-10 (the uniforms truncated to 24 bits, span = 1 - exp(-2 alpha)). This
test evaluates the same FP32 expression with numpy's float32 arithmetic (an independent
log1p / expm1 of comparable accuracy) on many random draws and checks the bound.
"""
import numpy as np


def _trunc24(u):
    """u rounded toward zero to 24 significant bits, as the kernel builds it."""
    m, e = np.frexp(u)
    return np.ldexp(np.floor(m * 2.0 ** 24) / 2.0 ** 24, e).astype(np.float32)


def test_fp32_predecision_error_bound():
    rng = np.random.default_rng(11)
    n = 400_000
    alpha = np.exp(rng.uniform(np.log(1e-6), np.log(60.0), n))
    u0 = (np.floor(rng.uniform(0, 2.0 ** 53, n)) + 1.0) * 2.0 ** -53
    span = -np.expm1(-2.0 * alpha)
    t = -np.log1p(-u0 * span) / alpha
    s2 = t * (2.0 - t)                               # exact 1 - b0^2 (FP64)
    af = alpha.astype(np.float32)
    span_f = (-np.expm1(np.float32(-2.0) * af)).astype(np.float32)
    xf = (_trunc24(u0) * span_f).astype(np.float32)
    ok = xf <= np.float32(1.0 - 2.0 ** -10)
    tf = (-np.log1p(-xf) / af).astype(np.float32)
    s2f = (tf * (np.float32(2.0) - tf)).astype(np.float32)
    err = np.abs(s2f[ok].astype(np.float64) - s2[ok])
    assert ok.mean() > 0.95
    assert err.max() < 2.2e-4, err.max()
    assert err.max() < 2.0 ** -11 / 2  # the margin leaves room to spare


def test_uniform_truncation():
    rng = np.random.default_rng(12)
    u = (np.floor(rng.uniform(0, 2.0 ** 53, 100_000)) + 1.0) * 2.0 ** -53
    rel = np.abs(_trunc24(u).astype(np.float64) - u) / u
    assert rel.max() < 2.0 ** -23
