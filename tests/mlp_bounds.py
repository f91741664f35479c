"""Error bounds for comparing the surrogate's tensor-core kernels with the
oracle (oracle/mlp.py).  Test infrastructure, used by tests/test_gpu_mlp.py.

Both sides take the same rounding points: BF16 weights and activations, FP32
accumulation of exact BF16 x BF16 products, FP32 bias, GELU and loss
arithmetic.  Two effects separate them, and each is bounded here:

1. FP32 accumulation order.  A K-term sum of exact products, added in any
   order with rounding or truncating FP32 adds, is within
   gamma_K = K 2^-23 of sum |a_k w_k| (the recursive-summation bound, with
   the unit roundoff 2^-24 doubled for truncation).  For K <= 256 that is
   3.05e-5 of the absolute sum.
2. BF16 rounding boundaries.  A value rounds to BF16 identically on both
   sides unless the two pre-rounding values straddle a rounding boundary; the
   flip then moves it by one BF16 step.  If an evaluation's pre-rounding
   value lies within t of a reference u, its BF16 value lies in
   [R(u - t), R(u + t)], R the round-to-nearest-even BF16 rounding.

Layer by layer (the GPU's own BF16 inputs of each GEMM fed to the
reference), only (1) enters an accumulator, and (2) its epilogue's rounding.

End to end, the oracle runs on its own.  Below the BF16 rounding points the
two sides' small differences are absorbed: a BF16 value differs only where a
flip happened, by one BF16 step.  An output is an FP32 accumulation over the
BF16 values of the last rounding point before it, so

  |GPU - oracle| <= |W|^T |d| + gamma_K (|a_GPU| + |a_oracle|) |W|,

d the two sides' differences at that rounding point (the flips), and the
flips at every rounding point must stay rare and small (flips()).  Sub-ulp differences
never compound; a flip moves the next layer's sums only through the |W| d
term, and the next rounding point absorbs it unless it flips too.
"""
from __future__ import annotations

import numpy as np

from oracle import mlp

U32 = 2.0 ** -24                  # FP32 unit roundoff


def gamma(K: int) -> float:
    """Accumulation bound of K exact products in FP32, any order, rounding or
    truncating adds (relative to the sum of the products' magnitudes)."""
    return K * 2.0 ** -23


def fn_err(z, u):
    """Bound on how far an FP32 evaluation of GELU or gelu' at z lies from its
    float64 value u.  GELU is z/2 (1 + erf(z / sqrt 2)) and gelu' is
    (1 + erf(z / sqrt 2))/2 + z phi(z): erff is within 2 ulp (2^-23 absolute
    below 1), which 1 + erf keeps as an absolute error (the cancellation for
    z < 0), times z/2 in GELU and 1/2 in gelu' -- so 2^-23 (|z| + 1) covers
    both, twice over; the few FP32 products and sums add 2^-22 |u|."""
    return 2.0 ** -23 * (np.abs(z) + 1.0) + 2.0 ** -22 * np.abs(u) + 2.0 ** -126


def bf16_round64(v):
    """Round float64 values to BF16 (8 significant bits, ties to even), in
    float64.  Equal to the FP32 -> BF16 rounding for FP32 inputs."""
    v = np.asarray(v, dtype=np.float64)
    m, e = np.frexp(v)
    return np.ldexp(np.rint(m * 256.0), e - 8)


def f64(a):
    return np.asarray(a, dtype=np.float64)


def check_acc(acc, A, W, what, transposed=True):
    """Tensor-core accumulator against the exact product of its own BF16
    operands.  acc [n][N] FP32; A [n][K] (BF16 values); W [N][K] when
    `transposed` (acc = A W^T) else [K][N] (acc = A W).  Every element must lie
    within gamma_K of its absolute sum, which for K <= 256 is 1e-3 of the
    element's own scale max(|z|, sum|a w| / 32).  Returns diagnostics."""
    A, W = f64(A), f64(W)
    Wt = W.T if transposed else W
    K = A.shape[1]
    ref = A @ Wt
    S = np.abs(A) @ np.abs(Wt)
    err = np.abs(f64(acc) - ref)
    bound = gamma(K) * S + 1e-38
    bad = err > bound
    assert not bad.any(), (what, int(bad.sum()), float((err / bound).max()))
    scale = np.maximum(np.abs(ref), S / 32.0)
    assert np.all(err <= 1e-3 * scale + 1e-38), what
    return {"max_err_over_gamma_bound": float((err / bound).max()),
            "max_rel_err": float((err / np.maximum(scale, 1e-30)).max())}


def check_rounded(got, u, tol, what, max_risk=0.02):
    """GPU's BF16 values `got` against the reference u (float64, before
    rounding) with |GPU pre-rounding value - u| <= tol: every element must lie
    in [R(u - tol), R(u + tol)], i.e. equal R(u) except at a rounding
    boundary within tol.  The share of such at-risk elements among those of
    magnitude >= 1% of the largest must stay below max_risk, so that the check
    is not vacuous.  (Smaller ones -- GELU's negative tail above all, whose
    FP32 value keeps only the absolute accuracy of 1 + erf -- are at risk far
    more often.)  Returns (at-risk share of those, flips)."""
    got, u = f64(got), f64(u)
    lo, hi = bf16_round64(u - tol), bf16_round64(u + tol)
    bad = (got < lo) | (got > hi)
    assert not bad.any(), (what, int(bad.sum()), got[bad][:5], u[bad][:5])
    big = np.abs(u) >= 1e-2 * np.abs(u).max()
    risk = float(np.mean((lo != hi)[big])) if big.any() else 0.0
    if big.sum() >= 4096:        # a share over a few rows only is noise
        assert risk <= max_risk, (what, risk)
    return risk, int(np.sum(got != bf16_round64(u)))


def weights16(params):
    return [f64(mlp.bf16_round(W)) for W, _ in params]


def flips(gpu, orc, what, max_share=0.1, max_mass=1e-3):
    """Elementwise |GPU - oracle| of the BF16 values at one rounding point,
    each side's own (the oracle run alone); they differ only where the two
    pre-rounding values straddled a rounding boundary.  The
    flips must stay rare (share of elements) and small (their summed size
    against the values' summed size), so that none compounds through the
    network.  GELU's negative tail flips most: there both sides' FP32 values
    keep only the absolute accuracy of 1 + erf."""
    g, o = f64(gpu), f64(orc)
    d = np.abs(g - o)
    share = float(np.mean(d > 0))
    mass = float(d.sum() / max(np.abs(o).sum(), 1e-300))
    assert share <= max_share and mass <= max_mass, (what, share, mass)
    return d


def last_layer_bound(d_in, a_gpu, a_orc, W):
    """Bound on |GPU - oracle| of acc = a W (W [K][N]) when the two sides'
    operands a differ by d_in elementwise (flips at the last rounding point)
    and each accumulates its own products in FP32: |W|^T d_in plus each
    side's gamma_K bound."""
    Wa = np.abs(f64(W))
    K = Wa.shape[0]
    return d_in @ Wa + gamma(K) * ((np.abs(f64(a_gpu)) + np.abs(f64(a_orc))) @ Wa)
