"""Property-based pins of the oracle (hypothesis draws the inputs): invariants
that follow from the definitions of Sec. 2 and Sec. 3, independent of how the
oracle computes them."""
import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings


def _img(seed, hi=255):
    return np.random.default_rng(seed).integers(0, hi + 1, (8, 16)).astype(np.uint8)


@settings(max_examples=60, deadline=None)
@given(st.integers(0, 2**32 - 1), st.integers(0, 2**32 - 1))
def test_forward_is_affine_in_the_pixels(sa, sb):
    """Z(X) = T (X - 128) T^T is affine: Z(A + B) = Z(A) + Z(B) + 8192 e0 e0^T
    (the level shift counted twice on the right; T 1 = 8 e0)."""
    a, b = _img(sa, 127), _img(sb, 128)
    za, zb, zab = oracle.forward(a), oracle.forward(b), oracle.forward((a + b).astype(np.uint8))
    e00 = np.zeros_like(za)
    e00[..., 0, 0] = 8192
    assert np.array_equal(zab, za + zb + e00)


@settings(max_examples=80, deadline=None)
@given(st.lists(st.integers(-8192, 8192), min_size=64, max_size=64), st.integers(1, 300))
def test_step_quantiser_is_odd_and_within_half_a_step(zs, Q):
    """Round half away from zero is an odd function, and q Q is within Q / 2 of Z."""
    Z = np.array(zs, np.int64).reshape(1, 1, 8, 8)
    Qt = np.full(64, Q, np.uint16)
    q = oracle.quantise(Z, oracle.MODE_STEP, Qt)
    assert np.array_equal(oracle.quantise(-Z, oracle.MODE_STEP, Qt), -q)
    assert np.all(2 * np.abs(q * Q - Z) <= Q)


@settings(max_examples=60, deadline=None)
@given(st.lists(st.integers(-8192, 8192), min_size=64, max_size=64), st.integers(0, 64))
def test_zonal_keeps_exactly_the_first_r_zigzag_positions(zs, r):
    Z = np.array(zs, np.int64).reshape(1, 1, 8, 8)
    q = oracle.quantise(Z, oracle.MODE_ZONAL, None, r)
    rank = oracle.zigzag_rank()
    keep = rank < r
    assert np.array_equal(q[0, 0][keep], Z[0, 0][keep])
    assert not np.any(q[0, 0][~keep])
    assert np.count_nonzero(q) <= r
