"""Pins of the oracle against what the paper and mathematics fix (CPU only).

Each test checks the oracle against something other than itself: the paper's
printed factorisation and scaling (Sec. 2), its operation count (Table 1) and
compression ratios (Sec. 3), closed forms (orthogonality, Parseval, identity
round trip), brute force (rounding) and finite differences (float adjoint).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from golden_io import paper_matrices, paper_numbers
from paper_1702_00817_gb300 import inputs

RNG = np.random.default_rng(20170202)


def _factor_T():
    m = paper_matrices()
    return m["P"] @ m["A3"] @ m["A2"] @ m["A1"]


def test_T_is_the_product_of_the_printed_factors():
    # Sec. 2: T = P A3 A2 A1.  Pins the oracle's transcription of T against a
    # different printed formula.
    m = paper_matrices()
    assert np.array_equal(oracle.matrix_T(), _factor_T())
    assert np.array_equal(oracle.matrix_T(), m["T"])


def test_T_orthogonality_gives_D_inverse_squared():
    # Sec. 2: C^ = D T is orthogonal, i.e. T T^T = D^-2.
    T = oracle.matrix_T()
    inv_d2 = np.array(paper_numbers()["inv_d2"][0], np.int64)
    assert np.array_equal(T @ T.T, np.diag(inv_d2))
    a = oracle.scale_exponents()
    assert np.array_equal(2 ** a.astype(np.int64), inv_d2)
    # Sec. 2: the entries of D^2 are negative powers of two {1/2, 1/4, 1/8}.
    dens = sorted(set(int(v) for v in inv_d2))
    assert dens == [int(v) for v in paper_numbers()["d2_denominators"][0]]
    # row L1 norms equal 2^a_i (bounds the integer ranges used by the codec)
    assert np.array_equal(np.abs(T).sum(axis=1), inv_d2)


def test_T_entries_need_no_multiplication():
    # Sec. 2: entries in {0, +1, -1}.
    assert set(np.unique(oracle.matrix_T())) <= {-1, 0, 1}


def test_zigzag_is_the_standard_sequence():
    # Sec. 3: "standard zigzag sequence".  Properties that fix the JPEG order:
    # a permutation of the 64 positions, starting (0,0) -> (0,1), each step to a
    # neighbouring cell, anti-diagonals visited in order and in alternating
    # direction.
    rank = oracle.zigzag_rank()
    assert sorted(rank.ravel()) == list(range(64))
    pos = {int(rank[i, j]): (i, j) for i in range(8) for j in range(8)}
    assert pos[0] == (0, 0) and pos[1] == (0, 1) and pos[2] == (1, 0) and pos[63] == (7, 7)
    for k in range(63):
        (i0, j0), (i1, j1) = pos[k], pos[k + 1]
        assert max(abs(i1 - i0), abs(j1 - j0)) == 1
        assert i1 + j1 >= i0 + j0
    for s in range(15):
        cells = [pos[k] for k in range(64) if sum(pos[k]) == s]
        rows = [c[0] for c in cells]
        assert rows == sorted(rows, reverse=(s % 2 == 0))


@pytest.mark.parametrize("r,printed", [tuple(v) for v in paper_numbers()["ratio"]])
def test_zonal_compression_ratio_matches_paper(r, printed):
    # Sec. 3: keeping r of 64 coefficients is a compression of 1 - r/64.  The
    # paper prints these rounded (45.310 for 45.3125, 29.690 for 29.6875).
    r = int(r)
    Z = RNG.integers(1, 500, size=(3, 5, 8, 8)) * RNG.choice([-1, 1], size=(3, 5, 8, 8))
    q = oracle.quantise(Z, oracle.MODE_ZONAL, None, r)
    kept = np.count_nonzero(q.reshape(-1, 64), axis=1)
    assert np.all(kept == r)
    ratio = 100.0 * (1.0 - kept[0] / 64.0)
    assert abs(ratio - printed) < 0.01
    # the kept ones are exactly the first r in zig-zag order
    rank = oracle.zigzag_rank().ravel()
    mask = (rank < r).reshape(8, 8)
    assert np.array_equal(q != 0, np.broadcast_to(mask, q.shape))


def test_cost_reductions_follow_table1():
    # Sec. 2: 14 additions against 18, 20 and 24 operations.
    ours = paper_numbers()["table1_proposed"][0]
    assert ours == [14.0, 0.0, 0.0]
    for other, pct in paper_numbers()["reduction"]:
        assert abs(100.0 * (1 - 14.0 / other) - pct) < 0.05


def _blocks(img):
    H, W = img.shape
    return img.reshape(H // 8, 8, W // 8, 8).transpose(0, 2, 1, 3).astype(np.int64)


def test_forward_equals_fast_factorisation_on_random_blocks():
    # Z computed with the printed factors (P A3 A2 A1) x (P A3 A2 A1)^T by numpy.
    img = inputs.synth_image(64, 96, seed=3)[0]
    Z = oracle.forward(img)
    F = _factor_T()
    x = _blocks(img) - 128
    expect = np.einsum("ik,abkl,jl->abij", F, x, F)
    assert np.array_equal(Z, expect)


def test_forward_constant_block_has_only_dc():
    for c in (0, 1, 127, 128, 200, 255):
        img = np.full((16, 24), c, np.uint8)
        Z = oracle.forward(img)
        expect = np.zeros_like(Z)
        expect[..., 0, 0] = 64 * (c - 128)
        assert np.array_equal(Z, expect)


def test_forward_parseval_exact():
    # C^ = D T orthonormal => sum_ij Z_ij^2 2^-(a_i+a_j) = sum x^2, exactly;
    # multiplied through by 64.
    a = oracle.scale_exponents().astype(np.int64)
    w = 2 ** (6 - a[:, None] - a[None, :])
    for seed in range(4):
        img = RNG.integers(0, 256, size=(32, 40), dtype=np.uint8)
        Z = oracle.forward(img)
        x = _blocks(img) - 128
        lhs = (Z * Z * w).sum(axis=(2, 3))
        rhs = 64 * (x * x).sum(axis=(2, 3))
        assert np.array_equal(lhs, rhs)


def test_forward_extremes_within_int16():
    # |Z_ij| <= 128 * 2^(a_i + a_j) <= 8192; the checkerboard hits large values.
    yy, xx = np.mgrid[0:16, 0:16]
    for img in (np.zeros((16, 16), np.uint8), np.full((16, 16), 255, np.uint8),
                (((yy + xx) % 2) * 255).astype(np.uint8)):
        Z = oracle.forward(img)
        assert np.abs(Z).max() <= 8192


def test_step_quantiser_brute_force_against_float64_division():
    # q = round half away from zero of Z/Q over |Z| <= 8192, Q in 1..1024.
    # Float64 Z/Q + 1/2 is exact enough here: ties are representable and the
    # nearest non-tie is at least 1/(2Q) away.
    Zs = np.arange(-8192, 8193, dtype=np.int64)
    for Q in list(range(1, 130)) + list(range(130, 1025, 7)) + [1024]:
        Zm = Zs
        pad = (-Zm.size) % 64
        Zp = np.concatenate([Zm, np.zeros(pad, np.int64)]).reshape(-1, 64)
        q = oracle.quantise(Zp, oracle.MODE_STEP, np.full(64, Q, np.uint16), 64).reshape(-1)
        q = q[: Zm.size]
        expect = np.sign(Zm) * np.floor(np.abs(Zm) / float(Q) + 0.5)
        assert np.array_equal(q, expect.astype(np.int64)), Q


def test_step_quantiser_rational_ties_and_samples():
    Qs = RNG.integers(1, 65536, size=2000)
    Zs = RNG.integers(-8192, 8193, size=2000)
    # add exact ties Z = (2k+1) Q / 2 for even Q
    even = np.arange(2, 200, 2)
    kk = RNG.integers(0, 40, size=even.size)
    Zt = ((2 * kk + 1) * even) // 2
    Zs = np.concatenate([Zs, Zt, -Zt])
    Qs = np.concatenate([Qs, even, even])
    for z, Q in zip(Zs.tolist(), Qs.tolist()):
        f = Fraction(abs(z), Q)
        m = math.floor(f + Fraction(1, 2))
        expect = -m if z < 0 else m
        Zb = np.zeros(64, np.int64)
        Zb[7] = z
        Qt = np.ones(64, np.uint16)
        Qt[7] = Q
        assert oracle.quantise(Zb, oracle.MODE_STEP, Qt, 64)[7] == expect


@pytest.mark.parametrize("mode,Q,r", [
    (oracle.MODE_NONE, None, 64),
    (oracle.MODE_ZONAL, None, 64),
    (oracle.MODE_STEP, np.ones(64, np.uint16), 64),
    (oracle.MODE_STEP_ZONAL, np.ones(64, np.uint16), 64),
])
def test_identity_round_trip_is_exact(mode, Q, r):
    # T^T D^2 T = I (Sec. 2): with nothing discarded the round trip is exact.
    yy, xx = np.mgrid[0:32, 0:48]
    imgs = [inputs.synth_image(40, 56, seed=11)[0], np.zeros((16, 16), np.uint8),
            np.full((16, 16), 255, np.uint8), (((yy + xx) % 2) * 255).astype(np.uint8),
            RNG.integers(0, 256, size=(24, 24), dtype=np.uint8)]
    for img in imgs:
        q, rec = oracle.roundtrip(img, mode, Q, r)
        assert np.array_equal(rec, img)


def test_step_round_trip_error_within_quantisation_bound():
    # Orthonormal C^: the pixel-domain error energy per block is at most the
    # coefficient-domain error energy (each |qQ - Z| <= Q/2, scaled by D^2) plus
    # the final rounding (1/2 per pixel); clamping only reduces it.
    a = oracle.scale_exponents().astype(np.float64)
    for s in (1, 4, 16):
        Q = inputs.step_table(s).astype(np.float64)
        coef_err = math.sqrt(((Q / 2) ** 2 * 2.0 ** (-a[:, None] - a[None, :])).sum())
        bound = (coef_err + math.sqrt(64 * 0.25)) ** 2
        img = inputs.synth_image(64, 64, seed=5)[0]
        q, rec = oracle.roundtrip(img, oracle.MODE_STEP, inputs.step_table(s), 64)
        err = (_blocks(rec) - _blocks(img)).astype(np.float64)
        assert np.all((err ** 2).sum(axis=(2, 3)) <= bound + 1e-9)
        # and the error is not trivially zero for coarse steps
        if s == 16:
            assert np.abs(err).max() > 0


def test_inverse_dequantisation_scale_matches_D_squared():
    # One nonzero coefficient q at (i, j): R = q Q 2^(6-a_i-a_j) T[:, i] T[:, j]^T,
    # i.e. (D^2 merged) the orthonormal basis image of Sec. 2 scaled by 64 q Q d_i^2 d_j^2.
    T = _factor_T()
    a = oracle.scale_exponents()
    for i in range(8):
        for j in range(8):
            q = np.zeros((1, 1, 8, 8), np.int64)
            q[0, 0, i, j] = 3
            Q = np.full(64, 2, np.uint16)
            rec = oracle.inverse(q, oracle.MODE_STEP, Q).astype(np.int64)
            basis = np.outer(T[i, :], T[j, :]) * Fraction(6, 2 ** (int(a[i]) + int(a[j])))
            expect = np.array([[min(255, max(0, math.floor(float(v) + 0.5) + 128)) for v in row]
                               for row in basis])
            assert np.array_equal(rec, expect)


def test_float_forward_is_orthonormal_and_invertible():
    x = inputs.normal_batch((2, 16, 24), seed=9).astype(np.float64)
    z, y = oracle.forward_f64(x, None, want_y=True)
    assert np.array_equal(z, y)
    F = _factor_T().astype(np.float64)
    d = 1.0 / np.sqrt(np.array(paper_numbers()["inv_d2"][0]))
    C = d[:, None] * F
    xb = x.reshape(2, 2, 8, 3, 8).transpose(0, 1, 3, 2, 4)
    yb = y.reshape(2, 2, 8, 3, 8).transpose(0, 1, 3, 2, 4)
    assert np.allclose(np.einsum("ik,pabkl,jl->pabij", C, xb, C), yb, atol=1e-12)
    assert np.allclose((yb ** 2).sum(axis=(3, 4)), (xb ** 2).sum(axis=(3, 4)), rtol=1e-12)
    # the adjoint applied to y returns x (C^ orthogonal)
    assert np.allclose(oracle.backward_f64(x, y, None), x, atol=1e-12)


def test_soft_quantiser_fixed_points():
    # z = y - (Q/2pi) sin(2 pi y / Q) leaves multiples of Q/2 unchanged.
    Q = inputs.step_table(1).astype(np.float64)
    x = np.zeros((1, 8, 8))
    z, y = oracle.forward_f64(x, Q, want_y=True)
    assert np.allclose(z, 0.0)


# Closed forms of the soft quantiser z(y) = y - (Q/2pi) sin(2 pi y / Q) and
# its derivative 1 - cos(2 pi y / Q) at y = f Q, written out by hand.
_SOFT_POINTS = [  # (f, z / Q, dz/dy)
    (0.25, 0.25 - 1 / (2 * math.pi), 1.0),
    (0.5, 0.5, 2.0),
    (0.75, 0.75 + 1 / (2 * math.pi), 1.0),
    (1.0, 1.0, 0.0),
    (-0.25, -0.25 + 1 / (2 * math.pi), 1.0),
]


def _orthonormal_rows():
    # C^ = D T from the printed factors and the printed D (Sec. 2), not from the oracle
    d = 1.0 / np.sqrt(np.array(paper_numbers()["inv_d2"][0]))
    return d[:, None] * _factor_T().astype(np.float64)


@pytest.mark.parametrize("Qv", [1.0, 3.0, 0.5, 37.0])
def test_soft_quantiser_constant_block_closed_form(Qv):
    # Sec. 2: T 1 = 8 e0 and d_0^2 = 1/8, so a constant block x = c gives
    # y_00 = 64 c / 8 = 8 c and y_ij = 0 elsewhere.  Choosing c = f Q / 8 puts
    # y_00 at f Q, where z_00 and dz/dy have the closed forms above; every
    # other z_ij is 0.  A dropped D, a sin(pi y / Q), a Q/pi factor or a sign
    # error in the soft term moves z_00 off these values.
    Q = np.full(64, Qv)
    for f, zq, dzdy in _SOFT_POINTS:
        x = np.full((1, 8, 8), f * Qv / 8.0)
        z, y = oracle.forward_f64(x, Q, want_y=True)
        assert abs(y[0, 0, 0] - f * Qv) <= 1e-12 * max(1.0, Qv)
        assert abs(z[0, 0, 0] - zq * Qv) <= 1e-12 * max(1.0, Qv)
        zz = z.copy()
        zz[0, 0, 0] = 0.0
        assert np.abs(zz).max() <= 1e-12 * max(1.0, Qv)
        # adjoint with g_z = e_00: g_x = C^T (e_00 dz/dy) C = dz/dy / 8 everywhere
        gz = np.zeros((1, 8, 8))
        gz[0, 0, 0] = 1.0
        gx = oracle.backward_f64(x, gz, Q)
        assert np.abs(gx - dzdy / 8.0).max() <= 1e-12


@pytest.mark.parametrize("i,j", [(0, 1), (2, 5), (3, 3), (7, 4), (6, 0)])
def test_soft_quantiser_single_coefficient_closed_form(i, j):
    # A basis block x = A C^[i]^T C^[j] (C^ = D T orthonormal, Sec. 2) has the
    # single coefficient y_ij = A.  With a different step at every position the
    # soft term must use Q_ij (a transposed table index fails); the adjoint of
    # g_z = e_ij is dz/dy * C^[i]^T C^[j].
    C = _orthonormal_rows()
    Q = 1.0 + 0.25 * np.arange(64)  # Q_ij = 1 + (8 i + j) / 4, no symmetry
    Qij = Q[8 * i + j]
    basis = np.outer(C[i], C[j])
    for f, zq, dzdy in _SOFT_POINTS:
        x = (f * Qij * basis)[None]
        z, y = oracle.forward_f64(x, Q, want_y=True)
        expect_y = np.zeros((8, 8))
        expect_y[i, j] = f * Qij
        assert np.abs(y[0] - expect_y).max() <= 1e-12 * Qij
        expect_z = np.zeros((8, 8))
        expect_z[i, j] = zq * Qij
        assert np.abs(z[0] - expect_z).max() <= 1e-12 * Qij
        gz = np.zeros((1, 8, 8))
        gz[0, i, j] = 1.0
        gx = oracle.backward_f64(x, gz, Q)
        assert np.abs(gx[0] - dzdy * basis).max() <= 1e-12


@pytest.mark.parametrize("Qkind", ["ones", "step1"])
def test_float_adjoint_matches_central_finite_differences(Qkind):
    # FP64 central differences, h = 1e-3, relative error < 1e-4.
    Q = np.ones(64) if Qkind == "ones" else inputs.step_table(1).astype(np.float64)
    rng = np.random.default_rng(77)
    x = rng.standard_normal((2, 16, 16))
    gz = rng.standard_normal(x.shape)
    gx = oracle.backward_f64(x, gz, Q)

    def f(v):
        return float((oracle.forward_f64(v, Q) * gz).sum())

    h = 1e-3
    idx = [tuple(rng.integers(0, s) for s in x.shape) for _ in range(64)]
    for ix in idx:
        e = np.zeros_like(x)
        e[ix] = h
        fd = (f(x + e) - f(x - e)) / (2 * h)
        assert abs(fd - gx[ix]) <= 1e-4 * max(1.0, abs(gx[ix])), (ix, fd, gx[ix])
    for _ in range(8):
        v = rng.standard_normal(x.shape)
        fd = (f(x + h * v) - f(x - h * v)) / (2 * h)
        an = float((gx * v).sum())
        assert abs(fd - an) <= 1e-4 * max(1.0, abs(an))


def test_float_adjoint_passes_torch_gradcheck():
    """The whole Jacobian of a 1x16x16 input, in float64, by torch's own
    numerical differentiation, against the oracle's analytic adjoint."""
    import torch
    Q = inputs.step_table(1).astype(np.float64)

    class Fp64(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x):
            ctx.save_for_backward(x)
            return torch.from_numpy(oracle.forward_f64(x.detach().numpy(), Q))

        @staticmethod
        def backward(ctx, g):
            (x,) = ctx.saved_tensors
            return torch.from_numpy(oracle.backward_f64(x.numpy(), g.contiguous().numpy(), Q))

    x = torch.from_numpy(np.random.default_rng(5).standard_normal((1, 16, 16))).requires_grad_(True)
    assert torch.autograd.gradcheck(Fp64.apply, (x,), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_dct_comparator_is_orthonormal_and_exact_at_r64():
    # the exact DCT of the Sec. 3 comparison: C C^T = I; keeping all 64
    # coefficients reproduces every image exactly (after rounding)
    C = oracle.dct_matrix()
    assert np.allclose(C @ C.T, np.eye(8), atol=1e-14)
    assert np.allclose(C[0], np.sqrt(1 / 8)) and abs(C[1, 0] - 0.5 * math.cos(math.pi / 16)) < 1e-15
    for img in (inputs.synth_image(64, 80, 21)[0], RNG.integers(0, 256, (32, 32), dtype=np.uint8)):
        assert np.array_equal(oracle.dct_zonal(img, 64), img)


def test_dct_comparator_dc_only_gives_block_means():
    # r = 1 keeps the DC term only: each block becomes its (rounded) mean
    img = inputs.synth_image(48, 64, 22)[0]
    rec = oracle.dct_zonal(img, 1)
    means = _blocks(img).mean(axis=(2, 3))
    expect = np.rint(means)
    got = _blocks(rec)
    assert np.all(got == got[..., :1, :1])
    assert np.array_equal(got[..., 0, 0], expect.astype(np.int64))


def test_zonal_quality_improves_with_r():
    # keeping more coefficients never hurts much: the proposed transform's
    # error at r = 64 is zero, and the error falls as r grows (synthetic image)
    img = inputs.synth_image(64, 64, 23)[0]
    errs = [oracle.sse(oracle.roundtrip(img, oracle.MODE_ZONAL, None, r)[1], img) for r in (1, 6, 16, 45, 64)]
    assert errs[-1] == 0 and errs[0] > errs[1] > errs[2] > errs[3]
