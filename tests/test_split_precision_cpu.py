"""The arithmetic behind the split-precision tolerances, emulated on the CPU.

The tensor-core path forms Y = B X with both operands split into 16-bit parts, x = hi + lo with
hi = rn16(x), lo = rn16(x - hi), after scaling every row of X and the operator B by powers of two
so that their largest entries lie in [2^14, 2^15); the product is X_hi B_hi + X_hi B_lo + X_lo B_hi
accumulated in FP32 (the lo x lo term is dropped).  Here the same splitting, in numpy, applied to
an operator of the method (the tet's nodal derivative matrices at N = 7, from the oracle), against
the FP64 product and against plain FP32 arithmetic:

* normwise (error of a row of Y over ||B||_2 ||x||): FP16 parts (11 significant bits) stay below
  2^-22 and within a small factor of plain FP32's error (FP32-class); BF16 parts (8 bits) below
  2^-17;
* rows like the GPU parity tests' inputs (random, no strong cancellation): the relative L2 error
  of a row stays below the GPU tests' tolerances, 1e-5 for FP16 x 3 (with a factor 10 to spare)
  and 3e-5 for BF16 x 3;
* rows of a large smooth field, whose derivatives cancel: the relative error grows by the
  cancellation for every format, FP32 included, and BF16 x 3 leaves its tolerance there (the
  tolerances hold for inputs without strong cancellation, as the parity tests use).

The emulation rounds to nearest even in both formats (numpy's float16 cast for FP16; BF16 by
rounding the FP32 bit pattern to its upper 16 bits)."""
import numpy as np

from oracle.elements import make_element


def rn_bf16(x):
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16        # round to nearest even
    return r.astype(np.uint32).view(np.float32)


def rn_fp16(x):
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float32)


def pow2_scale(m):
    """2^(14 - floor(log2 max|m|)) per row (the largest entry lands in [2^14, 2^15))."""
    mx = np.abs(m).max(axis=1)
    e = np.floor(np.log2(np.where(mx > 0, mx, 1.0)))
    return np.where(mx > 0, 2.0 ** (14 - e), 1.0).astype(np.float32)


def split(m, rn):
    hi = rn(m)
    lo = rn(m.astype(np.float32) - hi)
    return hi, lo


def emulate(X, B, rn):
    """Y = X B^T in the split form: per-row scales for X, one scale for B."""
    sx = pow2_scale(X)
    sb = np.float32(pow2_scale(B.reshape(1, -1))[0])
    xh, xl = split((X * sx[:, None]).astype(np.float32), rn)
    bh, bl = split((B * sb).astype(np.float32), rn)
    acc = (xh @ bh.T).astype(np.float32) + (xh @ bl.T).astype(np.float32) + (xl @ bh.T).astype(np.float32)
    return acc.astype(np.float64) / (sx[:, None].astype(np.float64) * float(sb))


def row_errors(Y, Y64):
    return np.linalg.norm(Y - Y64, axis=1) / np.linalg.norm(Y64, axis=1)


def operator_and_rows():
    el = make_element(3, 7)
    B = np.concatenate(list(el.grad(el.nodes)), axis=0)     # [D^r; D^s; D^t]: 360 x 120
    rng = np.random.default_rng(0)
    # random rows of very different magnitudes (the per-row scale removes them)
    X = rng.standard_normal((64, 120)) * 10.0 ** rng.uniform(-6, 6, (64, 1))
    # a large smooth field plus a unit perturbation: its derivatives cancel
    S = np.linspace(1.0, 2.0, 120)[None, :] * 1e3 + rng.standard_normal((8, 120))
    return B, X, S


def normwise(Y, Y64, B, X):
    return np.linalg.norm(Y - Y64, axis=1) / (np.linalg.norm(B, 2) * np.linalg.norm(X, axis=1))


def test_split_products_meet_the_tolerances():
    B, X, S = operator_and_rows()
    for rows in (X, S):
        Y64 = rows @ B.T
        y32 = (rows.astype(np.float32) @ B.T.astype(np.float32)).astype(np.float64)
        n32 = normwise(y32, Y64, B, rows).max()
        n16 = normwise(emulate(rows, B, rn_fp16), Y64, B, rows).max()
        nbf = normwise(emulate(rows, B, rn_bf16), Y64, B, rows).max()
        assert n16 < 2.0 ** -22 and n16 < 4 * n32, (n16, n32)
        assert nbf < 2.0 ** -17, nbf
    Y64 = X @ B.T
    e16 = row_errors(emulate(X, B, rn_fp16), Y64)
    ebf = row_errors(emulate(X, B, rn_bf16), Y64)
    assert e16.max() < 1e-5 / 10, e16.max()          # measured 1.4e-7
    assert ebf.max() < 3e-5, ebf.max()                # measured 5.3e-6
    assert np.median(ebf) > 4 * np.median(e16)
    ebf_s = row_errors(emulate(S, B, rn_bf16), S @ B.T)
    assert ebf_s.max() > 3e-5                         # measured 4.4e-4: cancellation


def test_dropping_the_lo_parts_breaks_the_fp32_class():
    """Control: with hi parts only (one 16-bit product) the FP16 error is far above the FP16 x 3
    tolerance, so the three-product form is what makes it FP32-class."""
    el = make_element(3, 7)
    B = np.concatenate(list(el.grad(el.nodes)), axis=0)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((32, 120))
    sx = pow2_scale(X)
    sb = np.float32(pow2_scale(B.reshape(1, -1))[0])
    xh = rn_fp16((X * sx[:, None]).astype(np.float32))
    bh = rn_fp16((B * sb).astype(np.float32))
    Y1 = (xh @ bh.T).astype(np.float64) / (sx[:, None].astype(np.float64) * float(sb))
    assert row_errors(Y1, X @ B.T).max() > 1e-4
