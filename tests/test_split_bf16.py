"""The split-bf16 arithmetic the float32 compressor's sketch and R^H GEMMs use
(hi = bf16(x), lo = bf16(x - hi)), emulated on the CPU with round-to-nearest-
even bf16: the error bounds that keep it inside the range finder's tol/3
margin (Sec. 5.2), and the real-matrix layouts that turn the complex products
into real GEMMs.  No library code is involved; this pins the arithmetic."""
import numpy as np


def bf16(x):
    """Round float32 to bf16 (nearest, ties to even), returned as float32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def split(x):
    x = np.asarray(x, np.float32)
    hi = bf16(x)
    lo = bf16(x - hi)
    return hi, lo


def test_bf16_rounding_is_round_to_nearest_even():
    # 1 + 2^-8 lies half way between 1 and 1 + 2^-7: ties go to the even 1.0
    assert bf16(np.float32(1 + 2 ** -8)) == 1.0
    assert bf16(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)
    x = np.random.default_rng(0).standard_normal(10000).astype(np.float32)
    assert np.all(np.abs(bf16(x) - x) <= 2.0 ** -8 * np.abs(x))


def test_split_carries_16_bits():
    x = np.random.default_rng(1).standard_normal(100000).astype(np.float32)
    hi, lo = split(x)
    err = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -16 * np.abs(x))
    assert np.all(bf16(hi) == hi) and np.all(bf16(lo) == lo)


def _planes(A):
    """m x n complex -> the split layout: column j holds [Re hi, Im hi, Re lo, Im lo]."""
    rh, rl = split(A.real)
    ih, il = split(A.imag)
    m, n = A.shape
    P = np.zeros((4 * m, n), np.float64)
    P[:m], P[m:2 * m], P[2 * m:3 * m], P[3 * m:] = rh, ih, rl, il
    return P


def test_sketch_two_products_within_margin():
    rng = np.random.default_rng(2)
    m, n, s = 96, 80, 24
    A = (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))).astype(np.complex64)
    W = (bf16(rng.standard_normal((n, s))) + 1j * bf16(rng.standard_normal((n, s)))).astype(np.complex128)
    P = _planes(A)
    # read with ld = m: an m x 4n matrix whose column 4j + p is plane p of column j
    Vm = P.T.reshape(4 * n, m).T
    B = np.zeros((4 * n, 2 * s))
    for h in range(2):
        B[2 * h::4, :s], B[2 * h::4, s:] = W.real, W.imag
        B[2 * h + 1::4, :s], B[2 * h + 1::4, s:] = -W.imag, W.real
    Yf = Vm @ B
    Y = Yf[:, :s] + 1j * Yf[:, s:]
    ref = A.astype(np.complex128) @ W
    rel = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
    assert rel < 1e-5            # representation error of A only (W is exact in bf16)
    assert rel > 1e-8            # and it is the split, not float64 rounding, that is measured


def test_rh_three_products_within_margin():
    rng = np.random.default_rng(3)
    m, n, r = 96, 80, 12
    A = (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))).astype(np.complex64)
    Q, _ = np.linalg.qr(rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r)))
    Q = Q.astype(np.complex64)
    P = _planes(A)                                           # read with ld = 4m: 4m x n
    qrh, qrl = split(Q.real)
    qih, qil = split(Q.imag)
    Bh = np.vstack([np.hstack([qrh, qih]), np.hstack([qih, -qrh])])
    Bh = np.vstack([Bh, Bh])                                 # hi parts against both hi and lo planes
    Bl = np.vstack([np.hstack([qrl, qil]), np.hstack([qil, -qrl])])
    F = P.T @ Bh + P[:2 * m].T @ Bl
    RH = F[:, :r] + 1j * F[:, r:]
    ref = A.astype(np.complex128).conj().T @ Q.astype(np.complex128)
    rel = np.linalg.norm(RH - ref) / np.linalg.norm(ref)
    assert rel < 1e-5            # only the lo.lo products are dropped
    # a sign error in either half of Bh would leave an O(1) error
    Bbad = Bh.copy()
    Bbad[:, r:] *= -1
    bad = (P.T @ Bbad + P[:2 * m].T @ Bl)
    assert np.linalg.norm(bad[:, :r] + 1j * bad[:, r:] - ref) / np.linalg.norm(ref) > 0.1
