"""The real formulation behind the tensor-core block-OSRC stream (CPU).

A row of T~ stored as interleaved (re, im) values is a real row of length
2 len; each complex input column x_q becomes two real columns,
(x_re, -x_im, ...) for the real part of T~ x_q and (x_im, x_re, ...) for the
imaginary part.  One real product then yields every complex product, in
columns 2 q + p, which is the order of the piece sums the combine kernel
reads (per right-hand side: Re/Im of T~ x_D, then of T~ x_N).  Checked in
FP64 with numpy on random data; the FP16 rounding of the kernel is covered by
the GPU parity tests."""
import numpy as np


def _real_operands(T, X):
    rows, L = T.shape
    A = np.empty((rows, 2 * L))
    A[:, 0::2], A[:, 1::2] = T.real, T.imag
    B = np.empty((2 * L, 2 * X.shape[1]))
    for q in range(X.shape[1]):
        x = X[:, q]
        B[0::2, 2 * q], B[1::2, 2 * q] = x.real, -x.imag          # real part column
        B[0::2, 2 * q + 1], B[1::2, 2 * q + 1] = x.imag, x.real   # imaginary part column
    return A, B


def test_real_product_gives_the_complex_products():
    rng = np.random.default_rng(5)
    for L, nc in ((8, 1), (640, 2), (37, 3), (96, 4)):
        T = rng.standard_normal((16, L)) + 1j * rng.standard_normal((16, L))
        X = rng.standard_normal((L, 2 * nc)) + 1j * rng.standard_normal((L, 2 * nc))
        A, B = _real_operands(T, X)
        C = A @ B
        Z = T @ X
        assert np.allclose(C[:, 0::2], Z.real, rtol=1e-12, atol=1e-10)
        assert np.allclose(C[:, 1::2], Z.imag, rtol=1e-12, atol=1e-10)
        # column v = 2 q + p, q = 2 c + slot: per right-hand side c the values
        # (Re, Im) of T~ x_D then of T~ x_N, as the combine kernel reads them
        for c in range(nc):
            for slot in range(2):
                q = 2 * c + slot
                v = 4 * c + 2 * slot
                assert np.allclose(C[:, v] + 1j * C[:, v + 1], T @ X[:, q], rtol=1e-12, atol=1e-10)


def test_zero_inputs_past_the_piece_cancel_any_padding():
    """Whole k16 chunks read up to 7 entries past a piece; the kernel zeroes
    the inputs there, so whatever the operator holds in those slots (the
    tiled copy stores zeros) does not reach the sums."""
    rng = np.random.default_rng(6)
    L, Lc = 37, 40
    T = rng.standard_normal((16, Lc)) + 1j * rng.standard_normal((16, Lc))
    X = rng.standard_normal((Lc, 4)) + 1j * rng.standard_normal((Lc, 4))
    X[L:] = 0.0
    A, B = _real_operands(T, X)
    C = A @ B
    Z = T[:, :L] @ X[:L]
    assert np.allclose(C[:, 0::2] + 1j * C[:, 1::2], Z, rtol=1e-12, atol=1e-10)
