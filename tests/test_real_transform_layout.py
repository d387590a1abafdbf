"""The index and spectrum identities the real-input transforms of the linear
advance rely on, checked with numpy's FFT (no library code here).

A real row x of length N = 2M is transformed as the M complex values
z[s] = x[2s] + i x[2s+1].  With Z = DFT_M(z), the row's spectrum is
X[k] = E[k] + W^k O[k] and X[k+M] = E[k] - W^k O[k] (W = e^{-2 pi i/N}),
E[k] = (Z[k] + conj Z[M-k]) / 2, O[k] = -i (Z[k] - conj Z[M-k]) / 2.  After the
product Y = X S the inverse is again an M-point transform of
A[k] + i W^{-k} B[k] with A = Y[k] + Y[k+M], B = Y[k] - Y[k+M], whose real and
imaginary parts are the even and odd output cells.  The transforms leave bins
in bit-reversed order; in blocks of 2^l slots, the block of bit-reversed
residue r holds bin M - k of each of its bins k in the block of residue -r, at
the slot with all l bits flipped (residues 0 and half the block count pair
within their own block)."""
import numpy as np
import pytest


def brev(v, bits):
    r = 0
    for _ in range(bits):
        r = (r << 1) | (v & 1)
        v >>= 1
    return r


@pytest.mark.parametrize("lgM,lti", [(3, 1), (5, 2), (6, 3), (8, 4), (10, 9), (11, 9), (12, 10)])
def test_mirror_blocks(lgM, lti):
    M = 1 << lgM
    nbl = lgM - lti
    nb, Bs = 1 << nbl, 1 << lti
    mask = Bs - 1
    pos = {brev(p, lgM): p for p in range(M)}        # bin -> bit-reversed position
    for b in range(nb):
        rb = brev(b, nbl)
        for s in range(Bs):
            k = rb + (brev(s, lti) << nbl)
            assert pos[k] == b * Bs + s
            j = (M - k) % M
            if rb == 0:
                assert pos[j] == b * Bs + brev((Bs - brev(s, lti)) & mask, lti)
            else:
                b2 = brev((nb - rb) % nb, nbl)
                assert pos[j] == b2 * Bs + (s ^ mask)
                assert (b2 == b) == (rb == nb // 2)


@pytest.mark.parametrize("lgN", [2, 3, 6, 11])
def test_split_product_merge(lgN):
    rng = np.random.default_rng(lgN)
    N = 1 << lgN
    M = N // 2
    x = rng.normal(size=N)
    S = np.fft.fft(rng.normal(size=N))                 # spectrum of a real kernel
    want = np.fft.ifft(np.fft.fft(x) * S).real
    z = x[0::2] + 1j * x[1::2]
    Z = np.fft.fft(z)
    k = np.arange(M)
    Zm = np.conj(Z[(M - k) % M])
    E = (Z + Zm) / 2
    O = -1j * (Z - Zm) / 2
    W = np.exp(-2j * np.pi * k / N)
    Y0, Y1 = (E + W * O) * S[:M], (E - W * O) * S[M:]
    A, B = Y0 + Y1, Y0 - Y1
    u = np.fft.ifft(A + 1j * np.conj(W) * B) / 2       # N/2-point inverse, scale 1/N overall
    got = np.empty(N)
    got[0::2], got[1::2] = u.real, u.imag
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
    # the kernel merges bin M-k from the pair of bin k (the product keeps Y
    # Hermitian): A[M-k] + i W^{-(M-k)} B[M-k] = conj A[k] + i W^k conj B[k]
    merged = A + 1j * np.conj(W) * B
    j = (M - k) % M
    assert np.allclose(merged[j], np.conj(A) + 1j * W * np.conj(B), rtol=0, atol=1e-12 * np.abs(merged).max())
