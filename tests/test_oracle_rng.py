"""Pins of the oracle's Gaussian test matrix (Fig. randQB_b line (2): Omega = randn(n, b)).

The method only requires Omega to have iid N(0, 1) entries; the generator is a
choice of this library (Philox4x32-10 + Box-Muller, indexed by global column).
Pins:
  * the Philox rounds against NVIDIA's independent host implementation of the
    same published generator (cuRAND's host Philox4_32_10 generator emits the
    block for counter (0, 0, j, 0) as its j-th output block);
  * bit-level uniformity and avalanche of the Philox output;
  * moments and a Kolmogorov-Smirnov test of the Gaussian entries (both
    evaluation precisions);
  * eq. (OmegaBlock): blocks drawn separately are slices of one matrix.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest


def _curand():
    cands = ["/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand") or ""]
    for c in cands:
        if c and os.path.exists(c):
            try:
                return ctypes.CDLL(c)
            except OSError:
                pass
    return None


def test_philox_matches_curand_host_generator(orc):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:  # CURAND_RNG_PSEUDO_PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    try:
        for seed in (0, 1, 0x123456789ABCDEF0, 2**64 - 1):
            assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(0)) == 0
            out = np.zeros(4 * 32, dtype=np.uint32)
            assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
            key = [seed & 0xFFFFFFFF, seed >> 32]
            for j in range(32):
                got = orc.philox4x32_10([0, 0, j, 0], key)
                np.testing.assert_array_equal(got, out[4 * j:4 * j + 4], err_msg=f"seed={seed} j={j}")
    finally:
        lib.curandDestroyGenerator(gen)


def test_philox_bits_uniform_and_avalanche(orc):
    rng = np.random.default_rng(0)
    key = [0xDEADBEEF, 0x01234567]
    words = np.array([orc.philox4x32_10([i, 7, 0, 0], key) for i in range(4000)], dtype=np.uint64)
    bits = ((words[..., None] >> np.arange(32, dtype=np.uint64)) & 1).astype(np.float64)
    freq = bits.reshape(-1, 32).mean(axis=0)
    N = words.size
    assert np.all(np.abs(freq - 0.5) < 6 * 0.5 / np.sqrt(N))
    # flipping one counter bit changes about half the output bits
    flips = []
    for t in range(300):
        c = [int(x) for x in rng.integers(0, 2**32, size=4, dtype=np.uint64)]
        a = orc.philox4x32_10(c, key)
        c2 = list(c)
        bit = int(rng.integers(0, 128))
        c2[bit // 32] ^= 1 << (bit % 32)
        b = orc.philox4x32_10(c2, key)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert abs(np.mean(flips) - 64.0) < 2.0


@pytest.mark.parametrize("prec", [64, 32, 19])
def test_omega_gaussian_moments_and_ks(orc, prec):
    from scipy import stats
    Om = orc.omega(seed=12345, n=4000, col0=0, ncols=256, prec=prec)
    x = Om.ravel()
    N = x.size
    assert abs(x.mean()) < 5 / np.sqrt(N)
    assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / N)
    kurt = np.mean(x ** 4)
    assert abs(kurt - 3.0) < 5 * np.sqrt(96.0 / N)
    assert stats.kstest(x, "norm").pvalue > 1e-4
    # the two entries of one Box-Muller pair, and neighbouring rows, are uncorrelated
    c = np.corrcoef(Om[:, 0::2].ravel(), Om[:, 1::2].ravel())[0, 1]
    assert abs(c) < 5 / np.sqrt(N / 2)
    c = np.corrcoef(Om[:-1, :].ravel(), Om[1:, :].ravel())[0, 1]
    assert abs(c) < 5 / np.sqrt(N)


@pytest.mark.parametrize("prec", [64, 32, 19])
def test_omega_blocks_slice_one_matrix(orc, prec):
    full = orc.omega(seed=99, n=300, col0=0, ncols=37, prec=prec)
    for c0, w in [(0, 5), (5, 3), (7, 12), (19, 18), (36, 1)]:
        part = orc.omega(seed=99, n=300, col0=c0, ncols=w, prec=prec)
        np.testing.assert_array_equal(part, full[:, c0:c0 + w])
    # different seeds give different matrices
    other = orc.omega(seed=100, n=300, col0=0, ncols=37, prec=prec)
    assert np.mean(other == full) < 1e-3


def test_omega_fp32_is_fp32_evaluation_of_same_draw(orc):
    """The binary32 evaluation uses the leading bits of the same Philox words, so it
    agrees with the binary64 entry to within binary32 resolution (bulk of entries)."""
    a = orc.omega(seed=5, n=2000, col0=0, ncols=64, prec=64)
    b = orc.omega(seed=5, n=2000, col0=0, ncols=64, prec=32)
    assert np.all(b == b.astype(np.float32).astype(np.float64))
    diff = np.abs(a - b)
    assert np.median(diff / np.maximum(np.abs(a), 1e-3)) < 1e-6
    assert np.quantile(diff, 0.999) < 2e-5


def test_round_tf32_closed_forms(orc):
    """11 significant bits, nearest, ties away from zero (cases fixed by the format)."""
    r = orc.round_tf32
    u = 2.0 ** -10                       # TF32 spacing on [1, 2)
    assert r(1.0) == 1.0 and r(0.0) == 0.0 and r(-3.0) == -3.0
    assert r(1.0 + u / 2) == 1.0 + u     # tie -> away from zero
    assert r(-(1.0 + u / 2)) == -(1.0 + u)
    assert r(1.0 + 3 * u / 2) == 1.0 + 2 * u
    assert r(1.0 + u / 4) == 1.0 and r(1.0 + 3 * u / 4) == 1.0 + u
    assert r(2.0 - u / 4) == 2.0         # carry into the next binade
    assert r(0.75 * 2.0 ** -30) == 0.75 * 2.0 ** -30
    x = (1.0 + 5 * u + u / 2) * 2.0 ** 40
    assert r(x) == (1.0 + 6 * u) * 2.0 ** 40


def test_omega_tf32_is_rounded_fp32_draw(orc):
    """prec 19 = the binary32 draw rounded to 11 significant bits: every value is
    representable in TF32 and within half a TF32 ulp of the binary32 value."""
    a = orc.omega(seed=5, n=2000, col0=0, ncols=64, prec=32)
    b = orc.omega(seed=5, n=2000, col0=0, ncols=64, prec=19)
    nz = a != 0
    e = np.floor(np.log2(np.abs(a[nz]))) + 1          # 2^(e-1) <= |a| < 2^e
    assert np.all(np.abs(b[nz] - a[nz]) <= 2.0 ** (e - 12) * (1 + 1e-12))
    scaled = b[nz] * 2.0 ** (11 - e)
    ok = np.abs(scaled - np.round(scaled)) == 0
    # values rounded up to 2^e carry one binade; they are powers of two
    assert np.all(ok | (np.abs(b[nz]) == 2.0 ** e))
    assert np.mean(b != a) > 0.99
