"""Pins of the oracle's primitives against published values and exact mathematics.

* Philox4x32-10: the known-answer vectors published with the Random123 library that accompanies
  Salmon et al., "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
* exp(-x): against the platform exp, within the error bound of scaling and squaring.
* Binomial / Poisson inversion (Sec. 3.1.3): the 32-bit CDF thresholds against exact rational
  (Binomial) or 50-digit (Poisson) CDFs; the split Poisson draw against Poisson moments.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from workloads.hypergraphs import uniform01

P32 = 1 << 32


def test_philox_known_answers(oracle):
    kat = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, want in kat:
        assert [int(x) for x in oracle.philox4x32_10(ctr, key)] == want


def test_philox_words_look_uniform(oracle):
    # 4096 blocks of consecutive counters: top byte histogram is flat (chi-square, 255 dof)
    words = np.concatenate([oracle.philox4x32_10([i, 7, 9, 11], [1, 0]) for i in range(4096)])
    hist = np.bincount(words >> np.uint32(24), minlength=256)
    exp = len(words) / 256
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 400  # p ~ 1e-7 for 255 dof


def test_exp_neg_accuracy(oracle):
    # scaling and squaring: s <= 11 squarings for x <= 64 amplify the Horner error by 2^s
    xs = np.concatenate([np.geomspace(1e-12, 64.0, 3000), np.linspace(0.001, 64.0, 3000), [64.0]])
    for x in xs:
        got = oracle.exp_neg(float(x))
        want = math.exp(-float(x))
        assert abs(got - want) <= 4e-12 * want, x


def _boundaries(fn, n):
    """T_h = least word w with fn(w) > h, for h = 0..n-1 (fn is non-decreasing in w)."""
    out = []
    for h in range(n):
        lo, hi = 0, P32  # fn(lo-1) <= h ... search the first w with fn(w) > h
        while lo < hi:
            mid = (lo + hi) // 2
            if fn(mid) > h:
                hi = mid
            else:
                lo = mid + 1
        out.append(lo)
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 7, 13, 20])
@pytest.mark.parametrize("thr", [1, 1 << 20, 214748364, 42949672, 1288490188, 3 << 30, P32 - 1])
def test_binomial_thresholds_exact(oracle, n, thr):
    p = Fraction(thr, P32)
    q = 1 - p
    cum = Fraction(0)
    exact = []
    for h in range(n):
        cum += math.comb(n, h) * p ** h * q ** (n - h)
        exact.append(math.floor(cum * P32))
    got = _boundaries(lambda w: oracle.binomial_h(n, thr, w), n)
    for h in range(n):
        e = min(exact[h], P32)
        assert abs(got[h] - e) <= 1, (n, thr, h, got[h], e)


def test_binomial_special_cases(oracle):
    for n in (0, 1, 5, 20):
        assert oracle.binomial_h(n, 0, 12345) == 0
        assert oracle.binomial_h(n, P32, 0) == n
        assert oracle.binomial_h(n, P32, P32 - 1) == n
    assert oracle.binomial_h(5, 1, 0) == 0
    assert oracle.binomial_h(5, P32 - 1, P32 - 1) == 5


@pytest.mark.parametrize("n,thr", [(21, 214748364), (1000, 2147483), (500, 171798691),
                                   (64, 4026531840), (100, 2576980377)])
def test_poisson_thresholds_exact(oracle, n, thr):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    lam = mpmath.mpf(n) * mpmath.mpf(thr) / P32
    assert lam <= 64
    term = mpmath.e ** (-lam)
    cum = mpmath.mpf(0)
    hmax = min(n, int(lam + 12 * mpmath.sqrt(lam) + 30))
    exact = []
    for h in range(hmax):
        cum += term
        term = term * lam / (h + 1)
        exact.append(int(mpmath.floor(cum * P32)))
    assert oracle.poisson_parts(n, thr) == 1
    got = _boundaries(lambda w: oracle.poisson_h(n, thr, [w])[0], hmax)
    for h in range(hmax):
        assert abs(got[h] - exact[h]) <= 2, (n, thr, h, got[h], exact[h])


@pytest.mark.parametrize("lam_target", [65.0, 200.0, 777.0])
def test_poisson_split_moments(oracle, lam_target):
    n = 100000
    thr = int(lam_target / n * P32)
    lam = n * thr / P32
    c = oracle.poisson_parts(n, thr)
    assert c == math.ceil(lam / 64)
    draws = 20000
    u = uniform01(99, int(lam_target), draws * c)
    words = (u * P32).astype(np.uint64).astype(np.uint32).reshape(draws, c)
    hs = np.array([oracle.poisson_h(n, thr, words[i])[0] for i in range(draws)], dtype=np.float64)
    se_mean = math.sqrt(lam / draws)
    assert abs(hs.mean() - lam) < 5 * se_mean
    se_var = lam * math.sqrt(2.0 / draws) + 1.0
    assert abs(hs.var() - lam) < 5 * se_var


def test_poisson_truncated_at_n(oracle):
    # lambda = n p with p close to 1: the draw never exceeds n
    n = 30
    thr = P32 - 10
    for w in (0, 1 << 31, P32 - 1):
        h, used = oracle.poisson_h(n, thr, [w])
        assert 0 <= h <= n and used == 1
