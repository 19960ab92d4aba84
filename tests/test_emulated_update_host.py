"""Error budget of the emulated-FP64 trailing update (the digit scheme of k_herk_emu.cu), checked
on the host with exact integer arithmetic: each panel component x of a row with max |x| < 2^e is
rounded to X = round(x 2^(63 - e)) and cut into seven balanced base-2^8 digits; the products of
digit pairs with p + q <= 6 (0-based) are summed per level.

Pinned here, on random and worst-case (all digits at their bound) panels:
* every digit is an integer of at most 8 significant bits (exact in BF16) with |d_1| <= 256 and
  |d_p| <= 128 after the first;
* every level's sum over K = 32 (64 real products per output) stays below 2^24 units, so FP32
  accumulation of each level is exact;
* the kept levels reproduce the exact complex product sum to 2^-47 of 2^(e_r + e_c).
"""
from fractions import Fraction

import numpy as np

K, DIG, BETA, NLEV = 32, 7, 8, 7


def row_digits(row):
    """Digits (DIG x K x 2 ints, Re/Im) and exponent e of one panel row (complex128, length K)."""
    comps = np.concatenate([row.real, row.imag])
    mx = float(np.max(np.abs(comps)))
    e = int(np.frexp(mx)[1]) if mx > 0 else 0          # mx < 2^e
    d = np.zeros((DIG, K, 2), dtype=object)
    for k in range(K):
        for c, x in enumerate((row[k].real, row[k].imag)):
            X = round(Fraction(x) * Fraction(2) ** (63 - e))
            for p in range(DIG):
                sh = 55 - BETA * p
                dp = (X + (1 << (sh - 1))) >> sh        # round half up
                X -= dp << sh
                d[p, k, c] = dp
    return d, e


def level_sums(dr, dc):
    """Per level s = p + q: (Re, Im) of sum_k a_p^r conj(a_q^c) in units of 2^(-8 s) (integers)."""
    out = []
    for s in range(NLEV):
        re = im = 0
        for p in range(s + 1):
            q = s - p
            if p >= DIG or q >= DIG:
                continue
            for k in range(K):
                pr, qr = dr[p, k]
                pc, qc = dc[q, k]
                re += pr * pc + qr * qc
                im += qr * pc - pr * qc
        out.append((re, im))
    return out


def emulated(dr, er, dc, ec):
    tot_re = tot_im = Fraction(0)
    for s, (re, im) in enumerate(level_sums(dr, dc)):
        w = Fraction(2) ** (-BETA * s)
        tot_re += re * w
        tot_im += im * w
    scale = Fraction(2) ** (er + ec - 2 * BETA)
    return tot_re * scale, tot_im * scale


def exact(r, c):
    re = sum(Fraction(a.real) * Fraction(b.real) + Fraction(a.imag) * Fraction(b.imag) for a, b in zip(r, c))
    im = sum(Fraction(a.imag) * Fraction(b.real) - Fraction(a.real) * Fraction(b.imag) for a, b in zip(r, c))
    return re, im


def check_pair(r, c):
    dr, er = row_digits(r)
    dc, ec = row_digits(c)
    for d in (dr, dc):
        # integers of magnitude <= 256 have at most 8 significant bits: exact in BF16
        assert max(abs(int(v)) for v in d[0].reshape(-1)) <= 256
        assert max(abs(int(v)) for v in d[1:].reshape(-1)) <= 128
    for re, im in level_sums(dr, dc):
        assert abs(re) < 2 ** 24 and abs(im) < 2 ** 24
    got = emulated(dr, er, dc, ec)
    want = exact(r, c)
    bound = Fraction(2) ** (er + ec - 47)
    assert abs(got[0] - want[0]) <= bound and abs(got[1] - want[1]) <= bound


def test_random_panels():
    rng = np.random.default_rng(7)
    for scale_r, scale_c in ((1.0, 1.0), (1e-3, 2.5), (3e-200, 1e150)):
        r = scale_r * (rng.standard_normal(K) + 1j * rng.standard_normal(K))
        c = scale_c * (rng.standard_normal(K) + 1j * rng.standard_normal(K))
        r[5] *= 1e-12   # components far below the row maximum keep their leading bits
        check_pair(r, c)


def test_worst_case_digits():
    """Every component with the digits 255, 127, 127, ... (as far as a double's 53 bits reach): all
    products of a level add with one sign, so the level sums come near their largest magnitudes
    (8.3e6 units at level 5; the bound for any input is 64 * 2^14 * 9 = 9.4e6 at level 6, under
    the 2^24 = 1.68e7 of exact FP32 accumulation)."""
    X = 255 * 2 ** 55 + sum(127 * 2 ** (55 - 8 * p) for p in range(1, DIG))
    x = float(Fraction(X, 2 ** 63))
    r = np.full(K, x + 1j * x)
    dr, _ = row_digits(r)
    assert int(dr[0, 0, 0]) == 255 and int(dr[3, 0, 0]) == 127
    sums = level_sums(dr, dr)
    assert max(abs(re) for re, _ in sums) > 8e6
    check_pair(r, r)
    check_pair(r, np.full(K, -x + 1j * x))
    x = 1.0 - 2.0 ** -53                      # all 53 mantissa bits set
    check_pair(np.full(K, x + 1j * x), np.full(K, x - 1j * x))


def test_zero_and_subnormal_rows():
    r = np.zeros(K, dtype=complex)
    c = np.full(K, 0.5 + 0.25j)
    check_pair(r, c)
    t = np.full(K, 5e-324 + 0j)              # the smallest subnormal
    t[3] = 3e-320
    check_pair(t, c)
