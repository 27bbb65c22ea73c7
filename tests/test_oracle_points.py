"""Pins of the oracle's point generators (Sec. 3.1) against things other than itself:
SciPy's Sobol and Halton (run as libraries), closed forms of the radical inverse,
the (0, m, 2)-net property by brute force, and the Philox known-answer vectors."""
import numpy as np
import pytest

from oracle import oracle as O


def _bitrev32(x):
    x = np.asarray(x, dtype=np.uint64)
    r = np.zeros_like(x)
    for b in range(32):
        r |= ((x >> np.uint64(b)) & np.uint64(1)) << np.uint64(31 - b)
    return r


def test_sobol_matches_scipy_gray_order():
    qmc = pytest.importorskip("scipy.stats.qmc")
    dims, n = 80, 1024
    ref = qmc.Sobol(dims, scramble=False, bits=32).random(n)
    ref_u32 = np.round(ref * 2.0 ** 32).astype(np.uint64)
    got = O.generate_points("sobol", dims, 0, n, "u32").astype(np.uint64)
    assert np.array_equal(got, ref_u32)


def test_sobol_random_access_far_index_matches_scipy():
    qmc = pytest.importorskip("scipy.stats.qmc")
    s = qmc.Sobol(5, scramble=False, bits=32)
    s.fast_forward(1_000_000)
    ref = np.round(s.random(64) * 2.0 ** 32).astype(np.uint64)
    got = O.generate_points("sobol", 5, 1_000_000, 64, "u32").astype(np.uint64)
    assert np.array_equal(got, ref)


def test_sobol_dim0_is_van_der_corput_of_gray_code():
    i = np.arange(1, 5000, dtype=np.uint64)
    g = i ^ (i >> np.uint64(1))
    got = O.generate_points("sobol", 1, 1, len(i), "u32")[:, 0].astype(np.uint64)
    assert np.array_equal(got, _bitrev32(g))


def _is_02_net(u32_2d, m):
    """Every elementary box 2^-a x 2^-(m-a) holds exactly one of the 2^m points."""
    x = u32_2d.astype(np.uint64)
    for a in range(m + 1):
        bx = x[:, 0] >> np.uint64(32 - a) if a > 0 else np.zeros(len(x), np.uint64)
        by = x[:, 1] >> np.uint64(32 - (m - a)) if m - a > 0 else np.zeros(len(x), np.uint64)
        cell = bx * np.uint64(1 << (m - a)) + by
        counts = np.bincount(cell.astype(np.int64), minlength=1 << m)
        if not np.all(counts == 1):
            return False
    return True


@pytest.mark.parametrize("kind,seed", [("sobol", 0), ("sobol_owen", 1), ("sobol_owen", 12345)])
def test_first_two_dims_form_0m2_net(kind, seed):
    m = 10
    pts = O.generate_points(kind, 2, 0, 1 << m, "u32", seed=seed)
    assert _is_02_net(pts, m)


def test_owen_scramble_is_nested():
    """Two values sharing their top j bits still share them after the scramble, and
    the scramble is a bijection on each level (it permutes the 2^j intervals)."""
    rng = np.random.default_rng(0)
    seed_d = O.owen_seed(7, 3)
    for j in (1, 4, 9, 17):
        ys = rng.integers(0, 2 ** 32, size=64, dtype=np.uint64)
        for y in ys:
            z = int(y) ^ int(rng.integers(0, 2 ** (32 - j)))  # same top j bits
            a, b = O.owen_scramble(int(y), seed_d), O.owen_scramble(z, seed_d)
            assert (a >> (32 - j)) == (b >> (32 - j))
        tops = {O.owen_scramble(t << (32 - j), seed_d) >> (32 - j) for t in range(min(1 << j, 512))}
        assert len(tops) == min(1 << j, 512)


def test_owen_scramble_changes_points_and_depends_on_seed():
    a = O.generate_points("sobol_owen", 3, 1, 256, "u32", seed=1)
    b = O.generate_points("sobol_owen", 3, 1, 256, "u32", seed=2)
    c = O.generate_points("sobol", 3, 1, 256, "u32")
    assert not np.array_equal(a, c)
    assert not np.array_equal(a, b)
    # stratification survives: each dim alone is a (0, 8, 1)-net on indices 0..255
    full = O.generate_points("sobol_owen", 3, 0, 256, "u32", seed=1)
    for d in range(3):
        assert len(np.unique(full[:, d] >> 24)) == 256


def test_radical_inverse_identities():
    for b in (2, 3, 5, 7, 11, 13):
        for k in range(0, 12):
            if b ** k >= 2 ** 40:
                break
            assert O.radical_inverse(b ** k, b) == float(b) ** (-k - 1)
        for i in range(1, 300):
            lhs = O.radical_inverse(b * i, b)
            rhs = O.radical_inverse(i, b) / b
            assert abs(lhs - rhs) <= 1e-16 * max(rhs, 1e-300) + np.spacing(rhs)


def test_radical_inverse_base2_is_bit_reversal():
    i = np.arange(1, 3000, dtype=np.uint64)
    ref = _bitrev32(i).astype(np.float64) / 2.0 ** 32
    got = np.array([O.radical_inverse(int(v), 2) for v in i])
    assert np.array_equal(got, ref)


def test_halton_is_exact_rational_correctly_rounded():
    from fractions import Fraction

    got = O.generate_points("halton", 6, 1, 700, "f64")
    for j in range(0, 700, 7):
        i = j + 1
        for d, b in enumerate((2, 3, 5, 7, 11, 13)):
            q, k, val = i, 1, Fraction(0)
            while q:
                q, r = divmod(q, b)
                val += Fraction(r, b ** k)
                k += 1
            assert got[j, d] == float(val)  # float(Fraction) rounds correctly


def test_halton_matches_scipy_within_two_ulp():
    # SciPy sums the digits in floating point (several roundings), so it may differ
    # from the correctly rounded value by a couple of units in the last place.
    qmc = pytest.importorskip("scipy.stats.qmc")
    dims, n = 20, 2048
    ref = qmc.Halton(dims, scramble=False).random(n)
    got = O.generate_points("halton", dims, 0, n, "f64")
    ulp = np.spacing(np.maximum(ref, 1e-300))
    assert np.all(np.abs(got - ref) <= 2 * ulp)


def test_first_primes():
    assert [O.prime(n) for n in range(10)] == [2, 3, 5, 7, 11, 13, 17, 19, 23, 29]
    assert O.prime(79) == 409


def test_hammersley_first_dim_is_i_over_n_and_rest_halton():
    N = 1000
    got = O.generate_points("hammersley", 4, 1, N, "f64", total_n=N)
    i = np.arange(1, N + 1)
    assert np.array_equal(got[:, 0], i / N)
    assert got[-1, 0] == 1.0
    hal = O.generate_points("halton", 3, 1, N, "f64")
    assert np.array_equal(got[:, 1:], hal)


def test_philox_known_answer_vectors():
    # Known-answer vectors for Philox4x32-10 published with the Random123 library
    # (Salmon, Moraes, Dror & Shaw, SC'11): (counter, key) -> output.
    kat = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, out in kat:
        assert O.philox4x32_10(ctr, key) == out


def test_philox_points_layout_and_uniformity():
    seed = 0x1234_5678_9ABC
    pts = O.generate_points("philox", 6, 10, 4096, "u32", seed=seed)
    # counter = (i_lo, i_hi, d / 4, 0), key = (seed_lo, seed_hi), word d % 4
    for j in (0, 17, 4095):
        i = 10 + j
        w0 = O.philox4x32_10([i & 0xFFFFFFFF, i >> 32, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
        w1 = O.philox4x32_10([i & 0xFFFFFFFF, i >> 32, 1, 0], [seed & 0xFFFFFFFF, seed >> 32])
        assert list(pts[j]) == w0 + w1[:2]
    # chi-square on 64 bins per dimension (df = 63; 99.99% quantile ~ 114)
    for d in range(6):
        counts = np.bincount((pts[:, d] >> 26).astype(np.int64), minlength=64)
        chi2 = np.sum((counts - 64.0) ** 2 / 64.0)
        assert chi2 < 114


@pytest.mark.parametrize("kind", ["sobol", "sobol_owen", "halton", "philox"])
def test_f32_is_f64_rounded_toward_zero(kind):
    f64 = O.generate_points(kind, 5, 1, 4096, "f64", seed=3)
    f32 = O.generate_points(kind, 5, 1, 4096, "f32", seed=3)
    near = f64.astype(np.float32)
    rz = np.where(near.astype(np.float64) > f64, np.nextafter(near, np.float32(0)), near)
    assert np.array_equal(f32, rz)
    assert np.all(f32 < 1.0)


def test_u32_points_scale_to_f64_exactly():
    u = O.generate_points("sobol_owen", 4, 1, 512, "u32", seed=9)
    f = O.generate_points("sobol_owen", 4, 1, 512, "f64", seed=9)
    assert np.array_equal(u.astype(np.float64) / 2.0 ** 32, f)


def test_halton_rejects_u32_format():
    with pytest.raises(ValueError):
        O.generate_points("halton", 2, 1, 4, "u32")


# --- Niederreiter base 2 and Faure (the paper's other two low-discrepancy sequences) ---

def _is_tms_net(u32, m, t):
    """(t, m, s)-net in base 2: for every split d_1 + ... + d_s = m - t, each elementary
    box (2^-d_1 x ... x 2^-d_s) holds exactly 2^t of the 2^m points."""
    import itertools

    x = u32.astype(np.uint64)
    s = x.shape[1]
    k = m - t
    for split in itertools.product(range(k + 1), repeat=s):
        if sum(split) != k:
            continue
        cell = np.zeros(len(x), np.uint64)
        for j, dj in enumerate(split):
            lead = x[:, j] >> np.uint64(32 - dj) if dj else np.zeros(len(x), np.uint64)
            cell = cell * np.uint64(1 << dj) + lead
        if not np.all(np.bincount(cell.astype(np.int64), minlength=1 << k) == (1 << t)):
            return False
    return True


def test_niederreiter_dim0_is_van_der_corput_in_natural_order():
    i = np.arange(0, 5000, dtype=np.uint64)
    got = O.generate_points("niederreiter", 1, 0, len(i), "u32")[:, 0].astype(np.uint64)
    assert np.array_equal(got, _bitrev32(i))


def test_niederreiter_dim1_is_the_pascal_matrix_of_sobol_dim1():
    """p = x + 1 gives the Pascal matrix mod 2, the generator of Sobol's second
    dimension: the Niederreiter point i equals the Sobol point whose Gray code is i."""
    i = np.arange(0, 4096, dtype=np.uint64)
    nied = O.generate_points("niederreiter", 2, 0, len(i), "u32")[:, 1]
    inv = i.copy()
    for sh in (1, 2, 4, 8, 16, 32):
        inv ^= inv >> np.uint64(sh)
    sob = np.array([O.lib().or_sobol_u32(O.sobol_directions(2).ctypes.data_as(O.C.POINTER(O.C.c_uint32)), 1, int(k))
                    for k in inv], dtype=np.uint32)
    assert np.array_equal(nied, sob)


@pytest.mark.parametrize("dims,t", [(3, 1), (5, 5)])
@pytest.mark.parametrize("block", [0, 5])
def test_niederreiter_aligned_blocks_are_tms_nets(dims, t, block):
    """t = sum of (degree - 1) over the polynomials x, x + 1, x^2 + x + 1, x^3 + x + 1,
    x^3 + x^2 + 1 bounds the quality parameter: a wrong polynomial order, a reducible
    polynomial or a transposed generator matrix breaks the net property.  In three
    dimensions the bound is attained (base 2 has no (0, m, 3)-net from these
    matrices)."""
    m = 10
    pts = O.generate_points("niederreiter", dims, block << m, 1 << m, "u32")
    assert _is_tms_net(pts, m, t)
    if dims == 3:
        assert not _is_tms_net(pts, m, t - 1)


def test_faure_base_is_the_smallest_prime_not_below_the_dimension():
    assert [O.faure_base(s) for s in (1, 2, 3, 4, 5, 6, 8, 80)] == [2, 2, 3, 5, 5, 7, 11, 83]


def test_faure_dim0_is_the_radical_inverse_and_values_are_exact():
    from fractions import Fraction

    b = O.faure_base(5)
    pts = O.generate_points("faure", 5, 0, 3000, "f64")
    for i in range(3000):
        assert pts[i, 0] == O.radical_inverse(i, b)
    # every coordinate is a fraction with denominator b^K, rounded once
    for i in (7, 124, 2999):
        K = len(np.base_repr(i, b))
        for d in range(5):
            frac = Fraction(pts[i, d]).limit_denominator(b ** K)
            assert float(frac) == pts[i, d] and (b ** K) % frac.denominator == 0


@pytest.mark.parametrize("dims,m", [(3, 4), (5, 3)])
def test_faure_is_a_0ms_net_in_base_b(dims, m):
    """Each elementary b-adic box of volume b^-m holds exactly one of the b^m points
    (Faure's (0, s)-sequence property), for every split of m over the dimensions."""
    import itertools

    b = O.faure_base(dims)
    n = b ** m
    pts = O.generate_points("faure", dims, 0, n, "f64")
    for split in itertools.product(range(m + 1), repeat=dims):
        if sum(split) != m:
            continue
        cell = np.zeros(n, np.int64)
        for j, dj in enumerate(split):
            cell = cell * (b ** dj) + np.floor(pts[:, j] * b ** dj + 1e-9).astype(np.int64)
        assert np.all(np.bincount(cell, minlength=n) == 1), split
