"""The numerics of the float64 force pass's sums (Eq. 3 as sum_j s_ij d_ij
with d_ij exact in fixed point and the products and totals in float32
pieces), restated step by step in numpy float32 (IEEE round-to-nearest
operations, FMA from the exact float64 product) and checked against exact
rational arithmetic: the split of s and of d, and the float-float totals of
54-term sums, against the error bounds the kernels rely on. CPU only; the
GPU tests compare the kernels themselves with the oracle."""
from fractions import Fraction

import numpy as np

F32 = np.float32
U32 = np.uint32


def f32_bits(u):
    return np.asarray(u, dtype=U32).view(F32)


def fma32(a, b, c):
    """fl32(a b + c): the product of two float32 values is exact in
    float64, and here so is its sum with c (the operands of the sums below
    lie within 2^53 of each other), so one rounding to float32 remains."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)


def ssplit(s):
    """s -> s_h (24 significant bits, truncated) + s_l (the remaining 29
    bits rounded to 23), from the float64 bit pattern."""
    b = np.asarray(s, dtype=np.float64).view(np.uint64)
    hi = (b >> np.uint64(32)).astype(U32)
    lo = (b & np.uint64(0xFFFFFFFF)).astype(U32)
    ab = hi & U32(0x7FFFFFFF)
    sg = hi & U32(0x80000000)
    inr = (ab - U32(923 << 20)) < U32((1151 - 923) << 20)
    adj = ab - U32(896 << 20)
    fb = (adj << U32(3)) | (lo >> U32(29))
    sh = f32_bits(fb | sg)
    F = ((fb & U32(0x7F800000)) - U32(23 << 23)) | sg
    sl = f32_bits(F + (((lo & U32(0x1FFFFFFF)) + U32(32)) >> U32(6))) - f32_bits(F)
    with np.errstate(over="ignore"):  # beyond the float32 range: the conversion's inf, as on the device
        sh = np.where(inr, sh, np.asarray(s).astype(F32))
    sl = np.where(inr, sl, F32(0.0))
    return sh.astype(F32), sl.astype(F32)


def dsplit_consts(kq, cb):
    sh = max(0, kq + cb - 54)
    rnd = (1 << (sh - 1)) if sh > 0 else 0
    mh = 0x4B400000 + (32 + sh - kq) * (1 << 23)
    mm = 0x4B000000 + (9 + sh - kq) * (1 << 23)
    ml = 0x4B000000 + (sh - kq) * (1 << 23)
    return dict(sh=sh, rnd=rnd, mh=mh, mm=mm, ml=ml)


def dsplit(dr, D):
    """d + rnd (int64, units 2^-kq) -> d_h + d_l: the high word, the next
    23 bits and the last 9 as exact float32 values, then Fast2Sum."""
    dr = np.asarray(dr, dtype=np.int64)
    sh = D["sh"]
    hi = (dr >> 32).astype(np.int32)
    lo = (dr & 0xFFFFFFFF).astype(U32)
    k = hi >> sh
    t = ((dr.view(np.uint64) >> np.uint64(9 + sh)) & np.uint64(0x7FFFFF)).astype(U32)
    u = (lo >> U32(sh)) & U32(0x1FF)
    a = (k.astype(np.int64) + D["mh"]).astype(U32).view(F32) - f32_bits(D["mh"])
    b = f32_bits(U32(D["mm"]) | t) - f32_bits(D["mm"])
    c = f32_bits(U32(D["ml"]) | u) - f32_bits(D["ml"])
    dh = a + b
    r = b - (dh - a)
    dl = r + c
    return dh.astype(F32), dl.astype(F32)


def add_term(A, c, sh, sl, dh, dl):
    """One component of ForceSumF::add: p = s_h d_h with its exact error
    and the small products in e; TwoSum of A + p; Fast2Sum renormalisation."""
    p = sh * dh
    e = fma32(sh, dh, -p)
    e = fma32(sl, dh, e)
    e = fma32(sh, dl, e)
    S = A + p
    bp = S - A
    err = (A - (S - bp)) + (p - bp)
    t = c + (err + e)
    An = S + t
    c = t - (An - S)
    return An, c


def random_s(rng, n):
    """s_ij over the magnitudes a force pass meets: 1e-4..1e4 eV/A^2, signs mixed."""
    return rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-4.0, 4.0, n)


def test_s_split_is_within_2_to_minus_47():
    rng = np.random.default_rng(11)
    s = rng.choice([-1.0, 1.0], 200000) * 10.0 ** rng.uniform(-25.0, 25.0, 200000)
    sh, sl = ssplit(s)
    err = np.abs((sh.astype(np.float64) + sl.astype(np.float64)) - s) / np.abs(s)
    assert err.max() <= 2.0 ** -47
    # the high part alone is s truncated to 24 significant bits
    assert np.all(np.abs(sh.astype(np.float64)) <= np.abs(s))
    z = np.array([0.0, -0.0, 1e-35, np.inf, -np.inf, 1e300])
    zh, zl = ssplit(z)
    assert list(zh[:2]) == [0.0, 0.0] and np.all(zl == 0.0)
    assert np.isinf(zh[3]) and np.isinf(zh[4]) and np.isinf(zh[5])
    assert np.isnan(ssplit(np.array([np.nan]))[0][0])


def test_separation_split_is_within_2_to_minus_47():
    rng = np.random.default_rng(12)
    cb = 3  # r_cut below 8 A
    for kq in (40, 45, 50, 51, 53, 55, 57, 59):  # box sides from ~1 A to ~1e6 A
        D = dsplit_consts(kq, cb)
        scale = float(2 ** kq)
        dv = np.concatenate([rng.uniform(-7.9, 7.9, 40000), rng.uniform(-1e-5, 1e-5, 4000),
                             rng.uniform(-0.6, 0.6, 4000), np.zeros(8)])
        d = np.round(dv * scale).astype(np.int64)
        dh, dl = dsplit(d + D["rnd"], D)
        got = dh.astype(np.float64) + dl.astype(np.float64)
        exact = d.astype(np.float64) / scale  # exact: |d| < 2^53 units here or a power-of-two scaling of it
        pre = (2.0 ** (D["sh"] - 1) / scale) if D["sh"] > 0 else 0.0  # the pre-shift's rounding
        assert np.all(np.abs(got - exact) <= 2.0 ** -47 * np.abs(exact) + pre + 1e-300), kq


def test_force_sums_of_54_terms_against_exact_sums():
    """Error of the float-float total against the exact rational sum: each
    term contributes at most about 2^-46 of itself (the rounding of its
    small parts), so 54 terms stay below 64 * 2^-46 = 2^-40 of the largest
    term, and the typical error lies near 2^-46."""
    rng = np.random.default_rng(13)
    kq, cb, n_sums, n_terms = 51, 3, 1500, 54
    D = dsplit_consts(kq, cb)
    s = random_s(rng, (n_terms, n_sums))
    d = np.round(rng.uniform(-5.3, 5.3, (n_terms, n_sums)) * 2.0 ** kq).astype(np.int64)
    A = np.zeros(n_sums, F32)
    c = np.zeros(n_sums, F32)
    for j in range(n_terms):
        sh, sl = ssplit(s[j])
        dh, dl = dsplit(d[j] + D["rnd"], D)
        A, c = add_term(A, c, sh, sl, dh, dl)
    got = A.astype(np.float64) + c.astype(np.float64)
    unit = Fraction(1, 2 ** kq)
    rel = np.empty(n_sums)
    for m in range(n_sums):
        exact = sum(Fraction(float(s[j, m])) * int(d[j, m]) for j in range(n_terms)) * unit
        big = max(abs(float(s[j, m])) * abs(int(d[j, m])) for j in range(n_terms)) / 2.0 ** kq
        rel[m] = abs(float(Fraction(float(got[m])) - exact)) / big
    assert rel.max() <= 2.0 ** -40, rel.max()
    # (seen: worst 2^-44.5, RMS 2^-46.5)
    assert np.sqrt(np.mean(rel ** 2)) <= 2.0 ** -45, np.sqrt(np.mean(rel ** 2))


def test_renormalised_total_is_exact_in_float64():
    """|c| <= ulp(A)/2 after each term, so A + c needs at most 49 bits."""
    rng = np.random.default_rng(14)
    D = dsplit_consts(51, 3)
    A = np.zeros(5000, F32)
    c = np.zeros(5000, F32)
    for _ in range(54):
        sh, sl = ssplit(random_s(rng, 5000))
        dh, dl = dsplit(np.round(rng.uniform(-5.3, 5.3, 5000) * 2.0 ** 51).astype(np.int64) + D["rnd"], D)
        A, c = add_term(A, c, sh, sl, dh, dl)
        ulp = np.spacing(np.abs(A)).astype(np.float64)
        assert np.all(np.abs(c.astype(np.float64)) <= 0.5 * ulp + 1e-300)
