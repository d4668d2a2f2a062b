"""Pins of two oracle pieces the sampler tests rely on: the structure factor
S(q) (Sec. IV.B, Eq. 11, reported per spin) and the bfloat16 rounding of the
learned proposal's net."""
import numpy as np
import pytest


def _ordered_states(R, C):
    fm = np.ones((R, C), np.int8)
    neel = np.fromfunction(lambda r, c: 1 - 2 * ((r + c) % 2), (R, C)).astype(np.int8)
    uud = np.tile(np.array([1, 1, -1], np.int8), (R, C // 3))
    return fm, neel, uud


@pytest.mark.parametrize("R,C", [(6, 6), (12, 12), (18, 12), (6, 18)])
def test_structure_factor_closed_forms(orc, R, C):
    """Ferromagnet: S(0) = N and S(q != 0) = 0.  Neel: S(pi, pi) = N and 0
    elsewhere.  Columns repeating up-up-down: N/9 at q = 0, 4N/9 at
    q = (0, +-2 pi/3), 0 elsewhere.  Every state: sum_q S(q) = N (Parseval)."""
    N = R * C
    fm, neel, uud = _ordered_states(R, C)
    s = orc.structure_factor(fm)
    ref = np.zeros((R, C))
    ref[0, 0] = N
    assert np.allclose(s, ref, atol=1e-9)
    s = orc.structure_factor(neel)
    ref = np.zeros((R, C))
    ref[R // 2, C // 2] = N
    assert np.allclose(s, ref, atol=1e-9)
    s = orc.structure_factor(uud)
    ref = np.zeros((R, C))
    ref[0, 0] = N / 9
    ref[0, C // 3] = ref[0, 2 * C // 3] = 4 * N / 9
    assert np.allclose(s, ref, atol=1e-9)
    for st in (fm, neel, uud):
        assert abs(orc.structure_factor(st).sum() - N) < 1e-8


def test_structure_factor_equals_the_fft_power(orc):
    """Random states: S(q) = |FFT(s)(q)|^2 / N at q = 2 pi (nR / R, nC / C)
    (numpy's FFT uses the opposite phase sign, which leaves |.|^2 unchanged);
    a transposed or sign-flipped phase would fail on rectangles."""
    rng = np.random.default_rng(12)
    for R, C in ((6, 6), (8, 12), (18, 18), (5, 7)):
        v = rng.choice(np.array([-1, 1], np.int8), size=(R, C))
        ref = np.abs(np.fft.fft2(v.astype(np.float64))) ** 2 / (R * C)
        assert np.allclose(orc.structure_factor(v), ref, rtol=1e-12, atol=1e-9)


def _bf16_exact(x):
    """Round-to-nearest-even of a float32 value to 8 significant bits, by
    integer arithmetic on the value's exact rational form (Python Fractions)."""
    from fractions import Fraction
    x = float(np.float32(x))
    if x == 0 or not np.isfinite(x):
        return x
    f = Fraction(x)
    sign = -1 if f < 0 else 1
    f = abs(f)
    e = 0
    while f >= 2:
        f /= 2
        e += 1
    while f < 1:
        f *= 2
        e -= 1
    e = max(e, -126)                     # bf16 shares float32's exponent range
    ulp = Fraction(2) ** (e - 7)
    q, r = divmod(abs(Fraction(x)), ulp)
    if r > ulp / 2 or (r == ulp / 2 and q % 2 == 1):
        q += 1
    val = q * ulp
    if val >= Fraction(2) ** 128:
        return sign * float("inf")
    return sign * float(val)


def _cases():
    f32 = np.float32
    ties = []
    for m in (0x3F80, 0x3F81, 0x4049, 0xC2F6, 0x0080, 0x7F7E):     # bf16 patterns
        base = np.array([m << 16], np.uint32).view(np.float32)[0]
        tie_bits = np.array([(m << 16) | 0x8000], np.uint32)
        tie = tie_bits.view(np.float32)[0]
        below = np.array([tie_bits[0] - 1], np.uint32).view(np.float32)[0]
        above = np.array([tie_bits[0] + 1], np.uint32).view(np.float32)[0]
        ties += [base, tie, below, above]
    sub = [np.array([b], np.uint32).view(np.float32)[0] for b in
           (0x00000001, 0x00008000, 0x00018000, 0x00007FFF, 0x0000C000, 0x007FFFFF, 0x80008000)]
    big = [f32(3.3895314e38), np.finfo(np.float32).max, -np.finfo(np.float32).max, f32(1e38)]
    return [float(x) for x in ties + sub + big + [0.0, -0.0, 1.0, -2.5, 1.0 / 3.0]]


def test_bf16_rounding_matches_independent_conversions(orc):
    """orc_bf16 against torch's float32 -> bfloat16 conversion and against
    exact rational round-to-nearest-even, on ties (both parities), one ulp
    either side of a tie, float32 subnormals, the largest values (rounding
    to infinity) and 10^5 random values over a wide exponent range."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    rnd = (rng.standard_normal(100000) * np.exp2(rng.integers(-40, 40, 100000))).astype(np.float32)
    xs = np.concatenate([np.array(_cases(), np.float32), rnd])
    ours = np.array([orc.bf16(float(x)) for x in xs])
    theirs = torch.from_numpy(xs).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, theirs)
    for x in _cases():
        assert orc.bf16(x) == _bf16_exact(x), (x, orc.bf16(x), _bf16_exact(x))
    # a truncating rounding would differ here: ties go to even, above-tie up
    one_tie = np.array([0x3F808000], np.uint32).view(np.float32)[0]     # 1 + 2^-8
    assert orc.bf16(float(one_tie)) == 1.0
    three_tie = np.array([0x3F818000], np.uint32).view(np.float32)[0]   # 1 + 3 * 2^-8
    assert orc.bf16(float(three_tie)) == 1.0 + 2.0 ** -6
    assert orc.bf16(float(np.finfo(np.float32).max)) == float("inf")
    assert np.isnan(orc.bf16(float("nan")))
