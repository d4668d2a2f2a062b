"""Host-side analysis helpers: closed forms of the structure factor."""
import numpy as np


def test_structure_factor_closed_forms():
    """S(q) of ordered patterns: ferromagnet -> N at q = 0; Neel -> N at
    (pi, pi); columns repeating up-up-down -> N/9 at q = 0 and 4N/9 at
    (0, +-2 pi/3); independent random spins -> about 1 everywhere."""
    from paper_2511_20911_gb300 import analysis
    R, C = 18, 12
    N = R * C
    fm = np.ones((1, R, C))
    s = analysis.structure_factor(fm)
    assert abs(s[0, 0] - N) < 1e-9 and abs(s.sum() - N) < 1e-9
    neel = np.fromfunction(lambda r, c: 1 - 2 * ((r + c) % 2), (R, C))[None]
    s = analysis.structure_factor(neel)
    assert abs(s[R // 2, C // 2] - N) < 1e-9
    uud = np.tile(np.array([1, 1, -1]), (R, C // 3))[None]
    s = analysis.structure_factor(uud)
    assert abs(s[0, 0] - N / 9) < 1e-9
    assert abs(s[0, C // 3] - 4 * N / 9) < 1e-9 and abs(s[0, 2 * C // 3] - 4 * N / 9) < 1e-9
    rng = np.random.default_rng(3)
    rnd = rng.choice([-1.0, 1.0], size=(4000, R, C))
    assert abs(analysis.structure_factor(rnd).mean() - 1.0) < 0.02
