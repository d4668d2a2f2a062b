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


def test_ss_counts_match_the_oracle(orc):
    from paper_2511_20911_gb300 import analysis
    rng = np.random.default_rng(9)
    for L, Lc in ((6, 6), (4, 8), (18, 18), (2, 4)):
        v = rng.choice(np.array([-1, 1], np.int8), size=(5, L, Lc))
        nJ, nP, M = analysis.ss_counts(v)
        for k in range(5):
            if L >= 3 and Lc >= 3:
                assert (nJ[k], nP[k], M[k]) == orc.counts(v[k], (L, Lc)), (L, Lc, k)


def test_ground_states_of_the_known_phases():
    """Per spin: FM 2J + J'/2 - h; Neel -2J + J'/2; dimer -J'/2 (J' > 2J);
    the 1/3 plateau (J' = J/2, h = 4): rows up-up-down, neighbouring rows
    shifted by one, so each row and each column pair contributes -1/3 of a
    bond per site (N_J = -2N/3), the dimers average -1/3 (N_J' = -N/6) and
    M = N/3: E/N = -2J/3 - J'/6 - h/3."""
    from paper_2511_20911_gb300 import analysis
    for L in (6, 12):
        N = L * L
        assert analysis.ground_state_energy(L, 1.0, 1.0, 7.0)[0] == 16 * N * (2 + 0.5 - 7)
        assert analysis.ground_state_energy(L, 1.0, 1.0, 0.0)[0] == 16 * N * (-2 + 0.5)
        assert analysis.ground_state_energy(L, 1.0, 2.5, 0.0)[0] == 16 * N * (-1.25)
        e, cell, pat = analysis.ground_state_energy(L, 1.0, 0.5, 4.0)
        assert e == round(16 * N * (-2 / 3 - 0.5 / 6 - 4 / 3)) and pat.sum() * 3 == pat.size


def test_phase_labels_of_the_known_ground_states():
    """Counts of the ideal states (N = 36): FM N_J = 2N, N_J' = N/2, M = N;
    Neel N_J = -2N, N_J' = N/2, M = 0; dimer N_J = 0, N_J' = -N/2, M = 0; the
    1/3 plateau of the closed form above (N_J = -2N/3, N_J' = -N/6, M = N/3)."""
    from paper_2511_20911_gb300 import analysis
    N = 36
    assert analysis.phase_label(2 * N, N // 2, -N, N) == "FM"
    assert analysis.phase_label(-2 * N, N // 2, 0, N) == "Neel"
    assert analysis.phase_label(0, -N // 2, 0, N) == "dimer"
    assert analysis.phase_label(-2 * N // 3, -N // 6, N // 3, N) == "1/3 plateau"
    assert analysis.phase_label(0, 0, N // 2, N) == "1/2 plateau"
    assert analysis.phase_label(0, 0, N // 9, N) == "m=1/9"
    for J, Jp, h, name in ((1.0, 1.0, 7.0, "FM"), (1.0, 1.0, 0.0, "Neel"), (1.0, 2.5, 0.0, "dimer"),
                           (1.0, 0.5, 4.0, "1/3 plateau")):
        L = 12
        e, (a, b), pat = analysis.ground_state_energy(L, J, Jp, h)
        nJ, nP, M = (int(x[0]) * (L * L // (a * b)) for x in analysis.ss_counts(pat[None]))
        assert analysis.phase_label(nJ, nP, M, L * L) == name
