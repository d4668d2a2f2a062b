"""Qualitative physics of the sampler at L = 18 (the paper's lattice size):
the Neel order of J' = J, h = 0 shows as the structure-factor peak at
q = (pi, pi) (Sec. IV.B, Eq. 11); at J' = J, h = 3 the chains sit on the 1/3
magnetisation plateau (Sec. III) with S(q) peaks at the plateau's
(pi, +-2 pi/3) wavevectors besides q = 0.  The paper's figures are missing,
so these are the qualitative statements of its text, checked on the GPU
sampler's own configurations."""
import numpy as np
import pytest

import paper_2511_20911_gb300 as crbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


L, N = 18, 324


def _run(Jp, h, beta, n=1024, burn=30000, meas=20000, seed=7):
    s = crbm.Sampler(L, dict(J=[1.0], Jp=[Jp], h=[h], beta=[beta]), n, seed=seed, measure_every=10,
                     sq_every=100, layout=crbm.CRBM_LAYOUT_SMEM)
    s.sweep(burn)
    s.reset_observables()
    s.sweep(meas)
    obs = s.observables()                      # per chain: n, sum NJ, sum NJ', sum M, ...
    m = obs[:, 3].sum() / obs[:, 0].sum() / N
    return s.structure_factor()[0] / N, m


def test_neel_order_peaks_at_pi_pi():
    """J' = J = 1, h = 0, beta = 3: the largest S(q) is at (pi, pi), and it
    holds a sizeable share of the weight (ordered domains)."""
    sq, m = _run(1.0, 0.0, 3.0)
    peak = np.unravel_index(np.argmax(sq), sq.shape)
    assert peak == (L // 2, L // 2), (peak, sq[peak])
    assert sq[L // 2, L // 2] > 0.1, sq[L // 2, L // 2]
    assert abs(m) < 0.02, m


def test_one_third_plateau():
    """J' = J = 1, h = 3, beta = 3: m within 0.05 of 1/3; S(0) = m^2 per spin
    up to fluctuations; the largest S(q) away from q = 0 sits at one of the
    plateau wavevectors (pi, +-2 pi/3) or (+-2 pi/3, pi)."""
    sq, m = _run(1.0, 3.0, 3.0)
    assert abs(m - 1.0 / 3.0) < 0.05, m
    assert abs(sq[0, 0] - m * m) < 0.02, (sq[0, 0], m)
    rest = sq.copy()
    rest[0, 0] = 0.0
    peak = tuple(int(x) for x in np.unravel_index(np.argmax(rest), rest.shape))
    plateau = {(L // 2, L // 3), (L // 2, 2 * L // 3), (L // 3, L // 2), (2 * L // 3, L // 2)}
    assert peak in plateau, (peak, rest[peak])
