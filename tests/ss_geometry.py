"""Independent test-side statements of the Shastry–Sutherland geometry and of
exact results, used to pin the oracle (never used by the oracle or library).

The SS lattice (Fig. 1(a)): a periodic square lattice of nearest-neighbour J
bonds plus one diagonal J' bond per site; the diagonals form orthogonal dimers
on alternating plaquettes -- "\\" on plaquettes whose top-left corner (R, C)
has R, C both even, "/" on plaquettes with R, C both odd.
"""
import numpy as np


def ss_pairs(L):
    """(J pairs, J' pairs) of the even-L periodic SS lattice, as site-index pairs."""
    assert L % 2 == 0
    nn, dia = [], []
    for R in range(L):
        for C in range(L):
            s = R * L + C
            nn.append((s, R * L + (C + 1) % L))
            nn.append((s, ((R + 1) % L) * L + C))
    for R in range(0, L, 2):
        for C in range(0, L, 2):
            dia.append((R * L + C, ((R + 1) % L) * L + (C + 1) % L))          # "\"
            dia.append(((R + 1) * L + (C + 2) % L, ((R + 2) % L) * L + C + 1))  # "/"
    return nn, dia


def ss_counts_batch(states, L):
    """(N_J, N_J', M) for a batch [n][L*L] of +-1 states (even L periodic)."""
    nn, dia = ss_pairs(L)
    s = np.asarray(states, dtype=np.int64)
    a = np.array(nn)
    d = np.array(dia)
    nJ = (s[:, a[:, 0]] * s[:, a[:, 1]]).sum(1)
    nJp = (s[:, d[:, 0]] * s[:, d[:, 1]]).sum(1)
    return nJ, nJp, s.sum(1)


def transfer_matrix_moments(L, J, Jp, h, beta):
    """Exact <E>, <E^2>, <M>, <M^2> of the even-L periodic SS Ising model by a
    row-to-row transfer matrix (every bond joins the same or adjacent rows),
    with first and second derivatives propagated through the matrix product.
    H = J sum_nn s s + J' sum_diag s s - h sum s."""
    assert L % 2 == 0 and L <= 8
    n = 1 << L
    rows = np.array([[1 if (x >> C) & 1 else -1 for C in range(L)] for x in range(n)],
                    dtype=np.float64)
    e_row = J * (rows * np.roll(rows, -1, axis=1)).sum(1) - h * rows.sum(1)
    m_row = rows.sum(1)
    vert = J * rows @ rows.T
    even = np.zeros((n, n))
    odd = np.zeros((n, n))
    for C in range(0, L, 2):
        # R even: (R, C) -- (R+1, C+1);  R odd: (R, C) -- (R+1, C-1) for even C
        even += Jp * np.outer(rows[:, C], rows[:, (C + 1) % L])
        odd += Jp * np.outer(rows[:, C], rows[:, (C - 1) % L])
    mats = []
    for R in range(L):
        e = e_row[:, None] + vert + (even if R % 2 == 0 else odd)
        mats.append((e, m_row[:, None] * np.ones((1, n))))
    emin = min(e.min() for e, _ in mats)

    def moments(which):
        P0 = np.eye(n)
        P1 = np.zeros((n, n))
        P2 = np.zeros((n, n))
        for e, m in mats:
            A = np.exp(-beta * (e - emin))
            x = -e if which == "E" else m
            B = x * A
            Cm = x * x * A
            P0, P1, P2 = P0 @ A, P1 @ A + P0 @ B, P2 @ A + 2 * P1 @ B + P0 @ Cm
            s = np.abs(P0).max()
            P0, P1, P2 = P0 / s, P1 / s, P2 / s
        Z = np.trace(P0)
        return np.trace(P1) / Z, np.trace(P2) / Z

    dE, d2E = moments("E")
    M1, M2 = moments("M")
    return {"E": -dE, "E2": d2E, "M": M1, "M2": M2}


def supercell_ground_energy(L, J, Jp, h, max_sites=18):
    """Minimum of H over all states periodic under a supercell a x b (a, b | L,
    a*b <= max_sites): brute force."""
    best = None
    divs = [d for d in range(1, L + 1) if L % d == 0]
    for a in divs:
        for b in divs:
            if a * b > max_sites:
                continue
            k = a * b
            x = np.arange(1 << k, dtype=np.int64)
            cell = ((x[:, None] >> np.arange(k)) & 1) * 2 - 1     # [2^k][a*b]
            R = np.arange(L)[:, None] % a
            C = np.arange(L)[None, :] % b
            idx = (R * b + C).reshape(-1)
            states = cell[:, idx]
            nJ, nJp, M = ss_counts_batch(states, L)
            E = J * nJ + Jp * nJp - h * M
            i = int(np.argmin(E))
            if best is None or E[i] < best[0]:
                best = (float(E[i]), states[i].reshape(L, L).copy())
    return best


def transfer_matrix_sample(L, J, Jp, h, beta, n, rng):
    """n independent exact samples [n][L][L] (+-1, int8) of the even-L
    periodic SS Ising model at (J, J', h, beta), drawn row by row from the
    same row transfer matrices as transfer_matrix_moments:
    P(r_0 .. r_{L-1}) is proportional to prod_R A_R(r_R, r_{R+1}) with
    r_L = r_0; r_0 is drawn from diag(A_0 ... A_{L-1}), then each r_R given
    r_{R-1} and r_0 from A_{R-1}(r_{R-1}, .) (A_R ... A_{L-1})(., r_0)."""
    assert L % 2 == 0 and L <= 8
    nr = 1 << L
    rows = np.array([[1 if (x >> C) & 1 else -1 for C in range(L)] for x in range(nr)],
                    dtype=np.float64)
    e_row = J * (rows * np.roll(rows, -1, axis=1)).sum(1) - h * rows.sum(1)
    vert = J * rows @ rows.T
    even = np.zeros((nr, nr))
    odd = np.zeros((nr, nr))
    for C in range(0, L, 2):
        even += Jp * np.outer(rows[:, C], rows[:, (C + 1) % L])
        odd += Jp * np.outer(rows[:, C], rows[:, (C - 1) % L])
    es = [e_row[:, None] + vert + (even if R % 2 == 0 else odd) for R in range(L)]
    emin = min(e.min() for e in es)
    A = [np.exp(-beta * (e - emin)) for e in es]
    suffix = [None] * (L + 1)             # suffix[R] = A_R ... A_{L-1}, normalised
    suffix[L] = np.eye(nr)
    for R in range(L - 1, -1, -1):
        m = A[R] @ suffix[R + 1]
        suffix[R] = m / m.max()
    out = np.zeros((n, L, L), np.int8)
    for i in range(n):
        p0 = np.clip(np.diag(suffix[0]), 0, None)
        r0 = rng.choice(nr, p=p0 / p0.sum())
        seq = [r0]
        for R in range(1, L):
            w = A[R - 1][seq[-1], :] * suffix[R][:, r0]
            seq.append(rng.choice(nr, p=w / w.sum()))
        out[i] = rows[seq].astype(np.int8)
    return out
