"""Pin of the oracle's first-passage sampler (training data of the learned exit
proposal) against the exact absorbing Markov chain of a small brick.

The DDMC walk inside a uniform b^3 brick is a finite Markov chain on
(cell, bin) whose one-step law is the categorical draw on the quantised
cumulative thresholds of the walk (Sec. 2.3).  Absorption in (exit face, exit
bin, exit position) has probabilities B = (I - Q)^-1 R and expected absorption
time (I - Q)^-1 1, computed here by dense linear algebra; the sampler's
frequencies must match within the multinomial error.  The fold of start cells
into the cube's fundamental domain is pinned separately: the exact law from a
cell equals the image, under the cube symmetry, of the law from its folded cell.
"""
import itertools

import numpy as np
import pytest

from oracle import analytic as A
from oracle import coracle as C
from paper_1709_10187_gb300 import workloads as W


def _rows(J=8, tau0=40.0):
    w = W.Workload("fp_pin", 3, (3, 3, 3), J, -6.0, 6.0, tau0, 1.0e4, 1, 1, R=1.5)
    return C.interior_rows(w)


def _other_axes(ax):
    return (1, 2) if ax == 0 else ((0, 2) if ax == 1 else (0, 1))


def _chain(rows, b):
    """Absorption matrix of the brick chain: (B [n_states x n_abs], keys of the
    absorbing states (face, bin, pos), mean absorption time per state,
    state index function)."""
    J = rows.shape[0]
    thr = rows[:, :7].astype(np.float64)
    cum = np.concatenate([np.zeros((J, 1)), thr, np.full((J, 1), 2.0 ** 32)], axis=1)
    p_out = np.diff(cum, axis=1) / 2.0 ** 32            # [J x 8]: bin-1, bin+1, -x, +x, -y, +y, -z, +z
    n_t = b ** 3 * J
    sid = lambda i, j: ((i[0] + b * (i[1] + b * i[2])) * J + j)
    Q = np.zeros((n_t, n_t))
    absorb, Rcols = {}, []
    for idx in itertools.product(range(b), repeat=3):
        for j in range(J):
            s = sid(idx, j)
            for o in range(8):
                p = p_out[j, o]
                if p == 0.0:
                    continue
                if o < 2:
                    jn = j + (1 if o else -1)
                    assert 0 <= jn < J, "the table leaks past the frequency grid"
                    Q[s, sid(idx, jn)] += p
                    continue
                f = o - 2
                ax, side = f // 2, (1 if f & 1 else -1)
                n = list(idx)
                n[ax] += side
                if 0 <= n[ax] < b:
                    Q[s, sid(n, j)] += p
                else:
                    u, v = _other_axes(ax)
                    key = (f, j, idx[u] + b * idx[v])
                    if key not in absorb:
                        absorb[key] = len(absorb)
                        Rcols.append(np.zeros(n_t))
                    Rcols[absorb[key]][s] += p
    R = np.stack(Rcols, axis=1)
    N = np.linalg.inv(np.eye(n_t) - Q)
    return N @ R, list(absorb), N @ np.ones(n_t), sid


def _fold(idx, b):
    c = [min(i, b - 1 - i) for i in idx]
    return tuple(sorted(c))


@pytest.mark.parametrize("b", [3, 4])
def test_first_passages_follow_the_absorbing_chain(b):
    rows = _rows()
    J = rows.shape[0]
    jlo, jhi = J // 2, J // 2 + 1
    n = 120_000
    out, steps = C.fp_samples(rows[None], b, [jlo], [jhi], 4242, 17, n, 1 << 40)
    assert np.all(out[:, 0] == 0) and np.all(out[:, 3] < 6) and np.all(out[:, 6:] == 0)
    Bm, keys, tmean, sid = _chain(rows, b)
    # start law: bin uniform on [jlo, jhi], cell uniform on the brick then folded
    start = np.zeros(Bm.shape[0])
    fold_p = {}
    for idx in itertools.product(range(b), repeat=3):
        c = _fold(idx, b)
        fold_p[c] = fold_p.get(c, 0.0) + 1.0 / b ** 3
    for c, pc in fold_p.items():
        for j in range(jlo, jhi + 1):
            start[sid(c, j)] += pc / (jhi - jlo + 1)
    # folded start cells appear with their orbit shares
    cells = out[:, 2]
    for c, pc in fold_p.items():
        k = c[0] + b * c[1] + b * b * c[2]
        cnt = int((cells == k).sum())
        assert abs(cnt - pc * n) <= 5.0 * np.sqrt(pc * n) + 3.0, (c, cnt, pc * n)
    probs = start @ Bm
    exact = {k: probs[i] for i, k in enumerate(keys)}
    obs = {}
    for f, j, q in out[:, [3, 4, 5]]:
        obs[(int(f), int(j), int(q))] = obs.get((int(f), int(j), int(q)), 0) + 1
    assert set(obs) <= set(keys), set(obs) - set(keys)
    chi2, dof = 0.0, 0
    for k in keys:
        e = exact[k] * n
        o = obs.get(k, 0)
        assert abs(o - e) <= 5.0 * np.sqrt(e) + 3.0, (k, o, e)
        if e >= 5.0:
            chi2 += (o - e) ** 2 / e
            dof += 1
    assert chi2 <= dof + 6.0 * np.sqrt(2.0 * dof), (chi2, dof)
    st = steps.astype(np.float64)
    assert abs(st.mean() - start @ tmean) <= 5.0 * st.std() / np.sqrt(n), (st.mean(), start @ tmean)


def test_fold_is_a_symmetry_of_the_brick_chain():
    """The exact exit law from a cell is the image of the law from its folded
    cell under the reflection + permutation that folds it.  The walk's six
    spatial probabilities are differences of cumulative thresholds rounded to
    2^-32 each, so they agree to about 2^-32 and the symmetry holds to that
    order (relative 1e-6 is a loose bound over a few dozen transitions)."""
    rows = _rows(J=6, tau0=25.0)
    b = 4
    Bm, keys, tmean, sid = _chain(rows, b)
    kidx = {k: i for i, k in enumerate(keys)}
    j0 = 3
    for idx in [(3, 0, 1), (2, 3, 0), (1, 2, 3), (0, 0, 3)]:
        flip = [idx[a] > b - 1 - idx[a] for a in range(3)]
        c = [b - 1 - idx[a] if flip[a] else idx[a] for a in range(3)]
        perm = sorted(range(3), key=lambda a: (c[a], a))   # canonical axis k <- world axis perm[k]
        folded = tuple(c[perm[k]] for k in range(3))
        assert folded == _fold(idx, b)
        law_w = Bm[sid(idx, j0)]
        law_c = Bm[sid(folded, j0)]
        assert abs(tmean[sid(idx, j0)] - tmean[sid(folded, j0)]) <= 1e-6 * tmean[sid(idx, j0)]
        for (f, j, q), i in kidx.items():
            ca, cs = f // 2, f & 1
            u, v = _other_axes(ca)
            cc = [0, 0, 0]
            cc[ca] = b - 1 if cs else 0
            cc[u], cc[v] = q % b, q // b
            # canonical -> world
            wl = [0, 0, 0]
            for k in range(3):
                wa = perm[k]
                wl[wa] = b - 1 - cc[k] if flip[wa] else cc[k]
            wa = perm[ca]
            wf = 2 * wa + (cs ^ int(flip[wa]))
            wu, wv = _other_axes(wa)
            wkey = (wf, j, wl[wu] + b * wl[wv])
            assert abs(law_c[i] - law_w[kidx[wkey]]) <= 1e-7, (idx, (f, j, q), wkey)


def test_exit_position_is_on_the_exit_face_and_cap_is_flagged():
    rows = _rows(tau0=400.0)
    J = rows.shape[0]
    b = 4
    out, steps = C.fp_samples(rows[None], b, [J // 2], [J // 2], 7, 0, 4000, 64)
    capped = out[:, 3] == 6
    assert capped.any() and (~capped).any()
    assert np.all(out[capped, 5] == -1) and np.all(steps[capped] == 64)
    ok = ~capped
    assert np.all((out[ok, 5] >= 0) & (out[ok, 5] < b * b)) and np.all(steps[ok] <= 64)
    c = out[:, 2]
    c0, c1, c2 = c % b, (c // b) % b, c // (b * b)
    assert np.all((c0 <= c1) & (c1 <= c2) & (2 * c2 <= b - 1))


# ---------------------------------------------------------------------------
# First passages out of a region of a medium that varies from cell to cell

def _region_chain(w, t, base, r):
    """Exact absorption law of the walk inside the region [base, base + r)^3 of
    grid w with table t (the oracle's dense table): transitions by the quantised
    thresholds, Doppler rebins across faces by (m, thr), exits recorded as
    (face, bin, cell on the face)."""
    J = w.J
    n0, n1 = w.n[0], w.n[1]
    thr = t["thr"].astype(np.float64)
    K = thr.shape[1] + 1
    cum = np.concatenate([np.zeros((thr.shape[0], 1)), thr, np.full((thr.shape[0], 1), 2.0 ** 32)], axis=1)
    p_out = np.diff(cum, axis=1) / 2.0 ** 32
    flags = t["flags"]
    nf = 6
    n_t = r ** 3 * J
    sid = lambda l, j: ((l[0] + r * (l[1] + r * l[2])) * J + j)
    Q = np.zeros((n_t, n_t))
    absorb, Rrows, Rcols, Rvals = {}, [], [], []
    for l in itertools.product(range(r), repeat=3):
        c = (base[0] + l[0]) + n0 * ((base[1] + l[1]) + n1 * (base[2] + l[2]))
        for j in range(J):
            s = sid(l, j)
            st = c * J + j
            for o in range(K):
                p = p_out[st, o]
                if p == 0.0:
                    continue
                if o < 2:
                    Q[s, sid(l, j + (1 if o else -1))] += p
                    continue
                f = o - 2
                ax, side = f // 2, (1 if f & 1 else -1)
                n = list(l)
                n[ax] += side
                if not (0 <= n[ax] < r):
                    u, v = _other_axes(ax)
                    key = (f, j, l[u] + r * l[v])
                    col = absorb.setdefault(key, len(absorb))
                    Rrows.append(s); Rcols.append(col); Rvals.append(p)
                    continue
                act = (int(flags[st]) >> (2 * o)) & 3
                if act == 3:  # Doppler rebin across the face
                    m = int(t["rebin_m"][c * nf + f])
                    pr = float(t["rebin_thr"][c * nf + f]) / 2.0 ** 32
                    for jn, pj in ((j + m, pr), (j + m + 1, 1.0 - pr)):
                        jn = min(max(jn, 0), J - 1)
                        if pj > 0:
                            Q[s, sid(n, jn)] += p * pj
                else:
                    assert act == 0
                    Q[s, sid(n, j)] += p
    R_ = np.zeros((n_t, len(absorb)))
    for a, b_, v in zip(Rrows, Rcols, Rvals):
        R_[a, b_] += v
    A = np.eye(n_t) - Q
    B = np.linalg.solve(A, R_)
    T = np.linalg.solve(A, np.ones(n_t))
    T2 = np.linalg.solve(A, 2.0 * T - 1.0)  # E[T^2] per start state
    return B, absorb, (T, T2), sid


def test_region_first_passages_match_the_exact_chain_of_a_moving_clumpy_region():
    # an 8^3 grid with a cell-resolution lognormal density and turbulent
    # velocity (so rows differ from cell to cell and crossings rebin); one
    # brick of 8^3 with a margin of 2: the region is the central 4^3 cells
    med = W.clumpy_medium(n=8, J=10, x_max=10.0, tau0=300.0, brick=1, sigma_v_kms=20.0, packets=1, seed=0x5EED0710)
    w = med.workload
    g = C.Grid(w, n_rel=med.n_rel)
    g.v = np.ascontiguousarray(med.v_kms, dtype=np.float64)
    g.g.v = C._ptr(g.v)
    t = g.table()
    assert len(set(map(tuple, t["thr"].reshape(w.ncell, -1)[:, :7].tolist()))) > 100  # cells differ
    bl, m, r = 8, 2, 4
    bins = np.arange(2, 8, dtype=np.int32)  # the listed start bins
    B, absorb, (T, T2), sid = _region_chain(w, t, (m, m, m), r)
    n = 120_000
    out, steps = C.fp_region_samples(g, t, bl, 0, m, 1, [0], [0, len(bins)], bins, 0xF00D, 0, n, 10_000_000)
    assert np.all(out[:, 0] == 0) and np.all(out[:, 3] < 6)
    assert out[:, 6].sum() > 0  # crossings inside the region were rebinned
    # start states: uniform over the region's cells and the listed bins
    cells = np.bincount(out[:, 2], minlength=r ** 3)
    assert abs(cells.std() / cells.mean()) < 0.06
    starts = [sid((c % r, (c // r) % r, c // (r * r)), j) for c in range(r ** 3) for j in bins]
    p_exit = B[starts].mean(axis=0)
    assert abs(p_exit.sum() - 1.0) < 1e-9
    keys = [(int(f), int(j), int(p)) for f, j, p in out[:, [3, 4, 5]]]
    cnt = np.zeros(len(absorb))
    for k in keys:
        cnt[absorb[k]] += 1
    zmax, frac, pval = A.compare_counts_to_probs(cnt, p_exit, n)
    assert zmax < 5.0 and frac <= 0.02 and pval > 1e-3, (zmax, frac, pval)
    # exit (face, bin) marginal, and the mean number of transitions
    fb = {}
    for (f, j, _), col in absorb.items():
        fb.setdefault((f, j), []).append(col)
    km = list(fb)
    pm = np.array([p_exit[fb[k]].sum() for k in km])
    cm = np.array([cnt[fb[k]].sum() for k in km])
    zmax, frac, pval = A.compare_counts_to_probs(cm, pm, n)
    assert zmax < 5.0 and pval > 1e-3, (zmax, pval)
    tm = T[starts].mean()
    var = T2[starts].mean() - tm * tm
    z = (steps.astype(np.float64).mean() - tm) / np.sqrt(var / n)
    assert abs(z) < 4.0, (steps.mean(), tm, z)
