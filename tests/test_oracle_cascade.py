"""Pins of the oracle's cascade search with target-decoy FDR (Section 3.4:
narrow search, FDR filter, wide search for the unidentified; Section 2.1:
target-decoy strategy, 1% FDR).

q-values are pinned by closed forms of ordered target/decoy sequences, by a
brute-force count over all thresholds on tiny inputs with ties, and by
invariants; each cascade level is pinned by an independent brute-force
top-1 (numpy unpackbits) on the queries still active at that level."""
import numpy as np
import pytest

import oracle
from tests.helpers import hamming_matrix

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_targets_then_decoys_closed_form():
    # k targets above m decoys: every target has q = 0; the j-th decoy has FDR j / k,
    # increasing, so its q is j / k
    k, m = 7, 5
    scores = np.arange(k + m)[::-1] + 100
    dec = np.r_[np.zeros(k), np.ones(m)]
    q = oracle.fdr_qvalues(scores, dec)
    assert np.all(q[:k] == 0.0)
    assert np.allclose(q[k:], np.arange(1, m + 1) / k, rtol=0, atol=0)


def test_alternating_closed_form():
    # T D T D ... (descending): target m+1 (m = 0..n-1) has FDR m / (m+1) and decoy m+1
    # has FDR 1; the FDR of the targets grows with m, so the q of target m+1 is
    # m / (m+1) and the q of decoy m+1 is that of the next target, (m+1) / (m+2) --
    # except the last decoy, below which no target lies: its q is its own FDR, 1
    n = 6
    scores = np.arange(2 * n)[::-1]
    dec = np.tile([0, 1], n)
    q = oracle.fdr_qvalues(scores, dec)
    m = np.arange(n)
    expect = np.empty(2 * n)
    expect[0::2] = m / (m + 1)
    expect[1::2] = (m + 1) / (m + 2)
    expect[-1] = 1.0
    assert np.array_equal(q, expect)


def test_all_targets_and_all_decoys():
    assert np.all(oracle.fdr_qvalues([9, 3, 3, 1], [0, 0, 0, 0]) == 0.0)
    # no target: the denominator is 1, so the FDR at the j-th threshold is j and q = j
    q = oracle.fdr_qvalues([9, 7, 5], [1, 1, 1])
    assert np.array_equal(q, [1.0, 2.0, 3.0])
    assert oracle.fdr_qvalues([], []).size == 0


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_count_with_ties(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    scores = rng.integers(0, 8, n)          # many ties
    dec = rng.integers(0, 2, n).astype(bool)
    q = oracle.fdr_qvalues(scores, dec)
    for i in range(n):
        best = np.inf
        for s in set(scores.tolist()):      # every threshold at or below this SSM's score
            if s > scores[i]:
                continue
            t = sum(1 for j in range(n) if scores[j] >= s and not dec[j])
            d = sum(1 for j in range(n) if scores[j] >= s and dec[j])
            best = min(best, d / max(t, 1))
        assert q[i] == best


@pytest.mark.parametrize("seed", range(4))
def test_invariants(seed):
    rng = np.random.default_rng(100 + seed)
    n = 200
    scores = rng.integers(0, 60, n)
    dec = rng.random(n) < 0.3
    q = oracle.fdr_qvalues(scores, dec)
    order = np.argsort(-scores, kind="stable")
    assert np.all(np.diff(q[order]) >= 0)                       # higher score, lower-or-equal q
    perm = rng.permutation(n)
    assert np.array_equal(oracle.fdr_qvalues(scores[perm], dec[perm]), q[perm])   # order-free
    q2 = oracle.fdr_qvalues(np.r_[scores, scores.min() - 1], np.r_[dec, True])
    assert np.array_equal(q2[:n], q)                            # a decoy below all leaves q unchanged


def _lib(rng, n_t, D):
    W = D // 64
    t_hv = rng.integers(-2**63, 2**63, (n_t, W), dtype=np.int64).view(np.uint64)
    d_hv = rng.integers(-2**63, 2**63, (n_t, W), dtype=np.int64).view(np.uint64)
    mz = rng.uniform(400, 1500, n_t)
    z = rng.integers(2, 4, n_t).astype(np.uint8)
    hv = np.concatenate([t_hv, d_hv])
    return hv, np.r_[mz, mz], np.r_[z, z], np.r_[np.zeros(n_t, np.uint8), np.ones(n_t, np.uint8)]


def _noisy(rng, hv, flips, D):
    bits = np.unpackbits(hv.view(np.uint8), bitorder="little").reshape(hv.shape[0], D)
    for r in range(hv.shape[0]):
        bits[r, rng.choice(D, flips[r], replace=False)] ^= 1
    return np.packbits(bits, axis=1, bitorder="little").view(np.uint64)


def test_cascade_levels_match_brute_force():
    rng = np.random.default_rng(5)
    D, n_t, n_q = 256, 300, 120
    hv, mz, z, dec = _lib(rng, n_t, D)
    src = rng.integers(0, n_t, n_q)
    shift = np.where(rng.random(n_q) < 0.4, 0.0, rng.uniform(-80, 80, n_q))
    q_mz = mz[src] + shift / z[src]
    q_z = z[src]
    q_hv = _noisy(rng, hv[src], rng.integers(10, 110, n_q), D)
    levels = [(20.0, "ppm"), (100.0, "da")]
    idx, dist, level, q = oracle.cascade(D, hv, mz, z, dec, q_hv, q_mz, q_z, levels, 0.01)

    dm = hamming_matrix(q_hv, hv)                    # [n_q, n_r] brute force
    active = np.ones(n_q, bool)
    for li, (tol, unit) in enumerate(levels):
        tq = tol if unit == "da" else q_mz * (tol * 1e-6)
        cand = (z[None, :] == q_z[:, None]) & (np.abs(mz[None, :] - q_mz[:, None]) <= np.broadcast_to(
            np.asarray(tq, np.float64).reshape(-1, 1), (n_q, 1)))
        key = np.where(cand, dm * (2 * hv.shape[0]) + np.arange(hv.shape[0])[None, :], np.iinfo(np.int64).max)
        best = key.argmin(axis=1)
        has = cand.any(axis=1)
        sel = active & has
        # a query reports the SSM of the last level it was searched at: the level that
        # identified it, else the last level
        here = sel & ((level == li) | ((level == 0xFF) & (li == len(levels) - 1)))
        assert here.any()
        assert np.array_equal(idx[here], best[here].astype(np.uint32))
        assert np.array_equal(dist[here], dm[here, best[here]].astype(np.uint16))
        # the level's identifications: targets with q <= 1%, computed over this level's SSMs only
        scores = D - dm[sel, best[sel]]
        qv = oracle.fdr_qvalues(scores, dec[best[sel]])
        ident = np.zeros(n_q, bool)
        ident[np.nonzero(sel)[0]] = (dec[best[sel]] == 0) & (qv <= 0.01)
        assert np.array_equal(level == li, ident)
        active &= ~ident
    assert np.all(level[active] == 0xFF)
    assert (level == 0).sum() > 0 and (level == 1).sum() > 0   # both levels identify something


def test_cascade_fdr_extremes():
    rng = np.random.default_rng(9)
    D, n_t, n_q = 128, 100, 60
    hv, mz, z, dec = _lib(rng, n_t, D)
    src = rng.integers(0, n_t, n_q)
    q_hv = _noisy(rng, hv[src], rng.integers(0, 50, n_q), D)
    args = (D, hv, mz, z, dec, q_hv, mz[src], z[src], [(10.0, "da")])
    idx, dist, level, q = oracle.cascade(*args, 1e9)           # any target SSM is accepted
    assert np.array_equal(level == 0, (idx != 0xFFFFFFFF) & (dec[np.minimum(idx, 2 * n_t - 1)] == 0))
    idx0, dist0, level0, q0 = oracle.cascade(*args, -1.0)       # nothing is accepted
    assert np.all(level0 == 0xFF)
    assert np.array_equal(idx0, idx) and np.array_equal(dist0, dist)
    assert np.array_equal(q0, q, equal_nan=True)


# ------------------------------------------------ multi-bit components (Section 4.3)
def _pm1(hv, D):
    """+-1 components of binary HVs (bit b -> 1 - 2b)."""
    bits = np.unpackbits(hv.view(np.uint8), bitorder="little").reshape(hv.shape[0], D)
    return (1 - 2 * bits.astype(np.int16)).astype(np.int8)


def test_cascade_dot_pm1_equals_binary_cascade():
    """For +-1 components S = D - 2 dist, a strictly increasing map of the
    Hamming similarity D - dist: the same SSMs, the same q-values, the same
    levels as the binary cascade."""
    rng = np.random.default_rng(21)
    D, n_t, n_q = 256, 300, 150
    hv, mz, z, dec = _lib(rng, n_t, D)
    src = rng.integers(0, n_t, n_q)
    shift = np.where(rng.random(n_q) < 0.4, 0.0, rng.uniform(-80, 80, n_q))
    q_mz, q_z = mz[src] + shift / z[src], z[src]
    q_hv = _noisy(rng, hv[src], rng.integers(10, 110, n_q), D)
    levels = [(20.0, "ppm"), (100.0, "da"), (5.0, "mass")]
    i1, d1, l1, q1 = oracle.cascade(D, hv, mz, z, dec, q_hv, q_mz, q_z, levels, 0.01)
    i2, s2, l2, q2 = oracle.cascade_dot(_pm1(hv, D), mz, z, dec, _pm1(q_hv, D), q_mz, q_z, levels, 0.01)
    assert np.array_equal(i1, i2) and np.array_equal(l1, l2)
    assert np.array_equal(q1, q2, equal_nan=True)
    ok = i1 != 0xFFFFFFFF
    assert np.array_equal(s2[ok], D - 2 * d1[ok].astype(np.int32))
    assert np.all(s2[~ok] == np.iinfo(np.int32).min)
    assert (l1 == 0).any() and (l1 == 1).any()


def _comp_lib(rng, n_t, D, m):
    t = rng.integers(-m, m + 1, (n_t, D)).astype(np.int8)
    d = rng.integers(-m, m + 1, (n_t, D)).astype(np.int8)
    mz = rng.uniform(400, 1500, n_t)
    z = rng.integers(2, 4, n_t).astype(np.uint8)
    return np.concatenate([t, d]), np.r_[mz, mz], np.r_[z, z], np.r_[np.zeros(n_t, np.uint8), np.ones(n_t, np.uint8)]


def _noisy_comp(rng, c, frac, m):
    out = c.copy()
    for r in range(c.shape[0]):
        sel = rng.random(c.shape[1]) < frac[r]
        out[r, sel] = rng.integers(-m, m + 1, int(sel.sum()))
    return out


@pytest.mark.parametrize("m", [1, 3, 15])
def test_cascade_dot_levels_match_brute_force(m):
    """Each level's SSMs against an int64 matrix product with (score
    descending, index ascending) top-1 on the queries still active; each
    level's identifications recomputed from its SSMs."""
    rng = np.random.default_rng(30 + m)
    D, n_t, n_q = 128, 250, 120
    R, mz, z, dec = _comp_lib(rng, n_t, D, m)
    src = rng.integers(0, n_t, n_q)
    shift = np.where(rng.random(n_q) < 0.4, 0.0, rng.uniform(-80, 80, n_q))
    q_mz, q_z = mz[src] + shift / z[src], z[src]
    Qc = _noisy_comp(rng, R[src], rng.uniform(0.2, 0.95, n_q), m)
    levels = [(20.0, "ppm"), (100.0, "da")]
    idx, score, level, q = oracle.cascade_dot(R, mz, z, dec, Qc, q_mz, q_z, levels, 0.01)
    S = Qc.astype(np.int64) @ R.astype(np.int64).T
    n_r = R.shape[0]
    active = np.ones(n_q, bool)
    for li, (tol, unit) in enumerate(levels):
        tq = np.full(n_q, tol) if unit == "da" else q_mz * (tol * 1e-6)
        cand = (z[None, :] == q_z[:, None]) & (np.abs(mz[None, :] - q_mz[:, None]) <= tq[:, None])
        key = np.where(cand, -S * (2 * n_r) + np.arange(n_r)[None, :], np.iinfo(np.int64).max)
        best = key.argmin(axis=1)
        has = cand.any(axis=1)
        sel = active & has
        here = sel & ((level == li) | ((level == 0xFF) & (li == len(levels) - 1)))
        assert here.any()
        assert np.array_equal(idx[here], best[here].astype(np.uint32))
        assert np.array_equal(score[here], S[here, best[here]].astype(np.int32))
        qv = oracle.fdr_qvalues(S[sel, best[sel]], dec[best[sel]])
        ident = np.zeros(n_q, bool)
        ident[np.nonzero(sel)[0]] = (dec[best[sel]] == 0) & (qv <= 0.01)
        assert np.array_equal(level == li, ident)
        active &= ~ident
    assert np.all(level[active] == 0xFF)
    assert (level == 0).sum() > 0 and (level == 1).sum() > 0


def test_cascade_dot_fdr_extremes():
    rng = np.random.default_rng(41)
    D, n_t, n_q, m = 128, 100, 60, 3
    R, mz, z, dec = _comp_lib(rng, n_t, D, m)
    src = rng.integers(0, n_t, n_q)
    Qc = _noisy_comp(rng, R[src], rng.uniform(0.0, 0.9, n_q), m)
    args = (R, mz, z, dec, Qc, mz[src], z[src], [(10.0, "da")])
    idx, score, level, q = oracle.cascade_dot(*args, 1e9)
    assert np.array_equal(level == 0, (idx != 0xFFFFFFFF) & (dec[np.minimum(idx, 2 * n_t - 1)] == 0))
    idx0, score0, level0, q0 = oracle.cascade_dot(*args, -1.0)
    assert np.all(level0 == 0xFF)
    assert np.array_equal(idx0, idx) and np.array_equal(score0, score)
    assert np.array_equal(q0, q, equal_nan=True)
