"""Pins of the oracle's windowed Hamming search (Section 3.4).

Distance = number of differing components (Hamming similarity is the count
of equal ones); candidates share the query's charge and lie within the
precursor m/z tolerance, bound inclusive; the best matches are the smallest
(distance, reference index) keys.  Checked against metric axioms, scipy's
Hamming distance, brute force on tiny inputs and exact window edges."""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from tests.helpers import bits, hamming_matrix

D = 256
W = D // 64


def _rand_hv(rng, n):
    return rng.integers(0, 2**63, (n, W), dtype=np.int64).astype(np.uint64) ^ \
        (rng.integers(0, 2, (n, W)).astype(np.uint64) << np.uint64(63))


def _all_distances(q, refs):
    n = refs.shape[0]
    mz = np.full(n, 500.0)
    z = np.full(n, 2, np.uint8)
    idx, dist = oracle.search(D, refs, mz, z, q[None], np.array([500.0]), np.array([2], np.uint8),
                              tol=1.0, k=n)
    out = np.empty(n, np.int64)
    out[idx[0]] = dist[0]
    return out


def test_metric_axioms():
    rng = np.random.default_rng(0)
    x = _rand_hv(rng, 6)
    refs = np.concatenate([x, ~x])
    dm = np.stack([_all_distances(x[i], refs) for i in range(6)])
    assert np.all(dm[np.arange(6), np.arange(6)] == 0)          # d(x,x)=0
    assert np.all(dm[np.arange(6), 6 + np.arange(6)] == D)      # d(x,~x)=D
    sq = dm[:, :6]
    assert np.array_equal(sq, sq.T)                             # symmetry
    for a in range(6):
        for b in range(6):
            assert np.all(sq[a, b] <= sq[a, :] + sq[:, b])      # triangle


def test_matches_scipy_hamming_all_pairs():
    rng = np.random.default_rng(1)
    refs, qs = _rand_hv(rng, 200), _rand_hv(rng, 30)
    # duplicate some references so that ties exercise the lowest-index rule
    refs[150:160] = refs[10:20]
    qs[:5] = refs[10:15]
    ref_d = (cdist(bits(qs), bits(refs), "hamming") * D).round().astype(np.int64)
    k = 7
    idx, dist = oracle.search(D, refs, np.full(200, 700.0), np.full(200, 3, np.uint8),
                              qs, np.full(30, 700.0), np.full(30, 3, np.uint8), tol=0.0, k=k)
    for q in range(30):
        order = np.lexsort((np.arange(200), ref_d[q]))[:k]
        assert np.array_equal(idx[q], order)
        assert np.array_equal(dist[q], ref_d[q, order])


def test_windowed_brute_force_tiny():
    rng = np.random.default_rng(2)
    nr, nq, k = 300, 40, 4
    refs, qs = _rand_hv(rng, nr), _rand_hv(rng, nq)
    rmz, qmz = rng.uniform(400, 600, nr), rng.uniform(400, 600, nq)
    rz, qz = rng.integers(1, 4, nr).astype(np.uint8), rng.integers(1, 4, nq).astype(np.uint8)
    dm = hamming_matrix(qs, refs)
    for unit, tol in (("da", 25.0), ("ppm", 40000.0)):
        idx, dist = oracle.search(D, refs, rmz, rz, qs, qmz, qz, tol=tol, unit=unit, k=k)
        for q in range(nq):
            t = tol if unit == "da" else qmz[q] * tol * 1e-6
            cand = [r for r in range(nr) if rz[r] == qz[q] and abs(rmz[r] - qmz[q]) <= t]
            best = sorted(cand, key=lambda r: (dm[q, r], r))[:k]
            got = [int(i) for i in idx[q] if i != 0xFFFFFFFF]
            assert got == best
            assert list(dist[q][:len(best)]) == [dm[q, r] for r in best]
            assert np.all(idx[q][len(best):] == 0xFFFFFFFF) and np.all(dist[q][len(best):] == 0xFFFF)


def test_window_edges_inclusive_exact():
    # 1000 +- 500 is exact in binary: 1500.0 and 500.0 are in, one ulp further is out
    rng = np.random.default_rng(3)
    refs = _rand_hv(rng, 6)
    rmz = np.array([1500.0, np.nextafter(1500.0, 2e3), 500.0, np.nextafter(500.0, 0.0), 1000.0, 1000.0])
    rz = np.array([2, 2, 2, 2, 2, 3], np.uint8)
    cnt = oracle.window_count(rmz, rz, np.array([1000.0]), np.array([2], np.uint8), 500.0)
    assert cnt[0] == 3
    idx, _ = oracle.search(D, refs, rmz, rz, refs[:1], np.array([1000.0]), np.array([2], np.uint8),
                           tol=500.0, k=6)
    assert sorted(int(i) for i in idx[0] if i != 0xFFFFFFFF) == [0, 2, 4]


def test_ppm_window_margins():
    q = 800.0
    tq = q * 20e-6
    rmz = np.array([q + 0.9 * tq, q - 0.9 * tq, q + 1.1 * tq, q - 1.1 * tq, q])
    rz = np.full(5, 2, np.uint8)
    cnt = oracle.window_count(rmz, rz, np.array([q]), np.array([2], np.uint8), 20.0, unit="ppm")
    assert cnt[0] == 3


def test_nan_query_has_no_candidates():
    rz = np.full(3, 2, np.uint8)
    cnt = oracle.window_count(np.array([1.0, 2.0, 3.0]), rz, np.array([np.nan]), np.array([2], np.uint8), 1e9)
    assert cnt[0] == 0


def test_subset_rows_match_full_run():
    rng = np.random.default_rng(4)
    refs, qs = _rand_hv(rng, 100), _rand_hv(rng, 20)
    rmz, qmz = rng.uniform(400, 500, 100), rng.uniform(400, 500, 20)
    rz, qz = np.full(100, 2, np.uint8), np.full(20, 2, np.uint8)
    full = oracle.search(D, refs, rmz, rz, qs, qmz, qz, tol=30.0, k=3, n_threads=3)
    which = np.array([19, 0, 7])
    sub = oracle.search(D, refs, rmz, rz, qs, qmz, qz, tol=30.0, k=3, which=which, n_threads=2)
    assert np.array_equal(sub[0], full[0][which]) and np.array_equal(sub[1], full[1][which])


def test_library_order_matches_lexsort():
    rng = np.random.default_rng(5)
    mz = np.round(rng.uniform(400, 410, 500), 1)      # many equal m/z values
    z = rng.integers(1, 5, 500).astype(np.uint8)
    order = oracle.library_order(mz, z)
    assert np.array_equal(order, np.lexsort((np.arange(500), mz, z)))


# ------------------------------------------------ neutral-mass windows (N4)
def test_mass_window_scales_mz_window_by_charge():
    """Within one charge z, neutral masses differ by z times the m/z
    difference, so the +-T Da mass window selects the references of m/z
    within T / z; checked away from the rounding boundary, for charges 1..4."""
    rng = np.random.default_rng(41)
    n = 4000
    mz = rng.uniform(400, 1500, n)
    z = rng.integers(1, 5, n).astype(np.uint8)
    qm = rng.uniform(450, 1450, 300)
    qz = rng.integers(1, 5, 300).astype(np.uint8)
    for T in (0.5, 20.0, 150.0, 500.0):
        got = oracle.window_count(mz, z, qm, qz, T, "mass")
        for i in range(qm.size):
            same = z == qz[i]
            d = np.abs(mz[same] - qm[i])
            lim = T / float(qz[i])
            if np.any(np.abs(d - lim) < 1e-9 * max(1.0, lim)):
                continue                                   # on the rounding boundary
            assert got[i] == int(np.count_nonzero(d <= lim)), (T, i)


def test_mass_window_charge_zero_and_charge_filter():
    # charge 0: every neutral mass is 0, so every charge-0 reference is a candidate
    mz = np.array([400.0, 900.0, 1400.0, 650.0])
    z = np.array([0, 0, 0, 2], np.uint8)
    assert list(oracle.window_count(mz, z, np.array([1000.0]), np.array([0], np.uint8), 0.0, "mass")) == [3]
    # another charge never matches, however wide the window
    assert list(oracle.window_count(mz, z, np.array([650.0]), np.array([3], np.uint8), 1e6, "mass")) == [0]


def test_mass_window_search_brute_force():
    rng = np.random.default_rng(42)
    n, m = 300, 40
    refs = _rand_hv(rng, n)
    mz = rng.uniform(400, 600, n)
    z = rng.integers(1, 4, n).astype(np.uint8)
    qs = _rand_hv(rng, m)
    qm = rng.uniform(400, 600, m)
    qz = rng.integers(1, 4, m).astype(np.uint8)
    idx, dist = oracle.search(D, refs, mz, z, qs, qm, qz, 30.0, "mass", k=4)
    dm = hamming_matrix(qs, refs)
    for i in range(m):
        cand = [r for r in range(n) if z[r] == qz[i] and abs((mz[r] - qm[i]) * float(qz[i])) <= 30.0 * (1 - 1e-12)]
        edge = [r for r in range(n) if z[r] == qz[i] and abs(abs((mz[r] - qm[i]) * float(qz[i])) - 30.0) < 1e-6]
        if edge:
            continue
        best = sorted(cand, key=lambda r: (dm[i, r], r))[:4]
        got = [int(x) for x in idx[i] if x != 0xFFFFFFFF]
        assert got == best
        assert [int(dm[i, r]) for r in best] == [int(x) for x in dist[i][:len(best)]]


def test_topk_prefix_and_reference_permutation():
    """The k1 best are the first k1 of the k2 best (k1 < k2); relabelling the
    references permutes indices but keeps every query's sorted distances."""
    rng = np.random.default_rng(17)
    n_ref, n_q = 400, 30
    refs = _rand_hv(rng, n_ref)
    refs[50] = refs[10]                       # ties
    qs = _rand_hv(rng, n_q)
    qs[0] = refs[10]
    mz = rng.uniform(500, 503, n_ref)
    z = rng.integers(2, 4, n_ref).astype(np.uint8)
    mz[50], z[50] = mz[10], z[10]
    q_mz = rng.uniform(500, 503, n_q)
    q_z = rng.integers(2, 4, n_q).astype(np.uint8)
    q_mz[0], q_z[0] = mz[10], z[10]
    i16, d16 = oracle.search(D, refs, mz, z, qs, q_mz, q_z, 1.0, "da", k=16)
    for k in (1, 3, 7):
        ik, dk = oracle.search(D, refs, mz, z, qs, q_mz, q_z, 1.0, "da", k=k)
        assert np.array_equal(ik, i16[:, :k]) and np.array_equal(dk, d16[:, :k])
    assert i16[0, 0] == 10 and i16[0, 1] == 50 and d16[0, 0] == d16[0, 1] == 0
    perm = rng.permutation(n_ref)
    ip, dp = oracle.search(D, refs[perm], mz[perm], z[perm], qs, q_mz, q_z, 1.0, "da", k=16)
    assert np.array_equal(dp, d16)
    ok = ip != 0xFFFFFFFF
    # the permuted run's rows map back to references with the same distances
    back = np.where(ok, perm[np.minimum(ip, n_ref - 1)], 0xFFFFFFFF)
    dist_of = lambda q, r: int(hamming_matrix(qs[q:q + 1], refs[r:r + 1])[0, 0])
    for q in range(n_q):
        for t in range(16):
            if ok[q, t]:
                assert dist_of(q, back[q, t]) == dp[q, t]
