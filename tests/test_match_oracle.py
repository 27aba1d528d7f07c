"""Pins of the matching/homography oracle (Sec. 4.2, Algorithm 3): Multi-Probe LSH against an
independent NumPy formulation, homography recovery from exact and contaminated correspondences,
and registration of two synthetic views against the rig's true relative homography."""
import numpy as np
import pytest

import oracle
import synth


def _numpy_lsh_matches(desc_a, desc_b, bits, max_dist, ratio):
    da = np.unpackbits(desc_a, axis=1, bitorder="little").astype(np.int64)
    db = np.unpackbits(desc_b, axis=1, bitorder="little").astype(np.int64)
    dist = (da[:, None, :] != db[None, :, :]).sum(axis=2)
    L, k = bits.shape
    weights = (1 << np.arange(k)).astype(np.int64)
    out = []
    for a in range(len(desc_a)):
        cand = np.zeros(len(desc_b), bool)
        for l in range(L):
            ka = int((da[a, bits[l]] * weights).sum())
            kb = (db[:, bits[l]] * weights).sum(axis=1)
            probes = [ka] + [ka ^ (1 << p) for p in range(k)]
            cand |= np.isin(kb, probes)
        if not cand.any():
            continue
        idx = np.nonzero(cand)[0]
        order = np.lexsort((idx, dist[a, idx]))
        b1, d1 = idx[order[0]], dist[a, idx[order[0]]]
        d2 = dist[a, idx[order[1]]] if len(idx) > 1 else None
        if d1 <= max_dist and (d2 is None or ratio[1] * d1 < ratio[0] * d2):
            out.append((a, b1, d1))
    out.sort(key=lambda m: (m[2], m[0]))
    return np.array(out, dtype=np.int64).reshape(-1, 3)


def _views(scale=0.5):
    cfg = synth.config_4x1080p(scale=scale, frames=1)
    fr = cfg.frame(0)
    pat = synth.brief_pattern(0)
    H, W = fr[0].shape[:2]
    fa = oracle.lorb(fr[0], [(W // 2, 0, W, H)], pat, max_points=600)
    fb = oracle.lorb(fr[1], [(0, 0, W // 2, H)], pat, max_points=600)
    Ht = np.linalg.inv(np.asarray(cfg.cameras[1].H)) @ np.asarray(cfg.cameras[0].H)
    return fa, fb, Ht / Ht[2, 2], (W, H)


@pytest.mark.parametrize("max_dist,ratio", [(80, (4, 5)), (40, (3, 4)), (256, (1, 1))])
def test_lsh_matches_independent_numpy_formulation(max_dist, ratio):
    fa, fb, _, _ = _views()
    bits = synth.lsh_bits(2, 6, 12)
    r = oracle.match_prosac(fa["xy"], fa["desc"], fb["xy"], fb["desc"], bits, np.zeros((0, 4)), max_dist, ratio)
    ref = _numpy_lsh_matches(fa["desc"], fb["desc"], bits, max_dist, ratio)
    assert len(ref) > 20
    np.testing.assert_array_equal(r["matches"], ref)


def test_homography_from_exact_and_contaminated_correspondences():
    rng = np.random.default_rng(5)
    Ht = np.array([[1.05, 0.02, 30.0], [-0.01, 0.97, -12.0], [2e-5, -1e-5, 1.0]])
    n, n_out = 120, 40
    a = rng.uniform(50, 900, (n, 2))
    xa = np.rint(a).astype(np.int32)
    xb = np.c_[xa, np.ones(n)] @ Ht.T
    xb = np.rint(xb[:, :2] / xb[:, 2:3]).astype(np.int32)
    xb[n - n_out:] = rng.integers(0, 900, (n_out, 2))  # outliers, last in the quality order (PROSAC's premise)
    # descriptors that match i <-> i exactly (a unique random pattern per point)
    desc = rng.integers(0, 256, (n, 32), dtype=np.uint8)
    r = oracle.match_prosac(xa, desc, xb, desc, synth.lsh_bits(0), synth.prosac_words(1, 512))
    m = r["matches"]
    assert len(m) == n and np.all(m[:, 0] == m[:, 1]) and np.all(m[:, 2] == 0)
    inl = np.zeros(n, bool)
    inl[m[r["inlier"], 0]] = True
    assert not inl[n - n_out:].any() and inl[:n - n_out].mean() > 0.95, inl.sum()
    p = np.array([[100.0, 100.0, 1], [800, 120, 1], [450, 700, 1]]).T
    pe, pt = r["H"] @ p, Ht @ p
    assert np.abs(pe[:2] / pe[2] - pt[:2] / pt[2]).max() < 0.5


def test_two_views_register_to_the_rig_geometry():
    fa, fb, Ht, (W, H) = _views()
    r = oracle.match_prosac(fa["xy"], fa["desc"], fb["xy"], fb["desc"], synth.lsh_bits(0), synth.prosac_words(0, 1024))
    assert r["inliers"] > 100
    p = np.array([[W * 0.6, H * 0.2, 1], [W * 0.9, H * 0.8, 1], [W * 0.75, H * 0.5, 1]]).T
    pe, pt = r["H"] @ p, Ht @ p
    assert np.abs(pe[:2] / pe[2] - pt[:2] / pt[2]).max() < 1.0


def test_too_few_matches_give_no_model():
    fa, fb, _, _ = _views()
    r = oracle.match_prosac(fa["xy"][:3], fa["desc"][:3], fb["xy"], fb["desc"], synth.lsh_bits(0),
                            synth.prosac_words(0, 64))
    assert r["inliers"] == 0 and np.array_equal(r["H"], np.eye(3))


@pytest.mark.parametrize("N,T", [(4, 50), (5, 300), (37, 2000), (255, 1000), (600, 5000), (2048, 20000)])
def test_prosac_schedule_from_the_definition(N, T):
    """Growth schedule against its definition in exact rationals: T_n = T_N prod_{i<m} (n-i)/(N-i)
    (m = 4, T_N = 200000), T'_m = 1, T'_{n+1} = T'_n + ceil(T_{n+1} - T_n); at t = T'_n the top n
    grows (up to N); sampling is uniform from the top n once t > T'_n."""
    from fractions import Fraction
    import math
    m, TN = 4, 200000

    def Tn(n):
        v = Fraction(TN)
        for i in range(m):
            v *= Fraction(n - i, N - i)
        return v

    n, Tp = m, 1
    want_n, want_u = [], []
    for t in range(1, T + 1):
        if t == Tp and n < N:
            Tp += math.ceil(Tn(n + 1) - Tn(n))
            n += 1
        want_n.append(n)
        want_u.append(Tp < t)
    nt, uni = oracle.prosac_schedule(N, T)
    np.testing.assert_array_equal(nt, want_n)
    np.testing.assert_array_equal(uni, want_u)
    if N > m and T > 10:
        assert nt[0] == m + 1 and nt.max() <= N  # the first growth happens at t = 1


def test_prosac_samples_from_the_definition():
    """The 4 indices of an iteration against the draw without replacement written out: word k picks
    the (word mod remaining)-th of the indices still free, in increasing order.  Before the schedule
    has passed, the newest match (index n - 1) is always taken and 3 come from the top n - 1; after,
    4 come from the top n."""
    rng = np.random.default_rng(3)
    for n in (4, 5, 9, 40, 300):
        for uniform in (False, True):
            for _ in range(50):
                w = rng.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
                free = list(range(n if uniform else n - 1))
                want = [] if uniform else [n - 1]
                for k in range(4 if uniform else 3):
                    want.append(free.pop(int(w[k]) % len(free)))
                np.testing.assert_array_equal(oracle.prosac_sample(n, uniform, w), want)


def _exact_pairs(Ht, a):
    b = np.c_[a, np.ones(len(a))] @ np.asarray(Ht).T
    return b[:, :2] / b[:, 2:3], b[:, 2]


def test_four_exact_matches_of_a_strongly_projective_homography():
    """With exactly 4 matches every hypothesis is the 4-point solve itself: it must reproduce a
    homography with large perspective terms (no refit can repair a wrong 4-point system)."""
    Ht = np.array([[0.9, 0.15, 40.0], [-0.1, 1.1, 25.0], [4e-4, -3e-4, 1.0]])
    a = np.array([[100, 120], [900, 80], [850, 700], [150, 650]], np.int32)
    b, w = _exact_pairs(Ht, a)
    assert (w > 0).all()
    # integer inputs: choose image-A points whose images are integers by scaling the homography
    # instead, compare with a sub-pixel tolerance on the rounded targets
    bi = np.rint(b).astype(np.int32)
    desc = np.random.default_rng(1).integers(0, 256, (4, 32), dtype=np.uint8)
    r = oracle.match_prosac(a, desc, bi, desc, synth.lsh_bits(0), synth.prosac_words(0, 8))
    assert r["inliers"] == 4
    pa = np.c_[a, np.ones(4)] @ r["H"].T
    np.testing.assert_allclose(pa[:, :2] / pa[:, 2:3], bi, atol=1e-6)


def test_inlier_threshold_is_in_image_b_pixels():
    """Image B four times larger than image A (H = diag(4, 4, 1) plus a shift): matches displaced by
    6 px in image B are outliers for inlier_px = 3, whatever the scale of image A."""
    rng = np.random.default_rng(2)
    Ht = np.array([[4.0, 0.0, 10.0], [0.0, 4.0, 20.0], [0.0, 0.0, 1.0]])
    a = rng.integers(0, 300, (60, 2)).astype(np.int32)
    b = (np.c_[a, np.ones(60)] @ Ht.T)[:, :2]
    b[40:] += 6.0 * np.array([0.6, 0.8])  # 6 px away in image B
    b = np.rint(b).astype(np.int32)
    desc = rng.integers(0, 256, (60, 32), dtype=np.uint8)
    r = oracle.match_prosac(a, desc, b, desc, synth.lsh_bits(0), synth.prosac_words(4, 256), inlier_px=3.0)
    m = r["matches"]
    inl = np.zeros(60, bool)
    inl[m[r["inlier"], 0]] = True
    assert inl[:40].all() and not inl[40:].any(), (inl[:40].sum(), inl[40:].sum())


def test_points_behind_the_camera_are_no_inliers():
    """Exact correspondences of a homography whose line w = 0 crosses the point set: the pairs with
    w < 0 satisfy the projection too but are behind the camera, so they are never inliers."""
    rng = np.random.default_rng(5)
    Ht = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [-2e-3, 0.0, 1.0]])  # w = 1 - x/500
    a = np.c_[rng.integers(10, 490, 50), rng.integers(0, 400, 50)]
    a = np.r_[a, np.c_[rng.integers(510, 1000, 20), rng.integers(0, 400, 20)]].astype(np.int32)
    bf, w = _exact_pairs(Ht, a)
    keep = np.abs(bf).max(axis=1) < 2e5
    a, bf, w = a[keep], bf[keep], w[keep]
    b = np.rint(bf).astype(np.int32)
    desc = rng.integers(0, 256, (len(a), 32), dtype=np.uint8)
    r = oracle.match_prosac(a, desc, b, desc, synth.lsh_bits(0), synth.prosac_words(6, 512), inlier_px=3.0)
    m = r["matches"]
    inl = np.zeros(len(a), bool)
    inl[m[r["inlier"], 0]] = True
    assert not inl[w < 0].any() and inl[w > 0].mean() > 0.9
