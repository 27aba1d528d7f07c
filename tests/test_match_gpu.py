"""Multi-Probe LSH matching and PROSAC on the GPU against the oracle (Sec. 4.2, Algorithm 3):
matches, inlier flags, inlier count and the homography bit-exact, on L-ORB features of two
synthetic views (several table shapes, ratio tests and iteration counts), on contaminated
correspondences at the maximum point count, with features chained from the GPU L-ORB, and on the
degenerate cases (no points, too few matches, no iterations, counts above the context's size)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=dtype))).cuda()


def _gpu(xy_a, desc_a, xy_b, desc_b, bits, rnd, max_dist=80, ratio=(4, 5), inlier_px=3.0, ctx=None,
         count_a=None, count_b=None, max_points=2048):
    import torch
    from paper_1810_03988_gb300 import Matcher
    own = ctx is None
    ctx = ctx or Matcher(max_points, max(len(rnd), 1))
    na = len(xy_a) if count_a is None else count_a
    nb = len(xy_b) if count_b is None else count_b
    args = [_dev(np.reshape(xy_a, (-1, 2)), np.int32), _dev(np.reshape(desc_a, (-1, 32)), np.uint8),
            _dev([na], np.int32), _dev(np.reshape(xy_b, (-1, 2)), np.int32),
            _dev(np.reshape(desc_b, (-1, 32)), np.uint8), _dev([nb], np.int32)]
    rw = _dev(np.asarray(rnd, np.uint32).view(np.int32).reshape(-1, 4), np.int32) if len(rnd) else None
    mt, nm, H, ni, inl = ctx.match(*args, bits, rw, max_dist, ratio, inlier_px)
    torch.cuda.synchronize()
    n = int(nm.cpu()[0])
    out = {"matches": mt[:n].cpu().numpy(), "H": H.cpu().numpy().reshape(3, 3), "inliers": int(ni.cpu()[0]),
           "inlier": inl[:n].cpu().numpy().astype(bool)}
    if own:
        ctx.close()
    return out


def _same(g, r):
    np.testing.assert_array_equal(g["matches"], r["matches"])
    np.testing.assert_array_equal(g["inlier"], r["inlier"])
    assert g["inliers"] == r["inliers"]
    np.testing.assert_array_equal(g["H"], r["H"])  # bit-exact: same operations in the same order


_VIEWS = {}


def _views(scale=0.5, n=600):
    key = (scale, n)
    if key not in _VIEWS:
        cfg = synth.config_4x1080p(scale=scale, frames=1)
        fr = cfg.frame(0)
        pat = synth.brief_pattern(0)
        H, W = fr[0].shape[:2]
        fa = oracle.lorb(fr[0], [(W // 2, 0, W, H)], pat, max_points=n)
        fb = oracle.lorb(fr[1], [(0, 0, W // 2, H)], pat, max_points=n)
        _VIEWS[key] = (fa, fb)
    return _VIEWS[key]


@pytest.mark.parametrize("L,k,max_dist,ratio,iters", [(8, 16, 80, (4, 5), 1024), (6, 12, 40, (3, 4), 333),
                                                      (1, 1, 256, (1, 1), 64), (32, 20, 80, (4, 5), 4096),
                                                      (4, 8, 60, (9, 10), 0)])
def test_views_match_oracle(L, k, max_dist, ratio, iters):
    fa, fb = _views()
    bits = synth.lsh_bits(L * 100 + k, L, k)
    rnd = synth.prosac_words(iters, iters)
    r = oracle.match_prosac(fa["xy"], fa["desc"], fb["xy"], fb["desc"], bits, rnd, max_dist, ratio)
    g = _gpu(fa["xy"], fa["desc"], fb["xy"], fb["desc"], bits, rnd, max_dist, ratio)
    _same(g, r)
    if iters >= 1024:
        assert r["inliers"] > 50


@pytest.mark.parametrize("inlier_px", [0.5, 3.0, 20.0])
def test_contaminated_correspondences_at_the_maximum_point_count(inlier_px):
    rng = np.random.default_rng(11)
    Ht = np.array([[0.98, 0.03, -40.0], [0.02, 1.01, 25.0], [-3e-5, 2e-5, 1.0]])
    n, n_out = 2048, 700
    xa = rng.integers(0, 2000, (n, 2)).astype(np.int32)
    xb = np.c_[xa, np.ones(n)] @ Ht.T
    xb = np.rint(xb[:, :2] / xb[:, 2:3]).astype(np.int32)
    xb[n - n_out:] = rng.integers(0, 2000, (n_out, 2))
    # few distinct descriptors plus noise bits: crowded buckets, equal distances, ties on index
    base = rng.integers(0, 256, (300, 32), dtype=np.uint8)
    da = base[rng.integers(0, 300, n)]
    flip = (rng.random((n, 32, 8)) < 0.03)
    db = da ^ np.packbits(flip, axis=2, bitorder="little").reshape(n, 32)
    bits, rnd = synth.lsh_bits(7), synth.prosac_words(7, 2000)
    r = oracle.match_prosac(xa, da, xb, db, bits, rnd, 80, (4, 5), inlier_px)
    g = _gpu(xa, da, xb, db, bits, rnd, 80, (4, 5), inlier_px)
    _same(g, r)
    assert len(r["matches"]) > 100


def test_gpu_lorb_features_chain_into_the_matcher():
    import torch
    from paper_1810_03988_gb300 import LORB, Matcher
    cfg = synth.config_4x1080p(scale=0.5, frames=1)
    fr = cfg.frame(0)
    pat = synth.brief_pattern(3)
    H, W = fr[0].shape[:2]
    areas_a, areas_b = [(W // 2, 0, W, H)], [(0, 0, W // 2, H)]
    bits, rnd = synth.lsh_bits(3), synth.prosac_words(3, 1000)
    with LORB(W, H, 800) as la, LORB(W, H, 800) as lb, Matcher(800, 1000) as m:
        xa, _, da, ca = la.detect(torch.from_numpy(fr[0]).cuda(), areas_a, pat, 20, 0, 800)
        xb, _, db, cb = lb.detect(torch.from_numpy(fr[1]).cuda(), areas_b, pat, 20, 0, 800)
        rw = torch.from_numpy(rnd.view(np.int32)).cuda()
        mt, nm, Hd, ni, inl = m.match(xa, da, ca, xb, db, cb, bits, rw)
        torch.cuda.synchronize()
        n = int(nm.cpu()[0])
        g = {"matches": mt[:n].cpu().numpy(), "H": Hd.cpu().numpy().reshape(3, 3), "inliers": int(ni.cpu()[0]),
             "inlier": inl[:n].cpu().numpy().astype(bool)}
    fa = oracle.lorb(fr[0], areas_a, pat, 20, 0, 800)
    fb = oracle.lorb(fr[1], areas_b, pat, 20, 0, 800)
    r = oracle.match_prosac(fa["xy"], fa["desc"], fb["xy"], fb["desc"], bits, rnd)
    _same(g, r)
    assert r["inliers"] > 50


def test_degenerate_cases():
    from paper_1810_03988_gb300 import Matcher
    fa, fb = _views()
    bits, rnd = synth.lsh_bits(0), synth.prosac_words(0, 200)
    with Matcher(600, 200) as ctx:
        # no points in A, none in B, too few matches for a model, no iterations
        for na, nb, it in [(0, len(fb["xy"]), 200), (len(fa["xy"]), 0, 200), (3, len(fb["xy"]), 200),
                           (len(fa["xy"]), len(fb["xy"]), 0)]:
            rw = rnd[:it]
            r = oracle.match_prosac(fa["xy"][:na], fa["desc"][:na], fb["xy"][:nb], fb["desc"][:nb], bits, rw)
            g = _gpu(fa["xy"], fa["desc"], fb["xy"], fb["desc"], bits, rw, ctx=ctx, count_a=na, count_b=nb)
            _same(g, r)
            assert g["inliers"] == 0 and np.array_equal(g["H"], np.eye(3))
    # counts above the context's size use the first max_points points of each image
    with Matcher(250, 200) as ctx:
        r = oracle.match_prosac(fa["xy"][:250], fa["desc"][:250], fb["xy"][:250], fb["desc"][:250], bits, rnd)
        g = _gpu(fa["xy"], fa["desc"], fb["xy"], fb["desc"], bits, rnd, ctx=ctx)
        _same(g, r)


def test_context_reuse_and_bad_arguments():
    from paper_1810_03988_gb300 import Matcher, StitchError
    fa, fb = _views()
    with Matcher(600, 100) as ctx:
        for seed in range(3):
            bits, rnd = synth.lsh_bits(seed), synth.prosac_words(seed, 100)
            r = oracle.match_prosac(fa["xy"], fa["desc"], fb["xy"], fb["desc"], bits, rnd)
            _same(_gpu(fa["xy"], fa["desc"], fb["xy"], fb["desc"], bits, rnd, ctx=ctx), r)
        with pytest.raises(StitchError):  # more iterations than the context holds
            _gpu(fa["xy"], fa["desc"], fb["xy"], fb["desc"], synth.lsh_bits(0), synth.prosac_words(0, 101), ctx=ctx)
        with pytest.raises(StitchError):  # 33 tables
            _gpu(fa["xy"], fa["desc"], fb["xy"], fb["desc"], synth.lsh_bits(0, 33, 8), synth.prosac_words(0, 10),
                 ctx=ctx)


def test_rig_registered_from_its_own_frames_stitches_like_the_true_rig():
    """The loop of Algorithm 4 on the GPU: L-ORB in the overlap halves of neighbouring views,
    matching and PROSAC per pair, the pairwise homographies chained outwards from camera 1 (placed
    as in the true rig), then stitch_rig_create with the estimates.  Each pair registers to a
    fraction of a pixel over its overlap; chained maps drift where they extrapolate (beyond the
    overlaps), so the canvases are compared between the camera centres."""
    import torch
    from paper_1810_03988_gb300 import LORB, Matcher, Rig
    cfg = synth.config_4x1080p(scale=0.5, frames=1)
    fr = cfg.frame(0)
    dfr = [torch.from_numpy(f).cuda() for f in fr]
    pat, bits = synth.brief_pattern(5), synth.lsh_bits(5)
    rw = torch.from_numpy(synth.prosac_words(5, 2000).view(np.int32)).cuda()
    H, W = fr[0].shape[:2]
    true = [np.asarray(c.H, dtype=np.float64) for c in cfg.cameras]
    pair = []
    with LORB(W, H, 1000) as la, LORB(W, H, 1000) as lb, Matcher(1000, 2000) as m:
        for i in range(len(fr) - 1):
            xa, _, da, ca = la.detect(dfr[i], [(W // 2, 0, W, H)], pat, 20, 0, 1000)
            xb, _, db, cb = lb.detect(dfr[i + 1], [(0, 0, W // 2, H)], pat, 20, 0, 1000)
            _, _, Hab, ni, _ = m.match(xa, da, ca, xb, db, cb, bits, rw)
            torch.cuda.synchronize()
            assert int(ni.cpu()[0]) > 200
            pair.append(Hab.cpu().numpy().reshape(3, 3))

    def err(Ha, Hb, pts):
        pa, pb = Ha @ pts, Hb @ pts
        return np.abs(pa[:2] / pa[2] - pb[:2] / pb[2]).max()

    grid = np.array([[x, y, 1.0] for x in np.linspace(0, W - 1, 24) for y in np.linspace(0, H - 1, 12)]).T
    for i, Hp in enumerate(pair):  # pairwise: over the points of view i that view i + 1 sees
        Ht = np.linalg.inv(true[i + 1]) @ true[i]
        q = Ht @ grid
        q = q[:2] / q[2]
        seen = (q[0] >= 0) & (q[0] < W) & (q[1] >= 0) & (q[1] < H)
        assert seen.sum() > 50 and err(Hp, Ht, grid[:, seen]) < 0.5
    ref = 1
    est = [None] * len(true)
    est[ref] = true[ref]
    for i in range(ref - 1, -1, -1):
        est[i] = est[i + 1] @ pair[i]
    for i in range(ref + 1, len(true)):
        est[i] = est[i - 1] @ np.linalg.inv(pair[i - 1])
    est = [h / h[2, 2] for h in est]
    for i in (ref - 1, ref + 1):  # neighbours of the reference, over their overlap with it
        q = np.linalg.inv(true[ref]) @ true[i] @ grid
        q = q[:2] / q[2]
        seen = (q[0] >= 0) & (q[0] < W) & (q[1] >= 0) & (q[1] < H)
        assert err(est[i], true[i], grid[:, seen]) < 1.0
    cams = [synth.Camera(c.width, c.height, h) for c, h in zip(cfg.cameras, est)]
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels) as rt, \
            Rig(cams, cfg.canvas_w, cfg.canvas_h, cfg.levels) as re:
        ot = rt.stitch(dfr).cpu().numpy().astype(np.float64)
        oe = re.stitch(dfr).cpu().numpy().astype(np.float64)
    both = (ot.sum(axis=2) > 0) & (oe.sum(axis=2) > 0)
    d = np.abs(ot - oe).mean(axis=2)
    cx = [int(round((h @ [W / 2, H / 2, 1])[0] / (h @ [W / 2, H / 2, 1])[2])) for h in true]
    for a in range(len(cx) - 1):  # between neighbouring camera centres: each seam region
        sl = slice(cx[a], cx[a + 1])
        assert d[:, sl][both[:, sl]].mean() < 2.5, a
