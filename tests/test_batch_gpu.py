"""S8: several rigs in one persistent launch (CUDA graph), against per-rig launches and the oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests import gpu_util

pytestmark = pytest.mark.gpu


def _rigs_and_frames(cfgs, out_float=False, band_fp16=False):
    from paper_1810_03988_gb300 import Rig
    rigs = [Rig(c.cameras, c.canvas_w, c.canvas_h, c.levels, out_float=out_float, band_fp16=band_fp16) for c in cfgs]
    frames = [gpu_util.gpu_frames(c.frame(0)) for c in cfgs]
    return rigs, frames


def _per_rig(rigs, frames):
    import torch
    outs = [r.stitch(f) for r, f in zip(rigs, frames)]
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


@pytest.mark.parametrize("out_float", [False, True])
def test_batch_equals_per_rig_launches(out_float):
    """16 uneven rigs (2-6 cameras, 720p/1080p/4K views, 4-6 levels) at 1/4 scale: the batched
    launch gives bit-identical canvases to one launch sequence per rig, on repeated calls."""
    from paper_1810_03988_gb300 import Batch
    cfgs = synth.config_batch(16, seed=0, scale=0.25)
    rigs, frames = _rigs_and_frames(cfgs, out_float=out_float)
    ref = _per_rig(rigs, frames)
    with Batch(rigs) as b:
        for _ in range(2):
            outs = b.stitch(frames)
            got = [o.cpu().numpy() for o in outs]
            for g, r in zip(got, ref):
                assert np.array_equal(g, r)
        sch = b.schedule()
        assert sch["tasks"] > 0 and sch["mode"] in ("persistent", "staged", "streams")
    for r in rigs:
        r.close()


def test_batch_full_size_equals_per_rig_launches():
    from paper_1810_03988_gb300 import Batch
    cfgs = synth.config_batch(16, seed=0)
    rigs, frames = _rigs_and_frames(cfgs)
    ref = _per_rig(rigs, frames)
    with Batch(rigs) as b:
        got = [o.cpu().numpy() for o in b.stitch(frames)]
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)
    for r in rigs:
        r.close()


def test_batch_matches_oracle():
    from paper_1810_03988_gb300 import Batch
    cfgs = synth.config_batch(5, seed=4, scale=0.125)
    rigs, frames = _rigs_and_frames(cfgs, out_float=True)
    with Batch(rigs) as b:
        got = [o.cpu().numpy() for o in b.stitch(frames)]
    for cfg, g in zip(cfgs, got):
        ref = oracle.forward(cfg.cameras, cfg.frame(0), cfg.canvas_w, cfg.canvas_h, cfg.levels)
        gpu_util.compare(g, ref, True)
    for r in rigs:
        r.close()


def test_batch_full_size_matches_oracle_windows():
    """The full-size 16-rig batch (2-6 cameras of 720p/1080p/4K, 4-6 levels): windows at every
    rig's seams, corners and random places against the oracle (each window evaluated exactly)."""
    from paper_1810_03988_gb300 import Batch
    cfgs = synth.config_batch(16, seed=0)
    rigs, frames = _rigs_and_frames(cfgs)
    with Batch(rigs) as b:
        got = [o.cpu().numpy() for o in b.stitch(frames)]
    for k, (cfg, g) in enumerate(zip(cfgs, got)):
        host = cfg.frame(0)
        for (x0, y0, w, h) in gpu_util.sample_windows(cfg, 6, 48, seed=k)[:10]:
            ref = oracle.forward(cfg.cameras, host, cfg.canvas_w, cfg.canvas_h, cfg.levels, window=(x0, y0, w, h))
            gpu_util.compare(g[y0:y0 + h, x0:x0 + w], ref, False)
    for r in rigs:
        r.close()


def test_batch_fp16_bands():
    from paper_1810_03988_gb300 import Batch
    cfgs = synth.config_batch(4, seed=2, scale=0.125)
    rigs, frames = _rigs_and_frames(cfgs, out_float=True, band_fp16=True)
    ref = _per_rig(rigs, frames)
    with Batch(rigs) as b:
        got = [o.cpu().numpy() for o in b.stitch(frames)]
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)
    for r in rigs:
        r.close()


@pytest.fixture
def forced_schedule(monkeypatch):
    def force(mode):
        monkeypatch.setenv("STITCH_TUNE", mode)
    return force


@pytest.mark.parametrize("mode", ["persistent", "staged", "streams"])
def test_each_schedule_equals_per_rig_launches(mode, forced_schedule):
    from paper_1810_03988_gb300 import Batch
    forced_schedule(mode)
    cfgs = synth.config_batch(6, seed=5, scale=0.25)
    rigs, frames = _rigs_and_frames(cfgs)
    ref = _per_rig(rigs, frames)
    with Batch(rigs) as b:
        for _ in range(2):
            got = [o.cpu().numpy() for o in b.stitch(frames)]
            for g, r in zip(got, ref):
                assert np.array_equal(g, r)
        assert b.schedule()["mode"] == mode
    for r in rigs:
        r.close()


def test_batch_bounded_wait_times_out_and_recovers(forced_schedule):
    """A stage target that is never reached makes the device wait of the persistent schedule give
    up: the asynchronous call's outcome, read by sync(), is STITCH_ETIMEOUT, and after restoring the
    target the same batch stitches correctly."""
    from paper_1810_03988_gb300 import Batch, StitchError, stitch
    forced_schedule("persistent")
    cfgs = synth.config_batch(3, seed=1, scale=0.125)
    rigs, frames = _rigs_and_frames(cfgs)
    ref = _per_rig(rigs, frames)
    with Batch(rigs) as b:
        b.stitch(frames)  # tune and build the graph first
        b.wait_test(2000, 0)
        with pytest.raises(StitchError) as e:
            b.stitch(frames)
            b.sync()
        assert e.value.status == stitch.STITCH_ETIMEOUT
        b.sync()  # reported once
        b.wait_test(1 << 22, -1)
        outs = b.stitch(frames)
        b.sync()
        got = [o.cpu().numpy() for o in outs]
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)
    for r in rigs:
        r.close()


def test_batch_rejects_unsupported_mixes():
    from paper_1810_03988_gb300 import Batch, Rig, StitchError, stitch
    cfg = synth.config_2cam(scale=0.2)
    a = Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels)
    p = Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, path="plain")
    h = Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, band_fp16=True)
    with pytest.raises(StitchError) as e:
        Batch([a, p])
    assert e.value.status == stitch.STITCH_EINVAL
    with pytest.raises(StitchError) as e:
        Batch([a, h])
    assert e.value.status == stitch.STITCH_EUNSUPPORTED
    for r in (a, p, h):
        r.close()


def test_tuning_cache_round_trip_and_every_tile_shape(tmp_path, monkeypatch):
    """STITCH_TUNE_CACHE: the first batch times the candidates and appends its choice; a second batch
    over the same rigs takes it from the file without timing.  A cache line naming each staged
    tile-shape combination (reduce 32x16 / 64x8, coarse 32x32 / 64x16) is taken as written, and
    every combination gives canvases bit-identical to per-rig launches."""
    import json
    from paper_1810_03988_gb300 import Batch
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("STITCH_TUNE_CACHE", str(cache))
    monkeypatch.delenv("STITCH_TUNE", raising=False)
    cfgs = synth.config_batch(5, seed=6, scale=0.25)
    rigs, frames = _rigs_and_frames(cfgs)
    ref = _per_rig(rigs, frames)
    with Batch(rigs) as b:
        b.stitch(frames)
        b.sync()
        first = b.schedule()
    assert not first["cached"]
    lines = [json.loads(x) for x in cache.read_text().splitlines()]
    assert len(lines) == 1 and lines[0]["mode"] == first["mode"]
    key = lines[0]["key"]
    with Batch(rigs) as b:
        got = [o.cpu().numpy() for o in b.stitch(frames)]
        assert b.schedule()["cached"] and b.schedule()["mode"] == first["mode"]
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)
    for shape in range(4):
        with open(cache, "a") as f:
            f.write(json.dumps({"key": key, "mode": "staged", "order": 1, "variant": 1, "chunk": 4, "shape": shape,
                                "ms": 0.0}) + "\n")
        with Batch(rigs) as b:
            outs = b.stitch(frames)
            b.sync()
            sch = b.schedule()
            assert sch["cached"] and sch["mode"] == "staged" and sch["shape"] == shape, sch
            for o, r in zip(outs, ref):
                assert np.array_equal(o.cpu().numpy(), r), shape
    for r in rigs:
        r.close()
