"""The debug build (libstitch_debug.so) as a memory-safety check: every rig allocation sits between
NaN guard bands and the fused kernels check their index arithmetic, recording a failure instead of
trapping.  Small and edge-case rigs run through it, in a child process that loads that build; the
guards must be intact, no check may fail, and the output must still match the oracle."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import oracle, synth
from synth import Camera
from tests import gpu_util
from tests.test_parity_gpu import _max_rig
from paper_1810_03988_gb300 import Rig, Batch, stitch
assert stitch.load()._name.endswith("libstitch_debug.so")
res = []

def check(name, cfg, frames, path, out_float=True, band_fp16=False):
    ref = oracle.forward(cfg.cameras, frames, cfg.canvas_w, cfg.canvas_h, cfg.levels, canvas=cfg.canvas)
    with Rig(cfg.cameras, cfg.canvas_w, cfg.canvas_h, cfg.levels, out_float=out_float, path=path,
             band_fp16=band_fp16, canvas=cfg.canvas) as rig:
        out = rig.stitch(gpu_util.gpu_frames(frames))
        torch.cuda.synchronize()
        dbg = rig.debug_check()
        got = out.cpu().numpy()
    tol = gpu_util.TOL_F16 if band_fp16 else None
    st = gpu_util.compare(got, ref, out_float, tol)
    res.append(dict(name=name, path=path, **dbg, **{k: v for k, v in st.items() if k != "excluded"}))

cfg = synth.config_2cam()
for path in ("fused", "plain"):
    for out_float in (True, False):
        check("2cam", cfg, cfg.frame(0), path, out_float)
rng = np.random.default_rng(7)
cams = [Camera(40, 30, np.array([[1.0, 0, gx * 25.3], [0, 1.0, gy * 18.7], [0, 0, 1.0]]))
        for gy in range(3) for gx in range(4)]
frames = [rng.integers(0, 256, (30, 40, 3), dtype=np.uint8) for _ in cams]
check("grid12", synth.RigConfig("grid", cams, 120, 70, 4, 1, None), frames, "fused")
mcfg, mframes = _max_rig()
check("max32x12", mcfg, mframes, "fused")
c8 = synth.config_8x4k(scale=0.1, frames=1)
check("8x4k/10", c8, c8.frame(0), "fused", True, True)
cc = synth.config_cyl(scale=0.25)
check("cyl/4", cc, cc.frame(0), "fused")
# a batch through its persistent and staged schedules
cfgs = synth.config_batch(4, seed=3, scale=0.125)
rigs = [Rig(c.cameras, c.canvas_w, c.canvas_h, c.levels, out_float=True) for c in cfgs]
fr = [gpu_util.gpu_frames(c.frame(0)) for c in cfgs]
import os
for mode in ("persistent", "staged"):
    os.environ["STITCH_TUNE"] = mode
    with Batch(rigs) as b:
        outs = b.stitch(fr)
        b.sync()
        for k, (c, r, o) in enumerate(zip(cfgs, rigs, outs)):
            ref = oracle.forward(c.cameras, c.frame(0), c.canvas_w, c.canvas_h, c.levels)
            st = gpu_util.compare(o.cpu().numpy(), ref, True)
            res.append(dict(name=f"batch-{mode}-{k}", path="fused", **r.debug_check(), max_abs=st["max_abs"]))
print("RESULT " + json.dumps(res))
'''


def test_debug_build_guards_and_index_checks():
    from paper_1810_03988_gb300 import _build
    assert os.path.exists(_build.DEBUG_LIB), "the debug build is made by build()"
    env = dict(os.environ, STITCH_LIBRARY=_build.DEBUG_LIB)
    env.pop("STITCH_TUNE", None)
    p = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env, capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
    line = [x for x in p.stdout.splitlines() if x.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    assert len(res) >= 14
    for r in res:
        assert r["damaged_words"] == 0 and r["failed_check"] == 0, r
