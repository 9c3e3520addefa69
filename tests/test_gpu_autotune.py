"""The launch-shape autotuner of the mixed-path SIMT sweep.

The first solve of a size class times the sweep at a few grid sizes and keeps the fastest in a
process-wide table; SFR_TUNE_FILE persists the table as a flat JSON object.  Each case runs in a
fresh interpreter so that the table starts empty.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1503_03004_gb300 import binding as B, synth
prob = synth.planted(2000, 360, 6, p=0.05, amp=50.0, seed=77, dtype="f32")
with B.Context(0) as ctx:
    sol = B.solve_torch(ctx, torch.from_numpy(prob.M).cuda(), 6, rho=1.5, mu0=0.05, tol=1e-9, max_iter=300,
                        precision=B.PREC_MIXED, s_dtype=B.F32)
    np.save({out!r}, np.concatenate([sol.U.cpu().numpy().ravel(), sol.B.cpu().numpy().ravel(), [sol.iters]]))
"""


def _child(tmp_path, name, env):
    out = str(tmp_path / f"{name}.npy")
    code = CHILD.format(root=ROOT, out=out)
    r = subprocess.run([sys.executable, "-c", code], env={**os.environ, **env}, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    import numpy as np
    return np.load(out)


def test_tuned_grid_is_persisted_and_reused(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    tune = tmp_path / "tune.json"
    first = _child(tmp_path, "a", {"SFR_TUNE_FILE": str(tune)})
    table = json.loads(tune.read_text())
    keys = [k for k in table if k.startswith("mx_sweep/")]
    assert len(keys) == 1 and table[keys[0]] in (2, 4, 8, 16)
    # a second process loads the choice instead of timing again, so it runs the same grid and
    # reproduces the first process's factors exactly
    second = _child(tmp_path, "b", {"SFR_TUNE_FILE": str(tune)})
    assert (first == second).all()
    assert json.loads(tune.read_text()) == table


def test_autotune_can_be_disabled(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    tune = tmp_path / "tune.json"
    _child(tmp_path, "c", {"SFR_TUNE_FILE": str(tune), "SFR_AUTOTUNE": "0"})
    table = json.loads(tune.read_text())
    assert list(table.values()) == [8]  # the untuned default: 8 CTAs per SM
