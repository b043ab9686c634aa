"""The Fourier CG solve as one persistent launch (each CTA loops its pair's steps, Alg. 1) against
one launch per step: the same operations in the same order, so the E-step's outputs, Lanczos
coefficients and step counts are bit-identical.  The two runs are separate processes because the
switch (CMCS_DFT_PERSIST) is read once per process."""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RUN = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2310_00420_gb300 import cmcs, synth
wl = synth.fourier_small()
out = {}
with cmcs.Context.from_fourier(wl, device=True, refine_max=8, refine_tol=1e-6, precond=int(sys.argv[3])) as ctx:
    ctx.em_iter(2)
    for k, v in dict(mu=cmcs.OUT_MU, s=cmcs.OUT_S, q=cmcs.OUT_Q, logdet=cmcs.OUT_LOGDET,
                     steps=cmcs.OUT_STEPS, gamma=cmcs.OUT_GAMMA, xi=cmcs.OUT_XI,
                     alpha=cmcs.OUT_ALPHA).items():
        out[k] = ctx.read(v)
np.savez(sys.argv[2], **out)
"""


@pytest.mark.parametrize("precond", [0, 1])
def test_persistent_fourier_solve_matches_per_step_launches(precond):
    with tempfile.TemporaryDirectory() as d:
        res = {}
        for persist in ("1", "0"):
            path = os.path.join(d, f"p{persist}.npz")
            env = dict(os.environ, CMCS_DFT_PERSIST=persist)
            r = subprocess.run([sys.executable, "-c", _RUN, ROOT, path, str(precond)], env=env,
                               capture_output=True, text=True, timeout=600)
            assert r.returncode == 0, r.stderr[-2000:]
            res[persist] = dict(np.load(path))
        for k in res["0"]:
            assert np.array_equal(res["1"][k], res["0"][k]), k
