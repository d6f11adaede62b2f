"""The debug build (LBM_DEBUG_BOUNDS=1: every computed index of the step
kernels' global accesses and of the general pull's ring columns checked
against its buffer, a violation raising device error flag 2) runs the
boundary-heavy cases without a single out-of-range index: ragged periodic and
walled domains, a solid mask, a variable force field, the open sides of the
cylinder channel, every storage format, and a batch.  It runs in a child
process, which loads the debug library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np
import workloads as wl
from paper_1806_10251_gb300 import lbm
assert lbm.debug_bounds() and lbm.library_path().endswith("liblbm_gb300_debug.so")
cases = [wl.random_periodic(300, 41, 0.45, 0.03, seed=11), wl.random_cavity_state(65, 37, 0.5, Re=80.0, seed=5),
         wl.channel_obstacle(nx=160, ny=48, D=8, Re=20.0, U0=0.05, gamma=0.4, xc=40),
         wl.square_cylinder(4, 20.0, 0.1, 0.5), wl.open_channel(129, 33, 0.05, 0.5, 0.05),
         wl.four_rolls_mill(33, 0.045, 20.0, 0.5), wl.cavity(3, 10.0, 0.1, 0.5, ny=130)]
for c in cases:
    for storage in (lbm.STORAGE_F32, lbm.STORAGE_F16, lbm.STORAGE_BF16, lbm.STORAGE_F64):
        for opts in ({}, {"fd": 1}, {"guard": 1}):
            g = lbm.solver_from_case(c, storage=storage, **opts)
            g.step(40)
            g.residual()  # raises on the device error flag
            g.close()
b = lbm.Batch(1 << 30, storage=lbm.STORAGE_F16)
b.set_option("check_every", 50)
ids = [b.submit_case(c, tol=1e-300, max_steps=200) for c in
       (wl.cavity(96, 100.0, 0.1, 0.5, ny=70), wl.cavity(33, 50.0, 0.1, 1.0),
        wl.channel_obstacle(nx=160, ny=48, D=8, Re=20.0, U0=0.05, gamma=0.4, xc=40))]
b.run()
assert all(b.poll(i)[1].state == lbm.REQ_NOT_CONVERGED for i in ids)
b.close()
print("debug bounds: clean")
"""


def test_debug_build_finds_no_out_of_range_index():
    env = dict(os.environ, LBM_DEBUG_BOUNDS="1")
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0 and "debug bounds: clean" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
