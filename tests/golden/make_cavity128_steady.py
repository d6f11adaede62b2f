"""Writes cavity128_re100_g05_steady.npz: the FP64 oracle's steady state of the
128 x 128 lid-driven cavity (U = 0.1, Re = 100, gamma = 0.5, Sec. 5 kernel,
omega3 = omega6 = omega7 = omega8 = 1), marched from rest until the relative L2
change of u between checks 1000 steps apart is below 1e-12.  Calls only the
oracle.  Stored in float32 (ample for the 1e-6 parity bound)."""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
import workloads as wl  # noqa: E402


def main():
    c = wl.cavity(128, 100.0, 0.1, 0.5)
    d = orc.Domain(c.nx, c.ny, c.nu, c.gamma, c.sides, gi_mode=orc.GI_FULL)
    d.init_equilibrium()
    t0 = time.time()
    hist = []
    while True:
        d.step(1000)
        r, _ = d.residual()
        hist.append((d.steps, r))
        print(d.steps, r, f"{time.time() - t0:.0f}s", flush=True)
        if r < 1e-12 or d.steps >= 2_000_000:
            break
    rho, u, v = d.fields()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cavity128_re100_g05_steady.npz")
    np.savez_compressed(out, rho=rho.astype(np.float32), ux=u.astype(np.float32), uy=v.astype(np.float32),
                        steps=d.steps, final_residual=hist[-1][1], history=np.array(hist))
    print("wrote", out)


if __name__ == "__main__":
    main()
