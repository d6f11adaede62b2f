"""Writes batch_sample_steady.npz: the FP64 oracle's steady states of the
smallest cavities of the seeded batch set (workloads.batch_cavities(256,
seed=0), indices listed in INDICES: sides 64, 96 and 128, Re 360-732, gamma
0.75-0.87; U = 0.1, Sec. 5 kernel, omega3 = omega6 = omega7 = omega8 = 1),
each marched from rest until the relative L2 change of u between checks 1000
steps apart is below 1e-11.  Calls only the oracle.  Fields stored in float32
(ample for the 1e-3 bound of the reduced-precision batch)."""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
import workloads as wl  # noqa: E402

INDICES = (7, 23, 5, 27, 6)


def main():
    cases = wl.batch_cavities(256, seed=0)
    out = {}
    for i in INDICES:
        c = cases[i]
        d = orc.Domain(c.nx, c.ny, c.nu, c.gamma, c.sides, gi_mode=orc.GI_FULL)
        d.init_equilibrium()
        t0 = time.time()
        while True:
            d.step(1000)
            r, _ = d.residual()
            if r < 1e-11 or d.steps >= 3_000_000:
                break
        _, u, v = d.fields()
        print(i, c.nx, c.meta["Re"], c.gamma, d.steps, r, f"{time.time() - t0:.0f}s", flush=True)
        out[f"ux_{i}"] = u.astype(np.float32)
        out[f"uy_{i}"] = v.astype(np.float32)
        out[f"steps_{i}"] = d.steps
        out[f"residual_{i}"] = r
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch_sample_steady.npz")
    np.savez_compressed(path, indices=np.array(INDICES), **out)
    print("wrote", path)


if __name__ == "__main__":
    main()
