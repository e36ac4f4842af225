"""Long oracle runs for the parity tests, in processes of their own.

The FP64 oracle is single-threaded and takes minutes on the larger lattices,
so a test starts its runs in spawned processes (never forked: the parent may
hold a CUDA context) before it touches the GPU, runs the same workloads on the
GPU meanwhile, and compares when both are done. A run records, on the oracle's
side only:

* every step: n_s of that step (``ns_last``);
* every ``hstride`` steps: the front heights h(x);
* at each checkpoint: density, velocity, occupancy mask, heights and the
  counters, written to ``<outdir>/<name>_<step>.npz`` (rows below ``rows``).

Nothing here touches the GPU or the CUDA library.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_oracle(name: str, params: dict, steps: int, checkpoints, hstride: int, rows: int, outdir: str) -> str:
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle.oracle import OracleSim
    t0 = time.time()
    o = OracleSim(params)
    ns = np.zeros(steps, dtype=np.int64)
    hs = []
    cps = set(int(c) for c in checkpoints)
    for t in range(1, steps + 1):
        o.step(1)
        st = o.stats()
        ns[t - 1] = st["ns_last"]
        if t % hstride == 0:
            hs.append(o.heights())
        if t in cps:
            rho, ux, uy = o.fields()
            np.savez(os.path.join(outdir, f"{name}_{t}.npz"), rho=rho[:rows], ux=ux[:rows], uy=uy[:rows],
                     mask=o.mask()[:rows], heights=o.heights(), stats=json.dumps(st))
    np.savez(os.path.join(outdir, f"{name}_series.npz"), ns=ns, heights=np.array(hs))
    o.close()
    return f"{name}: {steps} oracle steps in {time.time() - t0:.0f} s"
