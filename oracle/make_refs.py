"""Write FP64 oracle results of long runs that the GPU checks are compared with.

TEST INFRASTRUCTURE ONLY: calls nothing but ``oracle`` and the seeded input
generators in ``synth``.  The results are large (hundreds of MB) and take the
oracle tens of minutes, so they are written to a directory of the caller's
choice instead of the repository; each file carries the SHA-256 of the inputs
it was computed from, which the reader checks before use.

    python oracle/make_refs.py ring3d OUT_DIR      # 512x512x128, 31x31x21 template, 100 steps

Output: OUT_DIR/ring3d_x100.npz with X (the iterate after 100 accepted steps
of Steps 1-3 from the centre crop of Y, float32-rounded: 6e-8 relative at most),
f (the objective history), accepted, rejected, status, and the inputs Y and H
with their SHA-256 (input_sha256).  The inputs travel with the result because
the generator's library FFT blur and Poisson draws may differ in the last bits
between machines; a reader on another machine runs on the stored inputs.
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def input_sha256(P):
    """SHA-256 of the workload's observation, template and iteration count."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(P.Y, dtype=np.float32).tobytes())
    h.update(np.ascontiguousarray(P.H, dtype=np.float32).tobytes())
    h.update(str(int(P.K)).encode())
    return h.hexdigest()


def ring3d(out_dir, K=100):
    import oracle
    import synth
    P = synth.ring3d(K=K)
    t0 = time.time()
    ref = oracle.iterate(P.Y, P.H, oracle.x0_crop(P.Y, P.p), P.K)
    dt = time.time() - t0
    path = os.path.join(out_dir, "ring3d_x%d.npz" % K)
    np.savez(path, X=ref["X"].astype(np.float32), f=ref["f"], accepted=ref["accepted"],
             rejected=ref["rejected"], status=ref["status"], input_sha256=input_sha256(P),
             seconds=dt, threads=oracle.num_threads(), Y=P.Y, H=P.H, K=P.K)
    return path, dt


if __name__ == "__main__":
    if len(sys.argv) != 3 or sys.argv[1] != "ring3d":
        raise SystemExit(__doc__)
    os.makedirs(sys.argv[2], exist_ok=True)
    path, dt = ring3d(sys.argv[2])
    print("wrote %s (%.0f s)" % (path, dt))
