"""Write the golden digest of the full-size outdoor decimation (CPU oracle only).

Workload: the 10000 x 2000-ray outdoor scan (seed 0, 15 % dropout, ground
plane, 40 boxes, 20 spheres at 1-60 m), the k = 4 density cost (Eq. 11),
keep 10 % (m = floor(0.1 n), Eq. 1).  The script generates the scan with the
seeded generator, runs the oracle's sequential greedy (kd-tree kNN, binary
heap, section "Sub-sampling algorithm") and writes
tests/golden/outdoor_k4_keep10.txt with the SHA-256 of the input
coordinates, n, m and the SHA-256 of the keep mask.  It calls nothing but
the generator and oracle/; about 5 minutes on 8 cores.

    python tests/golden/make_outdoor_golden.py
"""
import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2311_17604_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "outdoor_k4_keep10.txt")


def main():
    s = synth.outdoor_scan(seed=0, n_az=10000, n_el=2000)
    m = oracle.target_count(s.n, 0.1)
    t0 = time.time()
    keep = oracle.decimate(s.xyz, 4, m)
    dt = time.time() - t0
    assert int(keep.sum()) == m
    with open(OUT, "w") as f:
        f.write("# full-size outdoor scan (seed 0, 10000x2000 rays, 15% dropout), k = 4 density\n")
        f.write("# cost (Eq. 11), keep 10 % (Eq. 1): sequential greedy of the CPU oracle\n")
        f.write("# written by tests/golden/make_outdoor_golden.py (oracle %.0f s)\n" % dt)
        f.write("xyz_sha256 %s\n" % hashlib.sha256(np.ascontiguousarray(s.xyz).tobytes()).hexdigest())
        f.write("n %d\nm %d\n" % (s.n, m))
        f.write("keep_sha256 %s\n" % hashlib.sha256(keep.astype(np.uint8).tobytes()).hexdigest())
    print(open(OUT).read())


if __name__ == "__main__":
    main()
