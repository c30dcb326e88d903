"""Writes the stored oracle results used by the full-size parity tests.

Calls only ``oracle`` (and the seeded ``workloads`` generators):
  c2_eigenvalues.npy -- all 8192 eigenvalues of config C2 (16^3 single vortex),
                        FP64 Householder + implicit QR, ascending.
Run:  python tests/golden/make_golden.py [threads]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as wk  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else 0
    w = wk.c2_single_vortex()
    t = time.time()
    H = oracle.build(w)
    ev = oracle.heev(H, vectors=False, threads=threads)
    dt = time.time() - t
    np.save(os.path.join(HERE, "c2_eigenvalues.npy"), ev)
    print(f"C2 N={w.N}: {dt:.1f} s with {threads or oracle.max_threads()} threads")


if __name__ == "__main__":
    main()
