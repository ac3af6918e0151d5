"""Write the generating-vector table used by both the oracle and the CUDA path.

    python -m oracle.make_genvec_table [--nmax 1024565021] [--s 10] [--out tables/...]

The paper ships its vectors as data (App. A.3, table of generating vectors); they are
not in this repository, so this script regenerates a table with the oracle's own CBC
(oracle/lattice.py): lattice sizes from the paper's size rule (next prime above
1020 * 1.1^i), Korobov-space kernel with alpha = 2, gamma_j = 1/s, beta_j = 1.  Sizes
up to 5000 are built with the naive CBC and larger ones with the FFT CBC; the two agree
on every prime where both were compared (tests/test_oracle_cbc.py).

The file is appended one line per size, "n z_1 ... z_s", so an interrupted run resumes.
Calls only oracle/ code.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle import lattice as L  # noqa: E402

DEFAULT_OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                           "tables", "cbc_korobov_a2_s10.txt")
NAIVE_MAX = 5000


def header(s: int) -> str:
    return (f"# rank-1 lattice generating vectors, CBC, Korobov space alpha=2, "
            f"omega(x)=2pi^2(x^2-x+1/6), gamma_j=1/{s}, beta_j=1, s={s}\n"
            f"# sizes: next prime above floor(1020*1.1^i); columns: n z_1 .. z_{s}\n")


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--nmax", type=int, default=1024565021)
    ap.add_argument("--nmin", type=int, default=0)
    ap.add_argument("--s", type=int, default=10)
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--only", type=int, nargs="*", default=None,
                    help="build just these sizes (must be table sizes)")
    args = ap.parse_args(argv)
    sizes = [n for n in L.lattice_sizes() if args.nmin <= n <= args.nmax]
    if args.only:
        sizes = [n for n in sizes if n in set(args.only)]
    done = set()
    if os.path.exists(args.out):
        for line in open(args.out):
            if line.strip() and not line.startswith("#"):
                done.add(int(line.split()[0]))
    else:
        os.makedirs(os.path.dirname(args.out), exist_ok=True)
        with open(args.out, "w") as fh:
            fh.write(header(args.s))
    for n in sizes:
        if n in done:
            continue
        t0 = time.time()
        z, e2 = (L.cbc_naive if n <= NAIVE_MAX else L.cbc_fast)(n, args.s)
        with open(args.out, "a") as fh:
            fh.write(" ".join(str(v) for v in [n] + list(z)) + "\n")
        print(f"n={n} z={z} e2={e2[-1]:.3e} {time.time() - t0:.1f}s", flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
