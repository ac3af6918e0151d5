"""Extend the generating-vector table past its largest size with the GPU fast CBC.

The table's sizes follow the paper's rule (App. A.2): the next prime above
floor(1020 * 1.1^i) for i = 0..152, and 2^31 - 1.  The shipped table was computed on the
CPU; this tool computes the rows for the sizes beyond its largest n with
qmc_cbc_korobov (s = 10 components, gamma = 1/10, beta = 1) and writes them, in the same
"n z_1 .. z_10" format, to the extension table that GenvecTable.load() reads after the
shipped one.

    python -m paper_1811_11720_gb300.extend_table [--max-n N] [--out PATH]
"""
from __future__ import annotations

import argparse
import os
import sys
import time


def _is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (the first 13 primes as bases)."""
    if n < 2:
        return False
    bases = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41)
    for p in bases:
        if n % p == 0:
            return n == p
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in bases:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def table_sizes(imax: int = 152) -> list[int]:
    """The next prime strictly above floor(1020 * 1.1^i), i = 0..imax, and 2^31 - 1."""
    out = set()
    for i in range(imax + 1):
        p = int(1020.0 * 1.1 ** i) + 1
        while not _is_prime(p):
            p += 1
        out.add(p)
    out.add(2 ** 31 - 1)
    return sorted(out)


def main(argv=None) -> int:
    import paper_1811_11720_gb300 as q

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--s", type=int, default=10)
    ap.add_argument("--max-n", type=int, default=2 ** 31 - 1)
    ap.add_argument("--out", default=q.EXTENSION_TABLE)
    args = ap.parse_args(argv)
    base = q.GenvecTable.load(extension=False)
    have = set(int(v) for v in base.n)
    if os.path.exists(args.out):
        have |= set(int(v) for v in q.GenvecTable.load(args.out).n)
    start = int(base.n.max())
    todo = [n for n in table_sizes() if start < n <= args.max_n and n not in have]
    new_file = not os.path.exists(args.out)
    with open(args.out, "a") as fh:
        if new_file:
            fh.write("# rank-1 lattice generating vectors beyond the shipped table, fast CBC on the GPU\n"
                     "# (qmc_cbc_korobov): Korobov space alpha=2, omega(x)=2pi^2(x^2-x+1/6), "
                     f"gamma=1/{args.s}, beta=1\n# columns: n z_1 .. z_{args.s}\n")
        for n in todo:
            t0 = time.perf_counter()
            z, e2 = q.cbc_korobov(n, args.s)
            dt = time.perf_counter() - t0
            fh.write(" ".join(str(int(v)) for v in [n] + list(z)) + "\n")
            fh.flush()
            print(f"n={n} e2={e2[-1]:.4e} {dt:.1f}s", file=sys.stderr)
    return 0


if __name__ == "__main__":
    sys.exit(main())
