"""Search for the Korobov generator a of the rank-1 lattice used by T_k, k>=3.

Figure of merit: P_2 of the lattice in the unweighted (gamma_d = 1) periodic
Korobov space of smoothness alpha = 2, the worst-case squared error of the
lattice rule for periodised integrands (Sloan & Joe, "Lattice Methods for
Multiple Integration", 1994):
    P_2(z) = -1 + (1/N) sum_i prod_d (1 + 2 pi^2 B_2({i z_d / N})),
B_2(x) = x^2 - x + 1/6.  z_d = a^d mod N.  The chosen a minimises the largest
P_2 over the dimensions 3..8 relative to the best a for that dimension.
Run: python oracle/korobov_search.py [N]
"""
import sys

import numpy as np


def p2(N, a, s):
    i = np.arange(N)
    z = [pow(a, d, N) for d in range(s)]
    prod = np.ones(N)
    for zd in z:
        x = (i * zd % N) / N
        prod *= 1.0 + 2.0 * np.pi ** 2 * (x * x - x + 1.0 / 6.0)
    return prod.mean() - 1.0


def search(N):
    cands = [a for a in range(3, N // 2, 2)]
    tab = np.array([[p2(N, a, s) for s in range(3, 9)] for a in cands])
    best = tab.min(axis=0)
    score = (tab / best).max(axis=1)
    k = int(np.argmin(score))
    return cands[k], score[k], tab[k]


if __name__ == "__main__":
    N = int(sys.argv[1]) if len(sys.argv) > 1 else 1024
    a, sc, row = search(N)
    print(f"N={N} a={a} worst ratio to per-dimension best={sc:.3f} P2(s=3..8)={row}")
