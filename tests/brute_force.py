"""A second, literal implementation of one gauge-fixing iteration, for pinning
the oracle on tiny lattices.

Written independently of ``oracle/lgf_oracle.py``: plain Python lists and
loops, coordinates as tuples with explicit periodic wrap-around, 3x3 complex
matrices multiplied entry by entry, the 4D Fourier transform as the full
V x V double sum with ``cmath.exp``, and Gram-Schmidt written out by hand.
Nothing here is vectorised or shared with the oracle.
"""
import cmath
import itertools
import math


def coords(L):
    Lx, Ly, Lz, Lt = L
    return [(x, y, z, t) for t in range(Lt) for z in range(Lz) for y in range(Ly) for x in range(Lx)]


def step(c, mu, d, L):
    c = list(c)
    c[mu] = (c[mu] + d) % L[mu]
    return tuple(c)


def zeros():
    return [[0j] * 3 for _ in range(3)]


def mat_mul(a, b):
    return [[sum(a[i][k] * b[k][j] for k in range(3)) for j in range(3)] for i in range(3)]


def dag(a):
    return [[a[j][i].conjugate() for j in range(3)] for i in range(3)]


def project_su3(m):
    r1 = list(m[0])
    r2 = list(m[1])
    n1 = math.sqrt(sum(abs(v) ** 2 for v in r1))
    r1 = [v / n1 for v in r1]
    ip = sum(r1[j].conjugate() * r2[j] for j in range(3))
    r2 = [r2[j] - ip * r1[j] for j in range(3)]
    n2 = math.sqrt(sum(abs(v) ** 2 for v in r2))
    r2 = [v / n2 for v in r2]
    r3 = [(r1[1] * r2[2] - r1[2] * r2[1]).conjugate(),
          (r1[2] * r2[0] - r1[0] * r2[2]).conjugate(),
          (r1[0] * r2[1] - r1[1] * r2[0]).conjugate()]
    return [r1, r2, r3]


def one_iteration(links, L, alpha):
    """links: dict (coord, mu) -> 3x3 list.  Returns (new_links, F, theta)."""
    sites = coords(L)
    V = len(sites)
    # gradient
    delta = {}
    for c in sites:
        a = zeros()
        for mu in range(4):
            back = links[(step(c, mu, -1, L), mu)]
            here = links[(c, mu)]
            for i in range(3):
                for j in range(3):
                    a[i][j] += back[i][j] - here[i][j]
        d = [[a[i][j] - a[j][i].conjugate() for j in range(3)] for i in range(3)]
        tr = (d[0][0] + d[1][1] + d[2][2]) / 3
        for i in range(3):
            d[i][i] -= tr
        delta[c] = d
    F = sum(links[(c, mu)][i][i].real for c in sites for mu in range(4) for i in range(3)) / (12 * V)
    theta = sum(abs(delta[c][i][j]) ** 2 for c in sites for i in range(3) for j in range(3)) / (3 * V)
    # momentum factor
    pmax = sum(max(4 * math.sin(math.pi * k / n) ** 2 for k in range(n)) for n in L)
    # full 4D DFT, V x V, entry by entry
    def phase(k, c, sign):
        return cmath.exp(sign * 2j * math.pi * sum(k[m] * c[m] / L[m] for m in range(4)))
    dk = {}
    for k in sites:
        p2 = sum(4 * math.sin(math.pi * k[m] / L[m]) ** 2 for m in range(4))
        fac = 0.0 if p2 == 0 else pmax / p2
        dk[k] = [[fac * sum(delta[c][i][j] * phase(k, c, -1) for c in sites) for j in range(3)]
                 for i in range(3)]
    g = {}
    for c in sites:
        dt = [[sum(dk[k][i][j] * phase(k, c, +1) for k in sites) / V for j in range(3)]
              for i in range(3)]
        m = [[(1.0 if i == j else 0.0) + 0.5 * alpha * dt[i][j] for j in range(3)] for i in range(3)]
        g[c] = project_su3(m)
    new = {}
    for c in sites:
        for mu in range(4):
            new[(c, mu)] = mat_mul(mat_mul(g[c], links[(c, mu)]), dag(g[step(c, mu, +1, L)]))
    return new, F, theta


def from_array(U):
    """oracle array U[t,z,y,x,mu,i,j] -> dict."""
    Lt, Lz, Ly, Lx = U.shape[:4]
    L = (Lx, Ly, Lz, Lt)
    out = {}
    for c in coords(L):
        x, y, z, t = c
        for mu in range(4):
            out[(c, mu)] = [[complex(U[t, z, y, x, mu, i, j]) for j in range(3)] for i in range(3)]
    return out, L


def max_diff(links, U):
    Lt, Lz, Ly, Lx = U.shape[:4]
    worst = 0.0
    for (c, mu), m in links.items():
        x, y, z, t = c
        for i, j in itertools.product(range(3), range(3)):
            worst = max(worst, abs(m[i][j] - U[t, z, y, x, mu, i, j]))
    return worst
