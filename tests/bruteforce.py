"""Brute-force references written in the tests, independent of the oracle's C code.

They restate the definitions of Sec. 2.1 with scipy's connected-component
labelling instead of the oracle's breadth-first search, and re-run the
subfield schedule in plain Python.  Only usable on tiny images.
"""
import numpy as np
from scipy import ndimage

EIGHT = np.ones((3, 3), dtype=int)
FOUR = np.array([[0, 1, 0], [1, 1, 1], [0, 1, 0]])
# ring order E, NE, N, NW, W, SW, S, SE as (row, col) in a 3x3 grid
RING_RC = [(1, 2), (0, 2), (0, 1), (0, 0), (1, 0), (2, 0), (2, 1), (2, 2)]
FOUR_NEIGHBOURS_RC = {(0, 1), (1, 0), (1, 2), (2, 1)}


def ring_values(grid):
    g = np.asarray(grid)
    return [int(g[r, c]) for r, c in RING_RC]


def grid_from_ring(center, nb):
    g = np.zeros((3, 3), dtype=np.int64)
    g[1, 1] = center
    for (r, c), v in zip(RING_RC, nb):
        g[r, c] = v
    return g


def _counted(labels, n_labels, n):
    """Components (sets of (r, c)) holding a point n-adjacent to the centre."""
    out = []
    for lab in range(1, n_labels + 1):
        pts = set(zip(*np.nonzero(labels == lab)))
        if n == 8 or pts & FOUR_NEIGHBOURS_RC:
            out.append(pts)
    return out


def local_numbers(grid, adj=0):
    """(T+, T--, list of lower components as sets of (r, c)) by scipy labelling;
    adj 0: (n, nbar) = (8, 4), adj 1: (4, 8)."""
    g = np.asarray(grid, dtype=np.int64)
    c = g[1, 1]
    n, nbar = (4, 8) if adj else (8, 4)
    upper = (g >= c)
    upper[1, 1] = False
    lower = (g < c)
    lower[1, 1] = False
    lu, nu = ndimage.label(upper, structure=FOUR if n == 4 else EIGHT)
    ll, nl = ndimage.label(lower, structure=FOUR if nbar == 4 else EIGHT)
    return len(_counted(lu, nu, n)), len(_counted(ll, nl, nbar)), _counted(ll, nl, nbar)


def point_step(grid, lam, rule, adj=0):
    """(lambda_destructible, alpha) of the centre of a 3x3 grid, from the definitions."""
    g = np.asarray(grid, dtype=np.int64)
    c = int(g[1, 1])
    tplus, tminus, comps = local_numbers(g, adj)
    lower = [(r, cc) for r in range(3) for cc in range(3) if (r, cc) != (1, 1) and g[r, cc] < c]
    if not lower:
        return False, c
    alpha = max(int(g[p]) for p in lower)
    if tplus == 1 and tminus == 1:
        return True, alpha
    if tminus > 1:
        f = max if rule == 0 else min
        ok = sum(1 for comp in comps if c - f(int(g[p]) for p in comp) <= lam)
        if ok >= tminus - 1:
            return True, alpha
    return False, alpha


def skeleton_step(grid, lam, rule, adj=0):
    """(lowerable by the lambda-skeleton, alpha) of the centre of a 3x3 grid,
    from the definitions of Sec. 2.1: lambda-deletable (lambda-destructible, or
    a peak point -- no neighbour in F_k, k = F(x) -- with F(x) - alpha <= lam)
    and not lambda-end (an end point -- exactly one neighbour in F_k -- with
    F(x) - alpha > lam)."""
    g = np.asarray(grid, dtype=np.int64)
    c = int(g[1, 1])
    near = FOUR_NEIGHBOURS_RC if adj else {rc for rc in RING_RC}  # Gamma_n^*(x)
    in_section = [int(v) >= c for (r, cc), v in np.ndenumerate(g) if (r, cc) in near]
    lower = [int(v) for (r, cc), v in np.ndenumerate(g) if (r, cc) != (1, 1) and v < c]
    if not lower:
        return False, c
    alpha = max(lower)
    tplus = local_numbers(g, adj)[0]
    deletable = point_step(g, lam, rule, adj)[0] or (tplus == 0 and c - alpha <= lam)
    lambda_end = sum(in_section) == 1 and c - alpha > lam
    return deletable and not lambda_end, alpha


def components(mask, structure):
    return ndimage.label(mask, structure=structure)[1]


def global_destructible(img, x, y, adj=0):
    """Removing (x, y) from F_k, k = F(x, y), keeps #n-components of F_k and
    #nbar-components of its complement (scipy labelling on the finite grid)."""
    a = np.asarray(img, dtype=np.int64)
    k = a[y, x]
    X = a >= k
    Xm = X.copy()
    Xm[y, x] = False
    sn, snbar = (FOUR, EIGHT) if adj else (EIGHT, FOUR)
    return (components(X, sn) == components(Xm, sn) and
            components(~X, snbar) == components(~Xm, snbar))


def schedule(img, lam, rule=0, use_global=False, max_rounds=10000, op=0, adj=0):
    """Subfield-schedule thinning in plain Python: phases 0,1,2,3,... visit the
    interior points of parity 2(y&1)+(x&1); each is lowered to alpha^- while it
    is lambda-destructible (op 0) or lambda-deletable and not lambda-end (op 1)
    (use_global: destructible by global component counts, lambda = 0 only;
    with op 1 an end point -- one neighbour in F_k -- is then kept).  Stops
    after a round with no change."""
    a = np.asarray(img, dtype=np.int64).copy()
    h, w = a.shape
    for _ in range(max_rounds):
        changed = False
        for p in range(4):
            for y in range(1, h - 1):
                for x in range(1, w - 1):
                    if 2 * (y & 1) + (x & 1) != p:
                        continue
                    while True:
                        g = a[y - 1:y + 2, x - 1:x + 2]
                        if use_global:
                            lower = [int(v) for (r, c), v in np.ndenumerate(g) if (r, c) != (1, 1) and v < g[1, 1]]
                            ok = bool(lower) and global_destructible(a, x, y, adj)
                            if op == 1:
                                near = FOUR_NEIGHBOURS_RC if adj else set(RING_RC)
                                ok = ok and sum(int(g[rc] >= g[1, 1]) for rc in near) != 1
                            alpha = max(lower) if lower else int(g[1, 1])
                        elif op == 1:
                            ok, alpha = skeleton_step(g, lam, rule, adj)
                        else:
                            ok, alpha = point_step(g, lam, rule, adj)
                        if not ok:
                            break
                        a[y, x] = alpha
                        changed = True
        if not changed:
            return a
    raise RuntimeError("no convergence")
