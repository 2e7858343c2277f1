"""The bound behind the remeshing stencils, checked on the CPU by brute force.

The remeshing (this library's form of Sec. 12's local interpolation) finds
the data of grid point g_k, the particles with scaled gnomonic radius
s < 2.2, through the cells of the particles' nearest grid points.  Its stencil
is the triangulation rings about g_k up to the first ring whose successor
lies at least twice the data-disc chord away, less every cell c with
|g_c - g_k| > chord + rho_c, rho_c being the largest chord from g_c to a vertex
of its Voronoi cell (a circumcentre of a triangle at c).  This test restates
that rule in numpy and checks, for particles moved by seeded random tangent
steps of up to one local spacing, that every datum of every grid point lies in
a kept cell, and that the pruning keeps well under half of the ring cells.
"""
import numpy as np
import pytest

from paper_2508_13550_gb300 import inputs as I

SC = 2.2


def _grid(kind, level):
    v, f = I.icosahedral_triangulation(level)
    x = v if kind == "icosahedral" else I.schmidt_transform(v, 0.5)
    off, nb = I.grid_adjacency(f, len(x))
    return x, [set(nb[off[k]:off[k + 1]].tolist()) for k in range(len(x))]


def _voronoi_radius(x, adj):
    rho = np.zeros(len(x))
    for c in range(len(x)):
        best = 0.0
        for a in adj[c]:
            for b in adj[a]:
                if b <= a or b not in adj[c]:
                    continue
                q = np.cross(x[a] - x[c], x[b] - x[c])
                q /= np.linalg.norm(q)
                if q @ x[c] < 0:
                    q = -q
                best = max(best, np.linalg.norm(q - x[c]))
        rho[c] = best
    return rho


def _chord(hk):
    return 2.0 * np.sin(0.5 * np.arctan(SC * hk)) * (1.0 + 1e-9)


def _stencil(k, x, adj, h, rho):
    need = 2.0 * _chord(h[k])
    S, seen, lo = [k], {k}, 0
    for _ in range(9):
        hi, dmin = len(S), np.inf
        for i in range(lo, hi):
            for w in adj[S[i]]:
                if w not in seen:
                    seen.add(w)
                    S.append(w)
                    dmin = min(dmin, np.linalg.norm(x[w] - x[k]))
        if dmin >= need:
            rings = S[:hi]
            kept = [c for c in rings
                    if np.linalg.norm(x[c] - x[k]) <= _chord(h[k]) + rho[c] * (1 + 1e-9)]
            return rings, kept
        lo = hi
    raise AssertionError("no ring holds the data disc")


@pytest.mark.parametrize("kind", ["icosahedral", "variable"])
def test_pruned_stencils_hold_every_datum(kind):
    from scipy.spatial import cKDTree
    x, adj = _grid(kind, 3)
    M = len(x)
    h = np.array([min(np.linalg.norm(x[j] - x[k]) for j in adj[k]) for k in range(M)])
    rho = _voronoi_radius(x, adj)
    # a Voronoi vertex of a near-regular grid sits about h/sqrt(3) from its point
    assert 0.5 < np.median(rho / h) < 0.75
    rng = np.random.default_rng(I.MASTER_SEED + 72)
    d = rng.normal(size=x.shape)
    d -= (d * x).sum(1, keepdims=True) * x
    d *= (h * rng.uniform(size=M) / np.linalg.norm(d, axis=1))[:, None]
    p = x + d
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    cell = cKDTree(x).query(p)[1]
    # the bound itself: a particle is within rho of its nearest grid point
    assert np.all(np.linalg.norm(p - x[cell], axis=1) <= rho[cell] * (1 + 1e-12))
    n_rings = n_kept = n_data = 0
    for k in range(M):
        rings, kept = _stencil(k, x, adj, h, rho)
        g = x[k]
        e1 = np.cross([0.0, 0.0, 1.0], g) if abs(g[2]) < 0.9 else np.cross([1.0, 0.0, 0.0], g)
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(g, e1)
        dot = p @ g
        with np.errstate(divide="ignore", invalid="ignore"):
            u, v = (p @ e1) / (dot * h[k]), (p @ e2) / (dot * h[k])
        data = np.nonzero((dot > 0) & (u * u + v * v < SC * SC))[0]
        assert len(data) >= 6
        assert set(cell[data].tolist()) <= set(kept), f"grid point {k}: a datum outside"
        n_rings += len(rings)
        n_kept += len(kept)
        n_data += len(data)
    print(f"\n{kind} level 3: ring cells {n_rings / M:.1f}, kept {n_kept / M:.1f}, "
          f"data {n_data / M:.1f} per grid point")
    assert n_kept < 0.45 * n_rings
