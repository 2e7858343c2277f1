"""Seeded synthetic inputs for the cubed-sphere FMM workloads.

This module only generates data: quadrature points on the unit sphere, cell
areas, data fields f and the weights w_j = f(x_j) A_j of the midpoint rule
(Sec. 1, Eq. (nbodysum)).  It contains none of the fast-summation method's
arithmetic (no tree, no interpolation, no kernel sums) and is the one module
that both the CUDA path's tests/benchmark and the CPU oracle draw inputs from.

Point sets: the equiangular gnomonic cubed-sphere grid of Sec. 3 (cell centres
are the images of uniform (xi, eta) grid points; Table "grids" lists
N = 6 m^2 for m = 2^L), and the icosahedral and latitude-longitude grids of
the same table.  Cell areas are exact: geodesic areas of the gnomonic cells,
of the spherical Voronoi cells of the icosahedral vertices, and of the
latitude-longitude bands.  Data fields: real spherical harmonics Y_{n,m} (Sec. 2.1),
the Rossby-Haurwitz wave-4 vorticity (Sec. 12, Eq. RH_initial), a land-masked
random field, and random spherical-harmonic combinations.

All randomness uses numpy's PCG64 generator with an explicit seed.
"""
from __future__ import annotations

import math

import numpy as np

MASTER_SEED = 2508135

# Face frames used only to lay out the input grid: (normal, e1, e2).  The
# order and orientation of the input points are arbitrary; the library sorts
# them itself.
_FACE_FRAMES = (
    ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)),
    ((0.0, 1.0, 0.0), (-1.0, 0.0, 0.0), (0.0, 0.0, 1.0)),
    ((-1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (0.0, 0.0, 1.0)),
    ((0.0, -1.0, 0.0), (1.0, 0.0, 0.0), (0.0, 0.0, 1.0)),
    ((0.0, 0.0, 1.0), (0.0, 1.0, 0.0), (-1.0, 0.0, 0.0)),
    ((0.0, 0.0, -1.0), (0.0, 1.0, 0.0), (1.0, 0.0, 0.0)),
)


def _gnomonic_cell_area(a1, a2, b1, b2):
    """Exact area of the spherical quadrilateral whose gnomonic face-plane
    image is [a1,a2] x [b1,b2] (a, b = tangents of the face angles)."""

    def F(a, b):
        return np.arctan(a * b / np.sqrt(1.0 + a * a + b * b))

    return F(a2, b2) - F(a1, b2) - F(a2, b1) + F(a1, b1)


def cubed_sphere_grid(m: int, shuffle_seed: int | None = None):
    """Equiangular gnomonic cubed-sphere grid with m x m cells per face.

    Returns (points [N,3] float64 unit vectors, areas [N] float64), N = 6 m^2.
    Cell centres sit at the equiangular midpoints
    xi_i = -pi/4 + (i + 1/2) (pi/2)/m.  If ``shuffle_seed`` is given the
    points are returned in a seeded random order.
    """
    if m < 1:
        raise ValueError("m must be >= 1")
    h = (math.pi / 2) / m
    edges = np.tan(-math.pi / 4 + h * np.arange(m + 1))
    mids = np.tan(-math.pi / 4 + h * (np.arange(m) + 0.5))
    A, B = np.meshgrid(mids, mids, indexing="ij")
    area2d = _gnomonic_cell_area(edges[:-1, None], edges[1:, None],
                                 edges[None, :-1], edges[None, 1:])
    pts = []
    areas = []
    for nrm, e1, e2 in _FACE_FRAMES:
        nrm, e1, e2 = (np.asarray(v) for v in (nrm, e1, e2))
        v = nrm[None, None, :] + A[..., None] * e1 + B[..., None] * e2
        v = v / np.linalg.norm(v, axis=-1, keepdims=True)
        pts.append(v.reshape(-1, 3))
        areas.append(area2d.reshape(-1))
    pts = np.ascontiguousarray(np.concatenate(pts))
    areas = np.ascontiguousarray(np.concatenate(areas))
    if shuffle_seed is not None:
        perm = np.random.default_rng(shuffle_seed).permutation(len(pts))
        pts = np.ascontiguousarray(pts[perm])
        areas = np.ascontiguousarray(areas[perm])
    return pts, areas


def _spherical_triangle_area(a, b, c):
    """Signed area of the spherical triangles (a, b, c) of unit vectors
    ([..., 3] arrays), by tan(E/2) = a.(b x c) / (1 + a.b + b.c + c.a)
    (Van Oosterom and Strackee, 1983); positive for counter-clockwise
    triangles seen from outside the sphere."""
    num = np.einsum("...i,...i->...", a, np.cross(b, c))
    den = 1.0 + np.einsum("...i,...i->...", a, b) + np.einsum("...i,...i->...", b, c) \
        + np.einsum("...i,...i->...", c, a)
    return 2.0 * np.arctan2(num, den)


def icosahedral_triangulation(level: int):
    """Vertices and faces of the icosahedron refined `level` times (each
    triangle split into four through its edge midpoints, new vertices
    projected to the sphere): N = 10 * 4^level + 2 vertices (Table "grids":
    2562 at level 4)."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(x, dtype=np.float64) / np.linalg.norm(x) for x in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        mid = {}

        def midpoint(i, j):
            key = (i, j) if i < j else (j, i)
            if key not in mid:
                x = verts[i] + verts[j]
                verts.append(x / np.linalg.norm(x))
                mid[key] = len(verts) - 1
            return mid[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts), np.array(faces, dtype=np.int64)


def grid_adjacency(faces, N: int):
    """Neighbour lists of a triangulated grid in CSR form: (offsets [N+1],
    neighbours int64), the vertices joined to each vertex by a triangle edge,
    ascending within each row."""
    f = np.asarray(faces, dtype=np.int64)
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    e = np.concatenate([e, e[:, ::-1]])
    e = np.unique(e, axis=0)
    offsets = np.zeros(N + 1, dtype=np.int64)
    np.add.at(offsets, e[:, 0] + 1, 1)
    return np.cumsum(offsets), np.ascontiguousarray(e[:, 1])


def icosahedral_grid(level: int):
    """Icosahedral grid of Table "grids": the cell centres are the vertices of
    the refined icosahedral triangulation and the cells are their spherical
    Voronoi (hexagonal, and 12 pentagonal) cells.  Returns (points [N, 3],
    exact cell areas [N]).  Each triangle (a, b, c) with circumcentre q adds
    to the cell of each vertex the quadrilateral (vertex, midpoint of one
    incident edge, q, midpoint of the other), bounded by the perpendicular
    bisectors through those midpoints; signed areas keep the sum exact."""
    verts, faces = icosahedral_triangulation(level)
    return verts, _dual_cell_areas(verts, faces)


def _dual_cell_areas(verts, faces):
    """Areas of the circumcentric dual cells of a spherical triangulation (the
    Voronoi cells of a Delaunay one): each triangle adds to the cell of each
    of its vertices the quadrilateral (vertex, midpoint of one incident edge,
    circumcentre, midpoint of the other), with signed areas."""
    a, b, c = verts[faces[:, 0]], verts[faces[:, 1]], verts[faces[:, 2]]
    q = np.cross(b - a, c - a)
    q /= np.linalg.norm(q, axis=1)[:, None]
    q *= np.sign(np.einsum("ij,ij->i", q, a + b + c))[:, None]

    def mid(x, y):
        m = x + y
        return m / np.linalg.norm(m, axis=1)[:, None]

    mab, mbc, mca = mid(a, b), mid(b, c), mid(c, a)
    areas = np.zeros(len(verts))
    T = _spherical_triangle_area
    np.add.at(areas, faces[:, 0], T(a, mab, q) + T(a, q, mca))
    np.add.at(areas, faces[:, 1], T(b, mbc, q) + T(b, q, mab))
    np.add.at(areas, faces[:, 2], T(c, mca, q) + T(c, q, mbc))
    return np.abs(areas)


def schmidt_transform(pts, stretch: float):
    """Schmidt's conformal map of the sphere, tan(theta'/2) = stretch tan(theta/2)
    with theta the co-latitude and the longitude kept: for stretch < 1 it
    draws points toward the north pole, refining the spacing there by 1/stretch
    and coarsening it at the south pole by stretch."""
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    r = np.hypot(x, y)
    south = 1.0 + z <= 1e-15
    t = np.where(south, np.inf, stretch * r / np.where(south, 1.0, 1.0 + z))  # tan(theta'/2)
    with np.errstate(invalid="ignore", divide="ignore"):
        zt = np.where(south, -1.0, (1.0 - t * t) / (1.0 + t * t))
        st = np.where(south, 0.0, 2.0 * t / (1.0 + t * t))
        ux = np.where(r > 0, x / np.where(r > 0, r, 1.0), 1.0)
        uy = np.where(r > 0, y / np.where(r > 0, r, 1.0), 0.0)
    out = np.stack([st * ux, st * uy, zt], axis=1)
    return out / np.linalg.norm(out, axis=1, keepdims=True)


def variable_resolution_grid(level: int, stretch: float = 0.5):
    """A variable-resolution grid in the manner of MPAS meshes (which the
    paper uses for SAL and are not available here): the icosahedral grid of
    the given level mapped by schmidt_transform(stretch), its cells the dual
    cells of the mapped triangulation.  With stretch 0.5 the spacing grows
    smoothly 4x from the north pole to the south pole.  Returns (points [N, 3],
    cell areas [N]) summing to 4 pi."""
    verts, faces = icosahedral_triangulation(level)
    pts = schmidt_transform(verts, stretch)
    return pts, _dual_cell_areas(pts, faces)


def latlon_grid(level: int):
    """Latitude-longitude grid of Table "grids": spacing 4 / 2^(level-4)
    degrees, 45 * 2^(level-4) latitude bands by 90 * 2^(level-4) longitudes;
    the cell centre is at the mean latitude and mean longitude of the cell
    edges.  Returns (points [N, 3], exact cell areas dlambda (sin phi2 -
    sin phi1) [N])."""
    nlat = 45 * 2 ** (level - 4)
    nlon = 2 * nlat
    phi = np.linspace(-0.5 * math.pi, 0.5 * math.pi, nlat + 1)
    lam = np.linspace(0.0, 2.0 * math.pi, nlon + 1)
    pc = 0.5 * (phi[:-1] + phi[1:])
    lc = 0.5 * (lam[:-1] + lam[1:])
    P, L = np.meshgrid(pc, lc, indexing="ij")
    pts = np.stack([np.cos(P) * np.cos(L), np.cos(P) * np.sin(L), np.sin(P)], axis=-1)
    band = (np.sin(phi[1:]) - np.sin(phi[:-1])) * (2.0 * math.pi / nlon)
    areas = np.repeat(band, nlon)
    return pts.reshape(-1, 3), areas


def random_sphere_points(N: int, seed: int):
    """N points drawn uniformly on the unit sphere (normalised Gaussians)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((N, 3))
    return np.ascontiguousarray(v / np.linalg.norm(v, axis=1, keepdims=True))


def random_rotation(seed: int):
    """A seeded random proper rotation matrix (QR of a Gaussian matrix)."""
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


# ----------------------------------------------------------------------------
# Real spherical harmonics, orthonormal on the unit sphere (Sec. 2.1):
#   Y_{n,0} = Pbar_n^0(z),  Y_{n,m} = sqrt(2) Pbar_n^m(z) cos(m lam)  (m > 0),
#   Y_{n,-m} = sqrt(2) Pbar_n^m(z) sin(m lam),
# with Pbar the associated Legendre functions normalised so that
# Pbar_n^m(cos th) e^{i m lam} has unit L2 norm on the sphere.
# ----------------------------------------------------------------------------

def _legendre_column(mm: int, nmax: int, z, s):
    """Pbar_n^mm(z) for n = mm..nmax (rows), using the standard three-term
    recurrence in n; s = sqrt(1 - z^2)."""
    out = np.empty((nmax - mm + 1,) + z.shape)
    p = np.full(z.shape, 1.0 / math.sqrt(4 * math.pi))
    for k in range(1, mm + 1):
        p = p * math.sqrt((2 * k + 1) / (2 * k)) * s
    out[0] = p
    if nmax == mm:
        return out
    out[1] = math.sqrt(2 * mm + 3) * z * p
    for n in range(mm + 2, nmax + 1):
        a = math.sqrt((4 * n * n - 1) / (n * n - mm * mm))
        b = math.sqrt(((n - 1) ** 2 - mm * mm) / (4 * (n - 1) ** 2 - 1))
        out[n - mm] = a * (z * out[n - mm - 1] - b * out[n - mm - 2])
    return out


def real_sph_harm(n: int, m: int, pts):
    """Orthonormal real spherical harmonic Y_{n,m} at unit vectors ``pts``."""
    if abs(m) > n or n < 0:
        raise ValueError("need |m| <= n")
    pts = np.asarray(pts, dtype=np.float64)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    lam = np.arctan2(y, x)
    p = _legendre_column(abs(m), n, z, s)[n - abs(m)]
    if m == 0:
        return p
    if m > 0:
        return math.sqrt(2.0) * p * np.cos(m * lam)
    return math.sqrt(2.0) * p * np.sin(-m * lam)


def sph_harm_combination(pts, coeffs: dict, nrhs: int | None = None,
                         chunk: int = 1 << 18):
    """Sum_{(n,m)} c[n,m] Y_{n,m}(pts).

    ``coeffs`` maps (n, m) -> scalar, or -> array of shape [nrhs] to build
    several fields at once (returned as [nrhs, N]).
    """
    pts = np.asarray(pts, dtype=np.float64)
    N = len(pts)
    multi = nrhs is not None
    out = np.zeros((nrhs, N) if multi else (N,))
    if not coeffs:
        return out
    nmax = max(n for n, _ in coeffs)
    by_m: dict[int, list] = {}
    for (n, m), c in coeffs.items():
        by_m.setdefault(abs(m), []).append((n, m, c))
    for lo in range(0, N, chunk):
        hi = min(N, lo + chunk)
        x, y, z = pts[lo:hi, 0], pts[lo:hi, 1], pts[lo:hi, 2]
        s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
        lam = np.arctan2(y, x)
        for am, items in by_m.items():
            col = _legendre_column(am, nmax, z, s)
            cos_ml = np.cos(am * lam)
            sin_ml = np.sin(am * lam)
            for n, m, c in items:
                p = col[n - am]
                if m == 0:
                    f = p
                elif m > 0:
                    f = math.sqrt(2.0) * p * cos_ml
                else:
                    f = math.sqrt(2.0) * p * sin_ml
                if multi:
                    out[:, lo:hi] += np.asarray(c)[:, None] * f[None, :]
                else:
                    out[lo:hi] += c * f
    return out


def random_sh_coeffs(nmax: int, nrhs: int, seed: int, nmin: int = 1):
    """Coefficients c_{n,m} ~ N(0, 1/n^2) for nmin <= n <= nmax, all m,
    for ``nrhs`` independent fields (n = 0 is excluded so Poisson data stays
    mean-free)."""
    rng = np.random.default_rng(seed)
    coeffs = {}
    for n in range(nmin, nmax + 1):
        for m in range(-n, n + 1):
            coeffs[(n, m)] = rng.standard_normal(nrhs) / max(n, 1)
    return coeffs


# ----------------------------------------------------------------------------
# Fields of the workloads
# ----------------------------------------------------------------------------

def rossby_haurwitz_vorticity(pts):
    """RH wave-4 initial vorticity (Sec. 12, Eq. RH_initial) with theta the
    latitude: zeta = (2 pi/7) sin(lat) + 30 sin(lat) cos^4(lat) cos(4 lam).
    On the unit sphere sin(lat) = z and cos^4(lat) cos(4 lam) = Re((x+iy)^4)."""
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    re4 = x ** 4 - 6 * x * x * y * y + y ** 4
    return (2 * math.pi / 7) * z + 30.0 * z * re4


def rossby_haurwitz_streamfunction(pts):
    """psi = int G_L zeta dS for the RH wave in closed form (-Lap psi = zeta):
    the solid-body part is degree 1 (eigenvalue 1/2) and the wave part
    degree 5 (eigenvalue 1/30), so psi = (pi/7) z + z Re((x+iy)^4)."""
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    re4 = x ** 4 - 6 * x * x * y * y + y ** 4
    return (math.pi / 7) * z + z * re4


def rossby_haurwitz_velocity(pts):
    """u = grad_S psi x x with psi = int G_L zeta (Sec. 2.3: the Biot-Savart
    kernel is grad_x G_L x x, so int K_BS zeta = grad psi x x).  The ambient gradient of the
    polynomial extension is projected onto the tangent plane."""
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    re4 = x ** 4 - 6 * x * x * y * y + y ** 4
    gx = z * (4 * x ** 3 - 12 * x * y * y)
    gy = z * (4 * y ** 3 - 12 * x * x * y)
    gz = (math.pi / 7) + re4
    g = np.stack([gx, gy, gz], axis=1)
    g = g - np.sum(g * pts, axis=1, keepdims=True) * pts
    return np.cross(g, pts)


def gaussian_vortex_vorticity(pts):
    """Gaussian vortex initial vorticity (Sec. 12, Eq. Gaussian_ic): a core
    4 pi exp(-16 |x - x_c|^2) at latitude pi/20, longitude 0, on the
    constant background -0.196353 printed with it (zero total vorticity)."""
    lat = math.pi / 20
    xc = np.array([math.cos(lat), 0.0, math.sin(lat)])
    d2 = np.sum((pts - xc) ** 2, axis=1)
    return 4 * math.pi * np.exp(-16.0 * d2) - 0.196353


def land_mask_field(pts, seed: int, land_fraction: float = 0.7,
                    nmax: int = 8):
    """Seeded 'land' field: U[0,1] values on the cells where a smooth random
    spherical-harmonic field (degree <= nmax) exceeds its
    (1 - land_fraction) quantile, 0 elsewhere."""
    rng = np.random.default_rng(seed)
    coeffs = {}
    for n in range(0, nmax + 1):
        for m in range(-n, n + 1):
            coeffs[(n, m)] = float(rng.standard_normal())
    s = sph_harm_combination(pts, coeffs)
    q = np.quantile(s, 1.0 - land_fraction)
    vals = rng.uniform(0.0, 1.0, size=len(pts))
    return np.where(s > q, vals, 0.0)


# ----------------------------------------------------------------------------
# The five workloads (points, weights and, where one exists, the closed form)
# ----------------------------------------------------------------------------

KERNEL_LAPLACE = 0
KERNEL_BIOT_SAVART = 1
KERNEL_NEWTON = 2
KERNEL_ONE = 100


def workload_poisson_y43(m: int = 32):
    """Poisson kernel, f = Y_{4,3}: returns (pts, areas, w[1,N], exact[1,N]).

    By the Funk-Hecke formula, int G_L(x,y) Y_{n,m}(y) dS(y) =
    Y_{n,m}(x)/(n(n+1)) for n >= 1 (G_L is the Green's function of -Lap,
    Sec. 2.1; Eq. (G_L_1) prints this relation with the opposite sign, while
    the n = 0 relation Eq. (G_L_2) agrees with the positive one).  So the
    kernel sum approximates exact = Y_{4,3}/20."""
    pts, areas = cubed_sphere_grid(m)
    f = real_sph_harm(4, 3, pts)
    w = (f * areas)[None, :]
    exact = (f / 20.0)[None, :]
    return pts, areas, np.ascontiguousarray(w), exact


def workload_rh_biot_savart(m: int = 256, noise: float = 1e-3,
                            seed: int = MASTER_SEED + 2):
    """Biot-Savart kernel, RH wave-4 vorticity plus seeded Gaussian noise of
    standard deviation noise * rms(zeta) per cell; returns
    (pts, areas, w[1,N], exact velocity of the noise-free field [1,N,3])."""
    pts, areas = cubed_sphere_grid(m)
    zeta = rossby_haurwitz_vorticity(pts)
    rng = np.random.default_rng(seed)
    rms = math.sqrt(float(np.mean(zeta * zeta)))
    zeta_n = zeta + noise * rms * rng.standard_normal(len(pts))
    w = (zeta_n * areas)[None, :]
    return pts, areas, np.ascontiguousarray(w), rossby_haurwitz_velocity(pts)[None]


BVE_OMEGA = 2 * math.pi  # rotation rate of the BVE runs, 2 pi per day (Sec. 12)
BVE_DT = 0.01            # RK4 time step of the BVE runs, in days (Sec. 12)


def workload_bve(level: int = 7, field: str = "rh", with_adjacency: bool = False):
    """Vortex-method particles for the barotropic vorticity equation (Sec. 12):
    icosahedral cell centres and areas of the given refinement level
    (N = 10 4^level + 2) with the RH wave-4 ("rh", Eq. RH_initial) or the
    Gaussian vortex ("gaussian", Eq. Gaussian_ic) vorticity; returns
    (x [N,3], zeta [N], area [N]), plus the grid's neighbour lists
    (offsets, neighbours) with with_adjacency."""
    pts, areas = icosahedral_grid(level)
    if field == "rh":
        zeta = rossby_haurwitz_vorticity(pts)
    elif field == "gaussian":
        zeta = gaussian_vortex_vorticity(pts)
    else:
        raise ValueError(f"unknown BVE field {field!r}")
    if with_adjacency:
        off, nb = grid_adjacency(icosahedral_triangulation(level)[1], len(pts))
        return pts, np.ascontiguousarray(zeta), areas, off, nb
    return pts, np.ascontiguousarray(zeta), areas


def workload_newton_land(m: int = 1024, seed: int = MASTER_SEED + 3):
    """Newtonian kernel, land-masked U[0,1] field; returns (pts, areas, w[1,N])."""
    pts, areas = cubed_sphere_grid(m)
    f = land_mask_field(pts, seed)
    return pts, areas, np.ascontiguousarray((f * areas)[None, :])


def workload_multi_rhs(m: int = 512, nrhs: int = 16, nmax: int = 32,
                       seed: int = MASTER_SEED + 4, with_exact: bool = True):
    """Poisson kernel, nrhs random spherical-harmonic combinations
    (n = 1..nmax, c ~ N(0, 1/n^2)); returns (pts, areas, w[nrhs,N],
    exact[nrhs,N] or None) with exact = sum c Y/(n(n+1)) (Funk-Hecke, see
    workload_poisson_y43)."""
    pts, areas = cubed_sphere_grid(m)
    coeffs = random_sh_coeffs(nmax, nrhs, seed)
    f = sph_harm_combination(pts, coeffs, nrhs=nrhs)
    w = np.ascontiguousarray(f * areas[None, :])
    exact = None
    if with_exact:
        ce = {k: np.asarray(v) / (k[0] * (k[0] + 1)) for k, v in coeffs.items()}
        exact = sph_harm_combination(pts, ce, nrhs=nrhs)
    return pts, areas, w, exact


def serving_requests(n_requests: int = 2000, rate_hz: float = 50.0,
                     seed: int = MASTER_SEED + 5,
                     ms=(64, 128, 256, 512, 1024),
                     kernels=(KERNEL_LAPLACE, KERNEL_BIOT_SAVART, KERNEL_NEWTON),
                     nrhs_range=(1, 8), degree_range=(8, 12)):
    """Seeded request stream: Poisson arrivals at ``rate_hz``; each request a
    cubed-sphere grid size m, a kernel, an RHS count and a degree drawn
    uniformly.  Returns a list of dicts sorted by arrival time (seconds)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests))
    reqs = []
    for i in range(n_requests):
        reqs.append(dict(
            id=i, arrival=float(t[i]),
            m=int(rng.choice(ms)),
            kernel=int(rng.choice(kernels)),
            nrhs=int(rng.integers(nrhs_range[0], nrhs_range[1] + 1)),
            degree=int(rng.integers(degree_range[0], degree_range[1] + 1)),
            seed=int(rng.integers(0, 2 ** 31 - 1)),
        ))
    return reqs
