"""Seeded synthetic inputs: fault meshes, right-hand sides and interface stiffness draws.

This module is the only code shared by the CUDA path, the CPU oracle, the tests and
the benchmark.  It lays out planar grids of rectangular constant-displacement-
discontinuity elements and draws seeded random numbers; it holds none of the method's
arithmetic (no influence coefficients, no tree, no compression, no solver).

Element description (one row per element, user order):
  c   (N,3) centroid (collocation point, Sec. 3.1)
  s1  (N,3), s2 (N,3), n (N,3)  local orthonormal frame (Sec. 2.2; the DOF order of
      every element is (s1, s2, n), Sec. 3.1)
  a   (N,)  half side along s1,  b (N,) half side along s2 (rectangles)
  shape (N,) 0 for a rectangle, 1 for a triangle (Sec. 3.1: the paper's element)
  tri (N,9) the three vertices of a triangle (global), unused for rectangles; its
      collocation point c is the centroid and (s1, s2) any orthonormal pair in its plane

Local in-plane axes of a plane with unit normal n: s1 = normalize(e3 x n), falling back
to s1 = e1 when n is parallel to e3, and s2 = n x s1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Elements:
    c: np.ndarray
    s1: np.ndarray
    s2: np.ndarray
    n: np.ndarray
    a: np.ndarray
    b: np.ndarray
    # plane id of every element (which fault / fracture it belongs to)
    plane: np.ndarray
    shape: np.ndarray = None
    tri: np.ndarray = None

    def __post_init__(self):
        if self.shape is None:
            self.shape = np.zeros(self.c.shape[0], dtype=np.int32)
        if self.tri is None:
            self.tri = np.zeros((self.c.shape[0], 9))

    @property
    def N(self) -> int:
        return int(self.c.shape[0])

    def subset(self, idx) -> "Elements":
        idx = np.asarray(idx)
        return Elements(*(np.ascontiguousarray(getattr(self, f.name)[idx])
                          for f in dataclasses.fields(self)))

    @staticmethod
    def concat(parts) -> "Elements":
        return Elements(*(np.ascontiguousarray(np.concatenate([getattr(p, f.name) for p in parts]))
                          for f in dataclasses.fields(Elements)))


def plane_axes(n):
    """Local in-plane axes (s1, s2) of a plane with unit normal n."""
    n = np.asarray(n, dtype=np.float64)
    n = n / np.linalg.norm(n)
    s1 = np.cross([0.0, 0.0, 1.0], n)
    if np.linalg.norm(s1) < 1e-12:
        s1 = np.array([1.0, 0.0, 0.0])
    s1 = s1 / np.linalg.norm(s1)
    s2 = np.cross(n, s1)
    return s1, s2, n


def plane_grid(n_cells1, n_cells2, lo1, hi1, lo2, hi2, normal, origin=(0.0, 0.0, 0.0),
               keep=None, plane_id=0) -> Elements:
    """Uniform grid of rectangles on a plane: cell centres at lo + (i + 1/2) h in the
    local (s1, s2) coordinates, mapped to 3D as origin + x1 s1 + x2 s2.
    `keep(x1, x2)` optionally selects cells by their local centre coordinates."""
    s1, s2, n = plane_axes(normal)
    h1 = (hi1 - lo1) / n_cells1
    h2 = (hi2 - lo2) / n_cells2
    x1 = lo1 + (np.arange(n_cells1) + 0.5) * h1
    x2 = lo2 + (np.arange(n_cells2) + 0.5) * h2
    X1, X2 = np.meshgrid(x1, x2, indexing="xy")  # row-major over (x2, x1)
    X1 = X1.ravel()
    X2 = X2.ravel()
    if keep is not None:
        m = keep(X1, X2)
        X1 = X1[m]
        X2 = X2[m]
    N = X1.size
    o = np.asarray(origin, dtype=np.float64)
    c = o[None, :] + X1[:, None] * s1[None, :] + X2[:, None] * s2[None, :]
    rep = lambda v: np.ascontiguousarray(np.broadcast_to(v, (N, 3)))
    return Elements(c=np.ascontiguousarray(c), s1=rep(s1), s2=rep(s2), n=rep(n),
                    a=np.full(N, 0.5 * h1), b=np.full(N, 0.5 * h2),
                    plane=np.full(N, plane_id, dtype=np.int32))


def triangles(V, normal, plane_id=0) -> Elements:
    """Triangle elements from their vertices V (T, 3, 3), all in the plane of the unit
    normal: centroid collocation points and the plane's (s1, s2, n) frame; a and b hold
    half the square root of the area (unused by the operator)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    s1, s2, n = plane_axes(normal)
    T = V.shape[0]
    c = V.mean(axis=1)
    area = 0.5 * np.linalg.norm(np.cross(V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]), axis=1)
    rep = lambda v: np.ascontiguousarray(np.broadcast_to(v, (T, 3)))
    half = 0.5 * np.sqrt(area)
    return Elements(c=np.ascontiguousarray(c), s1=rep(s1), s2=rep(s2), n=rep(n), a=half.copy(), b=half.copy(),
                    plane=np.full(T, plane_id, dtype=np.int32), shape=np.ones(T, dtype=np.int32),
                    tri=np.ascontiguousarray(V.reshape(T, 9)))


def tri_disk_mesh(n_grid, radius=1.0, normal=(0.0, 0.0, 1.0), origin=(0.0, 0.0, 0.0), jitter=0.2, seed=1620,
                  plane_id=0) -> Elements:
    """Triangulated disk: the vertices of an n_grid x n_grid lattice on [-R, R]^2, each
    moved by a seeded uniform offset of up to jitter h per coordinate (shared by the
    cells that meet there), every cell whose centre has r < R split into two triangles
    along alternating diagonals.  General triangles with conforming vertices, like the
    unstructured meshes of the paper's examples."""
    R = float(radius)
    h = 2.0 * R / n_grid
    s1, s2, n = plane_axes(normal)
    rng = np.random.Generator(np.random.PCG64(seed))
    g = -R + h * np.arange(n_grid + 1)
    P1, P2 = np.meshgrid(g, g, indexing="xy")
    P1 = P1 + rng.uniform(-jitter, jitter, P1.shape) * h
    P2 = P2 + rng.uniform(-jitter, jitter, P2.shape) * h
    o = np.asarray(origin, dtype=np.float64)
    X = o[None, None, :] + P1[..., None] * s1 + P2[..., None] * s2  # (n+1, n+1, 3), [row j, col i]
    tris = []
    for j in range(n_grid):
        for i in range(n_grid):
            xc, yc = -R + (i + 0.5) * h, -R + (j + 0.5) * h
            if xc * xc + yc * yc >= R * R:
                continue
            a, b, c_, d = X[j, i], X[j, i + 1], X[j + 1, i + 1], X[j + 1, i]
            if (i + j) % 2 == 0:
                tris += [(a, b, c_), (a, c_, d)]
            else:
                tris += [(a, b, d), (b, c_, d)]
    return triangles(np.array(tris), normal, plane_id)


def disk_mesh(n_grid, radius=1.0, normal=(0.0, 0.0, 1.0), origin=(0.0, 0.0, 0.0), plane_id=0):
    """n_grid x n_grid square grid on [-R, R]^2 keeping the cells whose centre has r < R."""
    R = float(radius)
    return plane_grid(n_grid, n_grid, -R, R, -R, R, normal, origin,
                      keep=lambda x1, x2: x1 * x1 + x2 * x2 < R * R, plane_id=plane_id)


# ---------------------------------------------------------------------------------------
# The five workloads.  Sizes and recipes follow the hot-path configurations: a single
# penny crack (dense check against Sneddon), a single H-matrix fault, three intersecting
# fractures, 64 uneven independent faults, and a height-confined crack across a fault.
# ---------------------------------------------------------------------------------------

def config_penny(n_grid=40):
    """Planar crack z = 0: n x n grid on [-1,1]^2, centroids with r < 1 (n=40: N=1264)."""
    return disk_mesh(n_grid)


def config_fault(n_grid=256):
    """Single disk fault r < 1 on a 256 x 256 grid (N = 51,468)."""
    return disk_mesh(n_grid)


def config_three_planes(n_grid=300, shift_third=True):
    """Three square fractures of side 2 through the origin with normals e3, e1 and
    (1,1,0)/sqrt(2), each on an n x n grid.  The third grid is shifted by h/4 along its
    s2 axis so that no collocation point of the first plane lies on one of its edges."""
    h = 2.0 / n_grid
    p1 = plane_grid(n_grid, n_grid, -1, 1, -1, 1, (0, 0, 1), plane_id=0)
    p2 = plane_grid(n_grid, n_grid, -1, 1, -1, 1, (1, 0, 0), plane_id=1)
    off = 0.25 * h if shift_third else 0.0
    p3 = plane_grid(n_grid, n_grid, -1, 1, -1 + off, 1 + off,
                    (1 / math.sqrt(2), 1 / math.sqrt(2), 0), plane_id=2)
    return Elements.concat([p1, p2, p3])


def config_crack_fault(h=0.01, crack=(4.0, 1.0), fault=(4.0, 4.0)):
    """Height-confined vertical crack in the plane y = 0 (x in [-2,2], z in [-1/2,1/2],
    normal e2) crossing a vertical fault in the plane x = 0 (y, z in [-2,2], normal e1)."""
    Lx, Hz = crack
    Ly, Lz = fault
    nx, nz = int(round(Lx / h)), int(round(Hz / h))
    ny, nz2 = int(round(Ly / h)), int(round(Lz / h))
    # crack: its local axes are s1 = e3 x e2 = -e1, s2 = e3; lay the grid in x, z
    ck = plane_grid(nx, nz, -Lx / 2, Lx / 2, -Hz / 2, Hz / 2, (0, 1, 0), plane_id=0)
    ft = plane_grid(ny, nz2, -Ly / 2, Ly / 2, -Lz / 2, Lz / 2, (1, 0, 0), plane_id=1)
    return Elements.concat([ck, ft])


def config_faults_batch(n_faults=64, seed=1604, h=2.0 / 256, n_min=2000, n_max=40000):
    """64 independent disk faults: element counts log-uniform in [2k, 40k] at a fixed
    spacing h, radius R_f = h sqrt(N_f / pi), seeded uniform random normals and
    Poisson ratios nu_f ~ U[0.2, 0.3].  Returns (list of Elements, nu array)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    faults, nus = [], []
    for f in range(n_faults):
        nf = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        R = h * math.sqrt(nf / math.pi)
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        nus.append(rng.uniform(0.2, 0.3))
        ng = 2 * int(math.ceil(R / h))
        el = plane_grid(ng, ng, -ng * h / 2, ng * h / 2, -ng * h / 2, ng * h / 2, v,
                        keep=lambda x1, x2, R=R: x1 * x1 + x2 * x2 < R * R, plane_id=f)
        faults.append(el)
    return faults, np.array(nus)


# ------------------------------------------------------------------ right-hand sides

def rhs_uniform_pressure(el: Elements, p=1.0):
    """Uniform internal pressure p: traction b_n = -p, b_s = 0 (DOF order s1, s2, n)."""
    b = np.zeros((el.N, 3))
    b[:, 2] = -p
    return b.ravel()


def rhs_shear_plus_bump(el: Elements, sigma=0.2):
    """Uniform unit shear along s1 plus a Gaussian pressure bump of unit amplitude:
    b_s1 = 1, b_s2 = 0, b_n = -exp(-r^2 / (2 sigma^2)), r the distance to the origin."""
    r2 = np.sum(el.c * el.c, axis=1)
    b = np.zeros((el.N, 3))
    b[:, 0] = 1.0
    b[:, 2] = -np.exp(-r2 / (2.0 * sigma * sigma))
    return b.ravel()


def rhs_normal(n_dof, seed, nrhs=1):
    """Seeded N(0,1) tractions, shape (n_dof,) or (nrhs, n_dof)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.normal(size=(nrhs, n_dof))
    return x[0] if nrhs == 1 else x


def k_loguniform(N, seed, E=1.0, h=0.01, lo=1e-3, hi=1e2):
    """Interface stiffness per element, log-uniform in [lo, hi] * E / h."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=N)) * (E / h)


def random_vector(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(size=n)


def lp_initial_weights(hidden=32, seed=1607, n_features=8, n_out=3):
    """Seeded initial parameters of the learned correction's network, in the order
    W1 (H x F), b1, W2 (H x H), b2, W3 (3 x H), b3: hidden weights uniform in
    +-1/sqrt(fan-in), biases zero, output layer zero (the untrained correction is the
    identity)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H, F = hidden, n_features
    W1 = rng.uniform(-1.0, 1.0, size=(H, F)) / math.sqrt(F)
    W2 = rng.uniform(-1.0, 1.0, size=(H, H)) / math.sqrt(H)
    parts = [W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), np.zeros(n_out * H), np.zeros(n_out)]
    return np.concatenate(parts)


# Interface material sets (Sec. 2.2 parameters in units of the traction scale and of the
# element size): an intact, softening joint; a pre-existing fault (no tensile strength or
# cohesion, w_c = 0); a brittle joint that reaches full damage within the states drawn
# below; a joint without softening.
INTERFACE_PARAMS = {
    "softening": dict(Ks=10.0, Kn=20.0, fp=0.6, fr=0.3, psip=0.1, dc=0.2, cp=0.1, sigp=0.5, wc=0.4, alphaR=0.5),
    "fault": dict(Ks=10.0, Kn=20.0, fp=0.6, fr=0.45, psip=0.05, dc=0.1, cp=0.0, sigp=0.0, wc=0.0, alphaR=0.0),
    "brittle": dict(Ks=10.0, Kn=20.0, fp=0.6, fr=0.3, psip=0.1, dc=0.2, cp=0.1, sigp=0.5, wc=0.03, alphaR=0.5),
    "perfect": dict(Ks=15.0, Kn=30.0, fp=0.6, fr=0.6, psip=0.1, dc=1e300, cp=0.2, sigp=1.0, wc=1e300,
                    alphaR=0.0),
}


def interface_states(n, seed, open_fraction=0.1):
    """Seeded states and increments of n interface points: effective traction T'^n (mostly
    compressive, some tensile), inelastic DD delta^p, (chi_s, chi_t, w_dil) consistent
    with it (each at least the magnitude it bounds) and a DD increment; a fraction of the
    points carries a normal inelastic opening beyond 0.05 (an open fracture), another an
    increment that is mostly opening.  Arrays
    (n, 3) FP64."""
    rng = np.random.default_rng(seed)
    T = np.empty((n, 3))
    T[:, :2] = rng.normal(size=(n, 2)) * 0.2
    T[:, 2] = -rng.uniform(-0.3, 1.5, size=n)
    dp = np.empty((n, 3))
    dp[:, :2] = rng.normal(size=(n, 2)) * 0.02
    dp[:, 2] = np.abs(rng.normal(size=n)) * 0.005
    op = rng.uniform(size=n) < open_fraction
    dp[op, 2] += rng.uniform(0.05, 0.2, size=int(op.sum()))
    T[op] *= rng.uniform(0.0, 0.2, size=(int(op.sum()), 1))
    chi = np.empty((n, 3))
    chi[:, 0] = np.hypot(dp[:, 0], dp[:, 1]) * rng.uniform(1.0, 1.5, size=n)
    chi[:, 1] = np.linalg.norm(dp, axis=1) * rng.uniform(1.0, 1.5, size=n)
    chi[:, 2] = np.abs(rng.normal(size=n)) * 0.002
    dd = np.empty((n, 3))
    dd[:, :2] = rng.normal(size=(n, 2)) * 0.08
    dd[:, 2] = rng.normal(size=n) * 0.025
    pull = rng.uniform(size=n) < 0.2                # mostly opening increments
    dd[pull, :2] *= 0.1
    dd[pull, 2] = rng.uniform(0.02, 0.08, size=int(pull.sum()))
    return T, dp, chi, dd


def node_connectivity(el: Elements, rel_tol=1e-9):
    """Vertex nodes of the elements: one node per distinct vertex position (positions
    closer than rel_tol times the largest half side are one node).  Returns conn (N, 4)
    int32 -- a rectangle's vertices in the order (-a, -b), (+a, -b), (+a, +b), (-a, +b)
    of its (s1, s2) frame, a triangle's three vertices in their given order and -1 --
    and the node count."""
    sg = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]], dtype=np.float64)
    V = (el.c[:, None, :] + sg[None, :, 0:1] * el.a[:, None, None] * el.s1[:, None, :]
         + sg[None, :, 1:2] * el.b[:, None, None] * el.s2[:, None, :])
    tri = np.asarray(el.shape) == 1
    V[tri, :3] = np.asarray(el.tri)[tri].reshape(-1, 3, 3)
    q = max(float(el.a.max()), float(el.b.max())) * rel_tol
    keep = np.ones((el.N, 4), dtype=bool)
    keep[tri, 3] = False
    keys = np.round(V[keep] / q).astype(np.int64)
    _, inv = np.unique(keys, axis=0, return_inverse=True)
    conn = np.full((el.N, 4), -1, dtype=np.int32)
    conn[keep] = inv.ravel()
    return np.ascontiguousarray(conn), int(inv.max()) + 1
