"""Seeded synthetic geometry generators.

These build the triangle meshes the operators are evaluated on: closed
icospheres, UV ellipsoid shells ("ore bodies") and swept tubes ("drill holes"),
plus random rigid placements.  They stand in for the mining data set of the
paper's evaluation (Sec. 4, "Use case"), which is not available here.

This module holds no part of the distance / intersection arithmetic: it only
produces vertex and index arrays, so both the CPU oracle and the CUDA path can
consume the very same inputs.  Every function is deterministic in its seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 1808


# ----------------------------------------------------------------------------
# primitives
# ----------------------------------------------------------------------------

def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform rotation on SO(3) from a normalised Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def random_unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def icosphere(subdiv: int, radius: float = 1.0, jitter: float = 0.0,
              seed: int | None = None, vertex_on_x: bool = False):
    """Icosahedron subdivided `subdiv` times, vertices pushed to the sphere.

    20 * 4**subdiv triangles, CCW seen from outside.  With `jitter` > 0 every
    vertex is scaled radially by (1 + U[-jitter, jitter]).  With `vertex_on_x`
    the base icosahedron is oriented so that (+-1, 0, 0) are vertices.
    Returns (V float64[nv,3], I uint32[nt,3]).
    """
    p = (1.0 + math.sqrt(5.0)) / 2.0
    if vertex_on_x:
        # cyclic permutation of the standard (0, +-1, +-p) set puts a vertex on x
        verts = [(p, 0, 1), (p, 0, -1), (-p, 0, 1), (-p, 0, -1),
                 (1, p, 0), (-1, p, 0), (1, -p, 0), (-1, -p, 0),
                 (0, 1, p), (0, -1, p), (0, 1, -p), (0, -1, -p)]
        # rotate about y so that the vertex (p, 0, 1) lands on +x exactly:
        # handled below by explicit re-normalisation of a rotated set.
        ang = math.atan2(1.0, p)
        c, s = math.cos(ang), math.sin(ang)
        verts = [(c * x + s * z, y, -s * x + c * z) for (x, y, z) in verts]
    else:
        verts = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
                 (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
                 (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    V = [np.array(v, dtype=np.float64) for v in verts]
    V = [v / np.linalg.norm(v) for v in V]
    # faces: find all triples of mutually adjacent vertices (edge length 2)
    P = np.array(V)
    d2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    emin = np.min(d2[d2 > 1e-9])
    adj = np.abs(d2 - emin) < 1e-6
    faces = []
    for i in range(12):
        for j in range(i + 1, 12):
            if not adj[i, j]:
                continue
            for k in range(j + 1, 12):
                if adj[i, k] and adj[j, k]:
                    a, b, c_ = P[i], P[j], P[k]
                    n = np.cross(b - a, c_ - a)
                    if np.dot(n, a + b + c_) < 0:
                        faces.append((i, k, j))
                    else:
                        faces.append((i, j, k))
    assert len(faces) == 20
    verts = list(V)
    for _ in range(subdiv):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            if key in cache:
                return cache[key]
            m = verts[a] + verts[b]
            m = m / np.linalg.norm(m)
            verts.append(m)
            cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for (a, b, c_) in faces:
            ab, bc, ca = mid(a, b), mid(b, c_), mid(c_, a)
            nf += [(a, ab, ca), (b, bc, ab), (c_, ca, bc), (ab, bc, ca)]
        faces = nf
    Vn = np.array(verts, dtype=np.float64)
    if vertex_on_x:
        # snap the two axis vertices exactly (they are within an ulp already)
        for i in range(len(Vn)):
            if abs(abs(Vn[i, 0]) - 1.0) < 1e-12:
                Vn[i] = (np.sign(Vn[i, 0]), 0.0, 0.0)
    Vn *= radius
    if jitter > 0:
        rng = np.random.default_rng(seed)
        Vn *= (1.0 + rng.uniform(-jitter, jitter, size=(len(Vn), 1)))
    return Vn, np.array(faces, dtype=np.uint32)


def uv_ellipsoid(axes=(40.0, 25.0, 15.0), n_lon: int = 1024, n_lat: int = 1024,
                 jitter: float = 0.0, seed: int | None = None):
    """Closed UV ellipsoid shell with pole fans.

    `n_lat` latitude bands -> n_lat - 1 vertex rings of `n_lon` vertices plus
    two poles; 2 * n_lon * (n_lat - 1) triangles, CCW seen from outside.
    Vertices are scaled radially by (1 + U[-jitter, jitter]).
    """
    a, b, c = axes
    th = np.pi * np.arange(1, n_lat) / n_lat
    ph = 2 * np.pi * np.arange(n_lon) / n_lon
    st, ct = np.sin(th)[:, None], np.cos(th)[:, None]
    ring = np.stack([a * st * np.cos(ph)[None, :], b * st * np.sin(ph)[None, :],
                     np.broadcast_to(c * ct, (n_lat - 1, n_lon))], axis=-1)
    V = np.concatenate([[[0.0, 0.0, c]], ring.reshape(-1, 3), [[0.0, 0.0, -c]]])
    if jitter > 0:
        rng = np.random.default_rng(seed)
        V *= (1.0 + rng.uniform(-jitter, jitter, size=(len(V), 1)))
    nr = n_lat - 1
    j = np.arange(n_lon)
    jn = (j + 1) % n_lon
    top = np.stack([np.zeros(n_lon, np.int64), 1 + j, 1 + jn], axis=1)
    # bands between ring r and r+1
    r = np.arange(nr - 1)[:, None]
    v00 = 1 + r * n_lon + j[None, :]
    v01 = 1 + r * n_lon + jn[None, :]
    v10 = v00 + n_lon
    v11 = v01 + n_lon
    t1 = np.stack([v00, v10, v11], axis=-1).reshape(-1, 3)
    t2 = np.stack([v00, v11, v01], axis=-1).reshape(-1, 3)
    bands = np.stack([t1.reshape(nr - 1, n_lon, 3), t2.reshape(nr - 1, n_lon, 3)],
                     axis=2).reshape(-1, 3)
    south = len(V) - 1
    last = 1 + (nr - 1) * n_lon
    bot = np.stack([np.full(n_lon, south), last + jn, last + j], axis=1)
    I = np.concatenate([top, bands, bot]).astype(np.uint32)
    return V, I


def uv_sphere_tris(T: int):
    """(n_lon, n_lat) of a UV sphere with about T triangles."""
    n = max(3, int(round(math.sqrt(T / 2.0))))
    return n, max(2, n)


def random_walk_polyline(n_steps: int, step: float, sigma: float,
                         rng: np.random.Generator) -> np.ndarray:
    """Persistent random walk: each step turns the heading by an angle
    ~ N(0, sigma) about a random axis perpendicular to it."""
    d = random_unit(rng)
    pts = np.empty((n_steps + 1, 3))
    pts[0] = 0.0
    ang = rng.normal(0.0, sigma, size=n_steps)
    g = rng.standard_normal((n_steps, 3))
    dx, dy, dz = d
    px = py = pz = 0.0
    for k in range(n_steps):
        gx, gy, gz = g[k]
        t = gx * dx + gy * dy + gz * dz
        ax, ay, az = gx - t * dx, gy - t * dy, gz - t * dz
        n = math.sqrt(ax * ax + ay * ay + az * az)
        ax, ay, az = ax / n, ay / n, az / n
        # rotate heading about the perpendicular axis: d' = d cos + (a x d) sin
        c, s = math.cos(ang[k]), math.sin(ang[k])
        cx = ay * dz - az * dy
        cy = az * dx - ax * dz
        cz = ax * dy - ay * dx
        dx, dy, dz = dx * c + cx * s, dy * c + cy * s, dz * c + cz * s
        n = math.sqrt(dx * dx + dy * dy + dz * dz)
        dx, dy, dz = dx / n, dy / n, dz / n
        px, py, pz = px + step * dx, py + step * dy, pz + step * dz
        pts[k + 1] = (px, py, pz)
    return pts


def tube(polyline: np.ndarray, radius: float, sides: int):
    """Open tube of `sides`-gon rings swept along a polyline with
    parallel-transport frames.  (len-1) * 2 * sides triangles."""
    P = np.asarray(polyline, np.float64)
    n = len(P)
    seg = P[1:] - P[:-1]
    seg /= np.linalg.norm(seg, axis=1, keepdims=True)
    T = np.empty_like(P)
    T[0], T[-1] = seg[0], seg[-1]
    if n > 2:
        t = seg[1:] + seg[:-1]
        T[1:-1] = t / np.linalg.norm(t, axis=1, keepdims=True)
    # initial normal: any perpendicular of T0
    a = np.array([1.0, 0.0, 0.0]) if abs(T[0, 0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    N = np.empty_like(P)
    v = a - np.dot(a, T[0]) * T[0]
    N[0] = v / np.linalg.norm(v)
    for k in range(1, n):
        v = N[k - 1] - np.dot(N[k - 1], T[k]) * T[k]
        N[k] = v / np.linalg.norm(v)
    B = np.cross(T, N)
    th = 2 * np.pi * np.arange(sides) / sides
    V = (P[:, None, :] + radius * (np.cos(th)[None, :, None] * N[:, None, :]
                                   + np.sin(th)[None, :, None] * B[:, None, :]))
    V = V.reshape(-1, 3)
    k = np.arange(n - 1)[:, None]
    j = np.arange(sides)[None, :]
    jn = (j + 1) % sides
    v00 = k * sides + j
    v01 = k * sides + jn
    v10 = v00 + sides
    v11 = v01 + sides
    t1 = np.stack([v00, v01, v11], axis=-1)
    t2 = np.stack([v00, v11, v10], axis=-1)
    I = np.stack([t1, t2], axis=2).reshape(-1, 3).astype(np.uint32)
    return V, I


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

@dataclass
class Mesh:
    V: np.ndarray        # float64 or float32 [nv, 3]
    I: np.ndarray        # uint32 [nt, 3]

    @property
    def nt(self) -> int:
        return int(self.I.shape[0])


def icosphere_pair(center_dist: float, subdiv: int = 3, seed: int = BASE_SEED):
    """Two jittered icospheres (r = 1, jitter 5 %) whose centres are
    `center_dist` apart along a random unit axis.  float64 vertices."""
    VA, I = icosphere(subdiv, 1.0, 0.05, seed)
    VB, _ = icosphere(subdiv, 1.0, 0.05, seed + 1)
    axis = random_unit(np.random.default_rng(seed + 1000))
    VB = VB + center_dist * axis[None, :]
    return Mesh(VA, I), Mesh(VB, I.copy())


def small_pairs(seed: int = BASE_SEED):
    """The small plain-method case: 1,280-triangle icospheres, pair A with
    centres 2.5 apart (separated) and pair B 1.8 apart (intersecting)."""
    return {"A": icosphere_pair(2.5, 3, seed), "B": icosphere_pair(1.8, 3, seed)}


def ore_body(n_lon=1024, n_lat=1024, seed: int = BASE_SEED + 1):
    V, I = uv_ellipsoid((40.0, 25.0, 15.0), n_lon, n_lat, jitter=0.01, seed=seed)
    return Mesh(V, I)


def box_mesh(a: float, b: float, c: float, origin=(0.0, 0.0, 0.0)):
    """Axis-aligned box [0, a] x [0, b] x [0, c] + origin: 8 vertices
    (index = x + 2 y + 4 z bits), 12 faces counter-clockwise seen from
    outside.  float64 vertices."""
    o = np.array(origin, np.float64)
    V = np.array([[x, y, z] for z in (0, c) for y in (0, b) for x in (0, a)], np.float64) + o
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    I = []
    for q in quads:
        I += [(q[0], q[1], q[2]), (q[0], q[2], q[3])]
    return V, np.array(I, np.uint32)


def small_ore_body(seed: int = BASE_SEED + 5) -> Mesh:
    """The ore shape of the paper's experiments: one closed mesh of 500
    faces (UV ellipsoid 40/25/15, 25 longitudes x 11 latitude bands with pole
    fans, 1 % radial jitter), float32 vertices."""
    V, I = uv_ellipsoid((40.0, 25.0, 15.0), 25, 11, jitter=0.01, seed=seed)
    return Mesh(V.astype(np.float32), I)


def drill_holes(n_holes: int, segs_per_hole: int = 100, step: float = 1.0, sigma: float = 0.02,
                seed: int = BASE_SEED + 6) -> np.ndarray:
    """Drill-hole line segments around the ore body: collars uniform on
    [-60, 60] x [-40, 40] at z = 40, initial heading downwards with a dip of
    up to ~17 degrees, then a persistent random walk of `segs_per_hole` steps
    of length `step` (heading turned by N(0, sigma) rad per step about a
    random perpendicular axis).  Returns float32 [n_holes * segs_per_hole, 6]
    = (P0, P1) per segment, hole after hole."""
    rng = np.random.default_rng(seed)
    P = np.empty((n_holes, 3))
    P[:, 0] = rng.uniform(-60.0, 60.0, n_holes)
    P[:, 1] = rng.uniform(-40.0, 40.0, n_holes)
    P[:, 2] = 40.0
    d = np.column_stack([rng.uniform(-0.3, 0.3, n_holes), rng.uniform(-0.3, 0.3, n_holes), -np.ones(n_holes)])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    out = np.empty((n_holes, segs_per_hole, 6), np.float32)
    for k in range(segs_per_hole):
        g = rng.standard_normal((n_holes, 3))
        a = g - (g * d).sum(1, keepdims=True) * d
        a /= np.linalg.norm(a, axis=1, keepdims=True)
        ang = rng.normal(0.0, sigma, n_holes)[:, None]
        d = d * np.cos(ang) + np.cross(a, d) * np.sin(ang)
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        Q = P + step * d
        out[:, k, :3] = P
        out[:, k, 3:] = Q
        P = out[:, k, 3:].astype(np.float64)  # continue from the stored (rounded) end point
    return out.reshape(-1, 6)


def drill_hole(n_steps=65536, sides=16, seed: int = BASE_SEED + 2):
    rng = np.random.default_rng(seed)
    P = random_walk_polyline(n_steps, 0.05, 0.05, rng)
    V, I = tube(P, 0.5, sides)
    return Mesh(V, I), P


def place_tube(tube_V: np.ndarray, ring_centres: np.ndarray, sides: int,
               ore_V: np.ndarray, intersect: bool, gap: float,
               rng: np.random.Generator) -> np.ndarray:
    """One rigid placement of the tube against the ore body (float64 out).

    intersect: a random ring centre of the tube is moved onto a random ore
      vertex, so the tube crosses the shell there.
    separated: for a random unit direction u, let q be the ore vertex of
      largest u.x and p the tube vertex of smallest u.(Rx).  Moving p to
      q + gap * u puts the plane u.x = u.q + gap/2 between the two meshes and
      the two vertices `gap` apart, so the true distance is `gap`.
    """
    R = random_rotation(rng)
    X = tube_V @ R.T
    if intersect:
        k = int(rng.integers(0, len(ring_centres)))
        qi = int(rng.integers(0, len(ore_V)))
        t = ore_V[qi] - R @ ring_centres[k]
        return X + t[None, :]
    u = random_unit(rng)
    q = ore_V[int(np.argmax(ore_V @ u))]
    p = X[int(np.argmin(X @ u))]
    t = q + gap * u - p
    return X + t[None, :]


def large_placements(n_place: int = 64, seed: int = BASE_SEED + 3,
                     n_steps: int = 65536, n_lon: int = 1024, n_lat: int = 1024):
    """The large plain-method case: drill-hole tube (~2.1 M tris) against an
    ore-body ellipsoid shell (~2.1 M tris), `n_place` rigid placements, the
    first half intersecting, the second half separated by a gap log-uniform
    in [0.01, 10].  Vertices are rounded to float32.

    Returns (ore Mesh f32, tube index array, list of f32 tube vertex arrays,
    list of dicts describing each placement)."""
    ore = ore_body(n_lon, n_lat)
    tube_m, P = drill_hole(n_steps)
    rng = np.random.default_rng(seed)
    oreV32 = ore.V.astype(np.float32)
    oreV64 = oreV32.astype(np.float64)
    out, info = [], []
    for k in range(n_place):
        inter = k < n_place // 2
        gap = 0.0 if inter else float(10 ** rng.uniform(-2, 1))
        X = place_tube(tube_m.V, P, 16, oreV64, inter, gap, rng)
        out.append(X.astype(np.float32))
        info.append({"intersect_by_construction": inter, "gap": gap})
    return Mesh(oreV32, ore.I), tube_m.I, out, info


def jittered_uv_sphere(T: int, radius: float, rng: np.random.Generator):
    n_lon, n_lat = uv_sphere_tris(T)
    V, I = uv_ellipsoid((radius, radius, radius), n_lon, n_lat, jitter=0.0)
    V *= (1.0 + rng.uniform(-0.02, 0.02, size=(len(V), 1)))
    return V, I


def small_tube(T: int, rng: np.random.Generator, sides: int = 8):
    n_seg = max(1, int(round(T / (2 * sides))))
    P = random_walk_polyline(n_seg, 0.05, 0.05, rng)
    return tube(P, 0.1, sides)


def tiny_random_mesh(nt: int, rng: np.random.Generator, spread: float = 1.0,
                     size: float = 0.3, dtype=np.float64) -> Mesh:
    """Triangle soup of `nt` random triangles (no shared vertices)."""
    c = rng.uniform(-spread, spread, size=(nt, 1, 3))
    V = (c + rng.uniform(-size, size, size=(nt, 3, 3))).reshape(-1, 3)
    I = np.arange(3 * nt, dtype=np.uint32).reshape(nt, 3)
    return Mesh(V.astype(dtype), I)


# ----------------------------------------------------------------------------
# batched workload: many independent pairs of small meshes
# ----------------------------------------------------------------------------

class TemplateBank:
    """Shapes reused across pairs: jittered UV spheres (radius 1) and 8-sided
    tubes (radius 0.1, persistent random walk of step 0.05), with face counts
    rounded to half-octave buckets of a log-uniform target."""

    def __init__(self, seed: int):
        self.seed = seed
        self.cache: dict = {}

    def get(self, kind: str, T: int, variant: int):
        b = int(round(2 * math.log2(max(T, 2))))
        key = (kind, b, variant)
        if key not in self.cache:
            Tb = 2.0 ** (b / 2)
            rng = np.random.default_rng((self.seed, b, variant, kind == "tube"))
            if kind == "sphere":
                V, I = jittered_uv_sphere(int(Tb), 1.0, rng)
            else:
                n_seg = max(1, int(round(Tb / 16)))
                P = random_walk_polyline(n_seg, 0.05, 0.05, rng)
                V, I = tube(P, 0.1, 8)
            self.cache[key] = (np.ascontiguousarray(V, np.float64), np.ascontiguousarray(I, np.uint32))
        return self.cache[key]


def batch_workload(n_pairs: int, seed: int = BASE_SEED + 4, t_min: int = 20, t_max: int = 65536,
                   p_intersect: float = 0.3, gap_range=(1e-3, 1.0), variants: int = 4):
    """Independent pairs: each mesh a jittered UV sphere or a tube (50/50),
    face count log-uniform in [t_min, t_max]; each pair rotated at random.
    With probability p_intersect a vertex of B is moved exactly onto a vertex
    of A (the meshes share a point); otherwise B is placed at a gap g
    log-uniform in gap_range along a random direction u, extreme vertices
    aligned, so the exact distance is g before float32 rounding.  Ops: 50 %
    distance, 50 % intersects.  Each (kind, size bucket) has `variants`
    different template shapes.

    Returns (meshes [(V float32, I uint32)], queries [(ia, ib, op)],
    info [dict])."""
    rng = np.random.default_rng(seed)
    bank = TemplateBank(seed)
    meshes, queries, info = [], [], []
    lo, hi = math.log(t_min), math.log(t_max)
    for p in range(n_pairs):
        tmpl = []
        for _ in range(2):
            kind = "sphere" if rng.random() < 0.5 else "tube"
            T = int(round(math.exp(rng.uniform(lo, hi))))
            tmpl.append(bank.get(kind, T, int(rng.integers(0, variants))))
        (VA0, IA), (VB0, IB) = tmpl
        VA = (VA0 @ random_rotation(rng).T).astype(np.float32)
        VAd = VA.astype(np.float64)
        RB = random_rotation(rng)
        XB = VB0 @ RB.T
        inter = rng.random() < p_intersect
        if inter:
            a = VAd[int(rng.integers(0, len(VAd)))]
            b = XB[int(rng.integers(0, len(XB)))]
            t = a - b
            gap = 0.0
        else:
            u = random_unit(rng)
            gap = float(math.exp(rng.uniform(math.log(gap_range[0]), math.log(gap_range[1]))))
            q = VAd[int(np.argmax(VAd @ u))]
            pb = XB[int(np.argmin(XB @ u))]
            t = q + gap * u - pb
        VB = (XB + t[None, :]).astype(np.float32)
        ia, ib = len(meshes), len(meshes) + 1
        meshes += [(VA, IA), (VB, IB)]
        op = int(rng.integers(0, 2))
        queries.append((ia, ib, op))
        info.append({"shares_vertex": inter, "gap": gap, "faces": (len(IA), len(IB))})
    return meshes, queries, info


# ----------------------------------------------------------------------------
# near-coplanar face pairs: inputs only exact orientation signs can decide
# ----------------------------------------------------------------------------

def near_coplanar_face_pairs(n: int, seed: int = BASE_SEED + 7):
    """Face pairs (float64) on which the intersects answer turns on
    orientation determinants far below double precision's forward error.

    Face A = (P, Q, R) has integer vertices in [2^19, 2^20)^3: a generic
    plane with edges of about 2^19.  Face B's first vertex is
    X = P + (a (Q - P) + b (R - P)) / 2^32 (exact in binary64: |X| < 2^20 on a
    2^-32 grid), shifted by e * 2^-32 along z with e in {-1, 0, +1} (e = +1
    towards the side of A's plane that B's other two vertices lie on).  Those
    two are X + D + r_k, where D is about 2^17 times the unit normal of A's
    plane and r_k are integer offsets below 2^14; both lie strictly on the
    positive side (checked with exact integer dot products).  A vertex
    2^-32 off a plane whose normal is about 2^38 long gives a determinant of
    at most 2^6 against a double-precision error bound of about 2^8, so no
    floating-point filter can decide it.

    Kinds (a, b): "interior" (both in [2^28, 2^31]), "edge" (b = 0, X on the
    edge PQ), "vertex" (a = b = 0, X = P), "far_edge" (a + b = 2^32, X on the
    edge QR), and "coplanar": all three vertices of B on A's plane (e = 0),
    B straddling or just outside the edge QR.

    Returns a list of (T1 float64[3, 3], T2 float64[3, 3], expected, kind);
    expected is the intersects answer that follows from the construction
    (None where it depends on how the crossing point falls against an edge):
    interior e = 0 touches (True), interior e = +1 is strictly on one side
    (False), interior e = -1 crosses the plane inside A (True).  Coplanar
    straddling (a + b < 2^32 at one vertex) meets A (True); coplanar with
    every vertex at a + b > 2^32 and a, b >= 0 lies outside the edge QR
    (False)."""
    rng = np.random.default_rng(seed)
    S = 1 << 32
    out = []

    def cross(u, v):
        return (u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0])

    def dot(u, v):
        return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]

    def on_plane(P, Q, R, a, b):
        # exact rational point P + (a (Q - P) + b (R - P)) / 2^32 as floats
        return [float(P[k]) + (a * (Q[k] - P[k]) + b * (R[k] - P[k])) / S for k in range(3)]

    kinds = ["interior", "edge", "vertex", "far_edge", "coplanar"]
    while len(out) < n:
        P, Q, R = [[int(x) for x in rng.integers(1 << 19, 1 << 20, size=3)] for _ in range(3)]
        N = cross([Q[k] - P[k] for k in range(3)], [R[k] - P[k] for k in range(3)])
        nn = math.sqrt(float(dot(N, N)))
        if nn < 2.0 ** 30 or N[2] == 0:
            continue
        kind = kinds[len(out) % len(kinds)]
        D = [int(round(N[k] / nn * 2.0 ** 17)) for k in range(3)]
        T1 = np.array([P, Q, R], np.float64)
        if kind == "coplanar":
            # three on-plane points near the edge QR (a + b close to 2^32)
            straddle = bool(rng.integers(0, 2))
            pts = []
            for v in range(3):
                a = int(rng.integers(S // 4, 3 * S // 4))
                over = int(rng.integers(1, 1 << 20))
                b = S - a + over if (v > 0 or not straddle) else S - a - over
                pts.append(on_plane(P, Q, R, a, b))
            T2 = np.array(pts, np.float64)
            exp = True if straddle else False
            # every coordinate must be exact (on the 2^-32 grid below 2^20)
            if not all(abs(x) < 2.0 ** 20 for x in T2.ravel()):
                continue
            out.append((T1, T2, exp, kind))
            continue
        if kind == "interior":
            a, b = int(rng.integers(1 << 28, 1 << 31)), int(rng.integers(1 << 28, 1 << 31))
        elif kind == "edge":
            a, b = int(rng.integers(1 << 28, 1 << 31)), 0
        elif kind == "vertex":
            a, b = 0, 0
        else:
            a = int(rng.integers(1 << 28, S - (1 << 28)))
            b = S - a
        X = on_plane(P, Q, R, a, b)
        e = int(rng.integers(-1, 2))
        sz = 1 if N[2] > 0 else -1  # +z raises N . (X - P) when N_z > 0
        X[2] += e * sz * 2.0 ** -32
        r1 = [int(x) for x in rng.integers(-(1 << 14), 1 << 14, size=3)]
        r2 = [int(x) for x in rng.integers(-(1 << 14), 1 << 14, size=3)]
        Y = [X[k] + D[k] + r1[k] for k in range(3)]
        Z = [X[k] + D[k] + r2[k] for k in range(3)]
        # both far vertices strictly on the positive side (integer check on
        # the offsets: X's own height is below 2^-32 |N|)
        if dot([D[k] + r1[k] for k in range(3)], N) <= 0 or dot([D[k] + r2[k] for k in range(3)], N) <= 0:
            continue
        if not all(abs(x) < 2.0 ** 20 for x in X):
            continue
        T2 = np.array([X, Y, Z], np.float64)
        exp = {1: False, 0: True, -1: True}[e] if kind == "interior" else None
        out.append((T1, T2, exp, kind))
    return out
