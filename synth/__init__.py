"""Seeded synthetic inputs shared by the CPU oracle tests and the CUDA path.

This module only builds *inputs*: triangulated approximations of the unit
sphere (the icosahedral discretization of Sec. 4.2), their random
perturbations and rotations, and the serving request stream. It holds none of
the method's arithmetic (no Fourier transform, no quadrature rule, no
distance), so both sides of every parity test can consume its arrays without
sharing any computation.

Vertices are float64 arrays of shape (V, 3); triangles are int32 arrays of
shape (T, 3). Triangle vertex order carries no meaning for the surface measure
(Sec. 2.2, remark after the affine-simplex definition), but faces are emitted
counter-clockwise seen from outside for readability.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN = (1.0 + math.sqrt(5.0)) / 2.0


def icosahedron():
    """The regular icosahedron inscribed in the unit sphere (T_0 of Sec. 4.2).

    Its 12 vertices are the normalised cyclic permutations of (0, +-1, +-phi);
    its 20 faces are the vertex triples that are pairwise one edge apart.
    """
    base = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            base.append((0.0, s1, s2 * GOLDEN))
            base.append((s1, s2 * GOLDEN, 0.0))
            base.append((s2 * GOLDEN, 0.0, s1))
    v = np.array(base, dtype=np.float64)
    edge2 = 4.0  # squared edge length before normalisation
    faces = []
    n = len(v)
    d2 = ((v[:, None, :] - v[None, :, :]) ** 2).sum(-1)
    adj = np.abs(d2 - edge2) < 1e-9
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    faces.append(_outward(v, (i, j, k)))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(faces, dtype=np.int32)
    assert f.shape == (20, 3)
    return v, f


def _outward(v, tri):
    i, j, k = tri
    nrm = np.cross(v[j] - v[i], v[k] - v[i])
    if np.dot(nrm, v[i] + v[j] + v[k]) < 0:
        return (i, k, j)
    return (i, j, k)


def icosphere_recursive(levels: int):
    """T_N: `levels` rounds of 4-way midpoint subdivision with projection.

    Each round inserts the midpoint of every edge, projects it to |x| = 1 and
    splits every triangle into four (Sec. 4.2). T_N has 10*4^N + 2 vertices
    and 20*4^N triangles.
    """
    v, f = icosahedron()
    verts = [tuple(p) for p in v]
    tris = [tuple(t) for t in f]
    for _ in range(levels):
        mid = {}
        new_tris = []

        def midpoint(a, b):
            key = (a, b) if a < b else (b, a)
            idx = mid.get(key)
            if idx is None:
                p = 0.5 * (np.asarray(verts[a]) + np.asarray(verts[b]))
                p = p / np.linalg.norm(p)
                idx = len(verts)
                verts.append(tuple(p))
                mid[key] = idx
            return idx

        for (a, b, c) in tris:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            new_tris += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        tris = new_tris
    return np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int32)


def icosphere_flat(n: int):
    """Flat-grid icosahedral mesh for any edge subdivision count n >= 1.

    Every face of the icosahedron carries the barycentric grid
    (i*A + j*B + k*C)/n, i+j+k = n, which is then projected to |x| = 1.
    Grid points on shared edges and corners are generated once from a
    canonical description, so the result is a closed mesh with 10 n^2 + 2
    vertices and 20 n^2 triangles. For n = 2 it coincides with T_1.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    v0, f0 = icosahedron()
    index = {}
    verts = []

    def vid(key, pos):
        idx = index.get(key)
        if idx is None:
            idx = len(verts)
            index[key] = idx
            verts.append(pos / np.linalg.norm(pos))
        return idx

    def point(face, i, j, k):
        a, b, c = (int(x) for x in f0[face])
        coords = {a: i, b: j, c: k}
        nz = [(w, cnt) for w, cnt in coords.items() if cnt > 0]
        if len(nz) == 1:
            w = nz[0][0]
            return vid(("v", w), v0[w].copy())
        if len(nz) == 2:
            (p, cp), (q, cq) = sorted(nz)
            # canonical edge point: position cq/n along p -> q, p < q
            return vid(("e", p, q, cq), (cp * v0[p] + cq * v0[q]) / n)
        return vid(("f", face, i, j), (i * v0[a] + j * v0[b] + k * v0[c]) / n)

    tris = []
    for face in range(20):
        grid = {}
        for i in range(n + 1):
            for j in range(n + 1 - i):
                k = n - i - j
                grid[(i, j)] = point(face, i, j, k)
        for i in range(n):
            for j in range(n - i):
                # "upward" triangle and, where it exists, the "downward" one
                tris.append((grid[(i + 1, j)], grid[(i, j + 1)], grid[(i, j)]))
                if i + j < n - 1:
                    tris.append((grid[(i + 1, j)], grid[(i + 1, j + 1)], grid[(i, j + 1)]))
    v = np.array(verts, dtype=np.float64)
    t = np.array(tris, dtype=np.int32)
    # orient every face outward (cosmetic: the measure ignores orientation)
    cen = v[t].mean(axis=1)
    nrm = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
    flip = (nrm * cen).sum(1) < 0
    t[flip] = t[flip][:, [0, 2, 1]]
    return v, t


def icosphere(n: int):
    """Icosahedral mesh with n edge subdivisions (20 n^2 triangles).

    Powers of two use the recursive midpoint construction (T_N with n = 2^N,
    Sec. 4.2); other n use the flat barycentric grid.
    """
    if n >= 1 and (n & (n - 1)) == 0:
        return icosphere_recursive(int(round(math.log2(n))))
    return icosphere_flat(n)


def mean_edge_length(verts, tris):
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    e.sort(axis=1)
    e = np.unique(e, axis=0)
    return float(np.linalg.norm(verts[e[:, 0]] - verts[e[:, 1]], axis=1).mean())


def jitter_radial(verts, sigma, seed):
    """Scale every vertex by (1 + sigma * z), z ~ N(0, 1), numpy PCG64(seed)."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(len(verts))
    return verts * (1.0 + sigma * z)[:, None]


def jitter_isotropic(verts, sigma, seed):
    """Add an isotropic Gaussian displacement sigma * N(0, I_3) to every vertex."""
    rng = np.random.default_rng(seed)
    return verts + sigma * rng.standard_normal(verts.shape)


def haar_rotation(seed):
    """Uniform (Haar) random rotation: QR of a Gaussian matrix with sign fix."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def rotation_z(angle):
    c, s = math.cos(angle), math.sin(angle)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


# ---------------------------------------------------------------- workloads
@dataclass(frozen=True)
class BallRule:
    """Parameters of a ball-centred frequency rule (radius R, node counts)."""
    R: float
    n_r: int
    n_polar: int
    n_azim: int
    hermitian: bool

    def n_eval(self):
        return self.n_r * (self.n_polar // 2 if self.hermitian else self.n_polar) * self.n_azim


# 320 triangles vs the unit sphere, s = 1, R = 32, 48 x 24 x 48 nodes.
SMALL_RULE = BallRule(32.0, 48, 24, 48, False)
SMALL_N = 4
SMALL_S = 1.0

# refinement sweep n = 8..64, s in {1, 2}, R = 128, 192 x 96 x 192 nodes, Hermitian halving
SWEEP_RULE = BallRule(128.0, 192, 96, 192, True)
SWEEP_NS = (8, 16, 32, 64)
SWEEP_SS = (1.0, 2.0)

# 327,680 triangles, radial jitter 1e-4 (seed 7), s = 1, R = 256, 256 x 128 x 256
LARGE_RULE = BallRule(256.0, 256, 128, 256, True)
LARGE_N = 128
LARGE_SIGMA = 1e-4
LARGE_SEED = 7
LARGE_S = 1.0

# adjoint batch: n = 16 and 32, isotropic jitter 0.01, seeds 0..63, s = 1, R = 128
ADJOINT_RULE = BallRule(128.0, 192, 64, 96, True)
ADJOINT_NS = (16, 32)
ADJOINT_SIGMA = 0.01
ADJOINT_SEEDS = tuple(range(64))

# the paper's own experiment (Sec. 4.2, Fig. 3b): icosahedral T_N, N = 0..7,
# against the unit sphere in H_{-10} on the cube trapezoid rule xi_max = 5,
# M = 128 (paper's 2 pi convention); this library's order s = 10
PAPER_XI_MAX = 5.0
PAPER_M = 128
PAPER_S = 10.0
PAPER_LEVELS = tuple(range(8))

# serving stream rules keyed by truncation radius
SERVE_RULES = {64.0: BallRule(64.0, 64, 32, 64, True), 128.0: BallRule(128.0, 128, 48, 96, True)}


def large_mesh():
    v, t = icosphere(LARGE_N)
    return jitter_radial(v, LARGE_SIGMA, LARGE_SEED), t


def adjoint_mesh(n, seed):
    v, t = icosphere(n)
    return jitter_isotropic(v, ADJOINT_SIGMA, seed), t


@dataclass
class Query:
    arrival_s: float
    n: int
    s: float
    R: float
    verts: np.ndarray
    tris: np.ndarray


def serve_stream(n_queries=2000, rate=500.0, seed=0, n_range=(2, 48), build_meshes=True):
    """Poisson stream of distance queries (exponential inter-arrival times).

    Each query: n ~ U{n_range}, a Haar-random rotation, isotropic jitter with
    sigma = 1e-3 * mean edge length, s ~ U{1, 2}, R ~ U{64, 128}.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    cache = {}
    out = []
    for q in range(n_queries):
        t += rng.exponential(1.0 / rate)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        s = float(rng.integers(1, 3))
        R = float((64.0, 128.0)[int(rng.integers(0, 2))])
        rot_seed = int(rng.integers(0, 2**31))
        jit_seed = int(rng.integers(0, 2**31))
        v = t_ = None
        if build_meshes:
            if n not in cache:
                vv, tt = icosphere(n)
                cache[n] = (vv, tt, mean_edge_length(vv, tt))
            vv, tt, h = cache[n]
            v = jitter_isotropic(vv @ haar_rotation(rot_seed).T, 1e-3 * h, jit_seed)
            t_ = tt
        out.append(Query(t, n, s, R, v, t_))
    return out
