"""Seeded synthetic triangle meshes (positions FP64 n x 3, faces int32 m x 3).

Every mesh is a consistently oriented 2-manifold: closed spheres and tori, or a
planar disk with one boundary loop.  The generators stand in for the artists'
models the paper evaluates on, which are not available here.
"""
import math

import numpy as np


# ---------------------------------------------------------------------------
# spheres
# ---------------------------------------------------------------------------
def icosahedron():
    """The regular icosahedron on the unit sphere, faces oriented outward."""
    g = (1.0 + math.sqrt(5.0)) / 2.0
    V = np.array([(-1, g, 0), (1, g, 0), (-1, -g, 0), (1, -g, 0),
                  (0, -1, g), (0, 1, g), (0, -1, -g), (0, 1, -g),
                  (g, 0, -1), (g, 0, 1), (-g, 0, -1), (-g, 0, 1)], dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = np.array([(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
                  (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
                  (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
                  (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)], dtype=np.int32)
    return V, _orient_outward(V, F)


def _orient_outward(V, F):
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    inward = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) < 0
    F = F.copy()
    F[inward] = F[inward][:, [0, 2, 1]]
    return F


def icosphere(k):
    """Icosahedron split k times (every edge at its midpoint, projected to the sphere).

    Vertex count 10 * 4**k + 2 and face count 20 * 4**k.
    """
    V, F = icosahedron()
    for _ in range(k):
        n = V.shape[0]
        e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
        key = np.minimum(e[:, 0], e[:, 1]).astype(np.int64) * n + np.maximum(e[:, 0], e[:, 1])
        uniq, inv = np.unique(key, return_inverse=True)
        a = (uniq // n).astype(np.int64)
        b = (uniq % n).astype(np.int64)
        mid = 0.5 * (V[a] + V[b])
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        m = F.shape[0]
        ab = (n + inv[:m]).astype(np.int32)
        bc = (n + inv[m:2 * m]).astype(np.int32)
        ca = (n + inv[2 * m:]).astype(np.int32)
        F = np.concatenate([np.stack([F[:, 0], ab, ca], 1),
                            np.stack([F[:, 1], bc, ab], 1),
                            np.stack([F[:, 2], ca, bc], 1),
                            np.stack([ab, bc, ca], 1)]).astype(np.int32)
        V = np.concatenate([V, mid])
    return V, F


def geodesic_sphere(freq):
    """Class-I geodesic sphere: each icosahedron face cut into freq**2 triangles.

    Vertex count 10 * freq**2 + 2, so sizes are not limited to powers of 4.
    """
    V0, F0 = icosahedron()
    f = int(freq)
    ij = [(i, j) for j in range(f + 1) for i in range(f + 1 - j)]
    local = {p: t for t, p in enumerate(ij)}
    keys = np.zeros((F0.shape[0] * len(ij), 6), dtype=np.int64)
    for fi, (A, B, C) in enumerate(F0):
        for t, (i, j) in enumerate(ij):
            pairs = sorted(p for p in [(int(A), f - i - j), (int(B), i), (int(C), j)] if p[1] > 0)
            row = []
            for vid, w in pairs:
                row += [vid, w]
            row += [-1, 0] * (3 - len(pairs))
            keys[fi * len(ij) + t] = row
    uniq, inv = np.unique(keys, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    P = np.zeros((uniq.shape[0], 3))
    for s in range(3):
        vid, w = uniq[:, 2 * s], uniq[:, 2 * s + 1]
        ok = vid >= 0
        P[ok] += (w[ok, None] / f) * V0[vid[ok]]
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    tris = []
    for j in range(f):
        for i in range(f - j):
            tris.append((local[(i, j)], local[(i + 1, j)], local[(i, j + 1)]))
            if i + j < f - 1:
                tris.append((local[(i + 1, j)], local[(i + 1, j + 1)], local[(i, j + 1)]))
    tris = np.array(tris, dtype=np.int64)
    F = np.concatenate([inv[fi * len(ij) + tris] for fi in range(F0.shape[0])]).astype(np.int32)
    return P, _orient_outward(P, F)


def _assoc_legendre(l, m, x):
    """Associated Legendre function P_l^m(x), m >= 0, by the three-term recurrence."""
    pmm = np.ones_like(x)
    if m > 0:
        s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
        fact = 1.0
        for _ in range(m):
            pmm = -pmm * fact * s
            fact += 2.0
    if l == m:
        return pmm
    pmm1 = x * (2 * m + 1) * pmm
    if l == m + 1:
        return pmm1
    pll = pmm1
    for ll in range(m + 2, l + 1):
        pll = ((2 * ll - 1) * x * pmm1 - (ll + m - 1) * pmm) / (ll - m)
        pmm, pmm1 = pmm1, pll
    return pll


def _real_sh(l, m, theta, phi):
    am = abs(m)
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    p = _assoc_legendre(l, am, np.cos(theta))
    if m > 0:
        return math.sqrt(2.0) * norm * p * np.cos(m * phi)
    if m < 0:
        return math.sqrt(2.0) * norm * p * np.sin(am * phi)
    return norm * p


def sh_noise(P, seed, nterms=8, lmax=6):
    """Smooth seeded noise on unit directions P: a sum of `nterms` real spherical
    harmonics with degree uniform in 1..lmax, order uniform in [-l, l] and N(0, 1)
    coefficients, scaled so that max |s| = 1 over the given points."""
    rng = np.random.default_rng(seed)
    u = P / np.linalg.norm(P, axis=1, keepdims=True)
    theta = np.arccos(np.clip(u[:, 2], -1.0, 1.0))
    phi = np.arctan2(u[:, 1], u[:, 0])
    s = np.zeros(P.shape[0])
    for _ in range(nterms):
        l = int(rng.integers(1, lmax + 1))
        m = int(rng.integers(-l, l + 1))
        c = float(rng.standard_normal())
        s += c * _real_sh(l, m, theta, phi)
    return s / np.max(np.abs(s))


def perturbed_icosphere(k, seed=0, amp=0.1):
    """Icosphere split k times with each vertex radius scaled by 1 + amp * s(p)."""
    V, F = icosphere(k)
    s = sh_noise(V, seed)
    return V * (1.0 + amp * s)[:, None], F


def perturbed_geodesic_sphere(freq, seed=0, amp=0.1):
    V, F = geodesic_sphere(freq)
    s = sh_noise(V, seed)
    return V * (1.0 + amp * s)[:, None], F


# ---------------------------------------------------------------------------
# torus and disk
# ---------------------------------------------------------------------------
def torus(nu, nv, R=1.0, r=0.3, noise=0.02, seed=0):
    """Torus from an nu x nv grid (nu around the big circle), every vertex moved
    along the surface normal by noise * r * U[-1, 1].  Valence 6 everywhere."""
    rng = np.random.default_rng(seed)
    a, b = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    phi = 2.0 * np.pi * a.reshape(-1) / nu
    th = 2.0 * np.pi * b.reshape(-1) / nv
    nrm = np.stack([np.cos(th) * np.cos(phi), np.cos(th) * np.sin(phi), np.sin(th)], 1)
    ctr = np.stack([R * np.cos(phi), R * np.sin(phi), np.zeros_like(phi)], 1)
    d = noise * r * rng.uniform(-1.0, 1.0, size=nu * nv)
    V = ctr + (r + d)[:, None] * nrm
    ia, ib = a.reshape(-1), b.reshape(-1)
    v00 = ia * nv + ib
    v10 = ((ia + 1) % nu) * nv + ib
    v11 = ((ia + 1) % nu) * nv + (ib + 1) % nv
    v01 = ia * nv + (ib + 1) % nv
    F = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)]).astype(np.int32)
    # orient outward: signed volume of the closed surface must be positive
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    if np.einsum("ij,ij->i", A, np.cross(B, C)).sum() < 0:
        F = F[:, [0, 2, 1]].copy()
    return V, F


def _concentric(a, b):
    """Shirley-Chiu concentric map of the square [-1, 1]^2 onto the unit disk."""
    x = np.zeros_like(a)
    y = np.zeros_like(a)
    big_a = np.abs(a) > np.abs(b)
    rr = np.where(big_a, a, b)
    with np.errstate(divide="ignore", invalid="ignore"):
        ang = np.where(big_a, (np.pi / 4) * (b / a), np.pi / 2 - (np.pi / 4) * (a / b))
    zero = (a == 0) & (b == 0)
    ang = np.where(zero, 0.0, ang)
    x = rr * np.cos(ang)
    y = rr * np.sin(ang)
    return x, y


def _cross2(u, v):
    return u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0]


def disk(N=400, jitter=0.01, seed=0):
    """Planar unit disk from an N x N grid on [-1, 1]^2 through the concentric map.

    Interior grid vertices are jittered in-plane by jitter * h * U[-1, 1]^2
    (h = 2 / (N - 1)) before mapping; each cell is split along the diagonal
    parallel to the map's kink line in its quadrant.  Returns (V with z = 0,
    F, boundary mask)."""
    rng = np.random.default_rng(seed)
    h = 2.0 / (N - 1)
    g = np.linspace(-1.0, 1.0, N)
    a, b = np.meshgrid(g, g, indexing="ij")
    a = a.reshape(-1).copy()
    b = b.reshape(-1).copy()
    ia, ib = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    ia, ib = ia.reshape(-1), ib.reshape(-1)
    bnd = (ia == 0) | (ia == N - 1) | (ib == 0) | (ib == N - 1)
    jit = jitter * h * rng.uniform(-1.0, 1.0, size=(N * N, 2))
    a[~bnd] += jit[~bnd, 0]
    b[~bnd] += jit[~bnd, 1]
    x, y = _concentric(a, b)
    V = np.stack([x, y, np.zeros_like(x)], 1)
    ca, cb = np.meshgrid(np.arange(N - 1), np.arange(N - 1), indexing="ij")
    ca, cb = ca.reshape(-1), cb.reshape(-1)
    v00 = ca * N + cb
    v10 = (ca + 1) * N + cb
    v11 = (ca + 1) * N + cb + 1
    v01 = ca * N + cb + 1
    # each cell is split along the diagonal parallel to the concentric map's
    # kink line (a = b or a = -b) in its quadrant, so no triangle straddles a
    # kink; alternating diagonals fold triangles there once jittered
    alt = ((g[ca] + h / 2) * (g[cb] + h / 2)) > 0
    t1 = np.where(alt[:, None], np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
    t2 = np.where(alt[:, None], np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
    F = np.concatenate([t1, t2]).astype(np.int32)
    # orientation from the unjittered grid; a fold after mapping is an error
    G = np.stack([g[ia], g[ib]], 1)
    sg = _cross2(G[F[:, 1]] - G[F[:, 0]], G[F[:, 2]] - G[F[:, 0]])
    F[sg < 0] = F[sg < 0][:, [0, 2, 1]]
    sv = _cross2(V[F[:, 1], :2] - V[F[:, 0], :2], V[F[:, 2], :2] - V[F[:, 0], :2])
    if np.any(sv <= 0):
        raise ValueError("jitter folds %d triangles" % int(np.sum(sv <= 0)))
    return V, F, bnd


# ---------------------------------------------------------------------------
# plain mesh facts (no solver arithmetic)
# ---------------------------------------------------------------------------
def sinusoidal_displacement(V, frame, seed=0, amp=0.05, nframes=100, nwaves=3):
    """Seeded smooth deformation field for per-frame re-solves:
    d_f(p) = amp * sum_k a_k sin(w_k . p + phi_k + 2 pi f / nframes) e_k with
    a_k >= 0 summing to 1, |w_k| <= 4 pi, phases phi_k in [0, 2 pi) and unit
    directions e_k.  Returns the moved positions V + d_f(V)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.2, 1.0, nwaves)
    a /= a.sum()
    w = rng.normal(size=(nwaves, 3))
    w *= (rng.uniform(0.25, 1.0, nwaves) * 4 * np.pi / np.linalg.norm(w, axis=1))[:, None]
    phi = rng.uniform(0, 2 * np.pi, nwaves)
    e = rng.normal(size=(nwaves, 3))
    e /= np.linalg.norm(e, axis=1)[:, None]
    V = np.asarray(V, dtype=np.float64)
    s = np.sin(V @ w.T + phi + 2 * np.pi * frame / nframes)  # n x nwaves
    return V + amp * (s * a) @ e


def mean_edge_length(V, F):
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    e = np.unique(np.sort(e, axis=1), axis=0)
    return float(np.linalg.norm(V[e[:, 0]] - V[e[:, 1]], axis=1).mean())


def boundary_mask(F, n):
    """Vertices that lie on an edge used by exactly one face."""
    e = np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), axis=1)
    uniq, cnt = np.unique(e, axis=0, return_counts=True)
    mask = np.zeros(n, dtype=bool)
    mask[uniq[cnt == 1].reshape(-1)] = True
    return mask


def euler_characteristic(n, F):
    e = np.unique(np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), axis=1), axis=0)
    return int(n - e.shape[0] + F.shape[0])
