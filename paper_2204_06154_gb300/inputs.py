"""Seeded synthetic workloads: point clouds on surfaces, their unit normals, and right-hand sides.

This module only makes inputs. It holds none of the method's arithmetic (no stencils, no weights,
no coarsening, no solver): the oracle and the CUDA path both take their inputs from here, so the
two sides see byte-identical point clouds.

Surfaces (paper Sec. 5 and Sec. 6 use icosahedral sphere nodes, Poisson-disk cyclide nodes and
scanned models; the scans are not available, so seeded synthetic stand-ins are generated):

* ``icosahedral_sphere(q)``: vertices of the q-times recursively subdivided icosahedron projected
  to the unit sphere, N = 10 * 4**q + 2 (q = 5 gives 10,242 and q = 8 gives 2,621,442, the node
  counts of the paper's sphere experiments, Sec. 5.2 Table 2).
* ``fibonacci_sphere(N, jitter, seed)``: spherical Fibonacci points with uniform tangential jitter.
* ``torus_grid(N, R, r, jitter, seed)``: parametric grid on a torus with uniform jitter.
* ``bumpy_sphere(N, seed)``: radial perturbation of the sphere by 5 seeded real spherical harmonics.

Right-hand sides: ``sh_real`` evaluates real orthonormal spherical harmonics on unit vectors,
``random_sh_rhs`` a seeded sum of them, ``y43``/``y54`` the closed-form harmonic polynomials.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = (1.0 + math.sqrt(5.0)) / 2.0


# ----------------------------------------------------------------------------------------------
# Icosahedral sphere
# ----------------------------------------------------------------------------------------------
def _icosahedron():
    t = GOLDEN
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v, f


def icosahedral_sphere(q: int):
    """Vertices (N x 3) and unit normals of the level-q icosahedral node set, N = 10*4**q + 2.

    Each level splits every triangle into four through its edge midpoints; each new midpoint is
    projected to the sphere. Vertex order: parents first, then midpoints in first-seen order of
    their (sorted) edge key, which is deterministic.
    """
    v, f = _icosahedron()
    for _ in range(q):
        nv = v.shape[0]
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        e.sort(axis=1)
        key = e[:, 0] * (nv + 1) + e[:, 1]
        uniq, first, inv = np.unique(key, return_index=True, return_inverse=True)
        order = np.argsort(first, kind="stable")           # first-seen order
        rank = np.empty_like(order)
        rank[order] = np.arange(order.size)
        mid_id = nv + rank[inv]
        a = e[first[order], 0]
        b = e[first[order], 1]
        mid = v[a] + v[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid], axis=0)
        nf = f.shape[0]
        m01 = mid_id[0:nf]
        m12 = mid_id[nf:2 * nf]
        m20 = mid_id[2 * nf:3 * nf]
        f = np.concatenate([np.stack([f[:, 0], m01, m20], 1), np.stack([f[:, 1], m12, m01], 1),
                            np.stack([f[:, 2], m20, m12], 1), np.stack([m01, m12, m20], 1)], 0)
    x = np.ascontiguousarray(v)
    return x, x.copy()


# ----------------------------------------------------------------------------------------------
# Spherical Fibonacci and torus clouds with jitter
# ----------------------------------------------------------------------------------------------
def _sphere_tangents(x):
    """Orthonormal (e_theta, e_phi) at unit vectors x (poles handled by a fixed fallback axis)."""
    z = np.array([0.0, 0.0, 1.0])
    a = np.cross(z, x)
    n = np.linalg.norm(a, axis=1)
    bad = n < 1e-12
    a[bad] = np.cross(np.array([1.0, 0.0, 0.0]), x[bad])
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = np.cross(x, a)
    return a, b


def fibonacci_sphere(N: int, jitter: float = 0.1, seed: int = 2):
    """N spherical-Fibonacci points on the unit sphere with uniform tangential jitter.

    z_i = 1 - (2i+1)/N, longitude 2*pi*i/golden; each point is then moved by U(-jitter*h,
    jitter*h) along each of two tangent directions (h = sqrt(4*pi/N)) and projected back to the
    sphere. Normals are the points themselves.
    """
    i = np.arange(N, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / N
    lon = np.mod(2.0 * np.pi * i / GOLDEN, 2.0 * np.pi)
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    x = np.stack([rho * np.cos(lon), rho * np.sin(lon), z], axis=1)
    if jitter > 0.0:
        h = math.sqrt(4.0 * math.pi / N)
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter * h, jitter * h, size=(N, 2))
        a, b = _sphere_tangents(x)
        x = x + d[:, :1] * a + d[:, 1:] * b
        x /= np.linalg.norm(x, axis=1, keepdims=True)
    x = np.ascontiguousarray(x)
    return x, x.copy()


def _torus_shape(N: int, R: float, r: float):
    """Grid shape nu x nv (nu around the central circle, nv around the tube) with nu/nv close to
    R/r: the exact factorisation N = nu * nv whose log-ratio is nearest to log(R/r), if it is within
    0.35 of it (2048 x 512 at N = 2^20); otherwise nv = round(sqrt(N r / R)), nu = N // nv, and
    nu * nv <= N points (an exact but lopsided factorisation, such as 7211 x 15, would leave a few
    points around the tube)."""
    best = None
    target = math.log(R / r)
    for nv in range(3, int(math.isqrt(N)) + 1):
        if N % nv:
            continue
        nu = N // nv
        s = abs(math.log(nu / nv) - target)
        if best is None or s < best[0]:
            best = (s, nu, nv)
    if best is None or best[0] > 0.35:
        nv = max(3, int(round(math.sqrt(N * r / R))))
        nu = max(3, N // nv)
        return nu, nv
    return best[1], best[2]


def torus_grid(N: int, R: float = 1.0, r: float = 1.0 / 3.0, jitter: float = 0.1, seed: int = 2):
    """Parametric grid on the torus ((R + r cos v) cos u, (R + r cos v) sin u, r sin v).

    nu * nv = N exactly when N has a suitable factorisation (otherwise nu*nv <= N points are
    returned). Jitter: each parameter pair is moved by U(-jitter*h, jitter*h) of arc length in
    each direction, h = sqrt(area/N), area = 4 pi^2 R r.
    """
    nu, nv = _torus_shape(N, R, r)
    u = 2.0 * np.pi * (np.arange(nu, dtype=np.float64) + 0.5) / nu
    v = 2.0 * np.pi * (np.arange(nv, dtype=np.float64) + 0.5) / nv
    U, V = np.meshgrid(u, v, indexing="ij")
    U = U.reshape(-1).copy()
    V = V.reshape(-1).copy()
    if jitter > 0.0:
        h = math.sqrt(4.0 * np.pi ** 2 * R * r / U.size)
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter * h, jitter * h, size=(U.size, 2))
        U = U + d[:, 0] / (R + r * np.cos(V))
        V = V + d[:, 1] / r
    cu, su, cv, sv = np.cos(U), np.sin(U), np.cos(V), np.sin(V)
    x = np.stack([(R + r * cv) * cu, (R + r * cv) * su, r * sv], axis=1)
    n = np.stack([cv * cu, cv * su, sv], axis=1)
    return np.ascontiguousarray(x), np.ascontiguousarray(n)


# ----------------------------------------------------------------------------------------------
# Real spherical harmonics (orthonormal on the unit sphere)
# ----------------------------------------------------------------------------------------------
def _legendre_all(lmax: int, ct: np.ndarray):
    """Normalised associated Legendre values Pbar_l^m(cos theta) for 0 <= m <= l <= lmax.

    Pbar includes sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) so that the real harmonics below are
    orthonormal. Standard three-term recurrence in l for fixed m, seeded by the sectoral terms.
    """
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    P = {}
    pmm = np.full_like(ct, math.sqrt(1.0 / (4.0 * math.pi)))
    for m in range(0, lmax + 1):
        if m > 0:
            pmm = -math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * st * pmm
        P[(m, m)] = pmm
        if m + 1 <= lmax:
            P[(m + 1, m)] = math.sqrt(2.0 * m + 3.0) * ct * pmm
        for l in range(m + 2, lmax + 1):
            a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            P[(l, m)] = a * (ct * P[(l - 1, m)] - b * P[(l - 2, m)])
    return P


def sh_real_all(x: np.ndarray, lmax: int):
    """Dict (l, m) -> real orthonormal Y_l^m at the directions of the rows of x, -l <= m <= l."""
    xn = x / np.linalg.norm(x, axis=1, keepdims=True)
    ct = np.clip(xn[:, 2], -1.0, 1.0)
    phi = np.arctan2(xn[:, 1], xn[:, 0])
    P = _legendre_all(lmax, ct)
    Y = {}
    for l in range(lmax + 1):
        Y[(l, 0)] = P[(l, 0)]
        for m in range(1, l + 1):
            Y[(l, m)] = math.sqrt(2.0) * P[(l, m)] * np.cos(m * phi)
            Y[(l, -m)] = math.sqrt(2.0) * P[(l, m)] * np.sin(m * phi)
    return Y


def sh_real(x: np.ndarray, l: int, m: int):
    return sh_real_all(x, l)[(l, m)]


def random_sh_rhs(x: np.ndarray, lmax: int = 20, seed: int = 2):
    """f = sum_{l <= lmax, |m| <= l} a_lm Y_l^m(x/|x|), a_lm ~ N(0, 1) drawn in (l, m) order.

    Evaluated with the same normalised recurrence as sh_real_all but keeping only two Legendre
    columns at a time, so memory stays O(N) for million-point clouds."""
    rng = np.random.default_rng(seed)
    a = {}
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            a[(l, m)] = rng.standard_normal()
    xn = x / np.linalg.norm(x, axis=1, keepdims=True)
    ct = np.clip(xn[:, 2], -1.0, 1.0)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    phi = np.arctan2(xn[:, 1], xn[:, 0])
    f = np.zeros(x.shape[0])
    pmm = np.full_like(ct, math.sqrt(1.0 / (4.0 * math.pi)))
    for m in range(0, lmax + 1):
        if m > 0:
            pmm = -math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * st * pmm
        cm, sm = (np.cos(m * phi), np.sin(m * phi)) if m > 0 else (None, None)

        def add(l, P):
            if m == 0:
                f.__iadd__(a[(l, 0)] * P)
            else:
                f.__iadd__(math.sqrt(2.0) * P * (a[(l, m)] * cm + a[(l, -m)] * sm))
        add(m, pmm)
        if m + 1 <= lmax:
            p1 = math.sqrt(2.0 * m + 3.0) * ct * pmm
            add(m + 1, p1)
            p0 = pmm
            for l in range(m + 2, lmax + 1):
                aa = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
                bb = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
                p2 = aa * (ct * p1 - bb * p0)
                add(l, p2)
                p0, p1 = p1, p2
    return f


def y43(x: np.ndarray):
    """Closed-form degree-4 harmonic polynomial z (x^3 - 3 x y^2): on the unit sphere it is a
    multiple of the real harmonic Y_4^3, so Lap_S y43 = -20 y43 there."""
    return x[:, 2] * (x[:, 0] ** 3 - 3.0 * x[:, 0] * x[:, 1] ** 2)


def y54(x: np.ndarray):
    """Closed-form z (x^4 - 6 x^2 y^2 + y^4) (paper Sec. 5.4): a multiple of Y_5^4 on the sphere,
    Lap_S y54 = -30 y54."""
    X, Yc, Z = x[:, 0], x[:, 1], x[:, 2]
    return Z * (X ** 4 - 6.0 * X ** 2 * Yc ** 2 + Yc ** 4)


# ----------------------------------------------------------------------------------------------
# Bumpy sphere: r(theta, phi) = 1 + amp * sum_{t<5} c_t Y_{l_t}^{m_t}, analytic normals
# ----------------------------------------------------------------------------------------------
def _bumpy_terms(seed: int, nterms: int = 5, lmax: int = 6):
    rng = np.random.default_rng(seed)
    terms = []
    for _ in range(nterms):
        l = int(rng.integers(1, lmax + 1))
        m = int(rng.integers(-l, l + 1))
        c = float(rng.uniform(-1.0, 1.0))
        terms.append((l, m, c))
    # scale so the perturbation stays within +-amp of the unit sphere
    return terms


def bumpy_sphere(N: int, seed: int = 3, amp: float = 0.2, jitter: float = 0.1):
    """Points r(x) x on a star-shaped surface, x from a jittered Fibonacci sphere.

    r(x) = 1 + amp * g(x) / max|g|, g = sum of 5 seeded c * Y_l^m (l <= 6). Normals come from the
    gradient of F(p) = |p| - r(p/|p|), using a centred finite difference of r along two tangent
    directions (step 1e-6), which is accurate to ~1e-10 and independent of the method.
    """
    x, _ = fibonacci_sphere(N, jitter=jitter, seed=seed)
    terms = _bumpy_terms(seed)

    def g(u):
        lm = max(t[0] for t in terms)
        Y = sh_real_all(u, lm)
        out = np.zeros(u.shape[0])
        for (l, m, c) in terms:
            out += c * Y[(l, m)]
        return out

    # normalise amplitude with a fixed dense probe set so the scale does not depend on N
    probe, _ = fibonacci_sphere(20000, jitter=0.0)
    scale = amp / np.max(np.abs(g(probe)))

    def r(u):
        return 1.0 + scale * g(u)

    rv = r(x)
    p = x * rv[:, None]
    a, b = _sphere_tangents(x)
    eps = 1e-6
    def surf(u):
        u = u / np.linalg.norm(u, axis=1, keepdims=True)
        return u * r(u)[:, None]
    ta = (surf(x + eps * a) - surf(x - eps * a)) / (2 * eps)
    tb = (surf(x + eps * b) - surf(x - eps * b)) / (2 * eps)
    n = np.cross(ta, tb)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    flip = np.sum(n * x, axis=1) < 0
    n[flip] *= -1.0
    return np.ascontiguousarray(p), np.ascontiguousarray(n)


def bumpy_torus(N: int, seed: int = 5, amp: float = 0.2, R: float = 1.0, r: float = 1.0 / 3.0, jitter: float = 0.1):
    """Torus whose tube radius varies: X(u, v) = ((R + rho cos v) cos u, (R + rho cos v) sin u,
    rho sin v) with rho(u, v) = r (1 + amp g(u, v) / max|g|), g = sum of 5 seeded modes
    c cos(a u + b v + phase) (a in 1..6, b in 1..4, c ~ N(0, 1)). The (u, v) samples are those of
    torus_grid (jittered parametric grid). Normals: cross product of centred finite differences
    of X in u and v (step 1e-6), oriented away from the tube's centre line."""
    rng = np.random.default_rng(seed)
    modes = [(int(rng.integers(1, 7)), int(rng.integers(1, 5)), float(rng.uniform(0, 2 * np.pi)),
              float(rng.standard_normal())) for _ in range(5)]

    def g(u, v):
        out = np.zeros(np.broadcast(u, v).shape)
        for (a, b, ph, c) in modes:
            out = out + c * np.cos(a * u + b * v + ph)
        return out

    pu = np.linspace(0, 2 * np.pi, 400, endpoint=False)
    PU, PV = np.meshgrid(pu, pu, indexing="ij")
    scale = amp / np.max(np.abs(g(PU, PV)))
    nu, nv = _torus_shape(N, R, r)
    u = 2.0 * np.pi * (np.arange(nu, dtype=np.float64) + 0.5) / nu
    v = 2.0 * np.pi * (np.arange(nv, dtype=np.float64) + 0.5) / nv
    U, V = np.meshgrid(u, v, indexing="ij")
    U = U.reshape(-1).copy()
    V = V.reshape(-1).copy()
    if jitter > 0.0:
        h = math.sqrt(4.0 * np.pi ** 2 * R * r / U.size)
        d = np.random.default_rng(seed + 1).uniform(-jitter * h, jitter * h, size=(U.size, 2))
        U = U + d[:, 0] / (R + r * np.cos(V))
        V = V + d[:, 1] / r

    def X(u, v):
        rho = r * (1.0 + scale * g(u, v))
        return np.stack([(R + rho * np.cos(v)) * np.cos(u), (R + rho * np.cos(v)) * np.sin(u), rho * np.sin(v)], axis=1)

    p = X(U, V)
    eps = 1e-6
    tu = (X(U + eps, V) - X(U - eps, V)) / (2 * eps)
    tv = (X(U, V + eps) - X(U, V - eps)) / (2 * eps)
    n = np.cross(tu, tv)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    centre = np.stack([R * np.cos(U), R * np.sin(U), np.zeros_like(U)], axis=1)
    flip = np.sum(n * (p - centre), axis=1) < 0
    n[flip] *= -1.0
    return np.ascontiguousarray(p), np.ascontiguousarray(n)


def mean_spacing(x: np.ndarray, area: float) -> float:
    return math.sqrt(area / x.shape[0])
