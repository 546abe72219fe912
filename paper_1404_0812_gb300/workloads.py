"""Seeded synthetic inputs: surface node sets, normals and initial states.

This module holds no arithmetic of the RBF-FD method itself. It only makes the
inputs that the CUDA path and the oracle both consume: scattered nodes on a
surface, unit normals at those nodes, stencil-size assignments and initial
fields. Every random draw goes through ``numpy.random.default_rng(seed)`` so a
(seed, size) pair always gives the same bytes.

Node sets and the sections of the paper they stand in for:

* icosahedral sphere (Section 6, "Diffusion on the sphere": N = 10*4^k + 2)
* staggered torus grid (Section 6, forced diffusion on a torus, Eq. torus and
  the four-step staggered-grid recipe; N = 6 m^2)
* spherical Fibonacci lattice (quasi-uniform sphere of any N; stands in for
  the maximal-determinant node sets of Section 5, which are not available)
* bumpy sphere r = 1 + 0.1 sin(3 theta) cos(4 phi) (theta colatitude, phi
  azimuth), analytic or PCA-estimated normals (stands in for the downloaded
  bumpy-sphere and scanned point clouds of Section 7)
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "NodeSet", "icosahedral_sphere", "fibonacci_sphere", "torus_staggered",
    "bumpy_sphere", "pca_normals", "uniform_field", "sph_harm_y32",
    "stencil_size_groups", "SCHNAKENBERG", "GRAY_SCOTT", "BARRIO_SPOTS",
    "schnakenberg_initial", "gray_scott_initial", "workload",
]


@dataclass
class NodeSet:
    """Nodes X (N x 3, float64, C-contiguous) and unit normals (N x 3)."""
    name: str
    X: np.ndarray
    normals: np.ndarray
    extra: dict

    @property
    def N(self) -> int:
        return int(self.X.shape[0])


# ----------------------------------------------------------------------------
# sphere node sets
# ----------------------------------------------------------------------------

def icosahedral_sphere(level: int) -> NodeSet:
    """Recursively subdivided icosahedron on the unit sphere.

    Each level splits every triangle into four at the edge midpoints and
    projects the new vertices radially onto the sphere.  N = 10*4^level + 2:
    level 3 -> 642, 4 -> 2562, 5 -> 10242, 6 -> 40962 (the N values used in
    Section 6).  Vertex order: the 12 icosahedron vertices, then new
    midpoints in creation order.  Exact normals are the positions.
    """
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    V = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                cache[key] = len(V) - 1
            return cache[key]

        new_faces = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = new_faces
    X = np.ascontiguousarray(np.array(V, dtype=np.float64))
    nrm = X / np.linalg.norm(X, axis=1, keepdims=True)
    return NodeSet(f"icosahedral_sphere_N{len(X)}", X, np.ascontiguousarray(nrm), {})


def _fibonacci_dirs(N: int) -> np.ndarray:
    i = np.arange(N, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / N
    golden = (1.0 + math.sqrt(5.0)) / 2.0
    az = 2.0 * math.pi * np.mod(i / golden, 1.0)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(az), s * np.sin(az), z], axis=1)


def fibonacci_sphere(N: int) -> NodeSet:
    """Spherical Fibonacci lattice: z_i = 1-(2i+1)/N, azimuth 2*pi*frac(i/golden).

    Quasi-uniform for any N; index order runs from the north to the south
    pole.  Exact normals are the positions.
    """
    X = np.ascontiguousarray(_fibonacci_dirs(N))
    return NodeSet(f"fibonacci_sphere_N{N}", X, X.copy(), {})


# ----------------------------------------------------------------------------
# torus (Section 6, Eq. torus, R = 1, r = 1/3)
# ----------------------------------------------------------------------------

def torus_staggered(m: int, R: float = 1.0, r: float = 1.0 / 3.0) -> NodeSet:
    """Staggered intrinsic grid on the torus of Eq. torus, N = 6 m^2.

    m angles in varphi and 3m in lambda on [-pi, pi) (the endpoint pi is
    dropped), their direct product, plus the same grid offset by pi/m in
    varphi and pi/(3m) in lambda.  x = (R + r cos vp) cos lam,
    y = (R + r cos vp) sin lam, z = r sin vp; unit normal
    (cos vp cos lam, cos vp sin lam, sin vp).  ``extra`` keeps (vp, lam).
    """
    vp1 = -math.pi + 2.0 * math.pi * np.arange(m) / m
    la1 = -math.pi + 2.0 * math.pi * np.arange(3 * m) / (3 * m)
    VP1, LA1 = np.meshgrid(vp1, la1, indexing="ij")
    VP2, LA2 = VP1 + math.pi / m, LA1 + math.pi / (3 * m)
    vp = np.concatenate([VP1.ravel(), VP2.ravel()])
    la = np.concatenate([LA1.ravel(), LA2.ravel()])
    rho = R + r * np.cos(vp)
    X = np.stack([rho * np.cos(la), rho * np.sin(la), r * np.sin(vp)], axis=1)
    nrm = np.stack([np.cos(vp) * np.cos(la), np.cos(vp) * np.sin(la), np.sin(vp)], axis=1)
    return NodeSet(f"torus_m{m}_N{len(X)}", np.ascontiguousarray(X),
                   np.ascontiguousarray(nrm), {"varphi": vp, "lam": la, "R": R, "r": r})


# ----------------------------------------------------------------------------
# bumpy sphere r = 1 + 0.1 sin(3 theta) cos(4 phi)
# ----------------------------------------------------------------------------

def _bumpy_radius(theta, phi):
    return 1.0 + 0.1 * np.sin(3.0 * theta) * np.cos(4.0 * phi)


def bumpy_sphere(N: int, jitter: float = 0.0, seed: int = 4,
                 normals: str = "analytic", pca_k: int = 20) -> NodeSet:
    """Bumpy sphere r(theta, phi) = 1 + 0.1 sin(3 theta) cos(4 phi).

    Directions come from the spherical Fibonacci lattice; with ``jitter`` > 0
    each direction is moved in its tangent plane by a Gaussian step of
    standard deviation ``jitter * h`` (h = sqrt(4 pi / N)) before the radius
    is applied.  ``normals="analytic"`` gives the unit normal of the
    parametric surface (defined at every sample, none of which sits exactly
    on a pole); ``normals="pca"`` estimates it from the ``pca_k`` nearest
    nodes (smallest principal axis of the local covariance), sign arbitrary.
    """
    d = _fibonacci_dirs(N)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        h = math.sqrt(4.0 * math.pi / N)
        g = rng.standard_normal((N, 3)) * (jitter * h)
        g -= np.sum(g * d, axis=1, keepdims=True) * d
        d = d + g
        d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
    phi = np.arctan2(d[:, 1], d[:, 0])
    r = _bumpy_radius(theta, phi)
    X = d * r[:, None]
    if normals == "analytic":
        st, ct = np.sin(theta), np.cos(theta)
        sp, cp = np.sin(phi), np.cos(phi)
        e_r = np.stack([st * cp, st * sp, ct], axis=1)
        e_t = np.stack([ct * cp, ct * sp, -st], axis=1)
        e_p = np.stack([-sp, cp, np.zeros_like(sp)], axis=1)
        r_t = 0.3 * np.cos(3.0 * theta) * np.cos(4.0 * phi)
        r_p = -0.4 * np.sin(3.0 * theta) * np.sin(4.0 * phi)
        nv = e_r - (r_t / r)[:, None] * e_t - (r_p / (r * st))[:, None] * e_p
        nrm = nv / np.linalg.norm(nv, axis=1, keepdims=True)
    elif normals == "pca":
        nrm = pca_normals(X, pca_k)
    else:
        raise ValueError(normals)
    tag = f"bumpy_sphere_N{N}" + (f"_jit{jitter}" if jitter > 0 else "") + f"_{normals}"
    return NodeSet(tag, np.ascontiguousarray(X), np.ascontiguousarray(nrm), {})


def pca_normals(X: np.ndarray, k: int = 20) -> np.ndarray:
    """Unit normals from the k nearest nodes: eigenvector of the smallest
    eigenvalue of the neighbourhood covariance.  Input preparation only."""
    from scipy.spatial import cKDTree
    tree = cKDTree(X)
    out = np.empty_like(X)
    chunk = 65536
    for s in range(0, len(X), chunk):
        _, nb = tree.query(X[s:s + chunk], k=k, workers=-1)
        P = X[nb]
        P = P - P.mean(axis=1, keepdims=True)
        C = np.einsum("nki,nkj->nij", P, P)
        _, vec = np.linalg.eigh(C)
        out[s:s + chunk] = vec[:, :, 0]
    out /= np.linalg.norm(out, axis=1, keepdims=True)
    return np.ascontiguousarray(out)


# ----------------------------------------------------------------------------
# fields and stencil-size groups
# ----------------------------------------------------------------------------

def uniform_field(N: int, seed: int = 1) -> np.ndarray:
    """u ~ U[-1, 1] (float64)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, N)


def sph_harm_y32(X: np.ndarray) -> np.ndarray:
    """Real degree-3 order-2 spherical harmonic up to normalisation:
    z (x^2 - y^2) on the unit sphere (eigenvalue -l(l+1) = -12)."""
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    return z * (x * x - y * y)


def sectoral_harmonic(X: np.ndarray, l: int) -> np.ndarray:
    """Real orthonormal sectoral spherical harmonic of degree and order l on
    the unit sphere, Y_ll = c_l cos(lat)^l cos(l lon) = c_l Re((x + i y)^l),
    c_l^2 = (2l+1)!! / (2 pi (2l)!!) (no Condon-Shortley sign).  A harmonic
    homogeneous polynomial: Delta_S2 Y_ll = -l(l+1) Y_ll."""
    c2 = 1.0 / (2.0 * np.pi)
    for k in range(1, l + 1):
        c2 *= (2.0 * k + 1.0) / (2.0 * k)
    w = (X[:, 0] + 1j * X[:, 1]) ** l
    return np.sqrt(c2) * w.real


def sphere_heat_series(X: np.ndarray, t: float, terms: int = 30) -> np.ndarray:
    """Section 6's heat-equation test on the unit sphere (from MacDonald and
    Ruuth): u(t) = 20/(3 pi) sum_{l=1}^{terms} exp(-l^2/9) exp(-t l(l+1)) Y_ll,
    the exact solution of u_t = Delta_S2 u, truncated after 30 terms."""
    u = np.zeros(X.shape[0])
    for l in range(1, terms + 1):
        u += np.exp(-l * l / 9.0 - t * l * (l + 1)) * sectoral_harmonic(X, l)
    return (20.0 / (3.0 * np.pi)) * u


def sphere_forced_centers(K: int = 23, seed: int = 6) -> np.ndarray:
    """K seeded uniformly random unit vectors (the centres xi_k of Section 6's
    forced sphere problem)."""
    v = np.random.default_rng(seed).normal(size=(K, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def sphere_forced(X: np.ndarray, centers: np.ndarray):
    """Section 6's manufactured forced-diffusion solution on the unit sphere,
    u(t, x) = exp(-5 t) g(x), g = sum_k exp(-10 theta_k^2), theta_k the
    geodesic distance arccos(xi_k . x) (the exponent read as squared: the
    printed exp(-10 theta_k) has a cusp at every centre, while the text calls
    the solution smooth).  Returns (g, h) with h = -5 g - Delta_S2 g, so that
    u_t = Delta u + exp(-5 t) h; for a zonal G(theta),
    Delta G = G'' + cot(theta) G'."""
    g = np.zeros(X.shape[0])
    lap = np.zeros(X.shape[0])
    for xi in centers:
        c = np.clip(X @ xi, -1.0, 1.0)
        th = np.arccos(c)
        G = np.exp(-10.0 * th * th)
        sn = np.sqrt(np.maximum(0.0, 1.0 - c * c))
        # theta cot(theta) -> 1 at the centre; the antipode's G is ~1e-43
        tcot = np.where(th < 1e-8, 1.0, np.where(sn > 1e-12, th * c / np.maximum(sn, 1e-300), 0.0))
        g += G
        lap += G * (-20.0 + 400.0 * th * th - 20.0 * tcot)
    return g, -5.0 * g - lap


def torus_angles(X: np.ndarray, R: float = 1.0):
    """Intrinsic coordinates (phi, lambda) of points on the torus of Eq. torus."""
    lam = np.arctan2(X[:, 1], X[:, 0])
    rho = np.sqrt(X[:, 0] ** 2 + X[:, 1] ** 2) - R
    return np.arctan2(X[:, 2], rho), lam


def torus_forced_centers(K: int = 23, seed: int = 7) -> np.ndarray:
    """(phi_k, lambda_k) uniformly random in [-pi, pi]^2 (seeded), K x 2."""
    return np.random.default_rng(seed).uniform(-np.pi, np.pi, size=(K, 2))


def torus_forced(X: np.ndarray, centers: np.ndarray, a: float = 9.0, b: float = 3.0):
    """Section 6's manufactured forced-diffusion solution on the torus (Eq.
    torus_forced): u = exp(-5 t) g, g = sum_k exp(-a^2 (1 - cos(lambda -
    lambda_k)) - b^2 (1 - cos(phi - phi_k))).  Returns (g, h), h = -5 g -
    Delta_M g with the intrinsic Laplacian of Section 6 (R = 1, r = 1/3):
    Delta f = f_ll / rho^2 + 9 (rho'/rho f_p + f_pp), rho = 1 + cos(phi)/3."""
    phi, lam = torus_angles(X)
    rho = 1.0 + np.cos(phi) / 3.0
    drho = -np.sin(phi) / 3.0
    g = np.zeros(X.shape[0])
    lap = np.zeros(X.shape[0])
    for pk_, lk in centers:
        L, P = lam - lk, phi - pk_
        E = np.exp(-a * a * (1.0 - np.cos(L)) - b * b * (1.0 - np.cos(P)))
        El = -a * a * np.sin(L) * E
        Ell = (-a * a * np.cos(L) + a ** 4 * np.sin(L) ** 2) * E
        Ep = -b * b * np.sin(P) * E
        Epp = (-b * b * np.cos(P) + b ** 4 * np.sin(P) ** 2) * E
        g += E
        lap += Ell / rho ** 2 + 9.0 * (drho / rho * Ep + Epp)
        del El
    return g, -5.0 * g - lap


def stencil_size_groups(N: int, sizes=(31, 50, 70, 101)) -> np.ndarray:
    """Per-node stencil size for the mixed-n batched build: the node index
    range is cut into len(sizes) contiguous blocks of (nearly) equal length;
    block g gets sizes[g].  On a Fibonacci lattice each block is a latitude
    band.  Returns int32 (N,)."""
    g = (np.arange(N, dtype=np.int64) * len(sizes)) // N
    return np.asarray(sizes, dtype=np.int32)[g]


# ----------------------------------------------------------------------------
# reaction models (parameters chosen for the synthetic workloads)
# ----------------------------------------------------------------------------

# Schnakenberg:  f = gamma (a - u + u^2 v),  g = gamma (b - u^2 v)
# steady state (a + b, b / (a + b)^2).  d = du/dv chosen inside the Turing
# space of the linearisation for a = 0.1, b = 0.9.
SCHNAKENBERG = dict(model="schnakenberg", a=0.1, b=0.9, gamma=1.0,
                    delta_u=2.5e-4, delta_v=1.0e-2, dt=0.01)
# Gray-Scott: f = -u v^2 + F (1 - u),  g = u v^2 - (F + k) v
GRAY_SCOTT = dict(model="gray_scott", F=0.04, k=0.06,
                  delta_u=2.0e-5, delta_v=1.0e-5, dt=1.0)
# Paper's Turing kinetics (Eqs. turing1/2, Table tur_param, bumpy sphere/spots)
BARRIO_SPOTS = dict(model="barrio", alpha=0.899, beta=-0.91, gamma=-0.899,
                    tau1=0.02, tau2=0.2, delta_v=4.5e-3,
                    delta_u=0.516 * 4.5e-3, dt=0.01)


def schnakenberg_initial(N: int, seed: int = 2, p=SCHNAKENBERG):
    """Steady state times (1 + 0.01 U[-1,1]) for each species (seeded)."""
    rng = np.random.default_rng(seed)
    u0 = p["a"] + p["b"]
    v0 = p["b"] / (p["a"] + p["b"]) ** 2
    u = u0 * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, N))
    v = v0 * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, N))
    return u, v


def gray_scott_initial(X: np.ndarray, seed: int = 5, spots: int = 50,
                       radius: float = 0.05):
    """u = 1, v = 0 with ``spots`` random discs (u = 0.5, v = 0.25) of the
    given chord radius around seeded random surface nodes."""
    rng = np.random.default_rng(seed)
    N = len(X)
    u = np.ones(N)
    v = np.zeros(N)
    centres = X[rng.choice(N, size=spots, replace=False)]
    for c in centres:
        m = np.sum((X - c) ** 2, axis=1) < radius * radius
        u[m] = 0.5
        v[m] = 0.25
    return u, v


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def workload(name: str) -> NodeSet:
    """Named node sets of the five benchmark configurations (and small ones).

    sphere2562      icosahedral unit sphere, N = 2562 (n = 31, Gaussian)
    torus40344      staggered torus m = 82, N = 40,344 (n = 50)
    fib1m           Fibonacci unit sphere, N = 1,000,000 (mixed n)
    bumpy500k       bumpy sphere N = 500,000, analytic normals (n = 50)
    bumpy2m         bumpy sphere N = 2,000,000, jitter 0.25 h, PCA normals
    """
    if name == "sphere2562":
        return icosahedral_sphere(4)
    if name == "torus40344":
        return torus_staggered(82)
    if name == "fib1m":
        return fibonacci_sphere(1_000_000)
    if name == "bumpy500k":
        return bumpy_sphere(500_000)
    if name == "bumpy2m":
        return bumpy_sphere(2_000_000, jitter=0.25, seed=4, normals="pca")
    raise KeyError(name)


# ----------------------------------------------------------------------------
# MLP parameter initialisation and flat layout (learned eps warm start)
# ----------------------------------------------------------------------------

MLP_HIDDEN = 64
MLP_KEYS = ("W1", "b1", "W2", "b2", "W3", "b3")


def mlp_shapes(D: int, hidden: int = MLP_HIDDEN):
    """Parameter shapes of the D -> hidden -> hidden -> 1 network."""
    return {"W1": (D, hidden), "b1": (hidden,), "W2": (hidden, hidden),
            "b2": (hidden,), "W3": (hidden, 1), "b3": (1,)}


def mlp_init(D: int, seed: int = 0, hidden: int = MLP_HIDDEN) -> dict:
    """Seeded initial parameters: W ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)),
    biases 0.  float64."""
    rng = np.random.default_rng(seed)
    out = {}
    for k, shp in mlp_shapes(D, hidden).items():
        if k.startswith("W"):
            lim = 1.0 / math.sqrt(shp[0])
            out[k] = rng.uniform(-lim, lim, shp)
        else:
            out[k] = np.zeros(shp)
    return out


def mlp_pack(params: dict) -> np.ndarray:
    """Flat layout shared by the C ABI: W1 (row-major D x H), b1, W2 (H x H),
    b2, W3 (H), b3 (1)."""
    return np.concatenate([np.asarray(params[k]).reshape(-1) for k in MLP_KEYS])


def mlp_unpack(flat: np.ndarray, D: int, hidden: int = MLP_HIDDEN) -> dict:
    out, o = {}, 0
    for k, shp in mlp_shapes(D, hidden).items():
        sz = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + sz], dtype=np.float64).reshape(shp)
        o += sz
    return out
