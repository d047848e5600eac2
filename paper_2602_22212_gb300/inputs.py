"""Seeded synthetic inputs: reference meshes, point-cloud sequences, MLP init.

This module serves both the CUDA path and the FP64 oracle and holds none of the
method's arithmetic: it only builds the data the method consumes (Sec. 3,
problem statement): a keyframe reference mesh (vertices in [-1, 1]^3, unit
vertex normals, triangles), T point clouds, the keyframe index, and the random
MLP initialisation with a zeroed last layer (Sec. 3.1).

The paper's datasets (DFAUST, AMA, DT4D) are not available; two generators
stand in for them with the shapes of the paper's workloads (17-120 frames,
2500-20000 points per frame, noise relative to the bounding-box diagonal):

* ``sphere_blob``: an icosphere under three smooth localized rotations plus a
  sinusoidal radial bulge.
* ``figure``: a five-limbed capsule figure (torso, head, two arms, two legs
  merged by a smooth union), meshed by radial projection of an icosphere and
  animated by linear blend skinning with per-joint sinusoidal angles.

All frames are scaled jointly into [-0.95, 0.95]^3. Points are area-uniform
samples of the posed mesh plus isotropic Gaussian noise.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# --------------------------------------------------------------- meshes

def icosphere(subdiv: int):
    """Unit icosphere: 10 * 4^subdiv + 2 vertices, outward-oriented faces."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    verts = [tuple(p) for p in v]
    for _ in range(subdiv):
        cache = {}
        vl = verts

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                p = (np.array(vl[a]) + np.array(vl[b])) * 0.5
                p /= np.linalg.norm(p)
                cache[key] = len(vl)
                vl.append(tuple(p))
            return cache[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        f = np.array(nf, dtype=np.int64)
    v = np.array(verts, dtype=np.float64)
    # orient outward
    n = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    flip = np.einsum("ij,ij->i", n, v[f[:, 0]]) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    return v, f.astype(np.int32)


def fibonacci_sphere(n: int):
    """n points on the unit sphere along the golden-angle spiral, triangulated
    by their convex hull (outward-oriented faces): a sphere mesh of any size."""
    from scipy.spatial import ConvexHull
    k = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(np.maximum(1.0 - z * z, 0.0))
    phi = np.pi * (3.0 - 5.0 ** 0.5) * k
    v = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    f = ConvexHull(v).simplices.astype(np.int64)
    nrm = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    flip = np.einsum("ij,ij->i", nrm, v[f[:, 0]]) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    return v, f.astype(np.int32)


def sphere_mesh(subdiv=4, n_vertices=None):
    """Icosphere of the given subdivision, or a Fibonacci sphere of n_vertices."""
    return icosphere(subdiv) if n_vertices is None else fibonacci_sphere(int(n_vertices))


def vertex_normals(v, f):
    """Area-weighted vertex normals (unit length)."""
    n = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    vn = np.zeros_like(v)
    for k in range(3):
        np.add.at(vn, f[:, k], n)
    nrm = np.linalg.norm(vn, axis=1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return vn / nrm


def sample_surface(v, f, M, rng):
    """M area-uniform samples on a triangle mesh (square-root barycentrics)."""
    a = np.linalg.norm(np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]]), axis=1)
    tri = rng.choice(len(f), size=M, p=a / a.sum())
    r1, r2 = rng.random(M), rng.random(M)
    s = np.sqrt(r1)
    w0, w1, w2 = 1.0 - s, s * (1.0 - r2), s * r2
    F = f[tri]
    return w0[:, None] * v[F[:, 0]] + w1[:, None] * v[F[:, 1]] + w2[:, None] * v[F[:, 2]]


def _rot(axis, ang):
    """Rotation matrices about unit axis (3,) by angles ang (...,): Rodrigues."""
    ang = np.asarray(ang, dtype=np.float64)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    s, c = np.sin(ang)[..., None, None], np.cos(ang)[..., None, None]
    return np.eye(3) + s * K + (1 - c) * (K @ K)


def _unit(rng, n=None):
    u = rng.normal(size=(3,) if n is None else (n, 3))
    return u / np.linalg.norm(u, axis=-1, keepdims=True)


# --------------------------------------------------------------- sequences

@dataclass
class Sequence:
    """One synthetic sequence: keyframe reference mesh + T point clouds."""
    x: np.ndarray            # N x 3 float32, reference vertices at t_key
    n: np.ndarray            # N x 3 float32, unit vertex normals
    faces: np.ndarray        # F x 3 int32
    points: np.ndarray       # sum(M_t) x 3 float32, frames concatenated
    offsets: np.ndarray      # T + 1 int64
    t_key: int
    gt_frames: np.ndarray = field(repr=False, default=None)  # T x N x 3, clean posed vertices

    @property
    def N(self):
        return len(self.x)

    @property
    def T(self):
        return len(self.offsets) - 1


def _finish(frames, f, t_key, M, noise_rel, noise_abs, rng):
    """Joint scaling into [-0.95, 0.95]^3, point sampling, noise."""
    T = len(frames)
    s = 0.95 / np.abs(frames).max()
    frames = frames * s
    Ms = [M] * T if np.isscalar(M) else list(M)
    clouds = [sample_surface(frames[t], f, Ms[t], rng) for t in range(T)]
    lo = np.min([c.min(0) for c in clouds], axis=0)
    hi = np.max([c.max(0) for c in clouds], axis=0)
    sigma = noise_abs if noise_abs is not None else noise_rel * float(np.linalg.norm(hi - lo))
    clouds = [c + rng.normal(scale=sigma, size=c.shape) for c in clouds]
    pts = np.concatenate(clouds).astype(np.float32)
    off = np.zeros(T + 1, dtype=np.int64)
    off[1:] = np.cumsum(Ms)
    x = frames[t_key]
    n = vertex_normals(x, f)
    return Sequence(x=x.astype(np.float32), n=n.astype(np.float32), faces=f.astype(np.int32),
                    points=pts, offsets=off, t_key=int(t_key), gt_frames=frames)


def sphere_blob(subdiv=4, T=8, M=4096, noise=0.005, seed=0, t_key=None, n_vertices=None):
    """Icosphere under three localized smooth rotations (centre c_k on the
    sphere, radius r_k ~ U(0.3, 0.8), random axis, angle 0.5 sin(2 pi t~ + phi_k)
    falling off as exp(-|x - c_k|^2 / r_k^2)) and a radial bulge of amplitude
    0.1; noise is an absolute standard deviation."""
    rng = np.random.default_rng(seed)
    v0, f = sphere_mesh(subdiv, n_vertices)
    cs = _unit(rng, 3)
    rs = rng.uniform(0.3, 0.8, size=3)
    axes = _unit(rng, 3)
    ph = rng.uniform(0, 2 * np.pi, size=3)
    u = _unit(rng)
    phb = rng.uniform(0, 2 * np.pi)
    frames = []
    for t in range(T):
        tt = t / (T - 1) if T > 1 else 0.0
        x = v0.copy()
        for k in range(3):
            th = 0.5 * np.sin(2 * np.pi * tt + ph[k])
            fall = np.exp(-np.sum((x - cs[k]) ** 2, axis=1) / rs[k] ** 2)
            R = _rot(axes[k], th * fall)
            x = cs[k] + np.einsum("nij,nj->ni", R, x - cs[k])
        x = x * (1.0 + 0.1 * np.sin(2 * np.pi * tt + phb) * np.sin(3.0 * (x @ u)))[:, None]
        frames.append(x)
    frames = np.array(frames)
    if t_key is None:
        t_key = T // 2
    return _finish(frames, f, t_key, M, None, noise, rng)


# capsule figure in a star pose: every limb is radial from the torso centre,
# so the smooth union is star-shaped about the origin
def _limb_defs():
    limbs = [((0.0, -0.30, 0.0), (0.0, 0.30, 0.0), 0.22)]
    dirs = [((0.0, 1.0, 0.0), 0.34, 0.62, 0.14),
            ((1.0, 0.35, 0.0), 0.15, 0.88, 0.07), ((-1.0, 0.35, 0.0), 0.15, 0.88, 0.07),
            ((0.35, -1.0, 0.0), 0.20, 0.92, 0.09), ((-0.35, -1.0, 0.0), 0.20, 0.92, 0.09)]
    for d, s0, s1, r in dirs:
        d = np.array(d) / np.linalg.norm(d)
        limbs.append((tuple(d * s0), tuple(d * s1), r))
    return [(np.array(a, dtype=np.float64), np.array(b, dtype=np.float64), r) for a, b, r in limbs]


def _seg_dist(p, a, b):
    ab = b - a
    h = np.clip(((p - a) @ ab) / (ab @ ab), 0.0, 1.0)
    return np.linalg.norm(p - (a + h[..., None] * ab), axis=-1)


def _figure_sdf(p, limbs, k=0.08):
    d = None
    for a, b, r in limbs:
        di = _seg_dist(p, a, b) - r
        if d is None:
            d = di
        else:  # polynomial smooth minimum
            h = np.maximum(k - np.abs(d - di), 0.0) / k
            d = np.minimum(d, di) - h * h * k * 0.25
    return d


def figure_mesh(subdiv=6, n_vertices=None):
    """Sphere mesh radially projected onto the capsule figure's zero level set."""
    limbs = _limb_defs()
    u, f = sphere_mesh(subdiv, n_vertices)
    rho = np.linspace(0.0, 1.6, 321)
    vals = np.stack([_figure_sdf(u * r, limbs) for r in rho], axis=1)  # N x S
    sign = vals > 0
    changes = np.count_nonzero(sign[:, 1:] != sign[:, :-1], axis=1)
    if np.any(changes != 1):
        raise RuntimeError("capsule figure is not star-shaped about its centre")
    k = np.argmax(sign, axis=1)  # first outside sample
    lo, hi = rho[k - 1].copy(), rho[k].copy()
    for _ in range(40):
        m = 0.5 * (lo + hi)
        out = _figure_sdf(u * m[:, None], limbs) > 0
        hi = np.where(out, m, hi)
        lo = np.where(out, lo, m)
    v = u * (0.5 * (lo + hi))[:, None]
    return v, f, limbs


def figure(subdiv=6, T=100, M=20000, noise_rel=0.003, seed=0, t_key=None, amp_deg=60.0,
           n_vertices=None):
    """Capsule figure animated by linear blend skinning: each limb rotates
    about its proximal joint by amp sin(2 pi f t~ + phi) about a random axis
    (amp <= amp_deg, f in {1, 2}); skinning weights softmax(-d_k^2 / s^2) over
    the distances to the capsule segments; plus a slow global sway."""
    rng = np.random.default_rng(seed)
    v, f, limbs = figure_mesh(subdiv, n_vertices)
    n_l = len(limbs)
    d2 = np.stack([_seg_dist(v, a, b) ** 2 for a, b, _ in limbs], axis=1)
    s2 = 0.08 ** 2
    wts = np.exp(-(d2 - d2.min(axis=1, keepdims=True)) / s2)
    wts /= wts.sum(axis=1, keepdims=True)
    axes = _unit(rng, n_l)
    amps = np.deg2rad(rng.uniform(0.3, 1.0, size=n_l) * amp_deg)
    freqs = rng.integers(1, 3, size=n_l)
    ph = rng.uniform(0, 2 * np.pi, size=n_l)
    sway_ax = _unit(rng)
    frames = []
    for t in range(T):
        tt = t / (T - 1) if T > 1 else 0.0
        x = wts[:, :1] * v  # torso: identity
        for k in range(1, n_l):
            j = limbs[k][0]
            R = _rot(axes[k], amps[k] * np.sin(2 * np.pi * freqs[k] * tt + ph[k]))
            x = x + wts[:, k:k + 1] * ((v - j) @ R.T + j)
        Rg = _rot(sway_ax, 0.25 * np.sin(2 * np.pi * tt))
        frames.append(x @ Rg.T)
    frames = np.array(frames)
    if t_key is None:
        t_key = T // 2
    return _finish(frames, f, t_key, M, noise_rel, None, rng)


def random_cloud_sequence(N=40, T=3, M=30, seed=0, faces_from_sphere=True):
    """Tiny problem for oracle self-tests and kernel edge cases: a small
    icosphere (subdiv 1: 42 vertices) jittered, with uniform random clouds."""
    rng = np.random.default_rng(seed)
    v, f = icosphere(1)
    v = 0.6 * v + rng.normal(scale=0.02, size=v.shape)
    n = vertex_normals(v, f)
    Ms = [M] * T if np.isscalar(M) else list(M)
    pts = np.concatenate([rng.uniform(-0.8, 0.8, size=(m, 3)) for m in Ms]).astype(np.float32)
    off = np.zeros(T + 1, dtype=np.int64)
    off[1:] = np.cumsum(Ms)
    return Sequence(x=v.astype(np.float32), n=n.astype(np.float32), faces=f, points=pts,
                    offsets=off, t_key=T // 2)


# --------------------------------------------------------------- parameters

def linear_resolutions(L, r_min, r_max):
    """Per-level node counts r_l = round(r_min + (r_max - r_min)(l-1)/(L-1))."""
    if L == 1:
        return [int(r_max)]
    return [int(round(r_min + (r_max - r_min) * l / (L - 1))) for l in range(L)]


def mlp_init(k_in, H, D, n_out, seed=0, zero_last=True):
    """Flat FP32 MLP parameters: layer 0 W (H x k_in) + b, hidden layers
    W (H x H) + b, output W (n_out x H) + b; entries ~ U(+-1/sqrt(fan_in));
    the output layer's weights and bias are zero (Sec. 3.1) unless
    zero_last is False."""
    rng = np.random.default_rng(seed)
    parts = []
    dims = [(H, k_in)] + [(H, H)] * (D - 1)
    for o, i in dims:
        b = 1.0 / np.sqrt(i)
        parts += [rng.uniform(-b, b, size=o * i), rng.uniform(-b, b, size=o)]
    b = 1.0 / np.sqrt(H)
    if zero_last:
        parts += [np.zeros(n_out * H), np.zeros(n_out)]
    else:
        parts += [rng.uniform(-b, b, size=n_out * H), rng.uniform(-b, b, size=n_out)]
    return np.concatenate(parts).astype(np.float32)


def random_grid(n, scale=0.1, seed=0):
    """Random grid values (for parity tests away from the zero initialisation)."""
    rng = np.random.default_rng(seed)
    return rng.normal(scale=scale, size=n).astype(np.float32)


# --------------------------------------------------------------- presets

def preset(name):
    """Workload presets (sizes, schedules and hyper-parameters)."""
    if name == "tiny":      # 2562 vertices, 8 frames, 4096 points per frame
        return dict(gen="sphere_blob", subdiv=4, T=8, M=4096, noise=0.005, L=4,
                    res=linear_resolutions(4, 8, 64), F=2, H=64, D=2, slope=0.0, iters=10)
    if name == "paper":     # 40962 vertices, 100 frames, 20000 points per frame
        return dict(gen="figure", subdiv=6, T=100, M=20000, noise_rel=0.003, L=8,
                    res=linear_resolutions(8, 16, 256), F=4, H=64, D=3, slope=0.01, iters=500,
                    w_iso=1.0)
    if name == "long":      # 20000 vertices, 1000 frames, 10000 points per frame, MLP 3 x 128
        return dict(gen="figure", n_vertices=20000, T=1000, M=10000, noise_rel=0.003, L=8,
                    res=linear_resolutions(8, 16, 256), F=4, H=128, D=3, slope=0.01, iters=300,
                    w_iso=1.0)
    if name == "stress":    # 100000 vertices, 200 frames, 100000 points per frame
        return dict(gen="figure", n_vertices=100000, T=200, M=100000, noise_rel=0.003, L=8,
                    res=linear_resolutions(8, 16, 256), F=4, H=64, D=3, slope=0.01, iters=500,
                    w_iso=1.0)
    if name == "profile":   # 10242 vertices, 10 frames, 20000 points: search kernels at moderate size
        return dict(gen="figure", subdiv=5, T=10, M=20000, noise_rel=0.003, L=4,
                    res=linear_resolutions(4, 16, 64), F=4, H=64, D=3, slope=0.01, iters=500,
                    w_iso=1.0)
    raise KeyError(name)


def batch_specs(n=16, seed=0):
    """Sizes of the uneven-sequence batch: N ~ U[5000, 50000] vertices (Fibonacci
    spheres), T ~ U[50, 500] frames, M ~ U[5000, 30000] points per frame; even
    sequences use the sphere-blob generator, odd ones the capsule figure."""
    rng = np.random.default_rng(seed)
    return [dict(gen="sphere_blob" if s % 2 == 0 else "figure",
                 n_vertices=int(rng.integers(5000, 50001)), T=int(rng.integers(50, 501)),
                 M=int(rng.integers(5000, 30001)), seed=1000 + s) for s in range(n)]


def make_batch_sequence(spec):
    if spec["gen"] == "sphere_blob":
        return sphere_blob(T=spec["T"], M=spec["M"], noise=0.005, seed=spec["seed"],
                           n_vertices=spec["n_vertices"])
    return figure(T=spec["T"], M=spec["M"], noise_rel=0.003, seed=spec["seed"],
                  n_vertices=spec["n_vertices"])


def make_sequence(p, seed=0):
    if p["gen"] == "sphere_blob":
        return sphere_blob(subdiv=p["subdiv"], T=p["T"], M=p["M"], noise=p["noise"], seed=seed)
    return figure(subdiv=p.get("subdiv", 6), T=p["T"], M=p["M"], noise_rel=p["noise_rel"],
                  seed=seed, n_vertices=p.get("n_vertices"))
