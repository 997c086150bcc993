"""Seeded synthetic flow windows shaped like VOLDOR's workloads.

Analytic ray casting against planar patches, axis-aligned boxes and infinite
planes (no graphics API). For every frame pair (t-1, t) the generator casts
the rays of camera t-1, moves the hit points (static scene, moving boxes and
image-space non-rigid patches) and projects them into camera t, which gives
the flow X_t on the grid of I_{t-1} (Sec. 3 of the paper). Residual noise is
drawn from the Fisk model of Sec. 4: a squared end-point error with
alpha = a1 exp(a2 n), beta = b1 n + b2 at the true flow magnitude n (capped at
40 px for drawing), in a uniformly random direction; the drawn end-point error
is capped at 1e4 px (the Fisk tail is unbounded, and a flow must stay finite in
FP16).

This module is an input generator only: it feeds the oracle and the CUDA path
alike and implements none of the inference.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FISK_A1, FISK_A2, FISK_B1, FISK_B2 = 0.01, 0.09, -0.0022, 1.0
NOISE_N_CAP = 40.0
EPE_CAP = 1.0e4


@dataclass
class Window:
    flows: np.ndarray          # (T, H, W, 2) float64, X_t at index t-1 on the grid of I_{t-1}
    K: tuple                   # (fx, fy, cx, cy)
    poses: np.ndarray          # (T, 4, 4) true T_t: camera t-1 -> camera t
    depth0: np.ndarray         # (H, W) true z-depth of I_0
    rigid: np.ndarray          # (T, H, W) bool: pixel of I_{t-1} follows the static scene
    inv_depth_range: tuple     # (inv_min, inv_max) for depth sampling
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def T(self):
        return self.flows.shape[0]

    @property
    def H(self):
        return self.flows.shape[1]

    @property
    def W(self):
        return self.flows.shape[2]


# ---------------------------------------------------------------------------
# primitives (world = camera-0 frame; x right, y down, z forward)
# ---------------------------------------------------------------------------
class _Plane:
    def __init__(self, point, normal, u=None, v=None, hu=None, hv=None):
        self.c = np.asarray(point, float)
        self.n = np.asarray(normal, float) / np.linalg.norm(normal)
        self.bounded = u is not None
        if self.bounded:
            self.u = np.asarray(u, float) / np.linalg.norm(u)
            self.v = np.asarray(v, float) / np.linalg.norm(v)
            self.hu, self.hv = float(hu), float(hv)

    def hit(self, o, d, frame):
        den = d @ self.n
        with np.errstate(divide="ignore", invalid="ignore"):
            t = ((self.c - o) @ self.n) / den
        t = np.where(np.abs(den) > 1e-12, t, np.inf)
        if self.bounded:
            # in-plane coordinates of o + t d relative to the centre, per axis
            qu = (o - self.c) @ self.u + t * (d @ self.u)
            qv = (o - self.c) @ self.v + t * (d @ self.v)
            ok = (np.abs(qu) <= self.hu) & (np.abs(qv) <= self.hv)
            t = np.where(ok, t, np.inf)
        return np.where(t > 1e-6, t, np.inf)

    def offset(self, frame):
        return np.zeros(3)

    def corners(self, frame):
        if not self.bounded:
            return None
        return np.array([self.c + su * self.hu * self.u + sv * self.hv * self.v
                         for su in (-1, 1) for sv in (-1, 1)])


class _Box:
    """Axis-aligned box; a moving box translates by `vel` per frame."""

    def __init__(self, lo, hi, vel=(0.0, 0.0, 0.0)):
        self.lo = np.asarray(lo, float)
        self.hi = np.asarray(hi, float)
        self.vel = np.asarray(vel, float)
        self.moving = bool(np.any(self.vel != 0))

    def offset(self, frame):
        return self.vel * frame

    def corners(self, frame):
        off = self.offset(frame)
        lo, hi = self.lo + off, self.hi + off
        return np.array([[(lo, hi)[i][0], (lo, hi)[j][1], (lo, hi)[k][2]]
                         for i in (0, 1) for j in (0, 1) for k in (0, 1)])

    def hit(self, o, d, frame):
        off = self.offset(frame)
        lo, hi = self.lo + off, self.hi + off
        tmin = tmax = None
        with np.errstate(divide="ignore", invalid="ignore"):
            for k in range(3):            # slab test per axis; fmax / fmin ignore NaN
                inv = 1.0 / d[:, k]
                t1 = (lo[k] - o[k]) * inv
                t2 = (hi[k] - o[k]) * inv
                a, b = np.minimum(t1, t2), np.maximum(t1, t2)
                tmin = a if tmin is None else np.fmax(tmin, a)
                tmax = b if tmax is None else np.fmin(tmax, b)
        ok = (tmax >= tmin) & (tmax > 1e-6)
        t = np.where(tmin > 1e-6, tmin, tmax)
        return np.where(ok, t, np.inf)


def _rot(axis, angle):
    axis = np.asarray(axis, float)
    axis = axis / np.linalg.norm(axis)
    Kx = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(angle) * Kx + (1 - np.cos(angle)) * Kx @ Kx


def _rand_dir(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def _fisk_noise(rng, n_true):
    """Squared EPE ~ Fisk(alpha(n), beta(n)) by inverse CDF, random direction."""
    n = np.minimum(n_true, NOISE_N_CAP)
    alpha = FISK_A1 * np.exp(FISK_A2 * n)
    beta = np.maximum(FISK_B1 * n + FISK_B2, 0.05)
    u = rng.uniform(1e-12, 1 - 1e-12, size=n.shape)
    xsq = alpha * (u / (1 - u)) ** (1.0 / beta)
    epe = np.minimum(np.sqrt(xsq), EPE_CAP)
    ang = rng.uniform(0, 2 * np.pi, size=n.shape)
    return np.stack([epe * np.cos(ang), epe * np.sin(ang)], axis=-1)


_RAYS = {}


def _camera_rays(K, W, H):
    """Ray directions (x/z, y/z, 1) of the pixel centres, cached per camera."""
    key = (K, W, H)
    if key not in _RAYS:
        fx, fy, cx, cy = K
        xs, ys = np.meshgrid(np.arange(W, dtype=float), np.arange(H, dtype=float))
        if len(_RAYS) > 8:
            _RAYS.clear()
        _RAYS[key] = np.stack([(xs - cx) / fx, (ys - cy) / fy, np.ones_like(xs)], -1).reshape(-1, 3)
    return _RAYS[key]


def _footprint(prim, K, R, t, W, H, frame):
    """Indices of the rays that can hit a bounded convex primitive (all rays:
    None). A ray's hit point has camera depth > 0, so a primitive entirely at
    depth <= 0 is hit by none; one entirely at depth > 0 projects inside the
    bounding box of its projected corners; otherwise every ray is tested."""
    C = prim.corners(frame)
    if C is None:
        return None
    Xc = C @ R.T + t
    z = Xc[:, 2]
    if np.all(z <= 0):
        return np.zeros(0, np.int64)
    if np.any(z <= 1e-6):
        return None
    fx, fy, cx, cy = K
    u = fx * Xc[:, 0] / z + cx
    v = fy * Xc[:, 1] / z + cy
    x0, x1 = max(int(np.floor(u.min())) - 1, 0), min(int(np.ceil(u.max())) + 1, W - 1)
    y0, y1 = max(int(np.floor(v.min())) - 1, 0), min(int(np.ceil(v.max())) + 1, H - 1)
    if x0 > x1 or y0 > y1:
        return np.zeros(0, np.int64)
    ys, xs = np.arange(y0, y1 + 1), np.arange(x0, x1 + 1)
    return (ys[:, None] * W + xs[None, :]).ravel()


def _render(prims, K, M, W, H, frame):
    """Cast the rays of a camera with world->camera transform M."""
    dc = _camera_rays(tuple(K), W, H)
    R, t = M[:3, :3], M[:3, 3]
    o = -R.T @ t
    d = dc @ R                       # rows: R^T dc
    best = np.full(dc.shape[0], np.inf)
    oid = np.full(dc.shape[0], -1)
    for i, p in enumerate(prims):
        idx = _footprint(p, K, R, t, W, H, frame)
        if idx is not None and idx.size == 0:
            continue
        sub = slice(None) if idx is None else idx
        ti = p.hit(o, d[sub], frame)
        better = ti < best[sub]
        best[sub] = np.where(better, ti, best[sub])
        oid[sub] = np.where(better, i, oid[sub])
    X = o[None, :] + best[:, None] * d
    return X, best.reshape(H, W), oid


def _make_window(prims, K, Ms, W, H, patches, rng, name, inv_range, noise=True):
    T = len(Ms) - 1
    fx, fy, cx, cy = K
    xs, ys = np.meshgrid(np.arange(W, dtype=float), np.arange(H, dtype=float))
    flows = np.zeros((T, H, W, 2))
    rigid = np.ones((T, H, W), bool)
    poses = np.zeros((T, 4, 4))
    depth0 = None
    for t in range(1, T + 1):
        Mp, Mt = Ms[t - 1], Ms[t]
        poses[t - 1] = Mt @ np.linalg.inv(Mp)
        X, depth, oid = _render(prims, K, Mp, W, H, t - 1)
        if t == 1:
            depth0 = depth.copy()
        # move hit points of moving boxes to their frame-t position
        Xt = X.copy()
        moving = np.zeros(X.shape[0], bool)
        for i, p in enumerate(prims):
            if isinstance(p, _Box) and p.moving:
                sel = oid == i
                Xt[sel] += p.offset(t) - p.offset(t - 1)
                moving |= sel
        Pc = Xt @ Mt[:3, :3].T + Mt[:3, 3]
        z = Pc[:, 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = fx * Pc[:, 0] / z + cx
            v = fy * Pc[:, 1] / z + cy
        fl = np.stack([u.reshape(H, W) - xs, v.reshape(H, W) - ys], -1)
        # points passing (almost) through camera t's image plane have no
        # meaningful flow: they get an outlier flow, as a flow network would
        bad = (~np.isfinite(fl).all(-1) | (z.reshape(H, W) <= 0.5)
               | (np.abs(fl).max(-1) > max(W, H)))
        fl[bad] = rng.uniform(-20.0, 20.0, size=(int(bad.sum()), 2))
        rig = ~moving.reshape(H, W) & ~bad
        for (x0, y0, x1, y1) in patches:
            disp = rng.uniform(-8.0, 8.0, size=2)
            fl[y0:y1, x0:x1] += disp
            rig[y0:y1, x0:x1] = False
        if noise:
            fl = fl + _fisk_noise(rng, np.linalg.norm(fl, axis=-1))
        flows[t - 1] = fl
        rigid[t - 1] = rig
    return Window(flows=flows, K=K, poses=poses, depth0=depth0, rigid=rigid,
                  inv_depth_range=inv_range, name=name)


def _patches(rng, W, H, n, total_frac):
    out = []
    for _ in range(n):
        frac = total_frac / n
        pw = int(round(np.sqrt(frac) * W))
        ph = int(round(np.sqrt(frac) * H))
        x0 = int(rng.integers(0, max(1, W - pw)))
        y0 = int(rng.integers(0, max(1, H - ph)))
        out.append((x0, y0, x0 + pw, y0 + ph))
    return out


def _trajectory(rng, T, step_fn):
    Ms = [np.eye(4)]
    for _ in range(T):
        R, t = step_fn(rng)
        rel = np.eye(4)
        rel[:3, :3] = R
        rel[:3, 3] = t
        Ms.append(rel @ Ms[-1])
    return Ms


def _random_rect(rng, K, W, H, zmin, zmax, max_tilt_deg=60.0):
    fx, fy, cx, cy = K
    z = rng.uniform(zmin, zmax)
    px = rng.uniform(0.1 * W, 0.9 * W)
    py = rng.uniform(0.1 * H, 0.9 * H)
    c = np.array([(px - cx) / fx * z, (py - cy) / fy * z, z])
    tilt = np.deg2rad(rng.uniform(0, max_tilt_deg))
    axis = np.array([rng.normal(), rng.normal(), 0.0])
    n = _rot(axis, tilt) @ np.array([0.0, 0.0, -1.0])
    u = np.cross(n, [0.0, 1.0, 0.0])
    if np.linalg.norm(u) < 1e-6:
        u = np.array([1.0, 0.0, 0.0])
    v = np.cross(n, u)
    hu = z * rng.uniform(0.15, 0.4) * W / fx
    hv = z * rng.uniform(0.15, 0.4) * H / fy
    return _Plane(c, n, u, v, hu, hv)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def small_planes(seed=1000, W=160, H=120, f=120.0, T=3, noise=True, nonrigid=True):
    """160x120 pinhole f=120; 4 random planar patches at depth U[2,20] m in
    front of a background plane at 20 m; 0.1 m/frame translation in a random
    direction, rotation <= 2 deg about a random axis; one non-rigid patch of
    10% of the pixels."""
    rng = np.random.default_rng(seed)
    K = (f, f, (W - 1) / 2.0, (H - 1) / 2.0)
    prims = [_random_rect(rng, K, W, H, 2.0, 20.0) for _ in range(4)]
    prims.append(_Plane([0, 0, 20.0], [0, 0, -1.0]))

    def step(r):
        return _rot(_rand_dir(r), np.deg2rad(r.uniform(0, 2.0))), 0.1 * _rand_dir(r)

    Ms = _trajectory(rng, T, step)
    patches = _patches(rng, W, H, 1, 0.10) if nonrigid else []
    return _make_window(prims, K, Ms, W, H, patches, rng, "small_planes_160x120_T3",
                        (1 / 40.0, 1 / 1.0), noise)


def handheld(seed=2000, W=640, H=480, f=525.0, T=5, noise=True, nonrigid=True):
    """640x480 f=525 handheld-like: 20 planar patches and axis-aligned boxes
    in [0.5, 8] m before a background plane at 8 m; random 6-DoF motion with
    |t| <= 0.05 m and rotation <= 5 deg per frame; 3 non-rigid patches
    totalling 20% of the pixels."""
    rng = np.random.default_rng(seed)
    K = (f, f, (W - 1) / 2.0, (H - 1) / 2.0)
    prims = [_random_rect(rng, K, W, H, 0.5, 8.0) for _ in range(14)]
    for _ in range(6):
        z = rng.uniform(1.0, 7.0)
        c = np.array([rng.uniform(-0.5, 0.5) * z, rng.uniform(-0.4, 0.4) * z, z])
        half = rng.uniform(0.1, 0.5, size=3) * z * 0.4
        prims.append(_Box(c - half, c + half))
    prims.append(_Plane([0, 0, 8.0], [0, 0, -1.0]))

    def step(r):
        return (_rot(_rand_dir(r), np.deg2rad(r.uniform(0, 5.0))),
                r.uniform(0.01, 0.05) * _rand_dir(r))

    Ms = _trajectory(rng, T, step)
    patches = _patches(rng, W, H, 3, 0.20) if nonrigid else []
    return _make_window(prims, K, Ms, W, H, patches, rng, "handheld_640x480_T5",
                        (1 / 16.0, 1 / 0.25), noise)


def driving(seed=3000, W=1242, H=375, f=718.0, T=8, noise=True, nonrigid=True):
    """1242x375 f=718 driving-like: ground plane 1.65 m below the camera,
    vertical facades along and across the road in [3, 80] m, a far wall at
    80 m; forward motion 1 m/frame with yaw <= 1 deg; car-sized boxes
    (1.8 x 1.5 x 4.5 m) moving on their own until ~15% of the pixels are
    non-rigid."""
    rng = np.random.default_rng(seed)
    K = (f, f, (W - 1) / 2.0 if W != 1242 else 620.5, 187.0 if H == 375 else (H - 1) / 2.0)
    cam_h = 1.65
    prims = [_Plane([0, cam_h, 0], [0, -1.0, 0])]
    for side in (-1, 1):
        z = 0.0
        while z < 80:
            seg = rng.uniform(6, 20)
            x = side * rng.uniform(5.0, 15.0)
            height = rng.uniform(4.0, 20.0)
            prims.append(_Plane([x, cam_h - height / 2, z + seg / 2], [-side, 0, 0],
                                [0, 0, 1.0], [0, 1.0, 0], seg / 2, height / 2))
            z += seg
    for _ in range(4):
        z = rng.uniform(25, 75)
        x = rng.uniform(-15, 15)
        hw = rng.uniform(2, 6)
        height = rng.uniform(4, 15)
        prims.append(_Plane([x, cam_h - height / 2, z], [0, 0, -1.0], [1.0, 0, 0], [0, 1.0, 0],
                            hw, height / 2))
    prims.append(_Plane([0, 0, 80.0], [0, 0, -1.0]))
    M0 = np.eye(4)
    # cars until ~15% of frame-0 pixels are non-rigid: each new car is tested
    # against the depth of everything placed so far
    _, depth, _ = _render(prims, K, M0, W, H, 0)
    depth = depth.ravel()
    car = np.zeros(depth.shape, bool)
    fx_, fy_, cx_, cy_ = K
    xs_, ys_ = np.meshgrid(np.arange(W, dtype=float), np.arange(H, dtype=float))
    dirs = np.stack([(xs_ - cx_) / fx_, (ys_ - cy_) / fy_, np.ones_like(xs_)], -1).reshape(-1, 3)
    for _ in range(16):
        if car.mean() >= 0.15:
            break
        x = rng.uniform(-5.0, 5.0)
        z = rng.uniform(8.0, 35.0)
        lo = np.array([x - 0.9, cam_h - 1.5, z])
        hi = np.array([x + 0.9, cam_h, z + 4.5])
        # same-direction traffic near the camera, oncoming traffic only far ahead
        vz = rng.uniform(0.2, 2.0) if z < 20 else rng.uniform(-1.0, 2.0)
        box = _Box(lo, hi, np.array([rng.uniform(-0.1, 0.1), 0.0, vz]))
        th = box.hit(np.zeros(3), dirs, 0)
        closer = th < depth
        depth = np.where(closer, th, depth)
        car |= closer
        prims.append(box)

    def step(r):
        return _rot([0, 1.0, 0], np.deg2rad(r.uniform(-1.0, 1.0))), np.array([0.0, 0.0, -1.0])

    Ms = _trajectory(rng, T, step)
    return _make_window(prims, K, Ms, W, H, [], rng, "driving_1242x375_T8",
                        (1 / 160.0, 1 / 1.5), noise)


WORKLOADS = {"small_planes": small_planes, "handheld": handheld, "driving": driving}
