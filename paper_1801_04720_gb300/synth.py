"""Seeded synthetic stereo quadruples for the scene-flow path.

The paper evaluates on the KITTI Scene Flow benchmark (Sec. 4), which is not
available here; these generators stand in for it with scenes of the same
shape: rectified 8-bit grayscale stereo pairs at t and t+1, a camera with
focal length f and baseline B, and a 2D optical-flow field that enters the
method as an input (Eq. 2).  The module renders images and ground truth only:
it holds none of the method's arithmetic (no census, no aggregation, no
combination), and both the CUDA path and the CPU oracle consume its output.

Two recipes:

* ``fronto_planes`` - textured fronto-parallel rectangles at integer
  disparities that translate by integer 2D shifts; the input flow is the exact
  shift.  Rendering is pure integer indexing, so ground truth is exact.
* ``automotive`` - slanted planar segments with gradient-noise texture in
  front of a far wall and a ground plane, each segment moving rigidly in 3D;
  images are ray cast, get Gaussian sensor noise and are rounded to uint8; the
  input flow is the induced flow plus Gaussian noise.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Camera:
    f: float
    B: float
    cx: float
    cy: float


@dataclass
class Quad:
    """One stereo quadruple with its input flow and ground truth."""
    left_t: np.ndarray        # uint8 [H][W]
    right_t: np.ndarray       # uint8 [H][W]
    left_t1: np.ndarray       # uint8 [H][W]
    right_t1: np.ndarray      # uint8 [H][W]
    flow: np.ndarray          # float32 [H][W][2], the method's input flow
    camera: Camera
    D: int
    gt_disp0: np.ndarray      # float32 [H][W], disparity at t of the visible surface
    gt_disp1: np.ndarray      # float32 [H][W], disparity at t+1 of the same 3D point
    gt_flow: np.ndarray       # float32 [H][W][2]
    surface_t: np.ndarray     # int16 [H][W], id of the visible surface in left_t
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.left_t.shape

    def images(self):
        return (self.left_t, self.right_t, self.left_t1, self.right_t1)


# --------------------------------------------------------------------------
# Recipe 1: fronto-parallel planes, integer disparities and shifts
# --------------------------------------------------------------------------

def _render_fronto(W, H, planes, textures, bg_tex, bg_disp, view_right, shifts):
    """Render one view.  planes: list of (x0, y0, w, h, d), nearest first;
    shifts: per-plane integer (sx, sy) applied to the rectangle."""
    img = np.empty((H, W), dtype=np.uint8)
    sid = np.full((H, W), -1, dtype=np.int16)
    ys, xs = np.mgrid[0:H, 0:W]
    # background: a static textured fronto-parallel plane at bg_disp
    xb = xs + (bg_disp if view_right else 0)
    img[:] = bg_tex[ys, xb]
    disp = np.full((H, W), float(bg_disp), dtype=np.float32)
    # far to near so nearer planes overwrite farther ones
    order = sorted(range(len(planes)), key=lambda k: planes[k][4])
    for k in order:
        x0, y0, w, h, d = planes[k]
        sx, sy = shifts[k]
        xl = xs + (d if view_right else 0)   # left-image column of this pixel's point
        u = xl - (x0 + sx)
        v = ys - (y0 + sy)
        inside = (u >= 0) & (u < w) & (v >= 0) & (v < h)
        img[inside] = textures[k][v[inside], u[inside]]
        sid[inside] = k
        disp[inside] = d
    return img, sid, disp


def fronto_planes(W=64, H=48, D=16, disparities=(3, 7, 12), seed=0, f=100.0, B=0.5,
                  max_shift=3, bg_disp=1, size_frac=(0.25, 0.5)):
    """Textured fronto-parallel rectangles (the tiny 64x48, D=16 recipe).

    Each plane has a uniform-integer texture in [0, 255] attached to its own
    coordinates, translates by an integer (sx, sy) between t and t+1 at
    constant depth, and the input flow is that exact shift.  The background is
    a static textured plane at disparity ``bg_disp``."""
    rng = np.random.default_rng(seed)
    planes, textures, shifts = [], [], []
    for d in disparities:
        w = int(rng.integers(int(size_frac[0] * W), int(size_frac[1] * W) + 1))
        h = int(rng.integers(int(size_frac[0] * H), int(size_frac[1] * H) + 1))
        x0 = int(rng.integers(0, W - w + 1))
        y0 = int(rng.integers(0, H - h + 1))
        planes.append((x0, y0, w, h, int(d)))
        textures.append(rng.integers(0, 256, size=(h, w), dtype=np.uint8))
        shifts.append((int(rng.integers(-max_shift, max_shift + 1)),
                       int(rng.integers(-max_shift, max_shift + 1))))
    bg_tex = rng.integers(0, 256, size=(H, W + bg_disp), dtype=np.uint8)
    zero = [(0, 0)] * len(planes)
    lt, sid_t, disp_t = _render_fronto(W, H, planes, textures, bg_tex, bg_disp, False, zero)
    rt, sid_rt, _ = _render_fronto(W, H, planes, textures, bg_tex, bg_disp, True, zero)
    lt1, sid_t1, disp_t1 = _render_fronto(W, H, planes, textures, bg_tex, bg_disp, False, shifts)
    rt1, sid_rt1, _ = _render_fronto(W, H, planes, textures, bg_tex, bg_disp, True, shifts)
    flow = np.zeros((H, W, 2), dtype=np.float32)
    for k, (sx, sy) in enumerate(shifts):
        m = sid_t == k
        flow[m, 0] = sx
        flow[m, 1] = sy
    cam = Camera(f=f, B=B, cx=(W - 1) / 2.0, cy=(H - 1) / 2.0)
    return Quad(lt, rt, lt1, rt1, flow, cam, D, disp_t, disp_t.copy(), flow.copy(), sid_t,
                extra={"planes": planes, "shifts": shifts, "bg_disp": bg_disp,
                       "sid_right_t": sid_rt, "sid_left_t1": sid_t1, "sid_right_t1": sid_rt1,
                       "disp_t1": disp_t1})


def batch_recipe(seed, sizes=((320, 240), (640, 480), (1024, 320), (1242, 375)),
                 Ds=(64, 128, 192)):
    """One instance of the uneven batch: size and D drawn from the given sets,
    scene drawn with the fronto-parallel recipe scaled to that size."""
    rng = np.random.default_rng(1_000_003 + seed)
    W, H = sizes[int(rng.integers(0, len(sizes)))]
    D = int(Ds[int(rng.integers(0, len(Ds)))])
    n = 6
    disparities = sorted(int(v) for v in rng.integers(2, min(D - 4, W // 4), size=n))
    return fronto_planes(W=W, H=H, D=D, disparities=disparities, seed=seed, f=721.5, B=0.54,
                         max_shift=8, bg_disp=1, size_frac=(0.12, 0.3))


# --------------------------------------------------------------------------
# Recipe 2: slanted segments, gradient-noise texture, rigid 3D motion
# --------------------------------------------------------------------------

class GradientNoise:
    """2D gradient noise after Perlin (lattice gradients, quintic fade,
    interpolation of corner dot products), seeded."""

    def __init__(self, rng, size=256):
        self.size = size
        self.perm = rng.permutation(size).astype(np.int64)
        ang = rng.uniform(0.0, 2.0 * np.pi, size=size)
        self.gx = np.cos(ang)
        self.gy = np.sin(ang)

    def _grad(self, ix, iy):
        h = self.perm[(self.perm[ix % self.size] + iy) % self.size]
        return self.gx[h], self.gy[h]

    @staticmethod
    def _fade(t):
        return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)

    def __call__(self, x, y):
        x0 = np.floor(x)
        y0 = np.floor(y)
        fx = x - x0
        fy = y - y0
        ix = x0.astype(np.int64)
        iy = y0.astype(np.int64)
        out = 0.0
        u = self._fade(fx)
        v = self._fade(fy)
        for cx, cy, wx, wy in ((0, 0, 1 - u, 1 - v), (1, 0, u, 1 - v), (0, 1, 1 - u, v), (1, 1, u, v)):
            gx, gy = self._grad(ix + cx, iy + cy)
            out = out + wx * wy * (gx * (fx - cx) + gy * (fy - cy))
        return out

    def fractal(self, x, y, octaves=4, lacunarity=2.0, gain=0.55):
        amp, freq, total = 1.0, 1.0, 0.0
        for o in range(octaves):
            total = total + amp * self(x * freq + 17.3 * o, y * freq - 9.1 * o)
            amp *= gain
            freq *= lacunarity
        return total


@dataclass
class _Surface:
    centre: np.ndarray    # (3,)
    e1: np.ndarray        # in-plane unit axis (texture s)
    e2: np.ndarray        # in-plane unit axis (texture t)
    half: tuple           # (half extent along e1, along e2); inf for unbounded
    tex_scale: float
    tex_offset: tuple
    tex_gain: float
    tex_bias: float

    @property
    def normal(self):
        n = np.cross(self.e1, self.e2)
        return n / np.linalg.norm(n)


def _yaw(theta):
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def _pitch(phi):
    c, s = np.cos(phi), np.sin(phi)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def _moved(surf: _Surface, R, T):
    return _Surface(centre=R @ surf.centre + T, e1=R @ surf.e1, e2=R @ surf.e2, half=surf.half,
                    tex_scale=surf.tex_scale, tex_offset=surf.tex_offset, tex_gain=surf.tex_gain,
                    tex_bias=surf.tex_bias)


def _cast(surfaces, W, H, cam: Camera, origin_x):
    """Ray cast all pixels of a camera at (origin_x, 0, 0) looking down +Z.
    Returns per pixel: nearest surface index, depth Z, texture coords."""
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    dx = (xs - cam.cx) / cam.f
    dy = (ys - cam.cy) / cam.f
    best_z = np.full((H, W), np.inf)
    best_k = np.full((H, W), -1, dtype=np.int16)
    best_s = np.zeros((H, W))
    best_t = np.zeros((H, W))
    o = np.array([origin_x, 0.0, 0.0])
    with np.errstate(divide="ignore", invalid="ignore"):
        for k, s in enumerate(surfaces):
            _hit_surface(k, s, o, dx, dy, best_z, best_k, best_s, best_t)
    return best_k, best_z, best_s, best_t


def _hit_surface(k, s, o, dx, dy, best_z, best_k, best_s, best_t):
    """Intersect every pixel ray with surface s; keep the nearest hit."""
    n = s.normal
    denom = n[0] * dx + n[1] * dy + n[2]
    num = float(n @ (s.centre - o))
    z = num / denom
    px = o[0] + dx * z - s.centre[0]
    py = o[1] + dy * z - s.centre[1]
    pz = z - s.centre[2]
    sc = px * s.e1[0] + py * s.e1[1] + pz * s.e1[2]
    tc = px * s.e2[0] + py * s.e2[1] + pz * s.e2[2]
    hit = (z > 0.5) & np.isfinite(z) & (np.abs(sc) <= s.half[0]) & (np.abs(tc) <= s.half[1])
    closer = hit & (z < best_z)
    best_z[closer] = z[closer]
    best_k[closer] = k
    best_s[closer] = sc[closer]
    best_t[closer] = tc[closer]


def _shade(surfaces, k, s, t, noise: GradientNoise):
    img = np.zeros(k.shape)
    for idx, surf in enumerate(surfaces):
        m = k == idx
        if not m.any():
            continue
        val = noise.fractal(s[m] * surf.tex_scale + surf.tex_offset[0],
                            t[m] * surf.tex_scale + surf.tex_offset[1])
        img[m] = surf.tex_bias + surf.tex_gain * val
    return img


def _automotive_scene(rng, W, H, f, B, n_segments, disp_range, max_translation, max_yaw_deg, frames=2):
    """Camera, texture noise, surfaces and per-surface rigid motions of the
    automotive recipe.  Segments are placed so that every one of `frames`
    poses (the motion applied 0 .. frames-1 times) stays inside the
    disparity range."""
    cam = Camera(f=f, B=B, cx=(W - 1) / 2.0, cy=(H - 1) / 2.0)
    fB = f * B
    noise = GradientNoise(rng)
    surfaces = []
    z_far = fB / disp_range[0]
    # far wall, fronto-parallel
    surfaces.append(_Surface(np.array([0.0, 0.0, z_far]), np.array([1.0, 0.0, 0.0]),
                             np.array([0.0, 1.0, 0.0]), (np.inf, np.inf), 0.35,
                             tuple(rng.uniform(0, 50, 2)), 110.0, 120.0))
    # ground plane y = cam_height (image y points down)
    cam_height = 1.65
    surfaces.append(_Surface(np.array([0.0, cam_height, 0.5 * z_far]), np.array([1.0, 0.0, 0.0]),
                             np.array([0.0, 0.0, 1.0]), (np.inf, 0.5 * z_far - 1.0), 1.2,
                             tuple(rng.uniform(0, 50, 2)), 100.0, 110.0))
    motions = [(np.eye(3), np.zeros(3))] * 2
    tries = 0
    while len(surfaces) < 2 + n_segments:
        tries += 1
        if tries > 10000:
            raise RuntimeError("could not place segments")
        d_c = rng.uniform(disp_range[0] + 4.0, 0.8 * disp_range[1])
        z = fB / d_c
        xi = rng.uniform(0.05 * W, 0.95 * W)
        yi = rng.uniform(cam.cy - 0.35 * H, cam.cy + 0.3 * H)
        centre = np.array([(xi - cam.cx) * z / f, (yi - cam.cy) * z / f, z])
        yaw = rng.uniform(-np.pi / 4, np.pi / 4)
        pitch = rng.uniform(-np.pi / 18, np.pi / 18)
        R0 = _yaw(yaw) @ _pitch(pitch)
        e1 = R0 @ np.array([1.0, 0.0, 0.0])
        e2 = R0 @ np.array([0.0, 1.0, 0.0])
        half = (rng.uniform(0.4, 2.2), rng.uniform(0.4, 1.5))
        surf = _Surface(centre, e1, e2, half, rng.uniform(1.5, 5.0), tuple(rng.uniform(0, 200, 2)),
                        rng.uniform(90.0, 130.0), rng.uniform(90.0, 160.0))
        theta = np.deg2rad(rng.uniform(-max_yaw_deg, max_yaw_deg))
        direction = rng.normal(size=3)
        direction /= np.linalg.norm(direction)
        T = direction * rng.uniform(0.0, max_translation)
        Rm = _yaw(theta)
        # rigid motion about the segment's centre: X' = Rm (X - c) + c + T
        Tm = centre - Rm @ centre + T
        poses = [surf]
        for _ in range(frames - 1):
            poses.append(_moved(poses[-1], Rm, Tm))
        ok = True
        for sf in poses:
            for a in (-1, 1):
                for b in (-1, 1):
                    corner = sf.centre + a * sf.half[0] * sf.e1 + b * sf.half[1] * sf.e2
                    if corner[2] <= 0.5:
                        ok = False
                        continue
                    dd = fB / corner[2]
                    if not (disp_range[0] + 0.5 <= dd <= disp_range[1] - 0.5):
                        ok = False
        if not ok:
            continue
        surfaces.append(surf)
        motions.append((Rm, Tm))

    return cam, fB, noise, surfaces, motions


def automotive(seed=0, W=1242, H=375, D=128, n_segments=20, f=721.5, B=0.54,
               disp_range=(2.0, 120.0), max_translation=1.5, max_yaw_deg=3.0,
               pixel_noise=2.0, flow_noise=0.5):
    """Automotive-shaped quadruple (the 1242x375, D=128 recipe).

    A far wall (disparity ``disp_range[0]``) and a ground plane form the
    static background; ``n_segments`` slanted textured rectangles with
    disparities inside ``disp_range`` each move rigidly (translation up to
    ``max_translation`` m, yaw up to ``max_yaw_deg``).  Images carry
    N(0, pixel_noise) sensor noise; the input flow is the induced flow plus
    N(0, flow_noise) px."""
    rng = np.random.default_rng(seed)
    cam, fB, noise, surfaces, motions = _automotive_scene(rng, W, H, f, B, n_segments, disp_range,
                                                          max_translation, max_yaw_deg)
    surfaces_t1 = [_moved(s, R, T) for s, (R, T) in zip(surfaces, motions)]
    views = {}
    for name, surfs, ox in (("left_t", surfaces, 0.0), ("right_t", surfaces, B),
                            ("left_t1", surfaces_t1, 0.0), ("right_t1", surfaces_t1, B)):
        k, z, s, t = _cast(surfs, W, H, cam, ox)
        img = _shade(surfs, k, s, t, noise) + rng.normal(0.0, pixel_noise, size=(H, W))
        views[name] = np.clip(np.rint(img), 0, 255).astype(np.uint8)
        if name == "left_t":
            k_t, z_t = k, z
    # ground truth at t: visible point, its motion and its projection at t+1
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    X = (xs - cam.cx) * z_t / f
    Y = (ys - cam.cy) * z_t / f
    P = np.stack([X, Y, z_t], axis=-1)
    P1 = np.empty_like(P)
    for idx, (R, T) in enumerate(motions):
        m = k_t == idx
        P1[m] = P[m] @ R.T + T
    x1 = f * P1[..., 0] / P1[..., 2] + cam.cx
    y1 = f * P1[..., 1] / P1[..., 2] + cam.cy
    gt_flow = np.stack([x1 - xs, y1 - ys], axis=-1).astype(np.float32)
    flow = (gt_flow + rng.normal(0.0, flow_noise, size=gt_flow.shape)).astype(np.float32)
    gt_d0 = (fB / z_t).astype(np.float32)
    gt_d1 = (fB / P1[..., 2]).astype(np.float32)
    return Quad(views["left_t"], views["right_t"], views["left_t1"], views["right_t1"], flow, cam,
                D, gt_d0, gt_d1, gt_flow, k_t.astype(np.int16),
                extra={"n_segments": n_segments, "seed": seed})


class Sequence:
    """K consecutive stereo frames of one scene: lefts[k], rights[k] uint8
    [H][W]; flows[k] float32 [H][W][2] from frame k to k+1 (induced flow plus
    noise); ground truth gt_disp[k] (disparity of the visible surface),
    gt_flow[k] and gt_next_disp[k] (the disparity at frame k+1 of the point
    visible at frame k); only the frames rendered are filled (others None)."""

    def __init__(self, K, camera, D):
        self.K, self.camera, self.D = K, camera, D
        self.lefts = [None] * K
        self.rights = [None] * K
        self.flows = [None] * (K - 1)
        self.gt_disp = [None] * K
        self.gt_flow = [None] * (K - 1)
        self.gt_next_disp = [None] * (K - 1)


def sequence(K, seed=0, W=2048, H=1024, D=256, n_segments=40, f=721.5, B=0.54, disp_range=(2.0, 120.0),
             max_translation=0.25, max_yaw_deg=1.0, pixel_noise=2.0, flow_noise=0.5, frames=None):
    """K consecutive frames of one evolving automotive-recipe scene: every
    segment repeats its rigid motion (translation up to ``max_translation`` m,
    yaw up to ``max_yaw_deg`` per frame) from frame to frame, and is placed so
    that it stays inside the disparity range over all K frames.  The scene
    depends on the seed alone and each frame's noise on (seed, frame), so a
    subset ``frames`` can be rendered on its own (e.g. in parallel workers)
    and the parts put together; the flow F_k needs frame k rendered."""
    rng = np.random.default_rng(seed)
    cam, fB, noise, surfaces, motions = _automotive_scene(rng, W, H, f, B, n_segments, disp_range,
                                                          max_translation, max_yaw_deg, frames=K)
    seq = Sequence(K, cam, D)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    for k in (range(K) if frames is None else frames):
        frng = np.random.default_rng([seed, k])
        surfs = list(surfaces)
        for _ in range(k):
            surfs = [_moved(s_, R, T) for s_, (R, T) in zip(surfs, motions)]
        for name, ox in (("left", 0.0), ("right", B)):
            kk, z, s_, t = _cast(surfs, W, H, cam, ox)
            img = _shade(surfs, kk, s_, t, noise) + frng.normal(0.0, pixel_noise, size=(H, W))
            img = np.clip(np.rint(img), 0, 255).astype(np.uint8)
            if name == "left":
                seq.lefts[k], k_t, z_t = img, kk, z
            else:
                seq.rights[k] = img
        seq.gt_disp[k] = (fB / z_t).astype(np.float32)
        if k + 1 < K:
            P = np.stack([(xs - cam.cx) * z_t / f, (ys - cam.cy) * z_t / f, z_t], axis=-1)
            P1 = np.empty_like(P)
            for idx, (R, T) in enumerate(motions):
                m = k_t == idx
                P1[m] = P[m] @ R.T + T
            x1 = f * P1[..., 0] / P1[..., 2] + cam.cx
            y1 = f * P1[..., 1] / P1[..., 2] + cam.cy
            gt = np.stack([x1 - xs, y1 - ys], axis=-1).astype(np.float32)
            seq.gt_flow[k] = gt
            seq.gt_next_disp[k] = (fB / P1[..., 2]).astype(np.float32)
            seq.flows[k] = (gt + frng.normal(0.0, flow_noise, size=gt.shape)).astype(np.float32)
    return seq


def stream(n_frames, seed=0, W=2048, H=1024, D=256, n_segments=40, **kw):
    """A sequence of quadruples from one evolving scene (large-stream recipe):
    frame k uses seed*1000+k so each frame is a fresh rigid-motion step of a
    scene drawn from the automotive recipe at this size."""
    return [automotive(seed=seed * 1000 + k, W=W, H=H, D=D, n_segments=n_segments, **kw)
            for k in range(n_frames)]


def confnet_init(seed, layers):
    """Seeded initial parameters of a 3x3 convolutional network: for each
    (in_channels, out_channels) in `layers`, He-normal weights [co][3][3][ci]
    (std sqrt(2 / (9 ci))) then zero biases, flattened, float32."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in layers:
        parts.append(rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), size=9 * ci * co))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def confidence_recipe(seed, W=1242, H=375, D=128, n_planes=6):
    """Scenes for training and evaluating the learned confidence: the
    fronto-parallel plane recipe rendered at W x H with n_planes rectangles at
    seeded disparities in [2, D - 5]."""
    rng = np.random.default_rng(2_000_003 + seed)
    disparities = sorted(int(v) for v in rng.integers(2, max(3, min(D - 4, W // 4)), size=n_planes))
    return fronto_planes(W=W, H=H, D=D, disparities=disparities, seed=seed, f=721.5, B=0.54,
                         max_shift=8, bg_disp=1, size_frac=(0.12, 0.3))
