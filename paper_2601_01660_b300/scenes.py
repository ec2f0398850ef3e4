"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs: Gaussian clouds (means, linear scales,
unit quaternions w,x,y,z, opacities, colours), light positions, shell radii,
and the cubemap samples (Y, D, w) that the HDRI probe fit of Sec. 3.4 consumes.
It holds none of the method's arithmetic (no line integral, no octahedral map,
no SH basis), so both the CUDA path and the oracle can take their inputs from
it.  Every array is float32 and C-contiguous.

The paper measures on captured 3DGS scenes and avatars (ScanNet++, DL3DV,
SuperSplat, AvatarX, ActorsHQ); none of those are available here, so the
generators below stand in for their shapes: an indoor room of flattened
surface Gaussians with boxes, and a human-sized body of ellipsoid limbs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Scene", "cube_scene", "room_scene", "avatar_body", "radii_linear",
    "radii_geometric", "four_lights", "cubemap_samples", "random_quats",
    "quat_mul", "concat", "subset", "workload",
]


@dataclass
class Scene:
    """A set of 3D Gaussians in SoA layout (all float32, C-contiguous)."""
    means: np.ndarray    # (N,3)
    scales: np.ndarray   # (N,3) linear (not log) standard deviations, metres
    quats: np.ndarray    # (N,4) unit quaternions (w,x,y,z)
    opac: np.ndarray     # (N,)  opacities alpha in (0,1)
    colors: np.ndarray   # (N,3) RGB in [0,1]
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def random_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random unit quaternions (normalised 4-D standard normal)."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Hamilton product a*b of (w,x,y,z) quaternions, row-wise."""
    aw, ax, ay, az = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    bw, bx, by, bz = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([
        aw * bw - ax * bx - ay * by - az * bz,
        aw * bx + ax * bw + ay * bz - az * by,
        aw * by - ax * bz + ay * bw + az * bx,
        aw * bz + ax * by - ay * bx + az * bw,
    ], axis=-1)


def _axis_angle_quat(axis, angle) -> np.ndarray:
    axis = np.asarray(axis, dtype=np.float64)
    angle = np.asarray(angle, dtype=np.float64)
    h = 0.5 * angle
    s = np.sin(h)
    q = np.zeros(np.broadcast(angle, axis[..., 0]).shape + (4,))
    q[..., 0] = np.cos(h)
    q[..., 1] = axis[..., 0] * s
    q[..., 2] = axis[..., 1] * s
    q[..., 3] = axis[..., 2] * s
    return q


def cube_scene(n: int, seed: int, centre=(0.0, 0.0, 3.0), side: float = 4.0,
               log_s_mean: float = math.log(0.05), log_s_std: float = 0.5,
               alpha=(0.05, 0.95)) -> Scene:
    """Anisotropic Gaussians with means uniform in an axis-aligned cube.

    Means ~ U(centre +- side/2), log-scales ~ N(log_s_mean, log_s_std^2) per
    axis, uniform random rotations, opacities ~ U(alpha), colours ~ U(0,1)^3.
    """
    rng = np.random.default_rng(seed)
    c = np.asarray(centre, dtype=np.float64)
    means = c + (rng.random((n, 3)) - 0.5) * side
    scales = np.exp(rng.normal(log_s_mean, log_s_std, (n, 3)))
    quats = random_quats(rng, n)
    opac = rng.uniform(alpha[0], alpha[1], n)
    colors = rng.random((n, 3))
    return Scene(_f32(means), _f32(scales), _f32(quats), _f32(opac), _f32(colors),
                 meta={"kind": "cube", "n": n, "seed": seed})


_Z = np.array([0.0, 0.0, 1.0])


def _surface_quats(rng, normals_axis_q: np.ndarray) -> np.ndarray:
    """Rotations whose local z axis is the surface normal, random in-plane spin."""
    n = normals_axis_q.shape[0]
    spin = _axis_angle_quat(np.broadcast_to(_Z, (n, 3)), rng.uniform(0, 2 * math.pi, n))
    return quat_mul(normals_axis_q, spin)


def _flat_scales(rng, n, thin=0.002, log_s_mean=math.log(0.05), log_s_std=0.5):
    s = np.empty((n, 3))
    s[:, :2] = np.exp(rng.normal(log_s_mean, log_s_std, (n, 2)))
    s[:, 2] = thin
    return s


def avatar_body(rng: np.random.Generator, n: int, base=(1.5, 0.0, 0.0), yaw: float = 0.0,
                height: float = 1.8) -> Scene:
    """A human-sized body: Gaussians on the surfaces of six ellipsoid limbs.

    Torso, head, two arms and two legs, scaled so the body is `height` tall,
    standing on z=0 at `base` and turned by `yaw` about +z.  Scales are
    log-normal N(log 0.01, 0.3^2) per axis with random rotations.
    """
    # (centre xyz, semi-axes xyz) in a body frame facing +x, feet at z=0.
    limbs = np.array([
        [0.00, 0.00, 1.15, 0.12, 0.18, 0.30],   # torso
        [0.00, 0.00, 1.65, 0.10, 0.09, 0.12],   # head
        [0.00, 0.25, 1.12, 0.05, 0.05, 0.32],   # left arm
        [0.00, -0.25, 1.12, 0.05, 0.05, 0.32],  # right arm
        [0.00, 0.10, 0.43, 0.07, 0.07, 0.43],   # left leg
        [0.00, -0.10, 0.43, 0.07, 0.07, 0.43],  # right leg
    ])
    top = max(l[2] + l[5] for l in limbs)
    limbs[:, :6] *= height / top
    a = limbs[:, 3:]
    # approximate ellipsoid surface areas to share the n points
    p = 1.6075
    area = 4 * math.pi * (((a[:, 0] * a[:, 1]) ** p + (a[:, 0] * a[:, 2]) ** p +
                           (a[:, 1] * a[:, 2]) ** p) / 3) ** (1 / p)
    counts = np.floor(n * area / area.sum()).astype(int)
    counts[0] += n - counts.sum()
    which = np.repeat(np.arange(len(limbs)), counts)
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    local = limbs[which, :3] + u * limbs[which, 3:]
    cy, sy = math.cos(yaw), math.sin(yaw)
    world = np.empty_like(local)
    world[:, 0] = cy * local[:, 0] - sy * local[:, 1] + base[0]
    world[:, 1] = sy * local[:, 0] + cy * local[:, 1] + base[1]
    world[:, 2] = local[:, 2] + base[2]
    scales = np.exp(rng.normal(math.log(0.01), 0.3, (n, 3)))
    quats = random_quats(rng, n)
    opac = rng.uniform(0.05, 0.95, n)
    colors = rng.random((n, 3))
    return Scene(_f32(world), _f32(scales), _f32(quats), _f32(opac), _f32(colors),
                 meta={"kind": "avatar", "n": n})


def room_scene(seed: int, n_flat: int = 900_000, n_box: int = 600_000,
               n_avatar: int = 100_000, avatar_base=(1.5, 0.0, 0.0),
               n_boxes: int = 30) -> Scene:
    """Indoor-scan-shaped scene: room surfaces, boxes and an avatar.

    * n_flat flattened Gaussians (thin axis 0.002 m along the surface normal,
      in-plane log-scales N(log 0.05, 0.5^2)) uniform by area on a 10x8 m floor
      (z=0) and four 3 m walls;
    * n_box Gaussians uniform by area on the five visible faces of n_boxes boxes
      (side U(0.3,1.5) m, on the floor, random yaw), log-scales
      N(log 0.05, 0.5^2), random rotations;
    * an n_avatar-Gaussian body (avatar_body) standing at avatar_base.
    meta['avatar'] holds the slice of the avatar Gaussians.
    """
    rng = np.random.default_rng(seed)
    X, Y, Hh = 5.0, 4.0, 3.0
    # surfaces: floor, walls x=+-5, y=+-4   (origin, u-edge, v-edge, normal quat)
    s2 = math.sqrt(0.5)
    surf = [
        (np.array([-X, -Y, 0.0]), np.array([2 * X, 0, 0]), np.array([0, 2 * Y, 0]), np.array([1.0, 0, 0, 0])),
        (np.array([X, -Y, 0.0]), np.array([0, 2 * Y, 0]), np.array([0, 0, Hh]), np.array([s2, 0, -s2, 0])),
        (np.array([-X, -Y, 0.0]), np.array([0, 2 * Y, 0]), np.array([0, 0, Hh]), np.array([s2, 0, s2, 0])),
        (np.array([-X, Y, 0.0]), np.array([2 * X, 0, 0]), np.array([0, 0, Hh]), np.array([s2, s2, 0, 0])),
        (np.array([-X, -Y, 0.0]), np.array([2 * X, 0, 0]), np.array([0, 0, Hh]), np.array([s2, -s2, 0, 0])),
    ]
    areas = np.array([np.linalg.norm(np.cross(e1, e2)) for _, e1, e2, _ in surf])
    which = rng.choice(len(surf), size=n_flat, p=areas / areas.sum())
    uv = rng.random((n_flat, 2))
    o = np.stack([s[0] for s in surf])[which]
    e1 = np.stack([s[1] for s in surf])[which]
    e2 = np.stack([s[2] for s in surf])[which]
    flat_means = o + uv[:, :1] * e1 + uv[:, 1:] * e2
    flat_q = _surface_quats(rng, np.stack([s[3] for s in surf])[which])
    flat_s = _flat_scales(rng, n_flat)

    # boxes
    side = rng.uniform(0.3, 1.5, n_boxes)
    cx = rng.uniform(-X + 1.0, X - 1.0, n_boxes)
    cy = rng.uniform(-Y + 1.0, Y - 1.0, n_boxes)
    yaw = rng.uniform(0, 2 * math.pi, n_boxes)
    face_area = np.repeat(side[:, None] ** 2, 5, axis=1)  # 4 sides + top
    fa = face_area.ravel()
    pick = rng.choice(fa.size, size=n_box, p=fa / fa.sum())
    b, f = pick // 5, pick % 5
    uv = rng.random((n_box, 2)) - 0.5
    h = side[b]
    local = np.zeros((n_box, 3))
    # faces: 0:+x 1:-x 2:+y 3:-y 4:top
    local[f == 0] = np.stack([0.5 * h[f == 0], uv[f == 0, 0] * h[f == 0], (uv[f == 0, 1] + 0.5) * h[f == 0]], 1)
    local[f == 1] = np.stack([-0.5 * h[f == 1], uv[f == 1, 0] * h[f == 1], (uv[f == 1, 1] + 0.5) * h[f == 1]], 1)
    local[f == 2] = np.stack([uv[f == 2, 0] * h[f == 2], 0.5 * h[f == 2], (uv[f == 2, 1] + 0.5) * h[f == 2]], 1)
    local[f == 3] = np.stack([uv[f == 3, 0] * h[f == 3], -0.5 * h[f == 3], (uv[f == 3, 1] + 0.5) * h[f == 3]], 1)
    local[f == 4] = np.stack([uv[f == 4, 0] * h[f == 4], uv[f == 4, 1] * h[f == 4], h[f == 4]], 1)
    c, s = np.cos(yaw[b]), np.sin(yaw[b])
    box_means = np.stack([c * local[:, 0] - s * local[:, 1] + cx[b],
                          s * local[:, 0] + c * local[:, 1] + cy[b], local[:, 2]], 1)
    box_s = np.exp(rng.normal(math.log(0.05), 0.5, (n_box, 3)))
    box_q = random_quats(rng, n_box)

    av = avatar_body(rng, n_avatar, base=avatar_base) if n_avatar > 0 else None
    n_scene = n_flat + n_box
    means = [flat_means, box_means]
    scales = [flat_s, box_s]
    quats = [flat_q, box_q]
    opac = rng.uniform(0.05, 0.95, n_scene)
    colors = rng.random((n_scene, 3))
    sc = Scene(_f32(np.concatenate(means)), _f32(np.concatenate(scales)),
               _f32(np.concatenate(quats)), _f32(opac), _f32(colors),
               meta={"kind": "room", "seed": seed})
    if av is not None:
        sc = concat(sc, av)
        sc.meta = {"kind": "room", "seed": seed, "avatar": slice(n_scene, n_scene + n_avatar)}
    return sc


def concat(*scenes: Scene) -> Scene:
    return Scene(*(np.ascontiguousarray(np.concatenate([getattr(s, k) for s in scenes]))
                   for k in ("means", "scales", "quats", "opac", "colors")), meta={})


def subset(sc: Scene, idx) -> Scene:
    return Scene(*(np.ascontiguousarray(getattr(sc, k)[idx])
                   for k in ("means", "scales", "quats", "opac", "colors")), meta={})


def radii_linear(r0: float, r1: float, k: int) -> np.ndarray:
    """Shell radii r_k = r0 + k (r1-r0)/(K-1), k = 0..K-1."""
    return _f32(np.linspace(r0, r1, k))


def radii_geometric(r0: float, r1: float, k: int) -> np.ndarray:
    """Shell radii r_k = r0 (r1/r0)^(k/(K-1)), k = 0..K-1."""
    return _f32(r0 * (r1 / r0) ** (np.arange(k) / (k - 1)))


def look_at_camera(eye, target, W: int, H: int, fov_y_deg: float = 60.0, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """A pinhole camera (16 float32: rotation rows image x, image y (down),
    forward; position; fx, fy, cx, cy) at `eye` looking at `target`."""
    eye, target, up = (np.asarray(a, dtype=np.float64) for a in (eye, target, up))
    f = target - eye
    f /= np.linalg.norm(f)
    x = np.cross(f, up)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    fy = 0.5 * H / math.tan(math.radians(fov_y_deg) / 2)
    return _f32(np.concatenate([x, y, f, eye, [fy, fy, 0.5 * W, 0.5 * H]]))


def four_lights() -> np.ndarray:
    """The four point lights used by the multi-light workloads."""
    return _f32([[0.0, 0.0, 0.0], [1.5, 1.5, -0.5], [-1.5, 1.5, -0.5], [0.0, -2.0, -0.5]])


def room_lights() -> np.ndarray:
    """Four ceiling lights of the room, 2.8 m high over the quarters of the floor."""
    return _f32([[-2.5, -2.0, 2.8], [2.5, -2.0, 2.8], [-2.5, 2.0, 2.8], [2.5, 2.0, 2.8]])


def avatar_crowd(seed: int, n_avatars: int = 8, n_each: int = 100_000):
    """Rest-pose avatars for the moving-avatar workload, and their motion.

    Each avatar is an avatar_body standing at the origin facing +x; they are
    stored back to back (offsets `seg`).  Avatar a walks a circle of radius
    r_a ~ U(1, 3) m at 1 m/s, centred so that the circle stays 0.3 m inside
    the room's walls, starting at a random phase and direction, turned to
    face its motion.  Returns (rest Scene, seg, motion dict)."""
    rng = np.random.default_rng(seed)
    bodies = [avatar_body(rng, n_each, base=(0.0, 0.0, 0.0)) for _ in range(n_avatars)]
    rest = concat(*bodies)
    seg = np.arange(n_avatars + 1, dtype=np.int64) * n_each
    r = rng.uniform(1.0, 3.0, n_avatars)
    cx = rng.uniform(-5.0 + r + 0.3, 5.0 - r - 0.3)
    cy = rng.uniform(-4.0 + r + 0.3, 4.0 - r - 0.3)
    motion = dict(radius=r, centre=np.stack([cx, cy], 1), phase=rng.uniform(0, 2 * math.pi, n_avatars),
                  direction=rng.choice([-1.0, 1.0], n_avatars), speed=1.0, fps=30.0)
    return rest, seg, motion


def avatar_poses(motion: dict, frame: int) -> np.ndarray:
    """(n_avatars, 8) float32 poses (qw, qx, qy, qz, tx, ty, tz, 0) at `frame`."""
    t = frame / motion["fps"]
    r, d = motion["radius"], motion["direction"]
    th = motion["phase"] + d * motion["speed"] * t / r
    px = motion["centre"][:, 0] + r * np.cos(th)
    py = motion["centre"][:, 1] + r * np.sin(th)
    yaw = np.arctan2(d * np.cos(th), -d * np.sin(th))   # along the tangent of travel
    n = r.shape[0]
    out = np.zeros((n, 8))
    out[:, 0] = np.cos(0.5 * yaw)
    out[:, 3] = np.sin(0.5 * yaw)
    out[:, 4], out[:, 5] = px, py
    return _f32(out)


def cubemap_samples(face: int, seed: int, noise: float = 0.01):
    """Samples (D, Y, w) of a synthetic environment on the six cube faces.

    Stands in for the six 90-degree renders of the scene at the avatar
    (Sec. 3.4): D are unit texel-centre directions (6*face^2, 3), w the exact
    texel solid angles, Y a smooth radiance (ambient + three coloured lobes)
    plus Gaussian noise, clipped at 0.
    """
    rng = np.random.default_rng(seed)
    e = (np.arange(face + 1) / face) * 2.0 - 1.0           # texel edges
    c = 0.5 * (e[:-1] + e[1:])                             # texel centres
    uu, vv = np.meshgrid(c, c, indexing="xy")
    ue0, ve0 = np.meshgrid(e[:-1], e[:-1], indexing="xy")
    ue1, ve1 = np.meshgrid(e[1:], e[1:], indexing="xy")

    def omega(x, y):  # solid angle of the face rectangle [0,x]x[0,y] at unit distance
        return np.arctan2(x * y, np.sqrt(x * x + y * y + 1.0))

    wface = omega(ue1, ve1) - omega(ue0, ve1) - omega(ue1, ve0) + omega(ue0, ve0)
    one = np.ones_like(uu)
    faces = [(one, -vv, -uu), (-one, -vv, uu), (uu, one, vv),
             (uu, -one, -vv), (uu, -vv, one), (-uu, -vv, -one)]
    D = np.concatenate([np.stack(f, -1).reshape(-1, 3) for f in faces])
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    w = np.tile(wface.ravel(), 6)
    lobes = rng.standard_normal((3, 3))
    lobes /= np.linalg.norm(lobes, axis=1, keepdims=True)
    cols = rng.uniform(0.2, 1.5, (3, 3))
    powers = np.array([1.0, 4.0, 16.0])
    Y = np.full((D.shape[0], 3), 0.15) + 0.05 * rng.random(3)
    for a, col, p in zip(lobes, cols, powers):
        Y += np.maximum(D @ a, 0.0)[:, None] ** p * col
    Y += noise * rng.standard_normal(Y.shape)
    Y = np.maximum(Y, 0.0)
    return _f32(D), _f32(Y), _f32(w)


def workload(name: str) -> dict:
    """Named workloads (the configurations the parity tests and bench use).

    'cube20k'     20k-Gaussian cube scene, 1 light at the origin, 64x64 atlas,
                  16 linear shells 0.1-8 m, 20k query Gaussians.
    'room1p6m'    1.5M-Gaussian indoor room + 100k avatar, 1 light at 2.8 m,
                  512x512 atlas, 64 geometric shells 0.05-12 m, order-2 SH
                  relight of the avatar from a 6x64^2 cubemap fit.
    'room550k'    the same room with 300k + 200k + 50k Gaussians.
    'cube3m4l'    cube generator at 3M Gaussians, 4 lights, 64x64x16.
    'crowd8'      the room without its avatar (1.5M static Gaussians; static
                  atlases for 4 ceiling lights at 512x512x64, geometric
                  0.05-12 m), 8 avatars of 100k walking for 120 frames
                  (dynamic atlases 256x256x32, geometric 0.05-12 m), all 2.3M
                  attenuated and the 800k avatar Gaussians relit per frame.
    'crowd8s'     the same at a tenth of the Gaussians (for parity tests).
    """
    if name == "cube20k":
        occ = cube_scene(20_000, seed=0)
        q = cube_scene(20_000, seed=1)
        return dict(name=name, occluders=occ, queries=q, lights=_f32([[0, 0, 0]]),
                    H=64, W=64, radii=radii_linear(0.1, 8.0, 16))
    if name == "room1p6m":
        sc = room_scene(seed=2)
        return dict(name=name, occluders=sc, queries=sc, lights=_f32([[0, 0, 2.8]]),
                    H=512, W=512, radii=radii_geometric(0.05, 12.0, 64),
                    relight=subset(sc, sc.meta["avatar"]), cubemap=cubemap_samples(64, seed=5))
    if name == "room550k":
        # the room at about a third of the size (for profiler captures)
        sc = room_scene(seed=2, n_flat=300_000, n_box=200_000, n_avatar=50_000)
        return dict(name=name, occluders=sc, queries=sc, lights=_f32([[0, 0, 2.8]]),
                    H=512, W=512, radii=radii_geometric(0.05, 12.0, 64),
                    relight=subset(sc, sc.meta["avatar"]), cubemap=cubemap_samples(64, seed=5))
    if name in ("crowd8", "crowd8s"):
        small = name == "crowd8s"
        room = room_scene(seed=2, n_flat=90_000 if small else 900_000,
                          n_box=60_000 if small else 600_000, n_avatar=0)
        rest, seg, motion = avatar_crowd(seed=6, n_each=10_000 if small else 100_000)
        return dict(name=name, static=room, avatars=rest, seg=seg, motion=motion, frames=120,
                    lights=room_lights(), H=512, W=512, radii=radii_geometric(0.05, 12.0, 64),
                    H_dyn=256, W_dyn=256, radii_dyn=radii_geometric(0.05, 12.0, 32),
                    cubemap=cubemap_samples(64, seed=5))
    if name == "cube3m4l":
        occ = cube_scene(3_000_000, seed=3)
        return dict(name=name, occluders=occ, queries=occ, lights=four_lights(),
                    H=64, W=64, radii=radii_linear(0.1, 8.0, 16))
    raise KeyError(name)
