"""Seeded synthetic scenes for inverse path tracing.

This module only builds inputs: triangle meshes split into object segments,
pinhole camera poses and ground-truth per-segment parameters.  It holds none of
the light-transport arithmetic, so both the CUDA path and the FP64 oracle read
the arrays it returns.

The paper's inputs are a triangle mesh with per-object segmentation, camera
poses and linear-colour images (Sec. 3.2, Sec. 4.2).  Its own indoor scenes are
not available, so the generators below build procedural stand-ins of the same
kind: a Cornell-style box and furnished box rooms with rectangular ceiling
lights.

Parameter layout per segment (10 floats, all normalised to roughly [0, 1]):
``[kd_r, kd_g, kd_b, ks_r, ks_g, ks_b, roughness, e_r, e_g, e_b]``.  Emitted
radiance is ``emission_scale * e`` (Sec. 4.1 asks for parameters with similar
ranges; the scale keeps emission of 10-20 inside [0, 1]).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PARAMS_PER_SEGMENT = 10
EMISSION_SCALE = 32.0
MASTER_SEED = 190307145


@dataclass
class Camera:
    """Pinhole camera.  ``cam_to_world`` is 3x4 row-major: columns are the
    camera's right, up and backward axes (it looks down its -z axis) and its
    position."""

    cam_to_world: np.ndarray
    fov_y_deg: float
    width: int
    height: int


@dataclass
class Scene:
    name: str
    positions: np.ndarray          # (V, 3) float32
    indices: np.ndarray            # (T, 3) uint32
    tri_segment: np.ndarray        # (T,) uint32
    n_segments: int
    cameras: list
    gt_params: np.ndarray          # (S, 10) float32
    normals: np.ndarray | None = None   # (V, 3) float32 or None (geometric)
    emission_scale: float = EMISSION_SCALE
    light_segments: list = field(default_factory=list)
    spp: int = 16
    max_depth: int = 3

    @property
    def n_tri(self) -> int:
        return int(self.indices.shape[0])

    @property
    def n_pixels(self) -> int:
        return sum(c.width * c.height for c in self.cameras)


class _MeshBuilder:
    def __init__(self):
        self.pos = []
        self.idx = []
        self.seg = []
        self.nv = 0

    def quad_grid(self, corner, u, v, nu, nv, seg):
        """Planar grid of nu x nv quads spanning corner + [0,1]u + [0,1]v.
        Triangles wind so that their face normal is along cross(u, v)."""
        corner = np.asarray(corner, np.float64)
        u = np.asarray(u, np.float64)
        v = np.asarray(v, np.float64)
        ii, jj = np.meshgrid(np.arange(nu + 1), np.arange(nv + 1), indexing="ij")
        p = corner + (ii[..., None] / nu) * u + (jj[..., None] / nv) * v
        base = self.nv
        self.pos.append(p.reshape(-1, 3))
        vid = lambda i, j: base + i * (nv + 1) + j
        i, j = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
        i = i.ravel()
        j = j.ravel()
        a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
        tris = np.empty((2 * a.size, 3), np.int64)
        tris[0::2] = np.stack([a, b, c], 1)
        tris[1::2] = np.stack([a, c, d], 1)
        self.idx.append(tris)
        self.seg.append(np.full(tris.shape[0], seg, np.int64))
        self.nv += (nu + 1) * (nv + 1)

    def cuboid(self, center_xz, base_y, size, yaw, nsub, seg, top_seg=None):
        """Closed cuboid (outward normals) standing at height base_y, rotated
        by yaw about +y.  size = (sx, sy, sz)."""
        c, s = math.cos(yaw), math.sin(yaw)
        ex = np.array([c, 0.0, -s])
        ey = np.array([0.0, 1.0, 0.0])
        ez = np.array([s, 0.0, c])
        sx, sy, sz = size
        ctr = np.array([center_xz[0], base_y + sy / 2, center_xz[1]])
        half = {"x": sx / 2, "y": sy / 2, "z": sz / 2}
        axes = {"x": ex, "y": ey, "z": ez}
        dims = {"x": sx, "y": sy, "z": sz}
        # (normal axis, sign, t1 axis, t2 axis) with cross(t1, t2) = sign * normal
        faces = [("x", 1, "y", "z"), ("x", -1, "z", "y"),
                 ("y", 1, "z", "x"), ("y", -1, "x", "z"),
                 ("z", 1, "x", "y"), ("z", -1, "y", "x")]
        for n_ax, sign, t1, t2 in faces:
            fc = ctr + sign * half[n_ax] * axes[n_ax]
            u = axes[t1] * dims[t1]
            v = axes[t2] * dims[t2]
            corner = fc - u / 2 - v / 2
            fseg = top_seg if (top_seg is not None and n_ax == "y" and sign > 0) else seg
            self.quad_grid(corner, u, v, nsub, nsub, fseg)

    def box_room(self, size, nsub, segs):
        """Inward-facing box [0,X]x[0,Y]x[0,Z]; segs = (floor, ceiling,
        long walls (z=0, z=Z), short walls (x=0, x=X))."""
        X, Y, Z = size
        floor, ceil, longw, shortw = segs
        self.quad_grid([0, 0, 0], [0, 0, Z], [X, 0, 0], nsub, nsub, floor)        # +y
        self.quad_grid([0, Y, 0], [X, 0, 0], [0, 0, Z], nsub, nsub, ceil)         # -y
        self.quad_grid([0, 0, 0], [X, 0, 0], [0, Y, 0], nsub, nsub, longw)        # +z
        self.quad_grid([0, 0, Z], [0, Y, 0], [X, 0, 0], nsub, nsub, longw)        # -z
        self.quad_grid([0, 0, 0], [0, Y, 0], [0, 0, Z], nsub, nsub, shortw)       # +x
        self.quad_grid([X, 0, 0], [0, 0, Z], [0, Y, 0], nsub, nsub, shortw)       # -x

    def down_facing_rect(self, center, sx, sz, seg):
        cx, cy, cz = center
        corner = [cx - sx / 2, cy, cz - sz / 2]
        self.quad_grid(corner, [sx, 0, 0], [0, 0, sz], 1, 1, seg)   # cross(x, z) = -y

    def finish(self):
        pos = np.concatenate(self.pos).astype(np.float32)
        idx = np.concatenate(self.idx).astype(np.uint32)
        seg = np.concatenate(self.seg).astype(np.uint32)
        return pos, idx, seg


def look_camera(position, yaw, pitch, fov_y_deg, width, height):
    """Camera at ``position`` looking along yaw (about +y) / pitch."""
    f = np.array([math.cos(pitch) * math.sin(yaw), math.sin(pitch),
                  -math.cos(pitch) * math.cos(yaw)])
    right = np.cross(f, [0.0, 1.0, 0.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, f)
    m = np.stack([right, up, -f, np.asarray(position, np.float64)], axis=1)
    return Camera(m.astype(np.float32), float(fov_y_deg), int(width), int(height))


def random_materials(rng, n_segments, light_segments, emission_scale=EMISSION_SCALE):
    """kd ~ U[0.1,0.9]^3, ks ~ U[0,0.3]^3, roughness ~ U[0.05,0.8];
    emission U[10,20]^3 on light segments, 0 elsewhere (stored / scale)."""
    p = np.zeros((n_segments, PARAMS_PER_SEGMENT), np.float64)
    p[:, 0:3] = rng.uniform(0.1, 0.9, (n_segments, 3))
    p[:, 3:6] = rng.uniform(0.0, 0.3, (n_segments, 3))
    p[:, 6] = rng.uniform(0.05, 0.8, n_segments)
    for s in light_segments:
        p[s, 7:10] = rng.uniform(10.0, 20.0, 3) / emission_scale
    return p.astype(np.float32)


def cornell_box(seed: int = 1000, width: int = 64, height: int = 64) -> Scene:
    """Unit box with an open front: floor, emissive ceiling, back, left and
    right walls (2 triangles each) plus two cuboids of 12 triangles, one of
    them rotated by 15 degrees.  34 triangles, 7 segments."""
    rng = np.random.default_rng(seed)
    mb = _MeshBuilder()
    mb.quad_grid([0, 0, 0], [0, 0, 1], [1, 0, 0], 1, 1, 0)   # floor  (+y)
    mb.quad_grid([0, 1, 0], [1, 0, 0], [0, 0, 1], 1, 1, 1)   # ceiling (-y), emissive
    mb.quad_grid([0, 0, 0], [1, 0, 0], [0, 1, 0], 1, 1, 2)   # back   (+z)
    mb.quad_grid([0, 0, 0], [0, 1, 0], [0, 0, 1], 1, 1, 3)   # left   (+x)
    mb.quad_grid([1, 0, 0], [0, 0, 1], [0, 1, 0], 1, 1, 4)   # right  (-x)
    mb.cuboid((0.32, 0.36), 1e-3, (0.28, 0.6, 0.28), math.radians(15.0), 1, 5)
    mb.cuboid((0.70, 0.64), 1e-3, (0.30, 0.3, 0.30), 0.0, 1, 6)
    pos, idx, seg = mb.finish()
    cam = Camera(np.array([[1, 0, 0, 0.5], [0, 1, 0, 0.5], [0, 0, 1, 2.2]], np.float32),
                 40.0, width, height)
    gt = random_materials(rng, 7, [1])
    return Scene("cornell_box_34tri", pos, idx, seg, 7, [cam], gt,
                 light_segments=[1], spp=16, max_depth=3)


def cornell_variant(k: int) -> Scene:
    """Scene k of a 64-scene family of Cornell boxes (seed 6000 + k): the
    box of cornell_box with its two cuboids resized, moved and yawed at
    random, new materials, and one view at one of 32^2, 48^2, 64^2, 96^2 or
    128^2 pixels.  34 triangles, 7 segments, the emitting ceiling in view."""
    rng = np.random.default_rng(6000 + k)
    mb = _MeshBuilder()
    mb.quad_grid([0, 0, 0], [0, 0, 1], [1, 0, 0], 1, 1, 0)
    mb.quad_grid([0, 1, 0], [1, 0, 0], [0, 0, 1], 1, 1, 1)
    mb.quad_grid([0, 0, 0], [1, 0, 0], [0, 1, 0], 1, 1, 2)
    mb.quad_grid([0, 0, 0], [0, 1, 0], [0, 0, 1], 1, 1, 3)
    mb.quad_grid([1, 0, 0], [0, 0, 1], [0, 1, 0], 1, 1, 4)
    a = (rng.uniform(0.22, 0.38), rng.uniform(0.25, 0.45))
    b = (rng.uniform(0.62, 0.78), rng.uniform(0.55, 0.75))
    mb.cuboid(a, 1e-3, (rng.uniform(0.2, 0.3), rng.uniform(0.3, 0.7), rng.uniform(0.2, 0.3)),
              math.radians(rng.uniform(-30.0, 30.0)), 1, 5)
    mb.cuboid(b, 1e-3, (rng.uniform(0.2, 0.3), rng.uniform(0.2, 0.4), rng.uniform(0.2, 0.3)),
              math.radians(rng.uniform(-30.0, 30.0)), 1, 6)
    pos, idx, seg = mb.finish()
    res = [32, 48, 64, 96, 128][int(rng.integers(0, 5))]
    cam = Camera(np.array([[1, 0, 0, 0.5], [0, 1, 0, 0.5], [0, 0, 1, 2.2]], np.float32), 40.0, res, res)
    gt = random_materials(rng, 7, [1])
    return Scene(f"cornell_variant_{k}", pos, idx, seg, 7, [cam], gt, light_segments=[1], spp=16, max_depth=3)


def cornell_textured(seed: int = 1000, sub: int = 16, width: int = 64, height: int = 64) -> Scene:
    """The Cornell box with its five walls split into sub x sub quads and a
    4 x 4 checker of two diffuse albedos on the floor and the back wall (a
    texture that per-segment parameters cannot represent); the segments are
    the objects, as in cornell_box.  gt_params holds the per-segment values
    (the checker's mean on the floor and back wall) and tri_albedo the
    per-triangle diffuse albedo the images are rendered with (see
    per_triangle)."""
    rng = np.random.default_rng(seed)
    mb = _MeshBuilder()
    mb.quad_grid([0, 0, 0], [0, 0, 1], [1, 0, 0], sub, sub, 0)
    mb.quad_grid([0, 1, 0], [1, 0, 0], [0, 0, 1], sub, sub, 1)
    mb.quad_grid([0, 0, 0], [1, 0, 0], [0, 1, 0], sub, sub, 2)
    mb.quad_grid([0, 0, 0], [0, 1, 0], [0, 0, 1], sub, sub, 3)
    mb.quad_grid([1, 0, 0], [0, 0, 1], [0, 1, 0], sub, sub, 4)
    mb.cuboid((0.32, 0.36), 1e-3, (0.28, 0.6, 0.28), math.radians(15.0), 1, 5)
    mb.cuboid((0.70, 0.64), 1e-3, (0.30, 0.3, 0.30), 0.0, 1, 6)
    pos, idx, seg = mb.finish()
    cam = Camera(np.array([[1, 0, 0, 0.5], [0, 1, 0, 0.5], [0, 0, 1, 2.2]], np.float32), 40.0, width, height)
    gt = random_materials(rng, 7, [1])
    gt[:, 3:6] = 0.0   # diffuse only: the texture is an albedo texture
    tri_kd = gt[seg, 0:3].astype(np.float64).copy()
    c = pos[idx].mean(axis=1)
    dark, light = rng.uniform(0.1, 0.3, 3), rng.uniform(0.6, 0.9, 3)
    for s_id, (a, b) in ((0, (0, 2)), (2, (0, 1))):
        on = seg == s_id
        check = ((np.floor(c[:, a] * 4) + np.floor(c[:, b] * 4)) % 2 == 1)
        tri_kd[on & check] = light
        tri_kd[on & ~check] = dark
        gt[s_id, 0:3] = tri_kd[on].mean(axis=0)
    sc = Scene("cornell_textured", pos, idx, seg, 7, [cam], gt, light_segments=[1], spp=16, max_depth=3)
    sc.tri_albedo = tri_kd.astype(np.float32)
    return sc


def per_triangle(scene: Scene, params: np.ndarray | None = None) -> Scene:
    """The same geometry with every triangle its own segment (the paper's
    refinement from per-object to per-triangle material parameters, App. E).
    Triangle t starts from the parameters of its old segment (params, or
    the ground truth); the new ground truth takes a per-triangle albedo when
    the scene carries one (tri_albedo).  Light segments map to their
    triangles."""
    T = scene.n_tri
    seg = np.asarray(scene.tri_segment, np.int64)
    gt = np.asarray(scene.gt_params, np.float32)[seg].copy()
    if getattr(scene, "tri_albedo", None) is not None:
        gt[:, 0:3] = scene.tri_albedo
    lights = [int(t) for t in np.nonzero(np.isin(seg, np.asarray(scene.light_segments, np.int64)))[0]]
    out = Scene(scene.name + "_per_triangle", scene.positions, scene.indices, np.arange(T, dtype=np.uint32), T,
                scene.cameras, gt, normals=scene.normals, emission_scale=scene.emission_scale,
                light_segments=lights, spp=scene.spp, max_depth=scene.max_depth)
    out.start_params = (np.asarray(params, np.float32)[seg].copy() if params is not None
                        else np.asarray(scene.gt_params, np.float32)[seg].copy())
    if getattr(scene, "tri_albedo", None) is not None:
        out.tri_albedo = scene.tri_albedo
    return out


def subdivide(scene: Scene, split: np.ndarray, params: np.ndarray | None = None) -> Scene:
    """Splits the triangles with split[t] into four at their edge midpoints
    (adaptive subdivision, App. B); every triangle stays its own segment and
    the four children inherit their parent's parameters (params, else
    start_params, else the ground truth) and ground truth.  A split
    triangle's midpoints lie on its neighbours' edges, so the surface is
    unchanged."""
    P = np.asarray(scene.positions, np.float64)
    I = np.asarray(scene.indices, np.int64)
    split = np.asarray(split, bool)
    base = params if params is not None else getattr(scene, "start_params", scene.gt_params)
    base = np.asarray(base, np.float32)
    gt = np.asarray(scene.gt_params, np.float32)
    new_pos = [P]
    mid_id = {}

    def mid(a, b):
        k = (min(a, b), max(a, b))
        if k not in mid_id:
            mid_id[k] = len(P) + len(mid_id)
            new_pos.append(((P[a] + P[b]) * 0.5)[None])
        return mid_id[k]

    tris, owner = [], []
    for t, (a, b, c) in enumerate(I):
        if not split[t]:
            tris.append((a, b, c))
            owner.append(t)
            continue
        ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
        for tri in ((a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)):
            tris.append(tri)
            owner.append(t)
    owner = np.asarray(owner, np.int64)
    lights = set(int(x) for x in scene.light_segments)
    out = Scene(scene.name + "_sub", np.concatenate(new_pos).astype(np.float32),
                np.asarray(tris, np.uint32), np.arange(len(tris), dtype=np.uint32), len(tris), scene.cameras,
                gt[owner].copy(), emission_scale=scene.emission_scale,
                light_segments=[i for i, o in enumerate(owner) if int(o) in lights], spp=scene.spp,
                max_depth=scene.max_depth)
    out.start_params = base[owner].copy()
    out.parent = owner
    return out


def _obb_overlap(a, b, margin=0.0):
    """Separating-axis test of two yawed rectangles (cx, cz, hx, hz, yaw)."""
    def axes(r):
        c, s = math.cos(r[4]), math.sin(r[4])
        return [np.array([c, -s]), np.array([s, c])]
    d = np.array([b[0] - a[0], b[1] - a[1]])
    for ax in axes(a) + axes(b):
        ra = sum(h * abs(ax @ e) for h, e in zip(a[2:4], axes(a)))
        rb = sum(h * abs(ax @ e) for h, e in zip(b[2:4], axes(b)))
        if abs(ax @ d) > ra + rb + margin:
            return False
    return True


def _rect_point_dist(r, p):
    c, s = math.cos(r[4]), math.sin(r[4])
    d = np.array([p[0] - r[0], p[1] - r[1]])
    lx = d @ np.array([c, -s])
    lz = d @ np.array([s, c])
    qx = max(abs(lx) - r[2], 0.0)
    qz = max(abs(lz) - r[3], 0.0)
    return math.hypot(qx, qz)


def indoor_room(seed: int, room=(8.0, 3.0, 6.0), n_cuboids=40, cuboid_sub=11,
                room_sub=16, n_lights=4, n_views=8, width=320, height=240,
                split_tops=0, spp=32, max_depth=5, name="room") -> Scene:
    """Box room (X x Y x Z metres, y up) with yawed cuboid furniture proxies
    standing on the floor and downward-facing rectangular ceiling lights.

    Segments: 0 floor, 1 ceiling, 2 long walls, 3 short walls, then one per
    light, one per cuboid, and, for the first ``split_tops`` cuboids, an extra
    segment for the top face.  Camera positions are drawn first; cuboid
    footprints are then placed by rejection so that they do not overlap each
    other and stay 0.3 m from every camera (sizes shrink by 10% after 200
    failed draws, so the requested count always fits)."""
    rng = np.random.default_rng(seed)
    X, Y, Z = room
    mb = _MeshBuilder()
    mb.box_room((X, Y, Z), room_sub, (0, 1, 2, 3))
    seg_next = 4
    light_segs = []
    gx = int(math.ceil(math.sqrt(n_lights * X / Z)))
    gz = int(math.ceil(n_lights / gx))
    k = 0
    for a in range(gx):
        for b in range(gz):
            if k == n_lights:
                break
            cx = (a + 0.5) * X / gx + rng.uniform(-0.2, 0.2)
            cz = (b + 0.5) * Z / gz + rng.uniform(-0.2, 0.2)
            mb.down_facing_rect((cx, Y - 0.01, cz), 0.6, 1.2, seg_next)
            light_segs.append(seg_next)
            seg_next += 1
            k += 1
    # camera positions first
    cam_xyz = []
    for _ in range(n_views):
        cam_xyz.append((rng.uniform(0.6, X - 0.6), rng.uniform(1.2, 1.8),
                        rng.uniform(0.6, Z - 0.6)))
    rects = []
    cub_segs = []
    top_segs = []
    for ci in range(n_cuboids):
        shrink = 1.0
        tries = 0
        while True:
            sx, sy, sz = rng.uniform(0.3, 2.0, 3) * np.array([shrink, 1.0, shrink])
            sy = min(sy, Y - 0.2)
            yaw = rng.uniform(0, 2 * math.pi)
            hx, hz = sx / 2, sz / 2
            rad = math.hypot(hx, hz)
            cx = rng.uniform(rad + 0.02, X - rad - 0.02) if X > 2 * rad + 0.04 else X / 2
            cz = rng.uniform(rad + 0.02, Z - rad - 0.02) if Z > 2 * rad + 0.04 else Z / 2
            r = (cx, cz, hx, hz, yaw)
            ok = all(not _obb_overlap(r, q, 0.02) for q in rects)
            ok = ok and all(_rect_point_dist(r, (p[0], p[2])) > 0.3 for p in cam_xyz)
            if ok:
                break
            tries += 1
            if tries % 200 == 0:
                shrink *= 0.9
        rects.append(r)
        seg = seg_next
        seg_next += 1
        top = None
        if ci < split_tops:
            top = seg_next
            seg_next += 1
            top_segs.append(top)
        cub_segs.append(seg)
        mb.cuboid((cx, cz), 1e-3, (sx, sy, sz), yaw, cuboid_sub, seg, top)
    pos, idx, seg = mb.finish()
    n_seg = seg_next
    cams = []
    for p in cam_xyz:
        cams.append(look_camera(p, rng.uniform(0, 2 * math.pi),
                                math.radians(rng.uniform(-15, 15)), 60.0, width, height))
    gt = random_materials(rng, n_seg, light_segs)
    return Scene(name, pos, idx, seg, n_seg, cams, gt, light_segments=light_segs,
                 spp=spp, max_depth=max_depth)


def room_60k(seed: int = 1001) -> Scene:
    """~61k triangles in 48 segments, 8 views of 320x240, 32 spp, depth 5."""
    return indoor_room(seed, name="room_61k_tri")


def room_500k(seed: int = 1002, n_views: int = 16, width: int = 640, height: int = 480) -> Scene:
    """~516k triangles in 150 segments (4 room + 8 lights + 120 cuboids + 18
    split tops) in a 16 x 4 x 12 m room; 16 views of 640x480, 16 spp, depth 6."""
    return indoor_room(seed, room=(16.0, 4.0, 12.0), n_cuboids=120, cuboid_sub=18,
                       room_sub=64, n_lights=8, n_views=n_views, width=width,
                       height=height, split_tops=18, spp=16, max_depth=6,
                       name="room_516k_tri")


def batch_room(k: int, res_div: int = 1) -> Scene:
    """Room k of the 64-scene batch (seed 5000 + k): triangles log-uniform in
    [5k, 500k], segments uniform in [10, 200], lights in [1, 8], views in
    [1, 8] at one of 160x120, 320x240, 640x480 (each divided by res_div).
    Segments = 4 room + lights + cuboids, so the cuboid count follows; the
    floor grows with it (3 m^2 per cuboid, at least 8 x 6 m, so that
    placement by rejection stays quick), and the cuboid and room-face
    subdivisions are set to land near the drawn triangle count."""
    rng = np.random.default_rng(5000 + k)
    tris = float(np.exp(rng.uniform(np.log(5e3), np.log(5e5))))
    n_seg = int(rng.integers(10, 201))
    n_lights = int(rng.integers(1, 9))
    n_views = int(rng.integers(1, 9))
    w, h = [(160, 120), (320, 240), (640, 480)][int(rng.integers(0, 3))]
    n_cub = max(1, n_seg - 4 - n_lights)
    area = max(48.0, 3.0 * n_cub)
    X, Z = math.sqrt(area * 4.0 / 3.0), math.sqrt(area * 3.0 / 4.0)
    room_sub = int(np.clip(round(math.sqrt(tris * 0.05 / 12.0)), 2, 64))
    rest = max(tris - 12 * room_sub ** 2 - 2 * n_lights, 12.0 * n_cub)
    cub_sub = max(1, int(round(math.sqrt(rest / (12.0 * n_cub)))))
    return indoor_room(5000 + k, room=(X, 3.0, Z), n_cuboids=n_cub, cuboid_sub=cub_sub, room_sub=room_sub,
                       n_lights=n_lights, n_views=n_views, width=max(8, w // res_div),
                       height=max(6, h // res_div), name=f"batch_room_{k}")


def furnace_box(size=1.0, nsub=1, rho=0.5, emission=0.25, width=8, height=8) -> Scene:
    """Closed box (all six faces inward, one segment), Lambertian albedo rho,
    no specular, uniform emission on every face; camera inside."""
    mb = _MeshBuilder()
    mb.box_room((size, size, size), nsub, (0, 0, 0, 0))
    pos, idx, seg = mb.finish()
    cam = look_camera((0.5 * size, 0.5 * size, 0.5 * size), 0.3, 0.2, 60.0, width, height)
    gt = np.zeros((1, PARAMS_PER_SEGMENT), np.float32)
    gt[0, 0:3] = rho
    gt[0, 6] = 0.5
    gt[0, 7:10] = emission
    return Scene("furnace_box", pos, idx, seg, 1, [cam], gt, light_segments=[0])


def to_arrays(scene: Scene):
    """Flat contiguous arrays in the order the C ABI takes them."""
    return (np.ascontiguousarray(scene.positions, np.float32),
            None if scene.normals is None else np.ascontiguousarray(scene.normals, np.float32),
            np.ascontiguousarray(scene.indices, np.uint32),
            np.ascontiguousarray(scene.tri_segment, np.uint32))


def config_scene(index: int) -> Scene:
    """Scene for the named workload: 0 Cornell box, 1 room ~61k triangles,
    2 room ~516k triangles."""
    if index == 0:
        return cornell_box(1000)
    if index == 1:
        return room_60k(1001)
    if index == 2:
        return room_500k(1002)
    raise ValueError(f"no scene for workload {index}")


DISNEY_VALUES = 16  # base rgb, subsurface, metallic, specular, spec tint, roughness, aniso,
                   # sheen, sheen tint, clearcoat, clearcoat gloss, emission rgb


def disney_materials(scene: Scene, seed: int) -> np.ndarray:
    """Random Disney parameter blocks (Sec. 4.1) for a scene: base colour
    U[0.1, 0.9]^3, every other material value U[0, 1] except roughness
    U[0.15, 0.9] (the model's GGX is near-singular towards 0), and the scene's
    own emission on its light segments (stored / emission scale)."""
    rng = np.random.default_rng(seed)
    S = scene.n_segments
    p = np.zeros((S, DISNEY_VALUES), np.float64)
    p[:, 0:3] = rng.uniform(0.1, 0.9, (S, 3))
    p[:, 3:13] = rng.uniform(0.0, 1.0, (S, 10))
    p[:, 7] = rng.uniform(0.15, 0.9, S)
    p[:, 13:16] = np.asarray(scene.gt_params, np.float64)[:, 7:10]
    return p.astype(np.float32)


def initial_params(scene: Scene, value: float = 0.5) -> np.ndarray:
    p = np.full((scene.n_segments, PARAMS_PER_SEGMENT), value, np.float32)
    return p


def random_rays(scene: Scene, n: int, seed: int):
    """Rays with origins uniform in the scene's bounding box (shrunk 5%) and
    isotropic directions (float32)."""
    rng = np.random.default_rng(seed)
    lo = scene.positions.min(0).astype(np.float64)
    hi = scene.positions.max(0).astype(np.float64)
    c = (lo + hi) / 2
    h = (hi - lo) / 2 * 0.95
    o = c + rng.uniform(-1, 1, (n, 3)) * h
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)
