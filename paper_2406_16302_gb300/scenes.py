"""Seeded procedural scenes and edits (input data only).

This module builds triangle meshes, materials, cameras and edits as plain
numpy arrays.  It holds none of the residual estimator's arithmetic: no ray
tracing, no sampling, no BSDF.  Both the CUDA library and the CPU oracle take
its arrays as input, so the two see bit-identical float32 geometry.

Conventions shared by every consumer of these arrays:

* Triangles are one-sided.  The front side is the direction of
  ``cross(v1 - v0, v2 - v0)``; box walls face inward, closed objects outward,
  the area light faces down into the box.
* A material row holds 12 float32:
  ``[type, albedo_rgb(3), alpha, f0_rgb(3), emission_rgb(3), pad]`` with
  ``type`` 0 = Lambert (albedo), 1 = GGX microfacet reflection (alpha, F0).
  Any triangle whose material has non-zero emission is an area emitter that
  radiates from its front side (the paper's x_L is sampled on these).
* The dynamic object is given in object space; an edit supplies one 3x4
  object-to-world transform and one material row per frame (frame 1 =
  original, frame 2 = edited).  A rigid motion keeps the material; a material
  edit keeps the transform.
* Camera: pinhole, ``(pos, look, up, vfov_deg, width, height)``; pixel row 0
  is the top row.

The synthetic scenes stand in for the paper's evaluation scenes (Cornell-box
style rooms with a moved or re-materialed object, Sec. 6), which are not
available here.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

LAMBERT = 0
GGX = 1


def material(kind=LAMBERT, albedo=(0.0, 0.0, 0.0), alpha=1.0, f0=(0.04, 0.04, 0.04),
             emission=(0.0, 0.0, 0.0)) -> np.ndarray:
    m = np.zeros(12, dtype=np.float32)
    m[0] = kind
    m[1:4] = albedo
    m[4] = alpha
    m[5:8] = f0
    m[8:11] = emission
    return m


@dataclass
class Camera:
    pos: tuple
    look: tuple
    up: tuple
    vfov_deg: float
    width: int
    height: int

    def as_array(self) -> np.ndarray:
        return np.array(list(self.pos) + list(self.look) + list(self.up) + [self.vfov_deg],
                        dtype=np.float32)


@dataclass
class Scene:
    static_vertices: np.ndarray      # (Vs, 3) float32, world space
    static_triangles: np.ndarray     # (Ts, 3) uint32
    static_material: np.ndarray      # (Ts,) uint32 index into materials
    dyn_vertices: np.ndarray         # (Vd, 3) float32, object space
    dyn_triangles: np.ndarray        # (Td, 3) uint32
    materials: np.ndarray            # (M, 12) float32
    camera: Camera
    max_depth: int                   # maximum number of path edges
    alpha_min: float = 0.1           # reconnection roughness threshold (Sec. 5)
    d_min: float = 0.0346            # reconnection distance threshold (Sec. 5)
    jacobian_max: float = 10.0       # mapped-path Jacobian threshold (Sec. 5)
    name: str = ""
    object_ranges: np.ndarray = None # (K, 2) uint32: movable objects 1..K as (first, count)
                                     # ranges of the static triangles
    dyn_instance: np.ndarray = None  # (Td,) int32: instance of each dynamic triangle when the
                                     # dynamic mesh is several objects edited together

    @property
    def n_static(self) -> int:
        return int(self.static_triangles.shape[0])

    @property
    def n_dyn(self) -> int:
        return int(self.dyn_triangles.shape[0])


@dataclass
class Edit:
    M1: np.ndarray                   # (3, 4) float32, object -> world in frame 1
    M2: np.ndarray                   # (3, 4) float32, object -> world in frame 2
    mat1: np.ndarray                 # (12,) float32, dynamic object material in frame 1
    mat2: np.ndarray                 # (12,) float32, dynamic object material in frame 2
    name: str = ""
    object: int = 0                  # 0: the dynamic mesh; k >= 1: movable object k

    @property
    def moves(self) -> bool:
        return not np.array_equal(self.M1, self.M2)


# ----------------------------------------------------------------------------
# mesh builders
# ----------------------------------------------------------------------------

class MeshBuilder:
    def __init__(self):
        self.v = []
        self.t = []
        self.m = []
        self.nv = 0

    def add(self, verts, tris, mat_id):
        verts = np.asarray(verts, dtype=np.float64)
        tris = np.asarray(tris, dtype=np.int64)
        self.v.append(verts)
        self.t.append(tris + self.nv)
        self.m.append(np.full(len(tris), mat_id, dtype=np.uint32))
        self.nv += len(verts)

    def arrays(self):
        if not self.v:
            return (np.zeros((0, 3), np.float32), np.zeros((0, 3), np.uint32),
                    np.zeros((0,), np.uint32))
        return (np.concatenate(self.v).astype(np.float32),
                np.concatenate(self.t).astype(np.uint32),
                np.concatenate(self.m).astype(np.uint32))


def quad(center, u, v):
    """Quad c +- u +- v; front side along cross(u, v)."""
    c, u, v = (np.asarray(a, dtype=np.float64) for a in (center, u, v))
    verts = np.stack([c - u - v, c + u - v, c + u + v, c - u + v])
    return verts, np.array([[0, 1, 2], [0, 2, 3]])


def icosphere(level: int):
    """Unit icosphere with outward winding; 20 * 4**level triangles."""
    p = (1.0 + 5.0 ** 0.5) / 2.0
    verts = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
             (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
             (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    for _ in range(level):
        cache = {}
        new_faces = []

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = new_faces
    return np.array(verts), np.array(faces)


def uv_sphere(n_seg: int, n_ring: int):
    """Unit UV sphere, outward winding, 2 * n_seg * (n_ring - 1) triangles."""
    verts = [(0.0, 1.0, 0.0)]
    for r in range(1, n_ring):
        th = math.pi * r / n_ring
        for s in range(n_seg):
            ph = 2 * math.pi * s / n_seg
            verts.append((math.sin(th) * math.cos(ph), math.cos(th), math.sin(th) * math.sin(ph)))
    verts.append((0.0, -1.0, 0.0))
    last = len(verts) - 1
    tris = []
    for s in range(n_seg):
        tris.append((0, 1 + (s + 1) % n_seg, 1 + s))
    for r in range(n_ring - 2):
        a0 = 1 + r * n_seg
        b0 = a0 + n_seg
        for s in range(n_seg):
            a, a1 = a0 + s, a0 + (s + 1) % n_seg
            b, b1 = b0 + s, b0 + (s + 1) % n_seg
            tris.append((a, a1, b1))
            tris.append((a, b1, b))
    base = 1 + (n_ring - 2) * n_seg
    for s in range(n_seg):
        tris.append((last, base + s, base + (s + 1) % n_seg))
    return np.array(verts), np.array(tris)


def box_mesh():
    """Unit cube [-1,1]^3, outward winding, 12 triangles."""
    faces = [((0, 1, 0), (0, 0, 1), (1, 0, 0)), ((0, -1, 0), (1, 0, 0), (0, 0, 1)),
             ((1, 0, 0), (0, 1, 0), (0, 0, 1)), ((-1, 0, 0), (0, 0, 1), (0, 1, 0)),
             ((0, 0, 1), (1, 0, 0), (0, 1, 0)), ((0, 0, -1), (0, 1, 0), (1, 0, 0))]
    vs, ts = [], []
    for c, u, v in faces:
        qv, qt = quad(c, u, v)
        ts.append(qt + len(vs) * 4)
        vs.append(qv)
    return np.concatenate(vs), np.concatenate(ts)


def torus(n_major: int, n_minor: int, R=1.0, r=0.35):
    verts = []
    for i in range(n_major):
        u = 2 * math.pi * i / n_major
        for j in range(n_minor):
            v = 2 * math.pi * j / n_minor
            verts.append(((R + r * math.cos(v)) * math.cos(u), r * math.sin(v),
                          (R + r * math.cos(v)) * math.sin(u)))
    tris = []
    for i in range(n_major):
        for j in range(n_minor):
            a = i * n_minor + j
            b = ((i + 1) % n_major) * n_minor + j
            c = ((i + 1) % n_major) * n_minor + (j + 1) % n_minor
            d = i * n_minor + (j + 1) % n_minor
            tris.append((a, d, c))
            tris.append((a, c, b))
    return np.array(verts), np.array(tris)


def cylinder(n_seg: int):
    """Closed unit cylinder (radius 1, y in [-1, 1]), outward winding."""
    verts = []
    for s in range(n_seg):
        ph = 2 * math.pi * s / n_seg
        verts.append((math.cos(ph), -1.0, math.sin(ph)))
        verts.append((math.cos(ph), 1.0, math.sin(ph)))
    verts.append((0.0, -1.0, 0.0))
    verts.append((0.0, 1.0, 0.0))
    cb, ct = 2 * n_seg, 2 * n_seg + 1
    tris = []
    for s in range(n_seg):
        a, b = 2 * s, 2 * s + 1
        c, d = 2 * ((s + 1) % n_seg), 2 * ((s + 1) % n_seg) + 1
        tris.append((a, b, d))
        tris.append((a, d, c))
        tris.append((cb, a, c))
        tris.append((ct, d, b))
    return np.array(verts), np.array(tris)


def orient_outward(verts, tris, center=None):
    """Flip triangles whose normal points toward the mesh centroid."""
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris).copy()
    c = verts.mean(axis=0) if center is None else np.asarray(center)
    a, b, cc = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    n = np.cross(b - a, cc - a)
    flip = np.einsum("ij,ij->i", n, (a + b + cc) / 3.0 - c) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return tris


def value_noise_3d(points, freq, rng_seed):
    """Smooth value noise in [-1, 1]: trilinear blend of seeded lattice values."""
    rng = np.random.RandomState(rng_seed)
    n = int(freq) + 3
    lattice = rng.uniform(-1.0, 1.0, size=(n, n, n))
    q = (np.asarray(points, dtype=np.float64) + 1.5) / 3.0 * freq
    i0 = np.clip(np.floor(q).astype(int), 0, n - 2)
    f = q - i0
    f = f * f * (3 - 2 * f)
    out = np.zeros(len(q))
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                w = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1])
                     * (f[:, 2] if dz else 1 - f[:, 2]))
                out += w * lattice[i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz]
    return out


def value_noise_2d(x, z, freq, rng_seed):
    rng = np.random.RandomState(rng_seed)
    n = int(freq) + 3
    lattice = rng.uniform(-1.0, 1.0, size=(n, n))
    qx = (np.asarray(x) + 1.0) / 2.0 * freq
    qz = (np.asarray(z) + 1.0) / 2.0 * freq
    ix = np.clip(np.floor(qx).astype(int), 0, n - 2)
    iz = np.clip(np.floor(qz).astype(int), 0, n - 2)
    fx, fz = qx - ix, qz - iz
    fx = fx * fx * (3 - 2 * fx)
    fz = fz * fz * (3 - 2 * fz)
    return ((1 - fx) * (1 - fz) * lattice[ix, iz] + fx * (1 - fz) * lattice[ix + 1, iz]
            + (1 - fx) * fz * lattice[ix, iz + 1] + fx * fz * lattice[ix + 1, iz + 1])


def translate(t) -> np.ndarray:
    M = np.zeros((3, 4), dtype=np.float32)
    M[:, :3] = np.eye(3)
    M[:, 3] = t
    return M


def rotate_y_translate(deg, t) -> np.ndarray:
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    M = np.zeros((3, 4), dtype=np.float64)
    M[:, :3] = [[c, 0, s], [0, 1, 0], [-s, 0, c]]
    M[:, 3] = t
    return M.astype(np.float32)


# ----------------------------------------------------------------------------
# the Cornell-style box shared by the small configurations
# ----------------------------------------------------------------------------

GREY = (0.7, 0.7, 0.7)
RED = (0.7, 0.1, 0.1)
GREEN = (0.1, 0.7, 0.1)


def _box_room(mb: MeshBuilder, mats: list, closed_front=False, light=True,
              light_radiance=15.0):
    grey = len(mats); mats.append(material(LAMBERT, GREY))
    red = len(mats); mats.append(material(LAMBERT, RED))
    green = len(mats); mats.append(material(LAMBERT, GREEN))
    walls = [((0, -1, 0), (0, 0, 1), (1, 0, 0), grey),    # floor, normal +y
             ((0, 1, 0), (1, 0, 0), (0, 0, 1), grey),     # ceiling, normal -y
             ((0, 0, -1), (1, 0, 0), (0, 1, 0), grey),    # back, normal +z
             ((-1, 0, 0), (0, 1, 0), (0, 0, 1), red),     # left, normal +x
             ((1, 0, 0), (0, 0, 1), (0, 1, 0), green)]    # right, normal -x
    if closed_front:
        walls.append(((0, 0, 1), (0, 1, 0), (1, 0, 0), grey))
    for c, u, v, m in walls:
        qv, qt = quad(c, u, v)
        mb.add(qv, qt, m)
    if light:
        lm = len(mats)
        mats.append(material(LAMBERT, (0, 0, 0), emission=(light_radiance,) * 3))
        qv, qt = quad((0, 0.99, 0), (0.25, 0, 0), (0, 0, 0.25))   # normal -y
        mb.add(qv, qt, lm)


def _box_camera(w, h):
    return Camera((0.0, 0.0, 3.4), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 40.0, w, h)


def cfg1_box_sphere(width=64, height=64, max_depth=4):
    """Tiny box: 5 Lambert walls, one 0.5x0.5 quad light (radiance 15), a
    level-3 icosphere (1280 triangles, albedo 0.8) that is translated by
    (0.1, 0, 0) between frames."""
    mb = MeshBuilder(); mats = []
    _box_room(mb, mats)
    sv, st, sm = mb.arrays()
    dv, dt = icosphere(3)
    dv = dv * 0.35
    c = np.array([-0.3, -0.64, -0.2])
    scene = Scene(sv, st, sm, dv.astype(np.float32), dt.astype(np.uint32),
                  np.stack(mats), _box_camera(width, height), max_depth,
                  d_min=0.01 * 2.0 * math.sqrt(3.0), name="cfg1_box_sphere")
    m = material(LAMBERT, (0.8, 0.8, 0.8))
    edit = Edit(translate(c), translate(c + np.array([0.1, 0.0, 0.0])), m, m.copy(),
                name="translate_x_0.1")
    return scene, edit


def box_objects(width=64, height=64, max_depth=4, n_objects=8, level=2, seed=2406):
    """The cfg1 box with n_objects movable icospheres (level 2: 320
    triangles each, radius 0.11-0.16, seeded Lambert albedo) spread over the
    floor on a 4 x 2 grid, for edits that move several objects at once (the
    paper's scenes with 1, 2, 4 and 8 moving objects, Sec. 6).  The scene's
    own dynamic mesh is a small sphere that appears only in edits that name
    object 0; the edits of `move_objects` move objects 1..k."""
    rng = np.random.RandomState(seed)
    mb = MeshBuilder(); mats = []
    _box_room(mb, mats)
    sv, st, sm = mb.arrays()
    verts = [np.asarray(sv, np.float64)]
    tris = [np.asarray(st, np.int64)]
    mids = [np.asarray(sm, np.int64)]
    nv, nt = len(sv), len(st)
    ranges = []
    grid = [(x, z) for z in (-0.45, 0.15) for x in (-0.6, -0.2, 0.2, 0.6)]
    for k in range(n_objects):
        v, t = icosphere(level)
        r = rng.uniform(0.11, 0.16)
        x, z = grid[k % len(grid)]
        c = np.array([x, -1.0 + r + 0.02, z - 0.3 * (k // len(grid))])
        m = len(mats)
        mats.append(material(LAMBERT, tuple(rng.uniform(0.3, 0.9, size=3))))
        verts.append(v * r + c)
        tris.append(t + nv)
        mids.append(np.full(len(t), m))
        ranges.append((nt, len(t)))
        nv += len(v)
        nt += len(t)
    dv, dt = icosphere(1)
    return Scene(np.concatenate(verts).astype(np.float32), np.concatenate(tris).astype(np.uint32),
                 np.concatenate(mids).astype(np.uint32), (dv * 0.1).astype(np.float32),
                 dt.astype(np.uint32), np.stack(mats).astype(np.float32),
                 _box_camera(width, height), max_depth, d_min=0.01 * 2.0 * math.sqrt(3.0),
                 name=f"box_objects_{n_objects}", object_ranges=np.array(ranges, dtype=np.uint32))


def move_objects(scene: Scene, k: int, displacement: float, seed=7, objects=None):
    """Edits moving objects 1..k of `scene` (or the listed `objects`)
    together, each translated by `displacement` along a seeded horizontal
    direction (its material kept); a list for rp_edit_multi / the oracle's
    several-object edit."""
    rng = np.random.RandomState(seed)
    edits = []
    for j in (objects if objects is not None else range(1, k + 1)):
        first, _ = (int(c) for c in scene.object_ranges[j - 1])
        m = np.asarray(scene.materials[int(scene.static_material[first])], np.float32)
        phi = rng.uniform(0.0, 2.0 * math.pi)
        t = displacement * np.array([math.cos(phi), 0.0, math.sin(phi)])
        edits.append(Edit(translate((0.0, 0.0, 0.0)), translate(t), m.copy(), m.copy(),
                          name=f"move_{j}_by_{displacement}", object=j))
    return edits


def displaced_icosphere(level, radius, amp, seed):
    v, t = icosphere(level)
    d = value_noise_3d(v, 4.0, seed)
    v = v * (radius * (1.0 + amp * d))[:, None]
    return v, t


def cfg2_box_blob(width=256, height=256, max_depth=8, blob_level=5):
    """The tiny box with a static sphere plus a seeded displaced icosphere blob
    (20480 triangles at level 5) whose material changes from Lambert albedo
    0.8 to GGX alpha 0.3, F0 0.04."""
    mb = MeshBuilder(); mats = []
    _box_room(mb, mats)
    sph = len(mats); mats.append(material(LAMBERT, (0.8, 0.8, 0.8)))
    sv, stt = icosphere(3)
    mb.add(sv * 0.35 + np.array([-0.3, -0.64, -0.2]), stt, sph)
    s_v, s_t, s_m = mb.arrays()
    bv, bt = displaced_icosphere(blob_level, 0.3, 0.1, seed=2406)
    c = np.array([0.35, -0.65, 0.1])
    scene = Scene(s_v, s_t, s_m, bv.astype(np.float32), bt.astype(np.uint32),
                  np.stack(mats), _box_camera(width, height), max_depth,
                  d_min=0.01 * 2.0 * math.sqrt(3.0), name="cfg2_box_blob")
    M = translate(c)
    edit = Edit(M, M.copy(), material(LAMBERT, (0.8, 0.8, 0.8)),
                material(GGX, (0, 0, 0), alpha=0.3, f0=(0.04, 0.04, 0.04)),
                name="lambert_to_ggx")
    return scene, edit


def box_blob_side_light(width=64, height=64, max_depth=8, blob_level=4, radiance=60.0):
    """The cfg2 box and material edit with the ceiling light replaced by a small
    quad light (0.3 x 0.3) that faces the back wall from 0.15 in front of it:
    the blob receives no direct light, only light from the lit wall patch and
    further bounces -- indirect illumination concentrated in a few directions."""
    mb = MeshBuilder(); mats = []
    _box_room(mb, mats, light=False)
    sph = len(mats); mats.append(material(LAMBERT, (0.8, 0.8, 0.8)))
    sv, stt = icosphere(3)
    mb.add(sv * 0.35 + np.array([-0.3, -0.64, -0.2]), stt, sph)
    lm = len(mats); mats.append(material(LAMBERT, (0, 0, 0), emission=(radiance,) * 3))
    qv, qt = quad((0.45, 0.35, -0.85), (0.15, 0, 0), (0, -0.15, 0))      # normal -z
    mb.add(qv, qt, lm)
    s_v, s_t, s_m = mb.arrays()
    bv, bt = displaced_icosphere(blob_level, 0.3, 0.1, seed=2406)
    c = np.array([0.35, -0.65, 0.1])
    scene = Scene(s_v, s_t, s_m, bv.astype(np.float32), bt.astype(np.uint32),
                  np.stack(mats), _box_camera(width, height), max_depth,
                  d_min=0.01 * 2.0 * math.sqrt(3.0), name="box_blob_side_light")
    M = translate(c)
    edit = Edit(M, M.copy(), material(LAMBERT, (0.8, 0.8, 0.8)),
                material(GGX, (0, 0, 0), alpha=0.3, f0=(0.04, 0.04, 0.04)),
                name="lambert_to_ggx")
    return scene, edit


def cfg3_terrain(width=1024, height=1024, max_depth=8, grid=708, n_instances=200,
                 seed=2406):
    """Terrain at scale: a grid x grid fBm height field (2 * grid^2 triangles),
    n_instances instanced primitives (icosphere / box / torus / cylinder) with
    seeded Lambert or GGX materials, a 50k-triangle displaced UV sphere that is
    rotated 10 degrees about +y and translated by 5% of the extent, and one
    0.4x0.4 quad light at height 1.5 (radiance 30)."""
    rng = np.random.RandomState(seed)
    mb = MeshBuilder(); mats = []
    ground = len(mats); mats.append(material(LAMBERT, (0.6, 0.6, 0.6)))
    xs = np.linspace(-1.0, 1.0, grid + 1)
    X, Z = np.meshgrid(xs, xs, indexing="ij")
    H = np.zeros_like(X)
    amp, freq = 0.08, 3.0
    for o in range(6):
        H += amp * value_noise_2d(X, Z, freq, seed + 17 * o)
        amp *= 0.5; freq *= 2.0
    verts = np.stack([X.ravel(), H.ravel() - 0.2, Z.ravel()], axis=1)
    idx = np.arange((grid + 1) ** 2).reshape(grid + 1, grid + 1)
    a, b = idx[:-1, :-1].ravel(), idx[1:, :-1].ravel()
    c, d = idx[1:, 1:].ravel(), idx[:-1, 1:].ravel()
    # normal +y: (a, d, c) and (a, c, b) with x along the first index, z second
    tris = np.concatenate([np.stack([a, d, c], 1), np.stack([a, c, b], 1)])
    mb.add(verts, tris, ground)
    bases = [icosphere(3), box_mesh(), torus(40, 20), cylinder(64)]
    for i in range(n_instances):
        kind = i % 4
        bv, bt = bases[kind]
        s = rng.uniform(0.02, 0.06)
        p = np.array([rng.uniform(-0.9, 0.9), 0.0, rng.uniform(-0.9, 0.9)])
        p[1] = -0.2 + s + 0.12
        ang = rng.uniform(0, 2 * math.pi)
        R = np.array([[math.cos(ang), 0, math.sin(ang)], [0, 1, 0],
                      [-math.sin(ang), 0, math.cos(ang)]])
        alb = rng.uniform(0.2, 0.9, size=3)
        if rng.uniform() < 0.5:
            m = material(LAMBERT, alb)
        else:
            m = material(GGX, (0, 0, 0), alpha=rng.uniform(0.05, 0.8), f0=alb)
        mid = len(mats); mats.append(m)
        mb.add((bv * s) @ R.T + p, bt, mid)
    lm = len(mats); mats.append(material(LAMBERT, (0, 0, 0), emission=(30.0,) * 3))
    qv, qt = quad((0, 1.5, 0), (0.2, 0, 0), (0, 0, 0.2))
    mb.add(qv, qt, lm)
    sv, st, sm = mb.arrays()
    dv, dt = uv_sphere(250, 101)
    dv = dv * (1.0 + 0.08 * value_noise_3d(dv, 6.0, seed + 5))[:, None] * 0.15
    dt = orient_outward(dv, dt)
    cam = Camera((0.0, 1.2, 2.2), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 45.0, width, height)
    scene = Scene(sv, st, sm, dv.astype(np.float32), dt.astype(np.uint32), np.stack(mats),
                  cam, max_depth, d_min=0.01 * 2.0 * math.sqrt(2.0 ** 2 * 2 + 1.7 ** 2),
                  name="cfg3_terrain")
    c0 = np.array([0.1, 0.05, 0.1])
    extent = 2.0 * math.sqrt(2.0)
    m = material(LAMBERT, (0.8, 0.8, 0.8))
    edit = Edit(rotate_y_translate(0.0, c0),
                rotate_y_translate(10.0, c0 + np.array([0.05 * extent / math.sqrt(2), 0.0,
                                                        0.0])),
                m, m.copy(), name="rotate10_translate5pct")
    return scene, edit


# ----------------------------------------------------------------------------
# tiny scenes with closed-form answers (used to pin the oracle)
# ----------------------------------------------------------------------------

def furnace_box(albedo=0.5, radiance=1.0, max_depth=4, width=8, height=8):
    """Closed box, every wall Lambert `albedo` and emitting `radiance`; the
    camera sits at the centre.  Every pixel equals
    radiance * sum_{j<max_depth} albedo^j."""
    mb = MeshBuilder()
    mats = [material(LAMBERT, (albedo,) * 3, emission=(radiance,) * 3)]
    walls = [((0, -1, 0), (0, 0, 1), (1, 0, 0)), ((0, 1, 0), (1, 0, 0), (0, 0, 1)),
             ((0, 0, -1), (1, 0, 0), (0, 1, 0)), ((-1, 0, 0), (0, 1, 0), (0, 0, 1)),
             ((1, 0, 0), (0, 0, 1), (0, 1, 0)), ((0, 0, 1), (0, 1, 0), (1, 0, 0))]
    for c, u, v in walls:
        qv, qt = quad(c, u, v)
        mb.add(qv, qt, 0)
    sv, st, sm = mb.arrays()
    dv, dt = icosphere(0)
    cam = Camera((0.0, 0.0, 0.0), (0.0, 0.0, -1.0), (0.0, 1.0, 0.0), 60.0, width, height)
    # the dynamic object is parked far outside the closed box (never seen)
    scene = Scene(sv, st, sm, (dv * 0.1).astype(np.float32), dt.astype(np.uint32),
                  np.stack(mats), cam, max_depth, name="furnace")
    m = material(LAMBERT, (0.5, 0.5, 0.5))
    far = translate((50.0, 50.0, 50.0))
    return scene, Edit(far, far.copy(), m, m.copy(), name="identity")


def wall_and_quad(width=16, height=16, max_depth=2, shift=0.1, light_radiance=10.0,
                  wall_albedo=0.6, quad_albedo=0.9):
    """Back wall (z = 0), a small dynamic quad in front of it and a quad light
    above the view.  The light's shadow of the small quad falls outside the
    view, so with max_depth 2 every pixel is (albedo/pi) * E(x) with E the
    closed-form irradiance of a polygonal Lambertian emitter."""
    mb = MeshBuilder()
    mats = [material(LAMBERT, (wall_albedo,) * 3),
            material(LAMBERT, (0, 0, 0), emission=(light_radiance,) * 3)]
    qv, qt = quad((0, 0, 0), (2.0, 0, 0), (0, 2.0, 0))            # normal +z
    mb.add(qv, qt, 0)
    # light at y = 1.5, z = 2, tilted to face (0, -1, -1)/sqrt2
    n = np.array([0.0, -1.0, -1.0]) / math.sqrt(2.0)
    u = np.array([0.25, 0.0, 0.0])
    v = np.cross(n, u)           # cross(u, v) must be along n
    v = -v if np.dot(np.cross(u, v), n) < 0 else v
    v = v / np.linalg.norm(v) * 0.25
    qv, qt = quad((0.0, 1.5, 2.0), u, v)
    mb.add(qv, qt, 1)
    sv, st, sm = mb.arrays()
    dv, dt = quad((0, 0, 0), (0.15, 0, 0), (0, 0.15, 0))          # normal +z
    cam = Camera((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 30.0, width, height)
    scene = Scene(sv, st, sm, dv.astype(np.float32), dt.astype(np.uint32), np.stack(mats),
                  cam, max_depth, d_min=0.02, name="wall_and_quad")
    m = material(LAMBERT, (quad_albedo,) * 3)
    c = np.array([0.0, -0.7, 0.5])
    edit = Edit(translate(c), translate(c + np.array([shift, 0.0, 0.0])), m, m.copy(),
                name="quad_shift")
    return scene, edit


def identity_edit(edit: Edit) -> Edit:
    return Edit(edit.M1.copy(), edit.M1.copy(), edit.mat1.copy(), edit.mat1.copy(),
                name="identity")


def light_quads(scene: Scene):
    """Emissive triangles of a scene, as (tri index, material row) pairs."""
    em = scene.materials[:, 8:11].sum(axis=1) > 0
    return np.nonzero(em[scene.static_material])[0]


# --- seeded networks for the learned proposal of technique (3) --------------

GUIDE_LAYER_SHAPES = [(64, 80), (64, 64), (64, 64), (64, 64), (48, 64)]   # (out, in)


def guide_box(vertices):
    """(center xyz, inverse half extent xyz) of an object-space vertex array:
    the normalisation of the proposal network's position input."""
    v = np.asarray(vertices, dtype=np.float64)
    lo, hi = v.min(axis=0), v.max(axis=0)
    c = 0.5 * (lo + hi)
    h = np.maximum(0.5 * (hi - lo), 1e-6)
    return np.concatenate([c, 1.0 / h]).astype(np.float32)


def random_int_guide(seed, box, shifts=(9, 9, 9, 10), out_exp=12):
    """A seeded integer network: weights uniform in [-127, 127], the given
    hidden requantisation shifts and output exponent."""
    rng = np.random.default_rng(seed)
    W = rng.integers(-127, 128, size=sum(o * i for o, i in GUIDE_LAYER_SHAPES)).astype(np.int32)
    return W, np.asarray(shifts, dtype=np.int32), int(out_exp), np.asarray(box, dtype=np.float32)


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), as float32."""
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    a = (a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000
    return a.astype(np.uint32).view(np.float32)


def random_float_guide(seed, gain=1.0):
    """Seeded float weights of the same network (He initialisation, rounded
    to bfloat16 so that both precisions start from the same values)."""
    rng = np.random.default_rng(seed)
    out = []
    for o, i in GUIDE_LAYER_SHAPES:
        out.append(rng.normal(0.0, gain * np.sqrt(2.0 / i), size=o * i))
    return bf16_round(np.concatenate(out).astype(np.float32)).astype(np.float64)


# --- several movable objects and batches of edits ----------------------------

def object_view(scene: Scene, k: int) -> Scene:
    """The same geometry with movable object k (k >= 1) as the dynamic mesh
    (its given coordinates as object space) and removed from the static
    triangles; k = 0 returns the scene itself.  Only array slicing."""
    if k == 0:
        return scene
    first, count = (int(v) for v in scene.object_ranges[k - 1])
    tri = np.asarray(scene.static_triangles)
    keep = np.ones(len(tri), dtype=bool)
    keep[first:first + count] = False
    ot = tri[first:first + count]
    used, inv = np.unique(ot.ravel(), return_inverse=True)
    return Scene(scene.static_vertices, tri[keep], np.asarray(scene.static_material)[keep],
                 np.asarray(scene.static_vertices)[used], inv.reshape(-1, 3).astype(np.uint32),
                 scene.materials, scene.camera, scene.max_depth, scene.alpha_min, scene.d_min,
                 scene.jacobian_max, scene.name + f"_object{k}")


def objects_view(scene: Scene, ks) -> Scene:
    """The same geometry with several objects as one dynamic mesh: the
    listed objects (0: the scene's dynamic mesh, k >= 1: movable object k),
    in that order, each an instance with its own transforms; movable objects
    are removed from the static triangles.  Only array slicing."""
    ks = [int(k) for k in ks]
    assert len(set(ks)) == len(ks) and len(ks) >= 1
    tri = np.asarray(scene.static_triangles)
    keep = np.ones(len(tri), dtype=bool)
    verts, tris, inst = [], [], []
    nv = 0
    for i, k in enumerate(ks):
        if k == 0:
            v = np.asarray(scene.dyn_vertices, np.float32)
            t = np.asarray(scene.dyn_triangles, np.int64)
        else:
            first, count = (int(c) for c in scene.object_ranges[k - 1])
            keep[first:first + count] = False
            ot = tri[first:first + count]
            used, inv = np.unique(ot.ravel(), return_inverse=True)
            v = np.asarray(scene.static_vertices, np.float32)[used]
            t = inv.reshape(-1, 3).astype(np.int64)
        verts.append(v)
        tris.append(t + nv)
        inst.append(np.full(len(t), i, np.int32))
        nv += len(v)
    return Scene(scene.static_vertices, tri[keep], np.asarray(scene.static_material)[keep],
                 np.concatenate(verts), np.concatenate(tris).astype(np.uint32),
                 scene.materials, scene.camera, scene.max_depth, scene.alpha_min, scene.d_min,
                 scene.jacobian_max, scene.name + "_objects" + "_".join(map(str, ks)),
                 dyn_instance=np.concatenate(inst))


def uv_sphere_fast(n_seg: int, n_ring: int):
    """uv_sphere(n_seg, n_ring) built with array operations (same vertices and
    triangles)."""
    th = math.pi * np.arange(1, n_ring) / n_ring
    ph = 2 * math.pi * np.arange(n_seg) / n_seg
    T, P = np.meshgrid(th, ph, indexing="ij")
    ring = np.stack([np.sin(T) * np.cos(P), np.cos(T), np.sin(T) * np.sin(P)], -1).reshape(-1, 3)
    verts = np.concatenate([[[0.0, 1.0, 0.0]], ring, [[0.0, -1.0, 0.0]]])
    last = len(verts) - 1
    s_ = np.arange(n_seg)
    top = np.stack([np.zeros(n_seg, int), 1 + (s_ + 1) % n_seg, 1 + s_], 1)
    r_ = np.arange(n_ring - 2)[:, None]
    a = 1 + r_ * n_seg + s_[None, :]
    a1 = 1 + r_ * n_seg + ((s_ + 1) % n_seg)[None, :]
    b, b1 = a + n_seg, a1 + n_seg
    mid = np.stack([np.stack([a, a1, b1], -1), np.stack([a, b1, b], -1)], 2).reshape(-1, 3)
    base = 1 + (n_ring - 2) * n_seg
    bot = np.stack([np.full(n_seg, last), base + s_, base + (s_ + 1) % n_seg], 1)
    return verts, np.concatenate([top, mid, bot])


def rigid_about(center, deg, axis, t) -> np.ndarray:
    """Rotation by deg about a unit axis through center, then translation t."""
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    a = math.radians(deg)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    R = np.eye(3) + math.sin(a) * K + (1 - math.cos(a)) * K @ K
    c = np.asarray(center, dtype=np.float64)
    M = np.zeros((3, 4))
    M[:, :3] = R
    M[:, 3] = c + np.asarray(t, dtype=np.float64) - R @ c
    return M.astype(np.float32)


def cfg4_batch(n_objects=32, seed=2406, min_tris=1000, max_tris=200000, max_depth=8,
               resolutions=(256, 512, 1024), spp_range=(64, 256)):
    """The cfg2 box and blob plus n_objects movable objects (displaced UV
    spheres of log-uniform 1k..200k triangles, seeded Lambert albedo), and
    one animation frame per object: an edit that moves it by a seeded rigid
    transform (rotation <= 10 degrees about a random axis through its center,
    translation <= 5% of the 2-unit extent), at a seeded resolution from
    `resolutions` and a log-uniform spp in spp_range.
    Returns (scene, [(edit, width, height, spp)])."""
    rng = np.random.RandomState(seed)
    base, _ = cfg2_box_blob(width=256, height=256, max_depth=max_depth, blob_level=5)
    mats = list(base.materials)
    verts = [np.asarray(base.static_vertices, np.float64)]
    tris = [np.asarray(base.static_triangles, np.int64)]
    mids = [np.asarray(base.static_material, np.int64)]
    nv = len(verts[0])
    nt = len(tris[0])
    ranges, centers, albedos = [], [], []
    for k in range(n_objects):
        target = math.exp(rng.uniform(math.log(min_tris), math.log(max_tris)))
        n_ring = max(4, int(round(math.sqrt(target / 4.0))))
        n_seg = max(6, int(round(target / (2.0 * (n_ring - 1)))))
        v, t = uv_sphere_fast(n_seg, n_ring)
        r = rng.uniform(0.06, 0.14)
        noise = value_noise_3d(v, 3.0, seed + 31 * k)
        v = v * (r * (1.0 + 0.15 * noise))[:, None]
        c = np.array([rng.uniform(-0.8, 0.8), rng.uniform(-0.85, 0.6), rng.uniform(-0.8, 0.6)])
        alb = rng.uniform(0.2, 0.9, size=3)
        m = len(mats)
        mats.append(material(LAMBERT, tuple(alb)))
        verts.append(v + c)
        tris.append(t + nv)
        mids.append(np.full(len(t), m))
        ranges.append((nt, len(t)))
        centers.append(c)
        albedos.append(m)
        nv += len(v)
        nt += len(t)
    scene = Scene(np.concatenate(verts).astype(np.float32), np.concatenate(tris).astype(np.uint32),
                  np.concatenate(mids).astype(np.uint32), base.dyn_vertices, base.dyn_triangles,
                  np.stack(mats).astype(np.float32), base.camera, max_depth,
                  d_min=base.d_min, name="cfg4_batch",
                  object_ranges=np.array(ranges, dtype=np.uint32))
    frames = []
    ident = translate((0.0, 0.0, 0.0))
    for k in range(n_objects):
        axis = rng.normal(size=3)
        deg = rng.uniform(-10.0, 10.0)
        tdir = rng.normal(size=3)
        tdir *= rng.uniform(0.0, 0.1) / np.linalg.norm(tdir)
        M2 = rigid_about(centers[k], deg, axis, tdir)
        mrow = scene.materials[albedos[k]]
        res = int(rng.choice(resolutions))
        spp = int(round(math.exp(rng.uniform(math.log(spp_range[0]), math.log(spp_range[1])))))
        e = Edit(ident.copy(), M2, mrow.copy(), mrow.copy(), name=f"move_object_{k + 1}",
                 object=k + 1)
        frames.append((e, res, res, spp))
    return scene, frames
