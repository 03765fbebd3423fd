"""Shared test helpers: closed forms, statistics and a spawn process pool.

Nothing here implements the estimator; the closed forms are textbook results
(Lambert's polygon irradiance) evaluated with numpy.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# ---------------------------------------------------------------------------
# closed-form irradiance of a Lambertian polygon (Lambert 1760; see e.g.
# Arvo 1995 "Applications of irradiance tensors"): E = (L/2) sum_i theta_i
# (gamma_i . n) for a polygon entirely above the receiver's tangent plane.
# ---------------------------------------------------------------------------

def polygon_irradiance(x, n, poly, radiance):
    """x: (P, 3) receiver points, n: (3,) receiver normal, poly: (V, 3)."""
    x = np.asarray(x, dtype=np.float64)
    acc = np.zeros(len(x))
    V = len(poly)
    for i in range(V):
        a = poly[i][None, :] - x
        b = poly[(i + 1) % V][None, :] - x
        an = a / np.linalg.norm(a, axis=1, keepdims=True)
        bn = b / np.linalg.norm(b, axis=1, keepdims=True)
        theta = np.arccos(np.clip(np.einsum("ij,ij->i", an, bn), -1.0, 1.0))
        g = np.cross(a, b)
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        acc += theta * (g @ np.asarray(n, dtype=np.float64))
    return 0.5 * radiance * np.abs(acc)


def polygon_irradiance_quadrature(x, n, poly, radiance, m=400):
    """Midpoint quadrature of L cos_x cos_L / r^2 over a planar quad."""
    p0, p1, p2, p3 = (np.asarray(p, dtype=np.float64) for p in poly)
    u = (np.arange(m) + 0.5) / m
    U, Vv = np.meshgrid(u, u, indexing="ij")
    pts = (p0[None, None] + U[..., None] * (p1 - p0)[None, None]
           + Vv[..., None] * (p3 - p0)[None, None]).reshape(-1, 3)
    nl = np.cross(p1 - p0, p3 - p0)
    area = np.linalg.norm(nl)
    nl /= area
    d = pts - x[None, :]
    r2 = np.einsum("ij,ij->i", d, d)
    r = np.sqrt(r2)
    cx = np.clip(d @ n / r, 0, None)
    cl = np.clip(-(d @ nl) / r, 0, None)
    return radiance * np.sum(cx * cl / r2) * area / (m * m)


def camera_basis(cam):
    pos = np.array(cam.pos, dtype=np.float64)
    fwd = np.array(cam.look, dtype=np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.array(cam.up, dtype=np.float64))
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    hh = np.tan(np.radians(cam.vfov_deg) / 2)
    hw = hh * cam.width / cam.height
    return pos, fwd, right, up, hw, hh


def film_rays(cam, sub=32):
    """Per pixel a sub x sub midpoint grid of unit ray directions:
    array (H, W, sub*sub, 3)."""
    pos, fwd, right, up, hw, hh = camera_basis(cam)
    W, H = cam.width, cam.height
    s = (np.arange(sub) + 0.5) / sub
    px = (np.arange(W)[:, None] + s[None, :]).ravel()      # W*sub
    py = (np.arange(H)[:, None] + s[None, :]).ravel()      # H*sub
    sx = (2 * px / W - 1) * hw
    sy = (1 - 2 * py / H) * hh
    SY, SX = np.meshgrid(sy, sx, indexing="ij")
    d = fwd[None, None] + SX[..., None] * right[None, None] + SY[..., None] * up[None, None]
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    d = d.reshape(H, sub, W, sub, 3).transpose(0, 2, 1, 3, 4).reshape(H, W, sub * sub, 3)
    return pos, d


def wall_and_quad_closed_form(scene, edit, frame, sub=32):
    """Direct-lighting image (max depth 2) of scenes.wall_and_quad: every
    visible point is unshadowed, so pixel = mean over the pixel of
    (albedo / pi) * E(x)."""
    cam = scene.camera
    pos, d = film_rays(cam, sub)
    M = (edit.M1 if frame == 1 else edit.M2).astype(np.float64)
    qv = scene.dyn_vertices.astype(np.float64) @ M[:, :3].T + M[:, 3]
    qz = qv[0, 2]
    qlo, qhi = qv.min(axis=0), qv.max(axis=0)
    light_ids = np.nonzero(scene.materials[scene.static_material, 8] > 0)[0]
    tri0 = scene.static_triangles[light_ids[0]]
    tri1 = scene.static_triangles[light_ids[1]]
    corners = [tri0[0], tri0[1], tri0[2], tri1[2]]
    poly = scene.static_vertices[corners].astype(np.float64)
    L = float(scene.materials[scene.static_material[light_ids[0]], 8])
    wall_rho = float(scene.materials[scene.static_material[0], 1])
    quad_rho = float((edit.mat1 if frame == 1 else edit.mat2)[1])
    tq = (qz - pos[2]) / d[..., 2]
    pq = pos + tq[..., None] * d
    inq = ((pq[..., 0] >= qlo[0]) & (pq[..., 0] <= qhi[0]) & (pq[..., 1] >= qlo[1])
           & (pq[..., 1] <= qhi[1]))
    tw = (0.0 - pos[2]) / d[..., 2]
    pw = pos + tw[..., None] * d
    pts = np.where(inq[..., None], pq, pw)
    rho = np.where(inq, quad_rho, wall_rho)
    E = polygon_irradiance(pts.reshape(-1, 3), np.array([0.0, 0.0, 1.0]), poly, L)
    val = rho / np.pi * E.reshape(rho.shape)
    img = val.mean(axis=-1)
    return np.repeat(img[..., None], 3, axis=-1)


# ---------------------------------------------------------------------------
# repeated independent estimates in a spawn pool
# ---------------------------------------------------------------------------

def _job(args):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    from paper_2406_16302_gb300 import scenes
    kind, builder, bargs, seed, spp, mask, edit_kind, guide, domain = args
    if isinstance(edit_kind, tuple) and edit_kind[0] == "objects":
        # objects 1..k of a several-object scene moved by d (one dynamic set)
        _, k, d = edit_kind
        full = getattr(scenes, builder)(**bargs)
        edit = scenes.move_objects(full, k, d)
        scene = scenes.objects_view(full, [e.object for e in edit])
    else:
        scene, edit = getattr(scenes, builder)(**bargs)
    if edit_kind == "identity":
        edit = scenes.identity_edit(edit)
    o = oracle.Oracle(scene, edit)
    if guide is not None:
        gseed, gkw = guide
        o.set_guide(scenes.random_int_guide(gseed, scenes.guide_box(scene.dyn_vertices), **gkw))
    if kind == "corr":
        return (o.render_primal(2, spp, seed, domain=domain)
                - o.render_primal(1, spp, seed, domain=domain))
    if kind == "p1":
        return o.render_primal(1, spp, seed)
    if kind == "p2":
        return o.render_primal(2, spp, seed)
    if kind == "res_nomap":
        o.set_mapping(0)
    if kind == "res_objmap":
        o.set_mapping(1)
    return o.render_residual(spp, seed, tech_mask=mask)


def run_many(kind, builder, bargs, seeds, spp, mask=15, edit_kind=None, procs=None, guide=None,
             domain=0):
    """Independent oracle renders, one per seed.  guide = (seed, kwargs) of
    a seeded integer proposal network for technique (3); domain restricts the
    correlated path-traced difference to the paths of some of techniques
    (1)-(3)."""
    jobs = [(kind, builder, bargs, s, spp, mask, edit_kind, guide, domain) for s in seeds]
    procs = procs or min(len(jobs), os.cpu_count() or 1)
    if procs <= 1:
        return np.array([_job(j) for j in jobs])
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        return np.array(pool.map(_job, jobs))


def zscores(a, b):
    """Per-element z of the difference of two sets of independent repeats
    (axis 0), and the z of their image sums."""
    ka, kb = len(a), len(b)
    ma, mb = a.mean(0), b.mean(0)
    va, vb = a.var(0, ddof=1) / ka, b.var(0, ddof=1) / kb
    z = (ma - mb) / np.sqrt(va + vb + 1e-300)
    sa, sb = a.reshape(ka, -1).sum(1), b.reshape(kb, -1).sum(1)
    zs = (sa.mean() - sb.mean()) / np.sqrt(sa.var(ddof=1) / ka + sb.var(ddof=1) / kb)
    return z, zs
