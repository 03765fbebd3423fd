"""ctypes front end of the CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` leg are the only callers.
The product library never imports this package.

The oracle is single-threaded plain C in double precision.  ``build()``
compiles it with gcc; ``Oracle`` wraps one scene + edit.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

TECH_PT, TECH_T1, TECH_T2, TECH_T3, TECH_T4, TECH_T5, TECH_T6, TECH_T7 = 0, 1, 2, 3, 4, 5, 6, 7
MASK_ALL = 0b1111                  # bit 0: T1, bit 1: T2, bit 2: T3, bit 3: T7
MASK_GHOSTS = 0b1110000            # bit 4: T4, bit 5: T5, bit 6: T6 (ghost techniques)
MASK_SEVEN = MASK_ALL | MASK_GHOSTS

# status codes of a base path's mapping (see oracle.c)
MAP_ACCEPT, MAP_INVALID, MAP_REJECT_NODYN, MAP_REJECT_MULTI, MAP_REJECT_INVERT, MAP_REJECT_JAC, \
    MAP_OFF = range(7)

RECORD_DTYPE = np.dtype([
    ("root", "<u4"), ("tech", "<i4"), ("frame", "<i4"), ("sa", "<i4"), ("sb", "<i4"),
    ("pix_a", "<i4"), ("pix_b", "<i4"), ("_pad0", "<i4"),
    ("va", "<f8", 3), ("vb", "<f8", 3), ("status", "<i4"), ("_pad1", "<i4"),
    ("Pg", "<f8"), ("Py", "<f8"), ("J", "<f8"),
])


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        P = C.c_void_p
        L.oracle_create.restype = P
        L.oracle_create.argtypes = [P, C.c_int, P, P, C.c_int, P, C.c_int, P, C.c_int, P, C.c_int,
                                    P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                    C.c_double]
        L.oracle_set_edit.argtypes = [P, P, P, P, P]
        L.oracle_set_edit_multi.restype = C.c_int
        L.oracle_set_edit_multi.argtypes = [P, C.c_int, P, P, P, P, P]
        L.oracle_set_brute_force.argtypes = [P, C.c_int]
        L.oracle_set_mapping.argtypes = [P, C.c_int]
        L.oracle_destroy.argtypes = [P]
        L.oracle_render_residual.argtypes = [P, C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint32,
                                             C.c_int, P, P]
        L.oracle_render_primal.argtypes = [P, C.c_int, C.c_uint32, C.c_uint64, C.c_uint32,
                                           C.c_uint32, P]
        L.oracle_render_primal_domain.argtypes = [P, C.c_int, C.c_uint32, C.c_uint64, C.c_uint32,
                                                  C.c_uint32, C.c_int, P]
        L.oracle_dump.restype = C.c_int64
        L.oracle_dump.argtypes = [P, C.c_int, C.c_int, C.c_uint32, C.c_uint64, C.c_uint32,
                                  C.c_uint32, C.c_int, P, C.c_int64]
        L.oracle_record_size.restype = C.c_int
        L.oracle_closest_hit.argtypes = [P, C.c_int, C.c_int, P, P, P, P, P, P]
        L.oracle_philox4x32_10.argtypes = [P, P, P]
        L.oracle_bsdf.argtypes = [P, P, P, P, P, P]
        L.oracle_bsdf_sample.restype = C.c_int
        L.oracle_bsdf_sample.argtypes = [P, P, P, C.c_double, C.c_double, P, P]
        L.oracle_tangent_frame.argtypes = [P, P, P]
        L.oracle_check_mapping.argtypes = [P, C.c_int, C.c_int, C.c_uint32, C.c_uint64,
                                           C.c_uint32, C.c_uint32, P]
        L.oracle_set_guide.argtypes = [P, P, P, C.c_int, P]
        L.oracle_guide_encode.argtypes = [P, P, P, P]
        L.oracle_guide_forward.argtypes = [P, P, C.c_int, P, C.c_int, P]
        L.oracle_vmf_pdf.restype = C.c_double
        L.oracle_vmf_pdf.argtypes = [P, C.c_double, P]
        L.oracle_vmf_sample.argtypes = [P, C.c_double, C.c_double, C.c_double, P]
        L.oracle_guide_mixture.argtypes = [P, P, P, P]
        L.oracle_mlp_forward.argtypes = [P, P, C.c_int, P]
        L.oracle_mlp_loss_grad.restype = C.c_double
        L.oracle_mlp_loss_grad.argtypes = [P, P, P, P, C.c_int, P]
        L.oracle_mis_terms.restype = C.c_int
        L.oracle_mis_terms.argtypes = [P, C.c_int, C.c_int, P, P, C.c_int, P, P, C.c_int]
        assert L.oracle_record_size() == RECORD_DTYPE.itemsize, "record layout mismatch"
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def philox4x32_10(counter, key):
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def bsdf(mat_row, n, wi, wo):
    m = np.ascontiguousarray(mat_row, dtype=np.float32)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (n, wi, wo)]
    rho = np.zeros(3)
    pdf = np.zeros(1)
    lib().oracle_bsdf(_p(m), _p(arrs[0]), _p(arrs[1]), _p(arrs[2]), _p(rho), _p(pdf))
    return rho, float(pdf[0])


def bsdf_sample(mat_row, n, wc, u1, u2):
    m = np.ascontiguousarray(mat_row, dtype=np.float32)
    n = np.ascontiguousarray(n, dtype=np.float64)
    wc = np.ascontiguousarray(wc, dtype=np.float64)
    wo = np.zeros(3)
    ub = np.zeros(2)
    ok = lib().oracle_bsdf_sample(_p(m), _p(n), _p(wc), float(u1), float(u2), _p(wo), _p(ub))
    return (wo, ub) if ok else (None, None)


def tangent_frame(n):
    n = np.ascontiguousarray(n, dtype=np.float64)
    t = np.zeros(3)
    b = np.zeros(3)
    lib().oracle_tangent_frame(_p(n), _p(t), _p(b))
    return t, b


# --- learned proposal (network of technique (3)'s light-side direction) ----

GUIDE_IN, GUIDE_HID, GUIDE_OUT, GUIDE_LOBES = 80, 64, 48, 8
GUIDE_LAYER_SHAPES = [(64, 80), (64, 64), (64, 64), (64, 64), (48, 64)]   # (out, in)
GUIDE_WEIGHTS = sum(o * i for o, i in GUIDE_LAYER_SHAPES)                   # 20480


def guide_encode(box, p, n):
    """Integer input features of an object-space point and unit normal."""
    b = np.ascontiguousarray(box, dtype=np.float32)
    m = np.zeros(GUIDE_IN, dtype=np.int32)
    lib().oracle_guide_encode(_p(b), _p(np.ascontiguousarray(p, dtype=np.float64)),
                              _p(np.ascontiguousarray(n, dtype=np.float64)), _p(m))
    return m


def guide_forward(W, shift, out_exp, m):
    """Integer network: W int32[20480], shift[4], inputs m[rows][80] -> outputs [rows][48]."""
    W = np.ascontiguousarray(W, dtype=np.int32)
    sh = np.ascontiguousarray(shift, dtype=np.int32)
    m = np.ascontiguousarray(np.atleast_2d(m), dtype=np.int32)
    out = np.zeros((len(m), GUIDE_OUT))
    lib().oracle_guide_forward(_p(W), _p(sh), int(out_exp), _p(m), len(m), _p(out))
    return out


def guide_mixture(o):
    o = np.ascontiguousarray(o, dtype=np.float64)
    pi = np.zeros(GUIDE_LOBES); mu = np.zeros((GUIDE_LOBES, 3)); kappa = np.zeros(GUIDE_LOBES)
    lib().oracle_guide_mixture(_p(o), _p(pi), _p(mu), _p(kappa))
    return pi, mu, kappa


def vmf_pdf(mu, kappa, w):
    return lib().oracle_vmf_pdf(_p(np.ascontiguousarray(mu, dtype=np.float64)), float(kappa),
                                _p(np.ascontiguousarray(w, dtype=np.float64)))


def vmf_sample(mu, kappa, u1, u2):
    w = np.zeros(3)
    lib().oracle_vmf_sample(_p(np.ascontiguousarray(mu, dtype=np.float64)), float(kappa),
                            float(u1), float(u2), _p(w))
    return w


def mlp_forward(W, x):
    W = np.ascontiguousarray(W, dtype=np.float64)
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    out = np.zeros((len(x), GUIDE_OUT))
    lib().oracle_mlp_forward(_p(W), _p(x), len(x), _p(out))
    return out


def mlp_loss_grad(W, x, omega, wt, grad=True):
    """Mean loss -wt log q(omega) of the float network and dLoss/dW."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    wt = np.ascontiguousarray(wt, dtype=np.float64)
    g = np.zeros(GUIDE_WEIGHTS) if grad else None
    loss = lib().oracle_mlp_loss_grad(_p(W), _p(x), _p(om), _p(wt), len(x),
                                      _p(g) if grad else None)
    return (loss, g) if grad else loss


class Oracle:
    """One scene with one edit, held by the C oracle."""

    def __init__(self, scene, edit=None, brute_force=False):
        self.scene = scene
        L = lib()
        self._keep = [np.ascontiguousarray(scene.static_vertices, dtype=np.float32),
                      np.ascontiguousarray(scene.static_triangles, dtype=np.uint32),
                      np.ascontiguousarray(scene.static_material, dtype=np.uint32),
                      np.ascontiguousarray(scene.dyn_vertices, dtype=np.float32),
                      np.ascontiguousarray(scene.dyn_triangles, dtype=np.uint32),
                      np.ascontiguousarray(scene.materials, dtype=np.float32),
                      scene.camera.as_array()]
        sv, st, sm, dv, dt, mats, cam = self._keep
        self.h = L.oracle_create(_p(sv), len(sv), _p(st), _p(sm), len(st), _p(dv), len(dv),
                                 _p(dt), len(dt), _p(mats), len(mats), _p(cam),
                                 scene.camera.width, scene.camera.height, scene.max_depth,
                                 scene.alpha_min, scene.d_min, scene.jacobian_max)
        if brute_force:
            L.oracle_set_brute_force(self.h, 1)
        if edit is not None:
            self.set_edit(edit)

    def set_edit(self, edit):
        """One edit of the whole dynamic mesh, or a list of edits of the
        instances of a several-object dynamic mesh (scene.dyn_instance)."""
        if isinstance(edit, (list, tuple)):
            inst = getattr(self.scene, "dyn_instance", None)
            if inst is None:
                inst = np.zeros(self.scene.n_dyn, np.int32)
            inst = np.ascontiguousarray(inst, dtype=np.int32)
            assert len(inst) == self.scene.n_dyn and int(inst.max()) < len(edit)
            arrs = [np.ascontiguousarray(np.stack([getattr(e, f) for e in edit]),
                                         dtype=np.float32).ravel()
                    for f in ("M1", "M2", "mat1", "mat2")]
            self._edit = arrs + [inst]
            r = lib().oracle_set_edit_multi(self.h, len(edit), _p(inst), *[_p(a) for a in arrs])
            assert r == 0, "bad several-object edit"
            return
        arrs = [np.ascontiguousarray(a, dtype=np.float32).ravel()
                for a in (edit.M1, edit.M2, edit.mat1, edit.mat2)]
        self._edit = arrs
        lib().oracle_set_edit(self.h, *[_p(a) for a in arrs])

    def set_mapping(self, mode):
        """Path mapping: 2 camera replay for dynamic first edges (default), 1 the
        object transform only, 0 / False off (each frame estimates its own paths)."""
        lib().oracle_set_mapping(self.h, int(mode))

    def set_guide(self, guide):
        """Attach an integer network (W, shift, out_exp, box) to technique (3); None detaches."""
        if guide is None:
            lib().oracle_set_guide(self.h, None, None, 0, None)
            self._guide = None
            return
        W, shift, out_exp, box = guide
        arrs = (np.ascontiguousarray(W, dtype=np.int32), np.ascontiguousarray(shift, dtype=np.int32),
                np.ascontiguousarray(box, dtype=np.float32))
        self._guide = arrs
        lib().oracle_set_guide(self.h, _p(arrs[0]), _p(arrs[1]), int(out_exp), _p(arrs[2]))

    def close(self):
        if self.h:
            lib().oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.scene.camera.height, self.scene.camera.width, 3)

    def n_roots(self, spp):
        return spp * self.scene.camera.width * self.scene.camera.height

    def render_residual(self, spp, seed, root_begin=0, root_end=None, tech_mask=MASK_ALL,
                        counters=False):
        img = np.zeros(self.shape)
        cnt = np.zeros(8, dtype=np.int64)
        r1 = self.n_roots(spp) if root_end is None else root_end
        lib().oracle_render_residual(self.h, spp, seed, root_begin, r1, tech_mask, _p(img),
                                     _p(cnt))
        return (img, cnt) if counters else img

    def render_primal(self, frame, spp, seed, root_begin=0, root_end=None, domain=0):
        """Path-traced image of `frame`; domain != 0 keeps only the paths with a
        dynamic vertex where a technique of the mask (bit 0: (1), bit 1: (2),
        bit 2: (3)) would sample it (Sec. 4.1)."""
        img = np.zeros(self.shape)
        r1 = self.n_roots(spp) if root_end is None else root_end
        lib().oracle_render_primal_domain(self.h, frame, spp, seed, root_begin, r1, domain,
                                          _p(img))
        return img

    def dump(self, tech, frame, spp, seed, root_begin, root_end, tech_mask=MASK_ALL,
             max_records=None):
        L = lib()
        n = L.oracle_dump(self.h, tech, frame, spp, seed, root_begin, root_end, tech_mask, None, 0)
        cap = n if max_records is None else min(n, max_records)
        rec = np.zeros(cap, dtype=RECORD_DTYPE)
        L.oracle_dump(self.h, tech, frame, spp, seed, root_begin, root_end, tech_mask, _p(rec),
                      cap)
        return rec

    def closest_hit(self, frame, origins, dirs):
        o = np.ascontiguousarray(origins, dtype=np.float64)
        d = np.ascontiguousarray(dirs, dtype=np.float64)
        n = len(o)
        t = np.zeros(n); prim = np.zeros(n, dtype=np.int32)
        b1 = np.zeros(n); b2 = np.zeros(n)
        lib().oracle_closest_hit(self.h, frame, n, _p(o), _p(d), _p(t), _p(prim), _p(b1), _p(b2))
        return t, prim, b1, b2

    def mis_terms(self, frame, prims, bary, tech_mask=MASK_SEVEN):
        """The balance-heuristic denominator's terms (technique, per-root area
        density) of the path camera -> (prims[i], bary[i]) ... in `frame`, the
        last vertex on an emitter (Sec. 4.3; ghost terms Sec. 4.2)."""
        prims = np.ascontiguousarray(prims, dtype=np.int32)
        bary = np.ascontiguousarray(bary, dtype=np.float64).reshape(-1, 2)
        k = len(prims) + 1
        cap = 64
        tech = np.zeros(cap, dtype=np.int32)
        dens = np.zeros(cap)
        n = lib().oracle_mis_terms(self.h, frame, k, _p(prims), _p(bary), tech_mask, _p(tech),
                                   _p(dens), cap)
        if n < 0:
            raise ValueError("bad path")
        return tech[:min(n, cap)].copy(), dens[:min(n, cap)].copy()

    def check_mapping(self, tech, frame, spp, seed, root_begin, root_end):
        out = np.zeros(6)
        lib().oracle_check_mapping(self.h, tech, frame, spp, seed, root_begin, root_end, _p(out))
        return dict(pairs=int(out[0]), bad_inverse=int(out[1]), max_pos_err=out[2],
                    max_jac_err=out[3], fd_checked=int(out[4]), max_fd_err=out[5])
