"""Python binding of librp (include/rp.h): argument marshalling only.

Every function here forwards to the C ABI of the same name; all computation
runs in the library's CUDA kernels.  Device buffers are torch CUDA tensors,
passed by ``data_ptr()``; streams are torch streams.  If ``librp.so`` has not
been built, or no CUDA device is present, calls raise: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("RP_LIBRARY") or os.path.join(HERE, "_build", "librp.so")

RP_OK = 0
RP_TECH_ALL = 15
RP_TECH_GHOSTS = 112           # techniques (4), (5), (6)
RP_TECH_SEVEN = 127
STATUS = {0: "RP_OK", 1: "RP_ERR_INVALID_ARG", 2: "RP_ERR_OOM", 3: "RP_ERR_CUDA",
          4: "RP_ERR_TIMEOUT", 5: "RP_ERR_UNSUPPORTED"}


class RPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class rp_scene_desc(C.Structure):
    _fields_ = [("static_vertices", C.c_void_p), ("n_static_vertices", C.c_uint32),
                ("static_triangles", C.c_void_p), ("static_material", C.c_void_p),
                ("n_static_triangles", C.c_uint32),
                ("dyn_vertices", C.c_void_p), ("n_dyn_vertices", C.c_uint32),
                ("dyn_triangles", C.c_void_p), ("n_dyn_triangles", C.c_uint32),
                ("materials", C.c_void_p), ("n_materials", C.c_uint32),
                ("camera", C.c_float * 10), ("width", C.c_uint32), ("height", C.c_uint32),
                ("max_depth", C.c_uint32), ("alpha_min", C.c_float), ("d_min", C.c_float),
                ("jacobian_max", C.c_float), ("n_objects", C.c_uint32),
                ("object_ranges", C.c_void_p)]


class rp_edit_desc(C.Structure):
    _fields_ = [("M1", C.c_float * 12), ("M2", C.c_float * 12),
                ("mat1", C.c_float * 12), ("mat2", C.c_float * 12), ("object", C.c_uint32)]


class rp_batch_item(C.Structure):
    _fields_ = [("edit", C.c_void_p), ("width", C.c_uint32), ("height", C.c_uint32),
                ("spp", C.c_uint32), ("seed", C.c_uint64), ("tech_mask", C.c_uint32),
                ("d_out", C.c_void_p)]


class rp_batch_config(C.Structure):
    _fields_ = [("wave_roots", C.c_uint32), ("streams", C.c_uint32), ("blocks_per_sm", C.c_uint32),
                ("persistent", C.c_uint32)]


class rp_stats(C.Structure):
    _fields_ = [(n, C.c_ulonglong) for n in ("roots", "paths", "rays_closest", "rays_shadow",
                                              "nodes_visited", "tris_tested", "accepted",
                                              "rejected", "nodes_closest", "tris_closest",
                                              "nodes_shadow", "tris_shadow")]


class rp_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_ulonglong), ("ms", C.c_double)]


RECORD_DTYPE = np.dtype([
    ("root", "<u4"), ("tech", "<i4"), ("frame", "<i4"), ("sa", "<i4"), ("sb", "<i4"),
    ("pix_a", "<i4"), ("pix_b", "<i4"), ("va", "<f4", 3), ("vb", "<f4", 3),
    ("status", "<i4"), ("Pg", "<f4"), ("Py", "<f4"), ("J", "<f4")])

# every symbol the header declares
EXPORTS = ["rp_scene_create", "rp_scene_destroy", "rp_edit", "rp_edit_multi", "rp_edit_destroy",
           "rp_render_residual", "rp_render_residual_f32", "rp_render_residual_f32_noalloc",
           "rp_render_residual_host",
           "rp_render_primal", "rp_dump_samples", "rp_trace_closest", "rp_philox",
           "rp_bvh_build_host",
           "rp_enable_stats", "rp_get_stats", "rp_sync_status", "rp_enable_timing",
           "rp_enable_timing_of",
           "rp_get_kernel_times",
           "rp_guide_create", "rp_guide_destroy", "rp_guide_set_weights", "rp_guide_get_weights",
           "rp_guide_set_int", "rp_guide_get_int", "rp_guide_infer", "rp_guide_encode", "rp_guide_loss_grad",
           "rp_guide_train_step", "rp_guide_status", "rp_guide_wait_selftest", "rp_scene_set_guide",
           "rp_batch_create", "rp_batch_destroy", "rp_batch_launch", "rp_batch_set_seeds",
           "rp_batch_info", "rp_batch_status", "rp_batch_autotune", "rp_scene_set_mapping",
           "rp_last_error"]

GUIDE_WEIGHTS, GUIDE_IN, GUIDE_OUT = 20480, 80, 48

_lib = None


def lib():
    """Load librp.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2406_16302_gb300.build` (there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    P, U32, U64, I = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
    sig = {
        "rp_scene_create": (I, [P, P]),
        "rp_scene_destroy": (None, [P]),
        "rp_edit": (I, [P, P, P]),
        "rp_edit_multi": (I, [P, P, C.c_uint32, P]),
        "rp_guide_encode": (I, [P, P, P, C.c_uint32, P, P]),
        "rp_edit_destroy": (None, [P]),
        "rp_render_residual": (I, [P, P, U32, U64, U32, P, P]),
        "rp_render_residual_f32": (I, [P, P, U32, U64, U32, P, P]),
        "rp_render_residual_f32_noalloc": (I, [P, P, U32, U64, U32, P, P]),
        "rp_render_residual_host": (I, [P, P, U32, U64, U32, P, P]),
        "rp_render_primal": (I, [P, P, I, U32, U64, P, P]),
        "rp_dump_samples": (I, [P, P, I, I, U32, U64, U32, U32, U32, P, U64, P, P]),
        "rp_trace_closest": (I, [P, P, I, U32, P, P, P, P, P, P, P]),
        "rp_philox": (I, [U32, P, P, P, P]),
        "rp_enable_stats": (I, [P, I]),
        "rp_get_stats": (I, [P, P]),
        "rp_sync_status": (I, [P]),
        "rp_bvh_build_host": (I, [P, C.c_uint32, P, C.c_uint32, P, C.c_uint32, P, P, P]),
        "rp_enable_timing": (I, [P, I]),
        "rp_enable_timing_of": (I, [P, C.c_char_p]),
        "rp_get_kernel_times": (I, [P, P, I, P]),
        "rp_guide_create": (I, [P, U32, U64, P]),
        "rp_guide_destroy": (None, [P]),
        "rp_guide_set_weights": (I, [P, P]),
        "rp_guide_get_weights": (I, [P, P]),
        "rp_guide_set_int": (I, [P, P, P, C.c_int32]),
        "rp_guide_get_int": (I, [P, P, P, P]),
        "rp_guide_infer": (I, [P, P, U32, P, P]),
        "rp_guide_loss_grad": (I, [P, P, P, P, U32, P, P, P]),
        "rp_guide_train_step": (I, [P, C.c_float, P, P]),
        "rp_guide_status": (I, [P]),
        "rp_guide_wait_selftest": (I, [P, U64]),
        "rp_scene_set_guide": (I, [P, P]),
        "rp_batch_create": (I, [P, P, U32, P, P]),
        "rp_batch_destroy": (None, [P]),
        "rp_batch_launch": (I, [P, P]),
        "rp_batch_set_seeds": (I, [P, P, P]),
        "rp_batch_info": (I, [P, P, P]),
        "rp_batch_status": (I, [P]),
        "rp_batch_autotune": (I, [P, P, U32, U32, P, P]),
        "rp_scene_set_mapping": (I, [P, I]),
        "rp_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status):
    if status != RP_OK:
        raise RPError(status, lib().rp_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def edit_desc(edit) -> rp_edit_desc:
    d = rp_edit_desc()
    d.M1[:] = [float(v) for v in np.asarray(edit.M1, np.float32).ravel()]
    d.M2[:] = [float(v) for v in np.asarray(edit.M2, np.float32).ravel()]
    d.mat1[:] = [float(v) for v in np.asarray(edit.mat1, np.float32).ravel()]
    d.mat2[:] = [float(v) for v in np.asarray(edit.mat2, np.float32).ravel()]
    d.object = int(getattr(edit, "object", 0))
    return d


class Scene:
    """rp_scene_create / rp_scene_destroy around a scenes.Scene."""

    def __init__(self, scene):
        self.src = scene
        arrs = [np.ascontiguousarray(scene.static_vertices, np.float32),
                np.ascontiguousarray(scene.static_triangles, np.uint32),
                np.ascontiguousarray(scene.static_material, np.uint32),
                np.ascontiguousarray(scene.dyn_vertices, np.float32),
                np.ascontiguousarray(scene.dyn_triangles, np.uint32),
                np.ascontiguousarray(scene.materials, np.float32)]
        sv, st, sm, dv, dt, mats = arrs
        d = rp_scene_desc()
        d.static_vertices = sv.ctypes.data
        d.n_static_vertices = len(sv)
        d.static_triangles = st.ctypes.data
        d.static_material = sm.ctypes.data
        d.n_static_triangles = len(st)
        d.dyn_vertices = dv.ctypes.data
        d.n_dyn_vertices = len(dv)
        d.dyn_triangles = dt.ctypes.data
        d.n_dyn_triangles = len(dt)
        d.materials = mats.ctypes.data
        d.n_materials = len(mats)
        d.camera[:] = [float(v) for v in scene.camera.as_array()]
        d.width, d.height = scene.camera.width, scene.camera.height
        d.max_depth = scene.max_depth
        d.alpha_min, d.d_min, d.jacobian_max = scene.alpha_min, scene.d_min, scene.jacobian_max
        ranges = getattr(scene, "object_ranges", None)
        if ranges is not None and len(ranges):
            self._ranges = np.ascontiguousarray(ranges, np.uint32)
            d.n_objects = len(self._ranges)
            d.object_ranges = self._ranges.ctypes.data
        h = C.c_void_p()
        _check(lib().rp_scene_create(C.byref(d), C.byref(h)))
        self.h = h
        self.width, self.height = scene.camera.width, scene.camera.height

    def close(self):
        if getattr(self, "h", None):
            lib().rp_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.height, self.width, 3)

    def n_roots(self, spp):
        return spp * self.width * self.height


class Edit:
    """rp_edit / rp_edit_destroy around a scenes.Edit, or rp_edit_multi
    around a list of them (one per edited object)."""

    def __init__(self, scene: Scene, edit):
        h = C.c_void_p()
        if isinstance(edit, (list, tuple)):
            descs = (rp_edit_desc * len(edit))(*[edit_desc(e) for e in edit])
            self.desc = descs
            _check(lib().rp_edit_multi(scene.h, descs, len(edit), C.byref(h)))
        else:
            self.desc = edit_desc(edit)
            _check(lib().rp_edit(scene.h, C.byref(self.desc), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().rp_edit_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rp_render_residual(scene: Scene, edit: Edit, spp, seed, out, tech_mask=RP_TECH_ALL,
                       stream=None):
    _check(lib().rp_render_residual(scene.h, edit.h, spp, seed, tech_mask, _ptr(out),
                                    _stream(stream)))


def rp_render_residual_f32(scene: Scene, edit: Edit, spp, seed, out, tech_mask=RP_TECH_ALL,
                           stream=None):
    _check(lib().rp_render_residual_f32(scene.h, edit.h, spp, seed, tech_mask, _ptr(out),
                                        _stream(stream)))


def rp_render_residual_f32_noalloc(scene: Scene, edit: Edit, spp, seed, out,
                                   tech_mask=RP_TECH_ALL, stream=None):
    """The float32 residual render with no device allocation (scratch lives in
    a fixed array inside the library; width * height <= 1048576; calls that
    overlap on the GPU race)."""
    _check(lib().rp_render_residual_f32_noalloc(scene.h, edit.h, spp, seed, tech_mask, _ptr(out),
                                                _stream(stream)))


def rp_render_residual_host(scene: Scene, edit, spp, seed, host_out: np.ndarray,
                            tech_mask=RP_TECH_ALL, stream=None):
    assert host_out.dtype == np.float64 and host_out.flags.c_contiguous
    d = edit_desc(edit)
    _check(lib().rp_render_residual_host(scene.h, C.byref(d), spp, seed, tech_mask,
                                         host_out.ctypes.data_as(C.c_void_p), _stream(stream)))


def rp_render_primal(scene: Scene, edit: Edit, frame, spp, seed, out, stream=None):
    _check(lib().rp_render_primal(scene.h, edit.h, frame, spp, seed, _ptr(out), _stream(stream)))


def rp_dump_samples(scene: Scene, edit: Edit, tech, frame, spp, seed, root_begin, root_end,
                    records, count, tech_mask=RP_TECH_ALL, stream=None):
    cap = 0 if records is None else records.numel() * records.element_size() // RECORD_DTYPE.itemsize
    _check(lib().rp_dump_samples(scene.h, edit.h, tech, frame, spp, seed, root_begin, root_end,
                                 tech_mask, _ptr(records), cap, _ptr(count), _stream(stream)))


def rp_trace_closest(scene: Scene, edit: Edit, frame, origins, dirs, t, prim, b1, b2,
                     stream=None):
    n = origins.shape[0]
    _check(lib().rp_trace_closest(scene.h, edit.h, frame, n, _ptr(origins), _ptr(dirs), _ptr(t),
                                  _ptr(prim), _ptr(b1), _ptr(b2), _stream(stream)))


def rp_philox(counters, keys, out, stream=None):
    _check(lib().rp_philox(counters.shape[0], _ptr(counters), _ptr(keys), _ptr(out),
                           _stream(stream)))


def rp_enable_stats(scene: Scene, on=True):
    _check(lib().rp_enable_stats(scene.h, 1 if on else 0))


def rp_get_stats(scene: Scene) -> dict:
    s = rp_stats()
    _check(lib().rp_get_stats(scene.h, C.byref(s)))
    return {n: int(getattr(s, n)) for n, _ in rp_stats._fields_}


def rp_bvh_build_host(vertices, triangles) -> dict:
    """The scene BVH of a mesh, built on the host: {"nodes": (n, 16) float32,
    "tris": (t, 12) float32 in leaf order, "depth": int}."""
    v = np.ascontiguousarray(vertices, dtype=np.float32)
    t = np.ascontiguousarray(triangles, dtype=np.uint32)
    n_nodes, depth = C.c_uint32(), C.c_int()
    L = lib()
    _check(L.rp_bvh_build_host(v.ctypes.data, len(v), t.ctypes.data, len(t), None, 0, None,
                               C.byref(n_nodes), C.byref(depth)))
    nodes = np.zeros((n_nodes.value, 16), dtype=np.float32)
    tris = np.zeros((len(t), 12), dtype=np.float32)
    _check(L.rp_bvh_build_host(v.ctypes.data, len(v), t.ctypes.data, len(t), nodes.ctypes.data,
                               n_nodes.value, tris.ctypes.data, C.byref(n_nodes), C.byref(depth)))
    return {"nodes": nodes, "tris": tris, "depth": depth.value}


def rp_sync_status(scene: Scene):
    """Waits for the scene's queued work; raises on a device-side failure."""
    _check(lib().rp_sync_status(scene.h))


def rp_enable_timing(scene: Scene, on=True):
    _check(lib().rp_enable_timing(scene.h, 1 if on else 0))


def rp_enable_timing_of(scene: Scene, kernel=None):
    """Time only the launches of one kernel (None: all)."""
    _check(lib().rp_enable_timing_of(scene.h, kernel.encode() if kernel else None))


def rp_get_kernel_times(scene: Scene) -> dict:
    """{kernel name: (launches, total ms)} since the previous call."""
    cap = 64
    arr = (rp_kernel_time * cap)()
    n = C.c_int()
    _check(lib().rp_get_kernel_times(scene.h, arr, cap, C.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].ms))
            for i in range(min(n.value, cap))}


class Guide:
    """rp_guide_create / rp_guide_destroy: the learned proposal of technique (3)."""

    def __init__(self, box, batch=1 << 20, seed=1):
        b = np.ascontiguousarray(box, dtype=np.float32)
        h = C.c_void_p()
        _check(lib().rp_guide_create(b.ctypes.data_as(C.c_void_p), int(batch), int(seed),
                                     C.byref(h)))
        self.h = h
        self.batch = int(batch)

    def close(self):
        if getattr(self, "h", None):
            lib().rp_guide_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rp_guide_set_weights(guide: Guide, W):
    w = np.ascontiguousarray(W, dtype=np.float32)
    assert w.size == GUIDE_WEIGHTS
    _check(lib().rp_guide_set_weights(guide.h, w.ctypes.data_as(C.c_void_p)))


def rp_guide_get_weights(guide: Guide):
    w = np.zeros(GUIDE_WEIGHTS, dtype=np.float32)
    _check(lib().rp_guide_get_weights(guide.h, w.ctypes.data_as(C.c_void_p)))
    return w


def rp_guide_set_int(guide: Guide, W, shift, out_exp):
    w = np.ascontiguousarray(W, dtype=np.int8)
    sh = np.ascontiguousarray(shift, dtype=np.int32)
    assert w.size == GUIDE_WEIGHTS and sh.size == 4
    _check(lib().rp_guide_set_int(guide.h, w.ctypes.data_as(C.c_void_p),
                                  sh.ctypes.data_as(C.c_void_p), int(out_exp)))


def rp_guide_get_int(guide: Guide):
    w = np.zeros(GUIDE_WEIGHTS, dtype=np.int8)
    sh = np.zeros(4, dtype=np.int32)
    e = C.c_int32()
    _check(lib().rp_guide_get_int(guide.h, w.ctypes.data_as(C.c_void_p),
                                  sh.ctypes.data_as(C.c_void_p), C.byref(e)))
    return w, sh, int(e.value)


def rp_guide_infer(guide: Guide, m_in, out, stream=None):
    """m_in: int8 tensor [n][80] on the device; out: float32 tensor [n][48]."""
    _check(lib().rp_guide_infer(guide.h, _ptr(m_in), m_in.shape[0], _ptr(out), _stream(stream)))


def rp_guide_encode(guide: Guide, points, normals, out, stream=None):
    """Input features of object-space points (float64 [n][3]) and unit
    normals (float32 [n][3]) into out (int8 [n][80]); device tensors."""
    _check(lib().rp_guide_encode(guide.h, _ptr(points), _ptr(normals), int(points.shape[0]),
                                 _ptr(out), _stream(stream)))


def rp_guide_loss_grad(guide: Guide, x, omega, wt, grad, loss, stream=None):
    """Adds the float network's mean loss and its weight gradient into loss / grad."""
    _check(lib().rp_guide_loss_grad(guide.h, _ptr(x), _ptr(omega), _ptr(wt), x.shape[0],
                                    _ptr(grad), _ptr(loss), _stream(stream)))


def rp_guide_train_step(guide: Guide, lr=2e-3, stream=None):
    loss = C.c_float()
    _check(lib().rp_guide_train_step(guide.h, float(lr), C.byref(loss), _stream(stream)))
    return float(loss.value)


def rp_guide_status(guide: Guide):
    _check(lib().rp_guide_status(guide.h))


RP_MAPPING_OFF, RP_MAPPING_OBJECT, RP_MAPPING_CAMERA = 0, 1, 2


def rp_guide_wait_selftest(guide: Guide, limit_ns=10_000_000):
    """Run the inference kernel with its tensor-core completion withheld and
    a wait bounded by limit_ns; raises RPError(RP_ERR_TIMEOUT) when the wait
    ran out, as it should."""
    _check(lib().rp_guide_wait_selftest(guide.h, limit_ns))


def rp_scene_set_mapping(scene: Scene, mode=RP_MAPPING_CAMERA):
    """Path mapping mode (True means the default camera mode, False off)."""
    if mode is True:
        mode = RP_MAPPING_CAMERA
    _check(lib().rp_scene_set_mapping(scene.h, int(mode)))


def rp_scene_set_guide(scene: Scene, guide):
    _check(lib().rp_scene_set_guide(scene.h, None if guide is None else guide.h))


def _batch_items(items):
    arr = (rp_batch_item * len(items))()
    for i, (edit, w, h, spp, seed, mask, out) in enumerate(items):
        arr[i].edit = edit.h.value
        arr[i].width, arr[i].height = int(w), int(h)
        arr[i].spp, arr[i].seed, arr[i].tech_mask = int(spp), int(seed), int(mask)
        arr[i].d_out = out.data_ptr()
    return arr


class Batch:
    """rp_batch_create / rp_batch_destroy.  items: list of
    (Edit, width, height, spp, seed, tech_mask, float64 device image);
    config: (wave_roots, streams, blocks_per_sm[, persistent])."""

    def __init__(self, scene: Scene, items, config=None):
        self.items = list(items)          # keeps edits and images alive
        arr = _batch_items(self.items)
        h = C.c_void_p()
        cfg = None
        if config is not None:
            cfg = rp_batch_config(*[int(v) for v in config])
        _check(lib().rp_batch_create(scene.h, arr, len(self.items),
                                     None if cfg is None else C.byref(cfg), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().rp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rp_batch_launch(batch: Batch, stream=None):
    _check(lib().rp_batch_launch(batch.h, _stream(stream)))


def rp_batch_set_seeds(batch: Batch, seeds, stream=None):
    a = np.ascontiguousarray(seeds, dtype=np.uint64)
    assert a.size == len(batch.items)
    _check(lib().rp_batch_set_seeds(batch.h, a.ctypes.data_as(C.c_void_p), _stream(stream)))
    if stream is None:
        import torch
        torch.cuda.current_stream().synchronize()


def rp_batch_info(batch: Batch):
    cfg = rp_batch_config()
    nodes = C.c_uint64()
    _check(lib().rp_batch_info(batch.h, C.byref(cfg), C.byref(nodes)))
    return (cfg.wave_roots, cfg.streams, cfg.blocks_per_sm, cfg.persistent), int(nodes.value)


def rp_batch_status(batch: Batch):
    """Raises RPError(RP_ERR_TIMEOUT) if a grid barrier of the persistent
    batch kernel gave up (synchronises the device)."""
    _check(lib().rp_batch_status(batch.h))


def rp_batch_autotune(scene: Scene, items, spp_divisor=4):
    arr = _batch_items(items)
    cfg = rp_batch_config()
    ms = C.c_double()
    _check(lib().rp_batch_autotune(scene.h, arr, len(items), int(spp_divisor), C.byref(cfg),
                                   C.byref(ms)))
    return (cfg.wave_roots, cfg.streams, cfg.blocks_per_sm, cfg.persistent), float(ms.value)


# ---------------------------------------------------------------------------
# conveniences built only from the calls above
# ---------------------------------------------------------------------------

def render_residual(scene: Scene, edit: Edit, spp, seed, tech_mask=RP_TECH_ALL):
    import torch
    out = torch.zeros(scene.shape, dtype=torch.float64, device="cuda")
    rp_render_residual(scene, edit, spp, seed, out, tech_mask)
    return out


def render_primal(scene: Scene, edit: Edit, frame, spp, seed):
    import torch
    out = torch.zeros(scene.shape, dtype=torch.float64, device="cuda")
    rp_render_primal(scene, edit, frame, spp, seed, out)
    return out


def dump_samples(scene: Scene, edit: Edit, tech, frame, spp, seed, root_begin, root_end,
                 tech_mask=RP_TECH_ALL, capacity=None):
    """Records as a numpy structured array (RECORD_DTYPE)."""
    import torch
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    if capacity is None:
        rp_dump_samples(scene, edit, tech, frame, spp, seed, root_begin, root_end, None, count,
                        tech_mask)
        capacity = int(count.item())
    nbytes = max(1, capacity) * RECORD_DTYPE.itemsize
    buf = torch.zeros(nbytes // 4, dtype=torch.int32, device="cuda")
    rp_dump_samples(scene, edit, tech, frame, spp, seed, root_begin, root_end, buf, count,
                    tech_mask)
    n = min(int(count.item()), capacity)
    return buf.cpu().numpy().view(RECORD_DTYPE)[:n].copy()
