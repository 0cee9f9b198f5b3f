"""Thin ctypes binding of libamrmhd.so (include/amrmhd.h): argument
marshalling only. Every step of the advance runs in the library's CUDA kernels;
PyTorch supplies the device arena and the stream. If the library is missing,
loading fails loudly: there is no fallback implementation."""
import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libamrmhd.so")
HEADER = os.path.join(HERE, "..", "include", "amrmhd.h")

OK, EINVAL, ENEST, EOVERLAP, ENOMEM, ECUDA, ENONPHYS, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7, -8
FP64, MIXED = 0, 1
MAPS = {
    "neighbors": 0, "ghost_cells": 1, "ghost_faces": 2, "cf_faces": 3, "cf_edges": 4,
    "emf_faces": 5, "restrict_cells": 6, "restrict_faces": 7, "reflux_cells": 8,
}
Q_NPATCH, Q_NLEVEL, Q_CELLS, Q_CELL_UPDATES_PER_STEP, Q_ARENA_BYTES, Q_KERNEL_LAUNCHES = range(6)
Q_REGRID_FLAG_US, Q_REGRID_CLUSTER_US, Q_REGRID_BUILD_US, Q_REGRID_TRANSFER_US, Q_REGRID_MAPS_US = range(6, 11)
Q_FLOOR_EVENTS = 11
Q_REGRID_TRANSFER_MAPS_US = 12
Q_MAPS_HOST_US, Q_MAPS_GHOST_US, Q_MAPS_REGISTERS_US = 13, 14, 15
OPT_ADVANCE, OPT_GRAPH, OPT_TILE, OPT_CONCURRENT, OPT_HOST_IO, OPT_DIRECT_HALO = 0, 1, 2, 3, 4, 5
OPT_QUEUE, OPT_QUEUE_TILE, OPT_QUEUE_WITHHOLD, OPT_QUEUE_BALANCE = 6, 7, 8, 9
OPT_DEVICE_MAPS, OPT_DEVICE_CLUSTER, OPT_ZCHUNK = 10, 11, 12


class AmrmhdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("amrmhd status %d: %s" % (status, msg))
        self.status = status


class Config(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("base", C.c_int32 * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("nghost", C.c_int32), ("ratio", C.c_int32), ("max_level", C.c_int32), ("precision", C.c_int32),
        ("bc", (C.c_int32 * 2) * 3), ("gamma", C.c_double), ("cfl", C.c_double), ("strict_fp64", C.c_int32),
        ("inflow", C.c_double * 8),
    ]


class Patch(C.Structure):
    _fields_ = [("level", C.c_int32), ("lo", C.c_int32 * 3), ("hi", C.c_int32 * 3)]


_lib = None


def lib():
    """Loads libamrmhd.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libamrmhd.so not built: run `python -m paper_1110_1616_gb300.build` "
                              "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "amrmhd_create": [C.POINTER(Config), vp, C.POINTER(vp)],
            "amrmhd_destroy": [vp],
            "amrmhd_set_hierarchy": [vp, C.POINTER(Patch), i32, C.POINTER(C.c_size_t)],
            "amrmhd_bind_arena": [vp, vp, C.c_size_t],
            "amrmhd_set_state": [vp, i32, i32, vp, i32],
            "amrmhd_get_state": [vp, i32, i32, vp, i32],
            "amrmhd_packed_size": [vp, i32, C.POINTER(i64)],
            "amrmhd_set_state_packed": [vp, i32, vp, i32],
            "amrmhd_get_state_packed": [vp, i32, vp, i32],
            "amrmhd_export_map": [vp, i32, vp, i64, C.POINTER(i64), C.POINTER(i32)],
            "amrmhd_fill_ghosts": [vp, i32, i32],
            "amrmhd_advance_level": [vp, i32, dbl, i32],
            "amrmhd_reflux_restrict": [vp, i32],
            "amrmhd_cfl_dt": [vp, C.POINTER(dbl)],
            "amrmhd_step": [vp, i32, vp],
            "amrmhd_step_dt": [vp, i32, vp],
            "amrmhd_set_state_all": [vp, vp, i32],
            "amrmhd_get_state_all": [vp, vp, i32],
            "amrmhd_set_state_all_f32": [vp, vp, i32],
            "amrmhd_get_state_all_f32": [vp, vp, i32],
            "amrmhd_backward": [vp, i32, vp, i32, vp, vp],
            "amrmhd_step_dt_ckpt": [vp, i32, vp, i32],
            "amrmhd_backward_recorded": [vp, vp, vp],
            "amrmhd_regrid": [vp, dbl, i32],
            "amrmhd_autotune": [vp, i32, vp],
            "amrmhd_tile_choice": [vp, i32, i32, C.POINTER(i32), C.POINTER(i32)],
            "amrmhd_step_async": [vp, i32],
            "amrmhd_sync": [vp],
            "amrmhd_get_patches": [vp, vp, i32, C.POINTER(i32)],
            "amrmhd_regrid_boxes": [vp, i32, vp, i64, vp, i32, C.POINTER(i32)],
            "amrmhd_query": [vp, i32, C.POINTER(i64)],
            "amrmhd_set_option": [vp, i32, i64],
            "amrmhd_local_vjp": [i32, i32, i64, vp, vp, dbl, vp, i32, vp],
            "amrmhd_fp_convert": [i32, i64, vp, vp, vp, vp, vp, vp],
            "amrmhd_recover_mixed": [i64, vp, vp, vp, dbl, vp],
            "amrmhd_alu_peak": [i32, C.POINTER(dbl), C.POINTER(i32)],
            "amrmhd_set_floors": [vp, dbl, dbl],
            "amrmhd_grad_velocity": [i64, vp, vp, vp, vp],
            "amrmhd_sm_partition_create": [i32, C.POINTER(vp), C.POINTER(i32), C.POINTER(vp)],
            "amrmhd_sm_partition_destroy": [vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.amrmhd_advance_patch_noalloc.argtypes = [vp, vp, i32, C.POINTER(i32), C.POINTER(dbl), dbl, dbl, i32, vp]
        L.amrmhd_advance_patch_noalloc.restype = C.c_int
        L.amrmhd_sm_partition_error.argtypes = []
        L.amrmhd_sm_partition_error.restype = C.c_char_p
        L.amrmhd_last_error.argtypes = [vp]
        L.amrmhd_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def local_vjp(which, x, g, gamma=5.0 / 3.0, dim=3, h=None, method=0):
    """gx = J^T g at every row of x (numpy float64, host) for the HLLD flux
    (which 0: rows of 15 inputs, 7 outputs) or the half-step predictor (which 1:
    rows of 8 + 8 dim inputs, 8 outputs, h = dt/(2 dx_d)); method 0 the
    hand-written transposes of the adjoint in FP64, 1 forward-mode dual numbers,
    2 the hand-written transposes in FP32 (the mixed-precision adjoint's)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    n = x.shape[0]
    gx = np.zeros_like(x)
    hh = np.ascontiguousarray(np.zeros(3) if h is None else np.asarray(h, dtype=np.float64).reshape(-1))
    st = lib().amrmhd_local_vjp(int(which), int(dim), n, x.ctypes.data_as(C.c_void_p), g.ctypes.data_as(C.c_void_p),
                                float(gamma), hh.ctypes.data_as(C.c_void_p), int(method),
                                gx.ctypes.data_as(C.c_void_p))
    if st != 0:
        raise RuntimeError("amrmhd_local_vjp failed: status %d" % st)
    return gx


def fp_convert(x, y, on_device=False):
    """The mixed recovery's bit-level conversions next to the compiler's casts:
    returns (narrow(x), widen(y), cast_f32(x), cast_f64(y)) for numpy arrays x
    (float64) and y (float32) of one length; on_device runs them in a kernel of
    the mixed-precision unit, else on the host."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float32)
    if x.shape != y.shape:
        raise ValueError("x and y must have one shape")
    n = x.size
    xn = np.empty(n, np.float32)
    xh = np.empty(n, np.float32)
    yw = np.empty(n, np.float64)
    yh = np.empty(n, np.float64)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    st = lib().amrmhd_fp_convert(int(bool(on_device)), n, p(x), p(y), p(xn), p(yw), p(xh), p(yh))
    if st != 0:
        raise RuntimeError("amrmhd_fp_convert failed: status %d" % st)
    return xn, yw, xh, yh


def alu_peak(fp64=False):
    """Measured multiply-add throughput of the device: (FLOP/s, SM count)."""
    v, n = C.c_double(0.0), C.c_int32(0)
    st = lib().amrmhd_alu_peak(int(bool(fp64)), C.byref(v), C.byref(n))
    if st != 0:
        raise RuntimeError("amrmhd_alu_peak failed: status %d" % st)
    return v.value, n.value


class SmPartition:
    """A stream whose kernels run on one group of at least sm_count SMs
    (amrmhd_sm_partition_create); .stream is the cudaStream_t handle, .sms the
    group's SM count. close() releases it."""

    def __init__(self, sm_count):
        s, h, n = C.c_void_p(), C.c_void_p(), C.c_int32(0)
        st = lib().amrmhd_sm_partition_create(int(sm_count), C.byref(s), C.byref(n), C.byref(h))
        if st != 0:
            raise AmrmhdError(st, "amrmhd_sm_partition_create(%d): %s"
                              % (sm_count, lib().amrmhd_sm_partition_error().decode()))
        self.stream, self.sms, self._h = s.value, n.value, h

    def close(self):
        if self._h:
            lib().amrmhd_sm_partition_destroy(self._h)
            self._h = None


def recover_mixed(u, bl, br, gamma=5.0 / 3.0):
    """The mixed-precision advance's primitive recovery of n cells on the GPU:
    u (n, 5), bl and br (n, 3) FP32 numpy arrays -> w (n, 8) FP32."""
    u = np.ascontiguousarray(u, dtype=np.float32)
    bl = np.ascontiguousarray(bl, dtype=np.float32)
    br = np.ascontiguousarray(br, dtype=np.float32)
    n = u.shape[0]
    w = np.empty((n, 8), np.float32)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    st = lib().amrmhd_recover_mixed(n, p(u), p(bl), p(br), float(gamma), p(w))
    if st != 0:
        raise RuntimeError("amrmhd_recover_mixed failed: status %d" % st)
    return w


def declared_symbols():
    """Names of the entry points declared in include/amrmhd.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:amrmhd_status|const char\*)\s+(amrmhd_\w+)\s*\(", txt, re.M)))


def make_config(dim, base, precision=FP64, max_level=10, gamma=5.0 / 3.0, cfl=0.4, lo=(0, 0, 0), hi=(1, 1, 1),
                strict_fp64=True, bc=None, inflow=None):
    """bc: 6 ints (x-low, x-high, y-low, ...), 0 periodic, 1 outflow, 2 inflow."""
    c = Config()
    c.dim = dim
    b = tuple(base) + (1,) * (3 - len(base))
    for d in range(3):
        c.base[d] = b[d] if d < dim else 1
        c.lo[d] = lo[d]
        c.hi[d] = hi[d]
        c.bc[d][0] = c.bc[d][1] = 0
        if bc is not None and d < dim:
            c.bc[d][0], c.bc[d][1] = int(bc[2 * d]), int(bc[2 * d + 1])
    for f in range(8):
        c.inflow[f] = 0.0 if inflow is None else float(inflow[f])
    c.nghost, c.ratio, c.max_level, c.precision = 4, 2, max_level, precision
    c.gamma, c.cfl, c.strict_fp64 = gamma, cfl, 1 if strict_fp64 else 0
    return c


class Context:
    """One amrmhd context. `stream` is an integer cudaStream_t (0/None: the
    library makes its own)."""

    def __init__(self, cfg, stream=None):
        self.cfg = cfg
        self.h = C.c_void_p()
        self._check(lib().amrmhd_create(C.byref(cfg), C.c_void_p(stream or 0), C.byref(self.h)), "create")
        self.arena = None
        self.patches = []

    def __del__(self):
        if getattr(self, "h", None) and self.h.value:
            lib().amrmhd_destroy(self.h)
            self.h = C.c_void_p()

    def _check(self, st, what):
        if st != OK:
            msg = lib().amrmhd_last_error(self.h).decode() if getattr(self, "h", None) and self.h.value else what
            raise AmrmhdError(st, "%s: %s" % (what, msg))

    # ------------------------------------------------------------ hierarchy and memory
    def set_hierarchy(self, patches):
        arr = (Patch * len(patches))()
        for i, (l, lo, hi) in enumerate(patches):
            arr[i].level = l
            for d in range(3):
                arr[i].lo[d] = lo[d]
                arr[i].hi[d] = hi[d]
        nb = C.c_size_t(0)
        st = lib().amrmhd_set_hierarchy(self.h, arr, len(patches), C.byref(nb))
        if st != OK:
            raise AmrmhdError(st, lib().amrmhd_last_error(self.h).decode())
        self.patches = list(patches)
        return nb.value

    def bind_arena(self, tensor_or_ptr, nbytes=None):
        if hasattr(tensor_or_ptr, "data_ptr"):
            self.arena = tensor_or_ptr
            ptr, nbytes = tensor_or_ptr.data_ptr(), tensor_or_ptr.numel() * tensor_or_ptr.element_size()
        else:
            ptr = tensor_or_ptr
        self._check(lib().amrmhd_bind_arena(self.h, C.c_void_p(ptr), nbytes), "bind_arena")

    def alloc_arena(self, device="cuda"):
        import torch
        nbytes = self.query(Q_ARENA_BYTES)
        t = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        off = (-t.data_ptr()) % 256
        self.bind_arena(t.data_ptr() + off, nbytes)
        self.arena = t
        return t

    # ------------------------------------------------------------ state I/O
    def packed_size(self, field):
        n = C.c_int64(0)
        self._check(lib().amrmhd_packed_size(self.h, field, C.byref(n)), "packed_size")
        return n.value

    def set_field_packed(self, field, arr):
        if hasattr(arr, "data_ptr"):
            self._check(lib().amrmhd_set_state_packed(self.h, field, C.c_void_p(arr.data_ptr()), 1), "set_state_packed")
        else:
            a = np.ascontiguousarray(arr, dtype=np.float64)
            self._check(lib().amrmhd_set_state_packed(self.h, field, a.ctypes.data_as(C.c_void_p), 0), "set_state_packed")

    def get_field_packed(self, field, out=None):
        if out is not None and hasattr(out, "data_ptr"):
            self._check(lib().amrmhd_get_state_packed(self.h, field, C.c_void_p(out.data_ptr()), 1), "get_state_packed")
            return out
        a = np.empty(self.packed_size(field), dtype=np.float64)
        self._check(lib().amrmhd_get_state_packed(self.h, field, a.ctypes.data_as(C.c_void_p), 0), "get_state_packed")
        return a

    def get_field(self, patch, field):
        l, lo, hi = self.patches[patch]
        shp = self.field_shape(patch, field)
        a = np.empty(shp, dtype=np.float64)
        self._check(lib().amrmhd_get_state(self.h, patch, field, a.ctypes.data_as(C.c_void_p), 0), "get_state")
        return a

    def set_field(self, patch, field, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.field_shape(patch, field))
        self._check(lib().amrmhd_set_state(self.h, patch, field, a.ctypes.data_as(C.c_void_p), 0), "set_state")

    def field_shape(self, patch, field):
        l, lo, hi = self.patches[patch]
        dim = self.cfg.dim
        n = [hi[d] - lo[d] if d < dim else 1 for d in range(3)]
        if field >= 5 and not (dim == 2 and field == 7):
            n[field - 5] += 1
        return (n[2], n[1], n[0])

    # packing of whole-level arrays (inputs format) into the library's packed layout
    def pack(self, state, field):
        parts = []
        for (l, lo, hi) in self.patches:
            a = state[l][field]
            shp_extra = [0, 0, 0]
            if field >= 5 and not (self.cfg.dim == 2 and field == 7):
                shp_extra[field - 5] = 1
            sl = tuple(slice(lo[d], hi[d] + shp_extra[d]) for d in (2, 1, 0))
            parts.append(a[sl].ravel())
        return np.concatenate(parts)

    def unpack(self, packed, field):
        out = []
        o = 0
        for p in range(len(self.patches)):
            shp = self.field_shape(p, field)
            n = int(np.prod(shp))
            out.append(packed[o:o + n].reshape(shp))
            o += n
        return out

    def load_state(self, state):
        for f in range(8):
            self.set_field_packed(f, self.pack(state, f))

    def read_state(self):
        """Per-patch arrays: out[field][patch]."""
        return [self.unpack(self.get_field_packed(f), f) for f in range(8)]

    # ------------------------------------------------------------ operations
    def fill_ghosts(self, level, substep=1):
        self._check(lib().amrmhd_fill_ghosts(self.h, level, substep), "fill_ghosts")

    def advance_level(self, level, dt, substep=1):
        self._check(lib().amrmhd_advance_level(self.h, level, float(dt), substep), "advance_level")

    def reflux_restrict(self, fine_level):
        self._check(lib().amrmhd_reflux_restrict(self.h, fine_level), "reflux_restrict")

    def cfl_dt(self):
        v = C.c_double(0)
        self._check(lib().amrmhd_cfl_dt(self.h, C.byref(v)), "cfl_dt")
        return v.value

    def step(self, n=1, want_dt=True):
        buf = np.zeros(max(n, 1), dtype=np.float64) if want_dt else None
        self._check(lib().amrmhd_step(self.h, n, buf.ctypes.data_as(C.c_void_p) if want_dt else None), "step")
        return buf

    def step_async(self, n=1):
        """n coarse steps queued on the context's stream (see amrmhd_step_async)."""
        self._check(lib().amrmhd_step_async(self.h, n), "step_async")

    def sync(self):
        """Waits for the context's stream; raises on a device error (amrmhd_sync)."""
        self._check(lib().amrmhd_sync(self.h), "sync")

    def autotune(self, trials=5):
        """Per-level fused-tile choice by timing (see amrmhd_autotune)."""
        n = self.query(Q_NLEVEL)
        out = np.zeros(max(n, 1), dtype=np.int32)
        self._check(lib().amrmhd_autotune(self.h, int(trials), out.ctypes.data_as(C.c_void_p)), "autotune")
        return out[:n].tolist()

    def tile_choice(self, level, kind):
        """(tile variant, z planes per CTA) of the fused advance of a level:
        kind 0 interior only, 1 with the extended ghost layers (see
        amrmhd_tile_choice)."""
        t, z = C.c_int32(0), C.c_int32(0)
        self._check(lib().amrmhd_tile_choice(self.h, int(level), int(kind), C.byref(t), C.byref(z)), "tile_choice")
        return t.value, z.value

    def regrid(self, theta, max_levels):
        """Rebuilds the levels above 0 from density-gradient flags (threshold
        theta) up to max_levels levels; the context then owns its arena.
        Returns the new patch list [(level, lo, hi)]."""
        self._check(lib().amrmhd_regrid(self.h, float(theta), int(max_levels)), "regrid")
        self.arena = None
        self.patches = self.get_patches()
        return self.patches

    def regrid_boxes(self, level, flags):
        """The clustering alone (host): level+1 boxes (n x 7) from flagged cells (n x 3)."""
        f = np.ascontiguousarray(np.asarray(flags, dtype=np.int32).reshape(-1, 3))
        n = C.c_int32(0)
        self._check(lib().amrmhd_regrid_boxes(self.h, level, f.ctypes.data_as(C.c_void_p), len(f), None, 0,
                                              C.byref(n)), "regrid_boxes")
        out = np.zeros(7 * max(n.value, 1), dtype=np.int32)
        self._check(lib().amrmhd_regrid_boxes(self.h, level, f.ctypes.data_as(C.c_void_p), len(f),
                                              out.ctypes.data_as(C.c_void_p), n.value, C.byref(n)), "regrid_boxes")
        return out[:7 * n.value].reshape(-1, 7)

    def get_patches(self):
        n = C.c_int32(0)
        self._check(lib().amrmhd_get_patches(self.h, None, 0, C.byref(n)), "get_patches")
        arr = (Patch * max(n.value, 1))()
        self._check(lib().amrmhd_get_patches(self.h, arr, n.value, C.byref(n)), "get_patches")
        return [(arr[i].level, tuple(arr[i].lo), tuple(arr[i].hi)) for i in range(n.value)]

    def step_dt(self, dts):
        """Coarse steps with the prescribed dt0 sequence (the map the adjoint differentiates)."""
        d = np.ascontiguousarray(dts, dtype=np.float64)
        self._check(lib().amrmhd_step_dt(self.h, len(d), d.ctypes.data_as(C.c_void_p)), "step_dt")

    # ---- the full state as one packed vector (8 fields one after the other)
    def packed_total(self):
        return sum(self.packed_size(f) for f in range(8))

    def field_offsets(self):
        o, out = 0, []
        for f in range(8):
            out.append(o)
            o += self.packed_size(f)
        return out

    def load_packed_all(self, vec):
        """vec: a float64 CUDA tensor (or numpy array) holding all 8 packed fields."""
        offs = self.field_offsets()
        for f in range(8):
            n = self.packed_size(f)
            if hasattr(vec, "data_ptr"):
                self._check(lib().amrmhd_set_state_packed(self.h, f, C.c_void_p(vec.data_ptr() + 8 * offs[f]), 1),
                            "set_state_packed")
            else:
                self.set_field_packed(f, vec[offs[f]:offs[f] + n])

    def read_packed_all(self, out):
        """Fills out (a float64 CUDA tensor of packed_total() entries)."""
        offs = self.field_offsets()
        for f in range(8):
            self._check(lib().amrmhd_get_state_packed(self.h, f, C.c_void_p(out.data_ptr() + 8 * offs[f]), 1),
                        "get_state_packed")
        return out

    def backward(self, dts, g_final, g0, ckpt_every=20):
        """dL/dU0 = (dU_final/dU0)^T dL/dU_final over len(dts) coarse steps with
        the dt0 sequence dts, starting from the current state (kept). g_final and
        g0 are float64 CUDA tensors in the packed_total() layout."""
        d = np.ascontiguousarray(dts, dtype=np.float64)
        self._check(lib().amrmhd_backward(self.h, len(d), d.ctypes.data_as(C.c_void_p), int(ckpt_every),
                                          C.c_void_p(g_final.data_ptr()), C.c_void_p(g0.data_ptr())), "backward")
        return g0

    def step_dt_ckpt(self, dts, ckpt_every=20):
        """step_dt recording checkpoints every ckpt_every coarse steps for
        backward_recorded (amrmhd_step_dt_ckpt)."""
        d = np.ascontiguousarray(dts, dtype=np.float64)
        self._check(lib().amrmhd_step_dt_ckpt(self.h, len(d), d.ctypes.data_as(C.c_void_p), int(ckpt_every)),
                    "step_dt_ckpt")

    def backward_recorded(self, g_final, g0):
        """The backward of the last step_dt_ckpt from its final state (the
        context then holds the initial state). Returns False, doing nothing, if
        no record matches the current state."""
        st = lib().amrmhd_backward_recorded(self.h, C.c_void_p(g_final.data_ptr()), C.c_void_p(g0.data_ptr()))
        if st == ESTATE:
            return False
        self._check(st, "backward_recorded")
        return True

    def query(self, what):
        v = C.c_int64(0)
        self._check(lib().amrmhd_query(self.h, what, C.byref(v)), "query")
        return v.value

    def set_option(self, opt, value):
        self._check(lib().amrmhd_set_option(self.h, opt, value), "set_option")

    def set_floors(self, rho_min, p_min):
        self._check(lib().amrmhd_set_floors(self.h, float(rho_min), float(p_min)), "set_floors")

    def export_map(self, which):
        if isinstance(which, str):
            which = MAPS[which]
        n, w = C.c_int64(0), C.c_int32(0)
        self._check(lib().amrmhd_export_map(self.h, which, None, 0, C.byref(n), C.byref(w)), "export_map")
        out = np.zeros(max(n.value, 1), dtype=np.int32)
        self._check(lib().amrmhd_export_map(self.h, which, out.ctypes.data_as(C.c_void_p), n.value, C.byref(n),
                                            C.byref(w)), "export_map")
        return out[: n.value].reshape(-1, w.value)


def advance_patch_noalloc(u_in, u_out, dim, n, dx, gamma, dt, w=0, stream=None):
    """One-patch advance that allocates nothing (see include/amrmhd.h):
    u_in/u_out are device float tensors in the ghosted single-patch layout."""
    ni = (C.c_int32 * 3)(*(list(n) + [1] * (3 - len(n))))
    dd = (C.c_double * 3)(*(list(dx) + [1.0] * (3 - len(dx))))
    st = lib().amrmhd_advance_patch_noalloc(C.c_void_p(u_in.data_ptr()), C.c_void_p(u_out.data_ptr()), dim, ni, dd,
                                             float(gamma), float(dt), w, C.c_void_p(stream or 0))
    if st != OK:
        raise AmrmhdError(st, "advance_patch_noalloc")


def context_for(problem, precision=FP64, strict_fp64=True, stream=None):
    """Context + hierarchy for an inputs.Problem (no device memory yet)."""
    cfg = make_config(problem.dim, problem.base, precision=precision, gamma=problem.gamma, cfl=problem.cfl,
                      lo=problem.lo, hi=problem.hi, strict_fp64=strict_fp64, bc=problem.bc, inflow=problem.inflow)
    ctx = Context(cfg, stream)
    ctx.set_hierarchy(problem.patches)
    return ctx
