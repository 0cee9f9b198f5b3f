"""ctypes binding of the oracle library (test infrastructure only)."""
import ctypes as C

import numpy as np

from . import build as _build

_lib = None

MAPS = {
    "neighbors": 0, "ghost_cells": 1, "ghost_faces": 2, "cf_faces": 3, "cf_edges": 4,
    "emf_faces": 5, "restrict_cells": 6, "restrict_faces": 7, "reflux_cells": 8,
}

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.oc_new.restype = C.c_void_p
        L.oc_new.argtypes = [C.c_int, _ip, _dp, _dp, C.c_int, C.c_double, C.c_double]
        L.oc_new2.restype = C.c_void_p
        L.oc_new2.argtypes = [C.c_int, _ip, _dp, _dp, C.c_int, C.c_double, C.c_double, _ip, _dp]
        L.oc_free.argtypes = [C.c_void_p]
        L.oc_set_patches.argtypes = [C.c_void_p, _ip, C.c_int]
        L.oc_field_size.restype = C.c_longlong
        L.oc_field_size.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.oc_set_field.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp]
        L.oc_get_field.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp]
        L.oc_cfl_dt.restype = C.c_double
        L.oc_cfl_dt.argtypes = [C.c_void_p]
        L.oc_step.restype = C.c_double
        L.oc_step.argtypes = [C.c_void_p, C.c_double]
        L.oc_cell_updates.restype = C.c_longlong
        L.oc_cell_updates.argtypes = [C.c_void_p]
        L.oc_set_flags.argtypes = [C.c_void_p, C.c_int]
        L.oc_get_masks.argtypes = [C.c_void_p, C.c_int, np.ctypeslib.ndpointer(dtype=np.int8),
                                   np.ctypeslib.ndpointer(dtype=np.int8)]
        L.oc_step_targets.argtypes = [C.c_void_p, C.c_double, _ip, C.c_int]
        L.oc_hlld.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double, _dp]
        L.oc_hlld_vjp.argtypes = [_dp, C.c_double, C.c_double, _dp, _dp]
        L.oc_predict.argtypes = [C.c_int, _dp, C.c_double, _dp, _dp]
        L.oc_predict_vjp.argtypes = [C.c_int, _dp, C.c_double, _dp, _dp, _dp]
        L.oc_flux.argtypes = [_dp, C.c_double, C.c_double, _dp]
        L.oc_recover.argtypes = [_dp, _dp, C.c_double, _dp]
        L.oc_minmod.restype = C.c_double
        L.oc_minmod.argtypes = [C.c_double, C.c_double]
        L.oc_fast_speed.restype = C.c_double
        L.oc_fast_speed.argtypes = [C.c_double] * 6
        L.oc_gs_edge.restype = C.c_double
        L.oc_gs_edge.argtypes = [_dp]
        L.oc_prolong_all.argtypes = [C.c_void_p, C.c_void_p]
        L.oc_restrict_all.argtypes = [C.c_void_p, C.c_void_p]
        L.oc_flops_per_cell_update.restype = C.c_double
        L.oc_flops_per_cell_update.argtypes = [C.c_int, C.c_int, C.c_uint]
        L.oc_flops_recovery.restype = C.c_longlong
        L.oc_build_map.restype = C.c_int
        L.oc_build_map.argtypes = [C.c_int, _ip, _ip, C.c_int, C.c_int, C.c_void_p, C.c_longlong,
                                   C.POINTER(C.c_longlong)]
        L.oc_state_size.restype = C.c_longlong
        L.oc_state_size.argtypes = [C.c_void_p]
        L.oc_backward.restype = C.c_longlong
        L.oc_backward.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp]
        L.oc_tangent.restype = C.c_int
        L.oc_tangent.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp]
        L.oc_regrid_boxes.restype = C.c_int
        L.oc_regrid_boxes.argtypes = [C.c_void_p, C.c_int, _ip, C.c_longlong, _ip, C.c_int, C.POINTER(C.c_int)]
        L.oc_regrid.restype = C.c_int
        L.oc_regrid.argtypes = [C.c_void_p, C.c_double, C.c_int, _ip, C.c_int, C.POINTER(C.c_int)]
        L.oc_build_map2.restype = C.c_int
        L.oc_build_map2.argtypes = [C.c_int, _ip, _ip, _ip, C.c_int, C.c_int, C.c_void_p, C.c_longlong,
                                    C.POINTER(C.c_longlong)]
        _lib = L
    return _lib


FIELDS = ["rho", "mx", "my", "mz", "E", "bx", "by", "bz"]


def patch_array(patches):
    """patches: iterable of (level, lo(3), hi(3)) -> int32 (n, 7)."""
    a = np.array([[p[0], *p[1], *p[2]] for p in patches], dtype=np.int32).reshape(-1, 7)
    return np.ascontiguousarray(a)


class OracleSim:
    """One hierarchy held by the oracle; fields are whole-level numpy arrays."""

    def __init__(self, dim, base, patches, nlev=None, lo=(0, 0, 0), hi=(1, 1, 1), gamma=5.0 / 3.0, cfl=0.4,
                 bc=None, inflow=None):
        self.dim = dim
        self.base = tuple(base) + (1,) * (3 - len(base))
        pa = patch_array(patches)
        if nlev is None:
            nlev = int(pa[:, 0].max()) + 1
        self.nlev = nlev
        bca = np.zeros(6, dtype=np.int32) if bc is None else np.ascontiguousarray(np.asarray(bc, dtype=np.int32).ravel())
        inf = np.zeros(8) if inflow is None else np.ascontiguousarray(np.asarray(inflow, dtype=np.float64))
        self.bc = bca
        self.h = lib().oc_new2(dim, np.array(self.base, dtype=np.int32), np.array(lo, dtype=np.float64),
                               np.array(hi, dtype=np.float64), nlev, gamma, cfl, bca, inf)
        self.status = lib().oc_set_patches(self.h, pa, len(pa))
        if self.status != 0:
            raise ValueError("oracle rejected the hierarchy: status %d" % self.status)

    def __del__(self):
        if getattr(self, "h", None):
            lib().oc_free(self.h)
            self.h = None

    def level_shape(self, level):
        n = [self.base[d] << level if d < self.dim else 1 for d in range(3)]
        return n

    def field_shape(self, level, f):
        n = self.level_shape(level)
        if f >= 5 and not (f == 7 and self.dim == 2):
            n[f - 5] += 1
        return (n[2], n[1], n[0])

    def set_field(self, level, f, a):
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(self.field_shape(level, f))
        lib().oc_set_field(self.h, level, f, a.ravel())

    def get_field(self, level, f):
        out = np.zeros(self.field_shape(level, f), dtype=np.float64)
        lib().oc_get_field(self.h, level, f, out.ravel())
        return out

    def set_state(self, state):
        """state: {level: [8 arrays]}"""
        for l, arrs in state.items():
            for f, a in enumerate(arrs):
                self.set_field(l, f, a)

    def get_state(self):
        return {l: [self.get_field(l, f) for f in range(8)] for l in range(self.nlev)}

    def cfl_dt(self):
        return lib().oc_cfl_dt(self.h)

    def step(self, dt0=0.0):
        return lib().oc_step(self.h, float(dt0))

    def set_flags(self, flags):
        lib().oc_set_flags(self.h, flags)

    def cell_updates(self):
        return lib().oc_cell_updates(self.h)

    def masks(self, level):
        n = self.level_shape(level)
        d = np.zeros(n[0] * n[1] * n[2], dtype=np.int8)
        c = np.zeros_like(d)
        lib().oc_get_masks(self.h, level, d, c)
        return d.reshape(n[2], n[1], n[0]), c.reshape(n[2], n[1], n[0])

    # ---- adjoint pins: the state as one vector (levels, then fields, each
    # array in the get_field layout; periodic face copies included)
    def flatten(self, state):
        return np.concatenate([np.ascontiguousarray(state[l][f], dtype=np.float64).ravel()
                               for l in range(self.nlev) for f in range(8)])

    def unflatten(self, vec):
        out, o = {}, 0
        for l in range(self.nlev):
            out[l] = []
            for f in range(8):
                shp = self.field_shape(l, f)
                n = int(np.prod(shp))
                out[l].append(vec[o:o + n].reshape(shp))
                o += n
        return out

    def backward(self, dts, lam_final):
        """(dU_final/dU0)^T lam_final over len(dts) coarse steps of the given
        dts, by a reverse sweep of the oracle's own operation tape; the
        simulation's state is left unchanged. Dicts {level: [8 arrays]}."""
        dts = np.ascontiguousarray(dts, dtype=np.float64)
        lam = self.flatten(lam_final)
        out = np.zeros_like(lam)
        lib().oc_backward(self.h, len(dts), dts, lam, out)
        return self.unflatten(out)

    def tangent(self, dts, v0):
        """(dU_final/dU0) v0 by forward-mode differentiation of the oracle."""
        dts = np.ascontiguousarray(dts, dtype=np.float64)
        v = self.flatten(v0)
        out = np.zeros_like(v)
        lib().oc_tangent(self.h, len(dts), dts, v, out)
        return self.unflatten(out)

    def regrid(self, theta, max_levels=None):
        """Rebuilds every level above 0 from density-gradient flags (threshold
        theta), coarse to fine up to max_levels levels (default: the current
        count), with the data transfer; returns the new patch list
        [(level, lo, hi)] and updates nlev."""
        if max_levels is None:
            max_levels = self.nlev
        cap = 1 << 20
        out = np.zeros(7 * cap, dtype=np.int32)
        n = C.c_int(0)
        st = lib().oc_regrid(self.h, float(theta), int(max_levels), out, cap, C.byref(n))
        if st != 0:
            raise ValueError("oracle regrid failed: %d" % st)
        rows = out[:7 * n.value].reshape(-1, 7)
        patches = [(int(r[0]), (int(r[1]), int(r[2]), int(r[3])), (int(r[4]), int(r[5]), int(r[6]))) for r in rows]
        self.nlev = max(p[0] for p in patches) + 1
        return patches

    def regrid_boxes(self, level, flags):
        """The clustering alone: level+1 boxes from flagged level cells (n x 3)."""
        f = np.ascontiguousarray(np.asarray(flags, dtype=np.int32).reshape(-1, 3))
        cap = 1 << 16
        out = np.zeros(7 * cap, dtype=np.int32)
        n = C.c_int(0)
        st = lib().oc_regrid_boxes(self.h, level, f.ravel(), len(f), out, cap, C.byref(n))
        if st != 0:
            raise ValueError("oracle clustering failed: %d" % st)
        return out[:7 * n.value].reshape(-1, 7).copy()

    def step_targets(self, dt, ijk):
        ijk = np.ascontiguousarray(np.asarray(ijk, dtype=np.int32).reshape(-1, 3))
        lib().oc_step_targets(self.h, float(dt), ijk.ravel(), len(ijk))


def build_map(dim, base, patches, which, bc=None):
    """Brute-force integer map; returns an (n_rows, width) int32 array. bc: 6
    ints (x-low, x-high, ...): 0 periodic, 1 outflow, 2 inflow."""
    if isinstance(which, str):
        which = MAPS[which]
    pa = patch_array(patches)
    b = np.array(tuple(base) + (1,) * (3 - len(base)), dtype=np.int32)
    bca = np.zeros(6, dtype=np.int32) if bc is None else np.ascontiguousarray(np.asarray(bc, dtype=np.int32).ravel())
    n = C.c_longlong(0)
    w = lib().oc_build_map2(dim, b, bca, pa, len(pa), which, None, 0, C.byref(n))
    out = np.zeros(max(n.value, 1), dtype=np.int32)
    lib().oc_build_map2(dim, b, bca, pa, len(pa), which, out.ctypes.data_as(C.c_void_p), n.value, C.byref(n))
    return out[: n.value].reshape(-1, w)


def flops_per_cell_update(dim=3, nsample=2000, seed=1):
    """Algorithmic FP operation count of one cell update (see opcount.cpp)."""
    return lib().oc_flops_per_cell_update(dim, nsample, seed)


def flops_recovery():
    return lib().oc_flops_recovery()


def hlld(ql, qr, bn, gamma=5.0 / 3.0, eps=1e-12):
    f = np.zeros(7)
    lib().oc_hlld(np.asarray(ql, dtype=np.float64), np.asarray(qr, dtype=np.float64), bn, gamma, eps, f)
    return f


def hlld_vjp(x, g, gamma=5.0 / 3.0, eps=1e-12):
    """J^T g of the HLLD flux at x = (ql[7], qr[7], bn), by the oracle's tape."""
    gx = np.zeros(15)
    lib().oc_hlld_vjp(np.ascontiguousarray(x, dtype=np.float64), gamma, eps,
                      np.ascontiguousarray(g, dtype=np.float64), gx)
    return gx


def predict(dim, x, h, gamma=5.0 / 3.0):
    """Half-step predictor wh = w - sum_d h_d A_d(w) s_d of one cell, x = (w, s_0, .., s_{dim-1})."""
    wh = np.zeros(8)
    lib().oc_predict(dim, np.ascontiguousarray(x, dtype=np.float64), gamma,
                     np.ascontiguousarray(np.resize(np.asarray(h, dtype=np.float64), 3)), wh)
    return wh


def predict_vjp(dim, x, h, g, gamma=5.0 / 3.0):
    """J^T g of the half-step predictor of one cell, by the oracle's tape."""
    gx = np.zeros(8 + 8 * dim)
    lib().oc_predict_vjp(dim, np.ascontiguousarray(x, dtype=np.float64), gamma,
                         np.ascontiguousarray(np.resize(np.asarray(h, dtype=np.float64), 3)),
                         np.ascontiguousarray(g, dtype=np.float64), gx)
    return gx


def mhd_flux(q, bn, gamma=5.0 / 3.0):
    f = np.zeros(7)
    lib().oc_flux(np.asarray(q, dtype=np.float64), bn, gamma, f)
    return f


def recover(u, bc, gamma=5.0 / 3.0):
    """Conservative -> primitive recovery of one cell: u = (rho, mx, my, mz, E),
    bc = cell-centred B; returns (rho, vx, vy, vz, p, Bx, By, Bz)."""
    w = np.zeros(8)
    lib().oc_recover(np.ascontiguousarray(u, dtype=np.float64), np.ascontiguousarray(bc, dtype=np.float64),
                     float(gamma), w)
    return w


def minmod(a, b):
    return lib().oc_minmod(a, b)


def fast_speed(rho, p, bn, bt, bu, gamma=5.0 / 3.0):
    return lib().oc_fast_speed(rho, p, bn, bt, bu, gamma)


def gs_edge(args):
    return lib().oc_gs_edge(np.asarray(args, dtype=np.float64))


def prolong_all(coarse, fine):
    lib().oc_prolong_all(coarse.h, fine.h)


def restrict_all(coarse, fine):
    lib().oc_restrict_all(coarse.h, fine.h)
