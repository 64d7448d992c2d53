"""Thin Python binding of libwd (C ABI in include/wd.h).

The functions below carry the C names and only marshal arguments: every step
of the computation runs in the CUDA library. Host arrays are numpy; the
`_dev` functions take torch CUDA tensors and the current torch stream (torch
is used for device memory and streams only). There is no CPU fallback: if the
shared library is missing this module raises at import.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

WD_OK, WD_EINVAL, WD_ENOMEM, WD_ECUDA, WD_EBUSY, WD_ETIMEOUT, WD_ENOTFOUND, WD_ECANCELLED = range(8)
WD_FP64, WD_MIXED = 0, 1
WD_RULE_BALL, WD_RULE_CUBE_TRAP, WD_RULE_EXPLICIT = 0, 1, 2
WD_NU_SPHERE, WD_NU_MESH = 0, 1
STATUS_NAMES = {0: "WD_OK", 1: "WD_EINVAL", 2: "WD_ENOMEM", 3: "WD_ECUDA", 4: "WD_EBUSY",
                5: "WD_ETIMEOUT", 6: "WD_ENOTFOUND", 7: "WD_ECANCELLED"}

LIB_PATH = _build.LIB
if not os.path.exists(LIB_PATH):
    raise ImportError("libwd.so is not built (%s); run __graft_entry__.build() or "
                      "python -m paper_2304_06340_b300._build" % LIB_PATH)
_lib = ctypes.CDLL(LIB_PATH)

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


class wd_rule_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("R", ctypes.c_double), ("n_r", ctypes.c_int),
                ("n_polar", ctypes.c_int), ("n_azim", ctypes.c_int), ("hermitian", ctypes.c_int)]


class wd_mesh(ctypes.Structure):
    _fields_ = [("verts", _vp), ("n_verts", _i64), ("tris", _vp), ("n_tris", _i64)]


class wd_measure(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("radius", ctypes.c_double), ("center", ctypes.c_double * 3),
                ("mesh", ctypes.POINTER(wd_mesh))]


WD_SERVE_MAX_SLOTS = 256


class wd_serve_config(ctypes.Structure):
    _fields_ = [("mem_cap_bytes", _i64), ("max_slots", ctypes.c_int), ("max_pending", ctypes.c_int),
                ("timeout_ms", ctypes.c_int), ("precision", ctypes.c_int), ("pairs_per_launch", _i64),
                ("n_rules", ctypes.c_int), ("rules", wd_rule_desc * 4)]


class wd_serve_stats_t(ctypes.Structure):
    _fields_ = [(k, _i64) for k in ("submitted", "admitted", "completed", "rejected", "timeouts", "cancelled",
                                    "failed", "launches", "pending", "active", "arena_used_bytes")] + \
               [(k, ctypes.c_double) for k in ("pairs", "p50_us", "p99_us", "max_us", "mean_us", "qps", "gpu_busy")]


def _sig(name, args, res=ctypes.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("wd_create", [ctypes.c_int, ctypes.POINTER(_vp)])
_sig("wd_destroy", [_vp], None)
_sig("wd_last_error", [_vp], ctypes.c_char_p)
_sig("wd_sync", [_vp, _vp])
_sig("wd_build_freq_rule", [_vp, ctypes.POINTER(wd_rule_desc), ctypes.POINTER(_vp)])
_sig("wd_build_freq_rule_shells", [_vp, ctypes.POINTER(wd_rule_desc), ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(_vp)])
_sig("wd_rule_from_nodes", [_vp, _dp, _dp, _i64, ctypes.POINTER(_vp)])
_sig("wd_rule_info", [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)])
_sig("wd_rule_copy_nodes", [_vp, _dp, _dp])
_sig("wd_rule_free", [_vp], None)
_sig("wd_mesh_ft", [_vp, _vp, ctypes.POINTER(wd_mesh), ctypes.c_int, _dp, _dp])
_sig("wd_mesh_ft_dev", [_vp, _vp, _vp, _i64, _vp, _i64, ctypes.c_int, _vp, _vp, _vp])
_sig("wd_mesh_ft_atoms", [_vp, _vp, ctypes.POINTER(wd_mesh), _dp, _dp])
_sig("wd_sphere_ft", [_vp, _vp, ctypes.c_double, _dp, _dp, _dp])
_sig("wd_sphere_ft_dev", [_vp, _vp, ctypes.c_double, _dp, _vp, _vp, _vp])
_sig("wd_distance", [_vp, _vp, ctypes.POINTER(wd_mesh), ctypes.POINTER(wd_measure), ctypes.c_double,
                     ctypes.c_int, _dp])
_sig("wd_distance_dev", [_vp, _vp, _vp, _i64, _vp, _i64, ctypes.POINTER(wd_measure), ctypes.c_double,
                         ctypes.c_int, _vp, _vp])
_sig("wd_distance_grad", [_vp, _vp, ctypes.POINTER(wd_mesh), ctypes.POINTER(wd_measure), ctypes.c_double,
                          ctypes.c_int, _dp, _dp])
_sig("wd_distance_grad_dev", [_vp, _vp, _vp, _i64, _vp, _i64, ctypes.POINTER(wd_measure), ctypes.c_double,
                              ctypes.c_int, _vp, _vp, _vp])
_sig("wd_launch_count", [_vp], _i64)
_sig("wd_serve_start", [_vp, ctypes.POINTER(wd_serve_config), ctypes.POINTER(_vp)])
_sig("wd_serve_submit", [_vp, ctypes.POINTER(wd_mesh), ctypes.c_double, ctypes.c_double,
                         ctypes.POINTER(ctypes.c_uint64)])
_sig("wd_serve_poll", [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), _dp, ctypes.POINTER(ctypes.c_int)])
_sig("wd_serve_wait", [_vp, ctypes.c_uint64, ctypes.c_int, _dp])
_sig("wd_serve_cancel", [_vp, ctypes.c_uint64])
_sig("wd_serve_stats", [_vp, ctypes.POINTER(wd_serve_stats_t)])
_sig("wd_serve_stop", [_vp])
_sig("wd_distance_dev_noalloc", [_vp, _vp, _i64, _vp, _i64, _vp, _i64, ctypes.c_double, ctypes.c_double, _dp,
                                 ctypes.c_int, _vp, _vp])


class WDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _check(status):
    if status != WD_OK:
        raise WDError(status, _lib.wd_last_error(None).decode(errors="replace"))


def library():
    """The loaded ctypes handle of libwd (for symbol checks and raw calls)."""
    return _lib


# ------------------------------------------------------------------ marshalling helpers
def _host_mesh(verts, tris):
    v = np.ascontiguousarray(verts, dtype=np.float64).reshape(-1, 3)
    t = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
    m = wd_mesh(v.ctypes.data if v.size else None, len(v), t.ctypes.data if t.size else None, len(t))
    return m, (v, t)


def _dev_ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _measure(nu, keep, device=False):
    """nu: None / ('sphere', radius[, center]) / ('mesh', verts, tris)."""
    m = wd_measure()
    if nu is None or nu[0] == "sphere":
        m.kind = WD_NU_SPHERE
        m.radius = 1.0 if nu is None else float(nu[1])
        c = (0.0, 0.0, 0.0) if nu is None or len(nu) < 3 else nu[2]
        for j in range(3):
            m.center[j] = float(c[j])
        m.mesh = None
        return m
    m.kind = WD_NU_MESH
    if device:
        v, t = nu[1], nu[2]
        mm = wd_mesh(v.data_ptr(), v.shape[0], t.data_ptr(), t.shape[0])
        keep.append((v, t))
    else:
        mm, arrays = _host_mesh(nu[1], nu[2])
        keep.append(arrays)
    keep.append(mm)
    m.mesh = ctypes.pointer(mm)
    return m


# ------------------------------------------------------------------ C-named functions
def wd_create(device=0):
    h = _vp()
    _check(_lib.wd_create(int(device), ctypes.byref(h)))
    return h


def wd_destroy(ctx):
    _lib.wd_destroy(ctx)


def wd_last_error(ctx=None):
    return _lib.wd_last_error(ctx).decode(errors="replace")


def wd_sync(ctx, stream=None):
    _check(_lib.wd_sync(ctx, _stream(stream)))


def wd_build_freq_rule(ctx, R, n_r, n_polar, n_azim, hermitian=False, kind=WD_RULE_BALL):
    """kind WD_RULE_BALL: (R, n_r, n_polar, n_azim); kind WD_RULE_CUBE_TRAP:
    R = xi_max and n_r = M of the paper's cube trapezoid rule (n_polar and
    n_azim ignored)."""
    d = wd_rule_desc(int(kind), float(R), int(n_r), int(n_polar), int(n_azim), int(bool(hermitian)))
    h = _vp()
    _check(_lib.wd_build_freq_rule(ctx, ctypes.byref(d), ctypes.byref(h)))
    return h


def wd_build_freq_rule_shells(ctx, R, n_r, n_polar, n_azim, hermitian, shell_begin, shell_end):
    """The ball rule (R, n_r, n_polar, n_azim) on its radial shells
    [shell_begin, shell_end)."""
    d = wd_rule_desc(WD_RULE_BALL, float(R), int(n_r), int(n_polar), int(n_azim), int(bool(hermitian)))
    h = _vp()
    _check(_lib.wd_build_freq_rule_shells(ctx, ctypes.byref(d), int(shell_begin), int(shell_end), ctypes.byref(h)))
    return h


def wd_build_cube_rule(ctx, xi_max, M, hermitian=True):
    """The paper's cube trapezoid rule (see WD_RULE_CUBE_TRAP in include/wd.h)."""
    return wd_build_freq_rule(ctx, xi_max, M, 0, 0, hermitian, kind=WD_RULE_CUBE_TRAP)


def wd_rule_from_nodes(ctx, xi, w_geom):
    """xi: (n, 3) nodes (converted to the ABI's SoA layout), w_geom: (n,)."""
    xi = np.asarray(xi, dtype=np.float64).reshape(-1, 3)
    soa = np.ascontiguousarray(xi.T)
    w = np.ascontiguousarray(w_geom, dtype=np.float64)
    h = _vp()
    _check(_lib.wd_rule_from_nodes(ctx, soa.ctypes.data_as(_dp), w.ctypes.data_as(_dp), len(w),
                                   ctypes.byref(h)))
    return h


def wd_rule_info(rule):
    a, b = _i64(), _i64()
    _check(_lib.wd_rule_info(rule, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def wd_rule_copy_nodes(rule):
    """Returns (xi (n, 3), w_geom (n,))."""
    n, _ = wd_rule_info(rule)
    soa = np.empty((3, n))
    w = np.empty(n)
    _check(_lib.wd_rule_copy_nodes(rule, soa.ctypes.data_as(_dp), w.ctypes.data_as(_dp)))
    return np.ascontiguousarray(soa.T), w


def wd_rule_free(rule):
    _lib.wd_rule_free(rule)


def wd_mesh_ft(ctx, rule, verts, tris, precision=WD_FP64):
    n, _ = wd_rule_info(rule)
    m, keep = _host_mesh(verts, tris)
    re = np.empty(n)
    im = np.empty(n)
    _check(_lib.wd_mesh_ft(ctx, rule, ctypes.byref(m), int(precision), re.ctypes.data_as(_dp),
                           im.ctypes.data_as(_dp)))
    return re + 1j * im


def wd_mesh_ft_atoms(ctx, rule, verts, tris):
    """The paper's 64-atom approximation of the mesh transform (float64)."""
    n, _ = wd_rule_info(rule)
    m, keep = _host_mesh(verts, tris)
    re = np.empty(n)
    im = np.empty(n)
    _check(_lib.wd_mesh_ft_atoms(ctx, rule, ctypes.byref(m), re.ctypes.data_as(_dp), im.ctypes.data_as(_dp)))
    return re + 1j * im


def wd_mesh_ft_dev(ctx, rule, verts, tris, precision, out_re, out_im, stream=None):
    _check(_lib.wd_mesh_ft_dev(ctx, rule, _dev_ptr(verts), verts.shape[0], _dev_ptr(tris), tris.shape[0],
                               int(precision), _dev_ptr(out_re), _dev_ptr(out_im), _stream(stream)))


def wd_sphere_ft(ctx, rule, radius=1.0, center=(0.0, 0.0, 0.0)):
    n, _ = wd_rule_info(rule)
    c = np.ascontiguousarray(center, dtype=np.float64)
    re = np.empty(n)
    im = np.empty(n)
    _check(_lib.wd_sphere_ft(ctx, rule, float(radius), c.ctypes.data_as(_dp), re.ctypes.data_as(_dp),
                             im.ctypes.data_as(_dp)))
    return re + 1j * im


def wd_sphere_ft_dev(ctx, rule, radius, center, out_re, out_im, stream=None):
    c = np.ascontiguousarray(center, dtype=np.float64)
    _check(_lib.wd_sphere_ft_dev(ctx, rule, float(radius), c.ctypes.data_as(_dp), _dev_ptr(out_re),
                                 _dev_ptr(out_im), _stream(stream)))


def wd_distance(ctx, rule, verts, tris, nu=None, s=1.0, precision=WD_FP64):
    keep = []
    m, arrays = _host_mesh(verts, tris)
    meas = _measure(nu, keep)
    out = ctypes.c_double()
    _check(_lib.wd_distance(ctx, rule, ctypes.byref(m), ctypes.byref(meas), float(s), int(precision),
                            ctypes.byref(out)))
    return out.value


def wd_distance_dev(ctx, rule, verts, tris, nu, s, precision, out, stream=None):
    """verts (V, 3) float64 and tris (T, 3) int32 CUDA tensors; out: one float64 element."""
    keep = []
    meas = _measure(nu, keep, device=True)
    _check(_lib.wd_distance_dev(ctx, rule, _dev_ptr(verts), verts.shape[0], _dev_ptr(tris), tris.shape[0],
                                ctypes.byref(meas), float(s), int(precision), _dev_ptr(out),
                                _stream(stream)))


def wd_distance_grad(ctx, rule, verts, tris, nu=None, s=1.0, precision=WD_FP64):
    keep = []
    m, arrays = _host_mesh(verts, tris)
    meas = _measure(nu, keep)
    out = ctypes.c_double()
    g = np.empty((m.n_verts, 3))
    _check(_lib.wd_distance_grad(ctx, rule, ctypes.byref(m), ctypes.byref(meas), float(s), int(precision),
                                 ctypes.byref(out), g.ctypes.data_as(_dp)))
    return out.value, g


def wd_distance_grad_dev(ctx, rule, verts, tris, nu, s, precision, out, grad, stream=None):
    keep = []
    meas = _measure(nu, keep, device=True)
    _check(_lib.wd_distance_grad_dev(ctx, rule, _dev_ptr(verts), verts.shape[0], _dev_ptr(tris),
                                     tris.shape[0], ctypes.byref(meas), float(s), int(precision),
                                     _dev_ptr(out), _dev_ptr(grad), _stream(stream)))


def wd_launch_count(ctx):
    return int(_lib.wd_launch_count(ctx))


def wd_distance_dev_noalloc(xi_soa, w_geom, verts, tris, s, radius, center, precision, out, stream=None):
    """Allocation-free distance (see include/wd.h): xi_soa is a (3, n) float64
    CUDA tensor, w_geom (n,), verts (V, 3) float64, tris (T, 3) int32, out one
    float64 element. Runs on the current CUDA device."""
    c = np.ascontiguousarray(center, dtype=np.float64)
    _check(_lib.wd_distance_dev_noalloc(_dev_ptr(xi_soa), _dev_ptr(w_geom), w_geom.shape[0], _dev_ptr(verts),
                                        verts.shape[0], _dev_ptr(tris), tris.shape[0], float(s), float(radius),
                                        c.ctypes.data_as(_dp), int(precision), _dev_ptr(out), _stream(stream)))


# ------------------------------------------------------------------ serving
def wd_serve_start(ctx, rules, precision=WD_MIXED, mem_cap_bytes=8 << 30, max_slots=64, max_pending=4096,
                   timeout_ms=0, pairs_per_launch=4_000_000_000):
    """rules: list of (R, n_r, n_polar, n_azim, hermitian[, kind]) tuples (at most 4); kind defaults to
    WD_RULE_BALL (WD_RULE_CUBE_TRAP: R = xi_max, n_r = M). Queries name their rule by R."""
    cfg = wd_serve_config()
    cfg.mem_cap_bytes = int(mem_cap_bytes)
    cfg.max_slots = int(max_slots)
    cfg.max_pending = int(max_pending)
    cfg.timeout_ms = int(timeout_ms)
    cfg.precision = int(precision)
    cfg.pairs_per_launch = int(pairs_per_launch)
    cfg.n_rules = len(rules)
    for i, r in enumerate(rules):
        R, n_r, n_p, n_a, herm = r[:5]
        kind = r[5] if len(r) > 5 else WD_RULE_BALL
        cfg.rules[i] = wd_rule_desc(int(kind), float(R), int(n_r), int(n_p), int(n_a), int(bool(herm)))
    h = _vp()
    _check(_lib.wd_serve_start(ctx, ctypes.byref(cfg), ctypes.byref(h)))
    return h


def wd_serve_submit(server, verts, tris, s, R):
    """Returns a ticket; raises WDError (status WD_EBUSY, WD_ENOMEM, WD_EINVAL) on refusal."""
    m, keep = _host_mesh(verts, tris)
    t = ctypes.c_uint64()
    _check(_lib.wd_serve_submit(server, ctypes.byref(m), float(s), float(R), ctypes.byref(t)))
    return t.value


def wd_serve_poll(server, ticket):
    """Returns (done, dist2, status)."""
    done = ctypes.c_int()
    d = ctypes.c_double()
    st = ctypes.c_int()
    _check(_lib.wd_serve_poll(server, ticket, ctypes.byref(done), ctypes.byref(d), ctypes.byref(st)))
    return bool(done.value), d.value, st.value


def wd_serve_wait(server, ticket, timeout_ms=60000):
    d = ctypes.c_double()
    _check(_lib.wd_serve_wait(server, ticket, int(timeout_ms), ctypes.byref(d)))
    return d.value


def wd_serve_cancel(server, ticket):
    _check(_lib.wd_serve_cancel(server, ticket))


def wd_serve_stats(server):
    st = wd_serve_stats_t()
    _check(_lib.wd_serve_stats(server, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in wd_serve_stats_t._fields_}


def wd_serve_stop(server):
    _check(_lib.wd_serve_stop(server))


class Context:
    """Owns one wd_ctx; methods forward to the C-named functions above."""

    def __init__(self, device=0):
        self.handle = wd_create(device)

    def close(self):
        if self.handle:
            wd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rule(self, R, n_r, n_polar, n_azim, hermitian=False):
        return wd_build_freq_rule(self.handle, R, n_r, n_polar, n_azim, hermitian)

    def rule_shells(self, R, n_r, n_polar, n_azim, hermitian, shell_begin, shell_end):
        return wd_build_freq_rule_shells(self.handle, R, n_r, n_polar, n_azim, hermitian, shell_begin, shell_end)

    def cube_rule(self, xi_max, M, hermitian=True):
        return wd_build_cube_rule(self.handle, xi_max, M, hermitian)

    def rule_from_nodes(self, xi, w_geom):
        return wd_rule_from_nodes(self.handle, xi, w_geom)

    def mesh_ft(self, rule, verts, tris, precision=WD_FP64):
        return wd_mesh_ft(self.handle, rule, verts, tris, precision)

    def mesh_ft_atoms(self, rule, verts, tris):
        return wd_mesh_ft_atoms(self.handle, rule, verts, tris)

    def sphere_ft(self, rule, radius=1.0, center=(0.0, 0.0, 0.0)):
        return wd_sphere_ft(self.handle, rule, radius, center)

    def distance(self, rule, verts, tris, nu=None, s=1.0, precision=WD_FP64):
        return wd_distance(self.handle, rule, verts, tris, nu, s, precision)

    def distance_grad(self, rule, verts, tris, nu=None, s=1.0, precision=WD_FP64):
        return wd_distance_grad(self.handle, rule, verts, tris, nu, s, precision)

    def launches(self):
        return wd_launch_count(self.handle)
