"""ctypes front end of the plain CPU oracle (wd_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline / reference leg of bench.py, never by the product package.
Everything here is argument marshalling; the arithmetic is in wd_oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.c_int64


def build(force=False):
    """Compile wd_oracle.c with gcc and OpenMP (no fast-math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.or_gauss_legendre.argtypes = [ctypes.c_int, _dp, _dp]
        L.or_ball_rule.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, _dp, _dp]
        L.or_ball_rule.restype = _i64
        L.or_cube_rule.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, _dp, _dp]
        L.or_cube_rule.restype = _i64
        L.or_triangle_ft.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp]
        L.or_divided_difference.argtypes = [_dp, ctypes.c_int, _dp, _dp]
        L.or_mesh_ft.argtypes = [_dp, _i64, _ip, _i64, _dp, _i64, _dp, _dp, ctypes.c_int]
        L.or_sphere_ft.argtypes = [_dp, _i64, ctypes.c_double, _dp, _dp, _dp]
        L.or_simplex_atoms.argtypes = [_dp, _dp, _dp]
        L.or_mesh_ft_atoms.argtypes = [_dp, _i64, _ip, _i64, _dp, _i64, _dp, _dp, ctypes.c_int]
        dist_args = [_dp, _dp, _i64, ctypes.c_double, ctypes.c_double, _dp, _i64, _ip, _i64, ctypes.c_int,
                     ctypes.c_double, _dp, _dp, _i64, _ip, _i64]
        L.or_distance.argtypes = dist_args + [_dp, _dp, ctypes.c_int]
        L.or_distance.restype = ctypes.c_double
        L.or_distance_grad.argtypes = dist_args + [_dp, ctypes.c_int]
        L.or_distance_grad.restype = ctypes.c_double
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def default_threads():
    return lib().or_num_threads()


def gauss_legendre(n):
    x = np.empty(n)
    w = np.empty(n)
    if lib().or_gauss_legendre(n, _d(x)[1], _d(w)[1]) != 0:
        raise ValueError("n must be >= 1")
    return x, w


def ball_rule(R, n_r, n_polar, n_azim, hermitian):
    """Nodes (N, 3) and s-free weights (N,) of the ball rule, oracle's own build."""
    n = lib().or_ball_rule(R, n_r, n_polar, n_azim, int(bool(hermitian)), None, None)
    if n < 0:
        raise ValueError("invalid rule")
    xi = np.empty((n, 3))
    w = np.empty(n)
    lib().or_ball_rule(R, n_r, n_polar, n_azim, int(bool(hermitian)), _d(xi)[1], _d(w)[1])
    return xi, w


# weight scale of the paper's convention: (1 + |eta|^2) = (1 + |xi|^2 / (4 pi^2)) at xi = 2 pi eta
PAPER_WSCALE = 1.0 / (4.0 * np.pi ** 2)


def cube_rule(xmax, M, hermitian):
    """Nodes (N, 3), angular xi = 2 pi eta, and weights (N,) of the paper's cube
    trapezoid rule on [-xmax, xmax]^3 in eta (oracle's own build)."""
    n = lib().or_cube_rule(xmax, M, int(bool(hermitian)), None, None)
    if n < 0:
        raise ValueError("invalid cube rule")
    xi = np.empty((n, 3))
    w = np.empty(n)
    lib().or_cube_rule(xmax, M, int(bool(hermitian)), _d(xi)[1], _d(w)[1])
    return xi, w


def triangle_ft(a, b, c, xi):
    re = ctypes.c_double()
    im = ctypes.c_double()
    args = [_d(np.asarray(v, dtype=np.float64)) for v in (a, b, c, xi)]
    lib().or_triangle_ft(args[0][1], args[1][1], args[2][1], args[3][1],
                         ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def divided_difference(t):
    """G[t_0..t_k] of G(t) = -exp(-i t), k = len(t) - 1 in {1, 2, 3}."""
    t = np.asarray(t, dtype=np.float64)
    re = ctypes.c_double()
    im = ctypes.c_double()
    tt = _d(t)
    lib().or_divided_difference(tt[1], len(t) - 1, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def mesh_ft(verts, tris, xi, nthreads=None):
    v, vp = _d(verts)
    t, tp = _i(tris)
    x, xp = _d(xi)
    n = len(x)
    re = np.empty(n)
    im = np.empty(n)
    rc = lib().or_mesh_ft(vp, len(v), tp, len(t), xp, n, _d(re)[1], _d(im)[1],
                          nthreads or default_threads())
    if rc != 0:
        raise ValueError("triangle index out of range")
    return re + 1j * im


def simplex_atoms():
    """The paper's 8 x 8 Gauss-Legendre atoms of the standard simplex: (u1, u2, q), 64 each."""
    u1, u2, q = np.empty(64), np.empty(64), np.empty(64)
    lib().or_simplex_atoms(_d(u1)[1], _d(u2)[1], _d(q)[1])
    return u1, u2, q


def mesh_ft_atoms(verts, tris, xi, nthreads=None):
    """mu^ of the mesh's atomic approximation (64 atoms per triangle) at the nodes xi (N, 3)."""
    v, vp = _d(verts)
    t, tp = _i(tris)
    x, xp = _d(xi)
    n = len(x)
    re = np.empty(n)
    im = np.empty(n)
    if lib().or_mesh_ft_atoms(vp, len(v), tp, len(t), xp, n, _d(re)[1], _d(im)[1],
                              nthreads or default_threads()) != 0:
        raise ValueError("triangle index out of range")
    return re + 1j * im


def sphere_ft(xi, radius=1.0, center=(0.0, 0.0, 0.0)):
    x, xp = _d(xi)
    c, cp = _d(np.asarray(center, dtype=np.float64))
    re = np.empty(len(x))
    im = np.empty(len(x))
    lib().or_sphere_ft(xp, len(x), radius, cp, _d(re)[1], _d(im)[1])
    return re + 1j * im


def _nu_args(nu):
    """nu: ('sphere', radius, center) or ('mesh', verts, tris)."""
    if nu is None or nu[0] == "sphere":
        radius = 1.0 if nu is None else float(nu[1])
        center = (0.0, 0.0, 0.0) if nu is None or len(nu) < 3 else nu[2]
        c = _d(np.asarray(center, dtype=np.float64))
        return (0, radius, c, (None, None), 0, (None, None), 0)
    v2 = _d(nu[1])
    t2 = _i(nu[2])
    return (1, 0.0, (None, None), v2, len(v2[0]), t2, len(t2[0]))


def distance(xi, w_geom, s, verts, tris, nu=None, nthreads=None, return_mu=False, wscale=1.0):
    """D = sum_k w_k (1 + wscale |xi_k|^2)^-s |mu^(xi_k) - nu^(xi_k)|^2 (long double)."""
    x, xp = _d(xi)
    w, wp = _d(w_geom)
    v, vp = _d(verts)
    t, tp = _i(tris)
    kind, radius, c, v2, nv2, t2, nt2 = _nu_args(nu)
    mu_re = np.empty(len(x)) if return_mu else None
    mu_im = np.empty(len(x)) if return_mu else None
    d = lib().or_distance(xp, wp, len(x), float(s), float(wscale), vp, len(v), tp, len(t), kind, radius, c[1],
                          v2[1], nv2, t2[1], nt2,
                          _d(mu_re)[1] if return_mu else None,
                          _d(mu_im)[1] if return_mu else None,
                          nthreads or default_threads())
    if np.isnan(d):
        raise ValueError("triangle index out of range")
    if return_mu:
        return d, mu_re + 1j * mu_im
    return d


def distance_grad(xi, w_geom, s, verts, tris, nu=None, nthreads=None, wscale=1.0):
    x, xp = _d(xi)
    w, wp = _d(w_geom)
    v, vp = _d(verts)
    t, tp = _i(tris)
    kind, radius, c, v2, nv2, t2, nt2 = _nu_args(nu)
    g = np.empty((len(v), 3))
    d = lib().or_distance_grad(xp, wp, len(x), float(s), float(wscale), vp, len(v), tp, len(t), kind, radius,
                               c[1], v2[1], nv2, t2[1], nt2, _d(g)[1],
                               nthreads or default_threads())
    if np.isnan(d):
        raise ValueError("triangle index out of range")
    return d, g
