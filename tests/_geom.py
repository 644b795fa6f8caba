"""Test-only geometry helpers: pinhole projection, polygon clipping, quadrature.

These are textbook constructions written independently of both the oracle and
the CUDA library; they give the tests expected values that neither side
computed.
"""
import math

import numpy as np


def camera_frame(view):
    eye = np.array(view.eye, np.float64)
    fwd = np.array(view.target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.array(view.up, np.float64))
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    th = math.tan(math.radians(view.fov_y_deg) / 2)
    return eye, fwd, right, up, th


def project(view, X):
    """Pixel coordinates (x right, y down, origin at the top-left corner) of world points X [n,3]."""
    eye, fwd, right, up, th = camera_frame(view)
    rel = np.atleast_2d(X) - eye
    z = rel @ fwd
    asp = view.width / view.height
    sx = (rel @ right) / (z * th * asp)
    sy = (rel @ up) / (z * th)
    return np.stack([(sx + 1) * view.width / 2, (1 - sy) * view.height / 2], -1)


def pixel_ray(view, px, py):
    """World-space ray through continuous pixel coordinates: the pinhole model inverted."""
    eye, fwd, right, up, th = camera_frame(view)
    asp = view.width / view.height
    sx = 2 * px / view.width - 1
    sy = 1 - 2 * py / view.height
    d = fwd + right * sx * th * asp + up * sy * th
    return eye, d / np.linalg.norm(d)


def clip_polygon(poly, x0, y0, x1, y1):
    """Sutherland-Hodgman clip of a convex polygon [n,2] against an axis-aligned box."""
    def clip(P, inside, inter):
        out = []
        n = len(P)
        for i in range(n):
            a, b = P[i], P[(i + 1) % n]
            ia, ib = inside(a), inside(b)
            if ia:
                out.append(a)
            if ia != ib:
                out.append(inter(a, b))
        return out

    P = [np.asarray(p, np.float64) for p in poly]
    for axis, bound, keep_ge in ((0, x0, True), (0, x1, False), (1, y0, True), (1, y1, False)):
        if not P:
            break

        def inside(p, axis=axis, bound=bound, keep_ge=keep_ge):
            return p[axis] >= bound if keep_ge else p[axis] <= bound

        def inter(a, b, axis=axis, bound=bound):
            t = (bound - a[axis]) / (b[axis] - a[axis])
            return a + t * (b - a)

        P = clip(P, inside, inter)
    return np.array(P) if P else np.zeros((0, 2))


def polygon_area(P):
    if len(P) < 3:
        return 0.0
    x, y = P[:, 0], P[:, 1]
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


# Degree-5, 7-point rule on a triangle (Stroud T2:5-1), barycentric form, closed-form nodes and weights.
_R15 = math.sqrt(15.0)
_A1, _B1 = (9 - 2 * _R15) / 21, (6 + _R15) / 21
_A2, _B2 = (9 + 2 * _R15) / 21, (6 - _R15) / 21
_TRI_PTS = np.array([[1 / 3, 1 / 3, 1 / 3],
                     [_A1, _B1, _B1], [_B1, _A1, _B1], [_B1, _B1, _A1],
                     [_A2, _B2, _B2], [_B2, _A2, _B2], [_B2, _B2, _A2]])
_TRI_W = np.array([9 / 40] + [(155 + _R15) / 1200] * 3 + [(155 - _R15) / 1200] * 3)


def polygon_quadrature(P, subdiv=2):
    """Points [m,2] and weights [m] integrating over a convex polygon (fan + midpoint subdivision)."""
    pts, wts = [], []
    if len(P) < 3:
        return np.zeros((0, 2)), np.zeros(0)
    c = P.mean(0)
    tris = [(c, P[i], P[(i + 1) % len(P)]) for i in range(len(P))]
    for _ in range(subdiv):
        nt = []
        for a, b, d in tris:
            ab, bd, da = (a + b) / 2, (b + d) / 2, (d + a) / 2
            nt += [(a, ab, da), (ab, b, bd), (da, bd, d), (ab, bd, da)]
        tris = nt
    for a, b, d in tris:
        area = 0.5 * abs((b[0] - a[0]) * (d[1] - a[1]) - (b[1] - a[1]) * (d[0] - a[0]))
        for bc, w in zip(_TRI_PTS, _TRI_W):
            pts.append(bc[0] * a + bc[1] * b + bc[2] * d)
            wts.append(w * area)
    return np.array(pts), np.array(wts)
