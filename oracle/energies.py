"""Residuals F(x) and explicit Jacobians J(x) in float64 (test infrastructure).

Each energy is a sum of squares E(x) = sum_r f_r(x)^2 = ||F(x)||^2 (Sec. 2,
Sec. 4 canonical form).  The unknown vector x is the concatenation of the
unknown planes, in the same order and layout the CUDA library uses for its
dense user buffers:

* warp:    [dx (H*W), dy (H*W), theta (H*W)], each plane row-major;
* poisson: [X_0, X_1, X_2, X_3] (each H*W), fixed pixels keep all-zero
           Jacobian columns (they are not solved for);
* mesh:    [dx, dy, dz, A_x, A_y, A_z] (each V);
* warp on a graph: [dx, dy, theta] (each V);
* volume:  [dx, dy, dz, A_x, A_y, A_z] (each W*H*D voxels, index (z*H + y)*W + x);
* embedded deformation: [dx, dy, dz, R00, R01, ..., R22] (each V; R row-major).

Weights: the configured weights multiply the *squared* residual, so residuals
carry their square roots (Fig. 3 caption: weights inside Energy() are square
roots); s_w = sqrt(w_reg), s_f = sqrt(w_fit).

The Jacobian is assembled row by row from hand-derived partial derivatives
(the paper derives them symbolically, Sec. 5.2; here they are written out)
and returned as a scipy CSR matrix.  It is pinned against central finite
differences of F in the tests.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

# Stencil directions of Fig. 24 / Fig. 27, as (offset x, offset y).
STENCIL = ((1, 0), (-1, 0), (0, 1), (0, -1))


def _csr(rows, cols, vals, shape):
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=shape)


def rot2d(theta):
    """Counter-clockwise rotation: R(t) = [[cos t, -sin t], [sin t, cos t]]."""
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, -s], [s, c]])


def euler_rotation(a):
    """Rotate3D of Fig. 25 read as R = Rz(a_z) Ry(a_y) Rx(a_x), radians.

    a: (..., 3) angles.  Returns (R, [dR/da_x, dR/da_y, dR/da_z]) with shape
    (..., 3, 3) each."""
    a = np.asarray(a, np.float64)
    cx, sx = np.cos(a[..., 0]), np.sin(a[..., 0])
    cy, sy = np.cos(a[..., 1]), np.sin(a[..., 1])
    cz, sz = np.cos(a[..., 2]), np.sin(a[..., 2])
    z, o = np.zeros_like(cx), np.ones_like(cx)

    def m(*e):
        return np.stack([np.stack(e[0:3], -1), np.stack(e[3:6], -1), np.stack(e[6:9], -1)], -2)

    Rx = m(o, z, z, z, cx, -sx, z, sx, cx)
    Ry = m(cy, z, sy, z, o, z, -sy, z, cy)
    Rz = m(cz, -sz, z, sz, cz, z, z, z, o)
    dRx = m(z, z, z, z, -sx, -cx, z, cx, -sx)
    dRy = m(-sy, z, cy, z, z, z, -cy, z, -sy)
    dRz = m(-sz, -cz, z, cz, -sz, z, z, z, z)
    R = Rz @ Ry @ Rx
    return R, [Rz @ Ry @ dRx, Rz @ dRy @ Rx, dRz @ Ry @ Rx]


class _Energy:
    N: int

    def energy(self, x) -> float:
        f = self.residuals(x)
        return float(f @ f)


class WarpEnergy(_Energy):
    """ARAP image warping, Fig. 24.

    Regularizer, for every pixel k and stencil direction d with k+d inside
    the image and both pixels unmasked (InBounds * eq(Mask,0) terms):
        r_{k,d} = s_w * ((O_k - O_{k+d}) - R(theta_k) (U_k - U_{k+d}))
    Fit, for every handle h:  s_f * (O_h - C_h).
    Offset O = UrShape + (dx, dy); the constraint C = UrShape + target.
    Both directions of each neighbour pair produce a residual (the stencil
    visits +-x and +-y from every centre).
    """

    def __init__(self, prob):
        self.prob = prob
        W, H = prob.W, prob.H
        self.W, self.H, self.n = W, H, W * H
        self.N = 3 * self.n
        self.s_w = math.sqrt(prob.w_reg)
        self.s_f = math.sqrt(prob.w_fit)
        self.U = prob.urshape.reshape(2, -1).astype(np.float64)
        mask = np.zeros((H, W), bool) if prob.mask is None else (prob.mask != 0)
        ys, xs = np.mgrid[0:H, 0:W]
        ks, js = [], []
        for ox, oy in STENCIL:
            nx, ny = xs + ox, ys + oy
            inb = (nx >= 0) & (nx < W) & (ny >= 0) & (ny < H)
            nxc, nyc = np.clip(nx, 0, W - 1), np.clip(ny, 0, H - 1)
            valid = inb & ~mask & ~mask[nyc, nxc]
            ks.append((ys * W + xs)[valid])
            js.append((nyc * W + nxc)[valid])
        self.k = np.concatenate(ks)
        self.j = np.concatenate(js)
        hidx = prob.handle_idx.astype(np.int64)
        hmask = ~mask.reshape(-1)[hidx]          # handles on excluded pixels are dropped
        self.h = hidx[hmask]
        self.C = self.U[:, self.h] + prob.handle_target.astype(np.float64)[hmask].T
        self.R = 2 * self.k.size + 2 * self.h.size

    def split(self, x):
        x = np.asarray(x, np.float64).reshape(3, self.n)
        return x[0:2], x[2]

    def residuals(self, x):
        d, th = self.split(x)
        O = self.U + d
        k, j = self.k, self.j
        v = self.U[:, k] - self.U[:, j]
        c, s = np.cos(th[k]), np.sin(th[k])
        Rv = np.stack([c * v[0] - s * v[1], s * v[0] + c * v[1]])
        reg = self.s_w * ((O[:, k] - O[:, j]) - Rv)
        fit = self.s_f * (O[:, self.h] - self.C)
        return np.concatenate([reg[0], reg[1], fit[0], fit[1]])

    def jacobian(self, x):
        d, th = self.split(x)
        n, k, j, h = self.n, self.k, self.j, self.h
        m = k.size
        v = self.U[:, k] - self.U[:, j]
        c, s = np.cos(th[k]), np.sin(th[k])
        sw, sf = self.s_w, self.s_f
        rx = np.arange(m)
        ry = m + np.arange(m)
        rfx = 2 * m + np.arange(h.size)
        rfy = 2 * m + h.size + np.arange(h.size)
        rows, cols, vals = [], [], []
        # d r / d O_k = s_w I, d r / d O_{k+d} = -s_w I
        for comp, rr in ((0, rx), (1, ry)):
            rows += [rr, rr]
            cols += [comp * n + k, comp * n + j]
            vals += [np.full(m, sw), np.full(m, -sw)]
        # d r / d theta_k = -s_w R'(theta_k) v,  R'(t) = [[-sin, -cos], [cos, -sin]]
        rows += [rx, ry]
        cols += [2 * n + k, 2 * n + k]
        vals += [-sw * (-s * v[0] - c * v[1]), -sw * (c * v[0] - s * v[1])]
        # fit: d / d O_h = s_f I
        rows += [rfx, rfy]
        cols += [0 * n + h, 1 * n + h]
        vals += [np.full(h.size, sf), np.full(h.size, sf)]
        return _csr(rows, cols, vals, (self.R, self.N))


class WarpGraphEnergy(_Energy):
    """ARAP image warping on an explicit graph (Sec. 4.1 "Graph-based Array
    Access"; the explicit-graph form of Fig. 18).  Per vertex the unknowns are
    (dx, dy, theta) and the rest position U; for every directed edge (a, b)
        r_e = s_w * ((O_a - O_b) - R(theta_a) (U_a - U_b))
    and for every handle h:  s_f * (O_h - C_h), O = U + displacement,
    C = U + target.  With the stencil pairs of an image as edges this is the
    energy of Fig. 24 (WarpEnergy) with its residuals in another order.
    """

    def __init__(self, prob):
        self.prob = prob
        self.V = self.n = prob.V
        self.N = 3 * self.V
        self.s_w = math.sqrt(prob.w_reg)
        self.s_f = math.sqrt(prob.w_fit)
        self.U = prob.urshape.astype(np.float64)
        self.a = prob.v0.astype(np.int64)
        self.b = prob.v1.astype(np.int64)
        self.h = prob.handle_idx.astype(np.int64)
        self.C = self.U[:, self.h] + prob.handle_target.astype(np.float64).T
        self.R = 2 * self.a.size + 2 * self.h.size

    def split(self, x):
        x = np.asarray(x, np.float64).reshape(3, self.V)
        return x[0:2], x[2]

    def residuals(self, x):
        d, th = self.split(x)
        O = self.U + d
        a, b = self.a, self.b
        v = self.U[:, a] - self.U[:, b]
        Rv = np.einsum('eij,je->ie', rot2d(th[a]).transpose(2, 0, 1), v)
        reg = self.s_w * ((O[:, a] - O[:, b]) - Rv)
        fit = self.s_f * (O[:, self.h] - self.C)
        return np.concatenate([reg[0], reg[1], fit[0], fit[1]])

    def jacobian(self, x):
        d, th = self.split(x)
        V, a, b, h = self.V, self.a, self.b, self.h
        m = a.size
        sw, sf = self.s_w, self.s_f
        v = self.U[:, a] - self.U[:, b]
        c, s = np.cos(th[a]), np.sin(th[a])
        rows, cols, vals = [], [], []
        for i in range(2):
            rr = i * m + np.arange(m)
            rows += [rr, rr]
            cols += [i * V + a, i * V + b]
            vals += [np.full(m, sw), np.full(m, -sw)]
        # d r / d theta_a = -s_w R'(theta_a) v
        dRv = np.stack([-s * v[0] - c * v[1], c * v[0] - s * v[1]])
        for i in range(2):
            rows.append(i * m + np.arange(m))
            cols.append(2 * V + a)
            vals.append(-sw * dRv[i])
        for i in range(2):
            rows.append(2 * m + i * h.size + np.arange(h.size))
            cols.append(i * V + h)
            vals.append(np.full(h.size, sf))
        return _csr(rows, cols, vals, (self.R, self.N))


class PoissonEnergy(_Energy):
    """Poisson image editing, Fig. 27 (4 channels, no weights).

    For every free pixel k (mask == 0; Exclude drops the rest) and stencil
    direction d with k+d inside the image (InBounds):
        r_{k,d} = (X_k - X_{k+d}) - (T_k - T_{k+d})     per channel.
    A fixed neighbour X_{k+d} is a constant (Dirichlet boundary).
    """

    def __init__(self, prob):
        self.prob = prob
        W, H = prob.W, prob.H
        self.W, self.H, self.n = W, H, W * H
        self.N = 4 * self.n
        self.T = prob.guide.reshape(4, -1).astype(np.float64)
        # no mask: nothing is excluded, every pixel is free
        free = np.ones(self.n, bool) if prob.mask is None else prob.mask.reshape(-1) == 0
        self.free = free
        ys, xs = np.mgrid[0:H, 0:W]
        ks, js = [], []
        for ox, oy in STENCIL:
            nx, ny = xs + ox, ys + oy
            inb = (nx >= 0) & (nx < W) & (ny >= 0) & (ny < H)
            valid = inb & free.reshape(H, W)
            ks.append((ys * W + xs)[valid])
            js.append((np.clip(ny, 0, H - 1) * W + np.clip(nx, 0, W - 1))[valid])
        self.k = np.concatenate(ks)
        self.j = np.concatenate(js)
        self.R = 4 * self.k.size

    def residuals(self, x):
        X = np.asarray(x, np.float64).reshape(4, self.n)
        k, j = self.k, self.j
        r = (X[:, k] - X[:, j]) - (self.T[:, k] - self.T[:, j])
        return r.reshape(-1)

    def jacobian(self, x=None):
        n, k, j = self.n, self.k, self.j
        m = k.size
        jf = self.free[j]
        rows, cols, vals = [], [], []
        for c in range(4):
            rr = c * m + np.arange(m)
            rows += [rr, rr[jf]]
            cols += [c * n + k, c * n + j[jf]]
            vals += [np.ones(m), -np.ones(int(jf.sum()))]
        return _csr(rows, cols, vals, (self.R, self.N))


class MeshEnergy(_Energy):
    """ARAP mesh deformation, Fig. 25.

    For every directed edge (a, b) of the graph:
        r_e = s_w * ((O_a - O_b) - Rotate3D(A_a) (U_a - U_b))
    and for every handle h:  s_f * (O_h - C_h).
    O = UrShape + displacement; C = UrShape + target.
    """

    def __init__(self, prob):
        self.prob = prob
        self.V = self.n = prob.V
        self.N = 6 * self.V
        self.s_w = math.sqrt(prob.w_reg)
        self.s_f = math.sqrt(prob.w_fit)
        self.U = prob.urshape.astype(np.float64)
        self.a = prob.v0.astype(np.int64)
        self.b = prob.v1.astype(np.int64)
        self.h = prob.handle_idx.astype(np.int64)
        self.C = self.U[:, self.h] + prob.handle_target.astype(np.float64).T
        self.R = 3 * self.a.size + 3 * self.h.size

    def split(self, x):
        x = np.asarray(x, np.float64).reshape(6, self.V)
        return x[0:3], x[3:6]

    def residuals(self, x):
        d, A = self.split(x)
        O = self.U + d
        a, b = self.a, self.b
        v = (self.U[:, a] - self.U[:, b]).T                  # (E, 3)
        R, _ = euler_rotation(A[:, a].T)
        Rv = np.einsum('eij,ej->ie', R, v)
        reg = self.s_w * ((O[:, a] - O[:, b]) - Rv)
        fit = self.s_f * (O[:, self.h] - self.C)
        return np.concatenate([reg.reshape(-1), fit.reshape(-1)])

    def jacobian(self, x):
        d, A = self.split(x)
        V, a, b, h = self.V, self.a, self.b, self.h
        m = a.size
        sw, sf = self.s_w, self.s_f
        v = (self.U[:, a] - self.U[:, b]).T
        _, dR = euler_rotation(A[:, a].T)
        dRv = [np.einsum('eij,ej->ie', dRm, v) for dRm in dR]   # 3 x (3, E)
        rows, cols, vals = [], [], []
        for i in range(3):
            rr = i * m + np.arange(m)
            rows += [rr, rr]
            cols += [i * V + a, i * V + b]
            vals += [np.full(m, sw), np.full(m, -sw)]
            for mm in range(3):
                rows.append(rr)
                cols.append((3 + mm) * V + a)
                vals.append(-sw * dRv[mm][i])
        for i in range(3):
            rr = 3 * m + i * h.size + np.arange(h.size)
            rows.append(rr)
            cols.append(i * V + h)
            vals.append(np.full(h.size, sf))
        return _csr(rows, cols, vals, (self.R, self.N))


class VolumeEnergy(_Energy):
    """Volumetric ARAP deformation, Fig. 31, on the W x H x D voxel array.

    For every voxel k and stencil direction d in {+-x, +-y, +-z} with k+d
    inside the grid (InBounds):
        r_{k,d} = s_w * ((O_k - O_{k+d}) - Rotate3D(A_k) (U_k - U_{k+d}))
    and for every constrained voxel h:  s_f * (O_h - C_h).
    O = UrShape + displacement; C = UrShape + target.  The stencil is walked
    on the 3-D array (shifted slices), not through an edge list.
    """

    def __init__(self, prob):
        self.prob = prob
        W, H, D = prob.W, prob.H, prob.D
        self.shape = (D, H, W)
        self.V = self.n = W * H * D
        self.N = 6 * self.V
        self.s_w = math.sqrt(prob.w_reg)
        self.s_f = math.sqrt(prob.w_fit)
        self.U = prob.urshape.astype(np.float64)
        idx = np.arange(self.V).reshape(D, H, W)
        ks, js = [], []
        for axis in range(3):                    # numpy axes: 0 = z, 1 = y, 2 = x
            for step in (1, -1):
                src = [slice(None)] * 3
                dst = [slice(None)] * 3
                if step == 1:
                    src[axis], dst[axis] = slice(0, -1), slice(1, None)
                else:
                    src[axis], dst[axis] = slice(1, None), slice(0, -1)
                ks.append(idx[tuple(src)].reshape(-1))
                js.append(idx[tuple(dst)].reshape(-1))
        self.a = np.concatenate(ks)
        self.b = np.concatenate(js)
        self.h = prob.handle_idx.astype(np.int64)
        self.C = self.U[:, self.h] + prob.handle_target.astype(np.float64).T
        self.R = 3 * self.a.size + 3 * self.h.size

    def split(self, x):
        x = np.asarray(x, np.float64).reshape(6, self.V)
        return x[0:3], x[3:6]

    def residuals(self, x):
        d, A = self.split(x)
        O = self.U + d
        a, b = self.a, self.b
        v = (self.U[:, a] - self.U[:, b]).T
        R, _ = euler_rotation(A[:, a].T)
        Rv = np.einsum('eij,ej->ie', R, v)
        reg = self.s_w * ((O[:, a] - O[:, b]) - Rv)
        fit = self.s_f * (O[:, self.h] - self.C)
        return np.concatenate([reg.reshape(-1), fit.reshape(-1)])

    def jacobian(self, x):
        d, A = self.split(x)
        V, a, b, h = self.V, self.a, self.b, self.h
        m = a.size
        sw, sf = self.s_w, self.s_f
        v = (self.U[:, a] - self.U[:, b]).T
        _, dR = euler_rotation(A[:, a].T)
        rows, cols, vals = [], [], []
        for i in range(3):
            rr = i * m + np.arange(m)
            rows += [rr, rr]
            cols += [i * V + a, i * V + b]
            vals += [np.full(m, sw), np.full(m, -sw)]
            for mm in range(3):
                rows.append(rr)
                cols.append((3 + mm) * V + a)
                vals.append(-sw * np.einsum('ej,ej->e', dR[mm][:, i, :], v))
        for i in range(3):
            rows.append(3 * m + i * h.size + np.arange(h.size))
            cols.append(i * V + h)
            vals.append(np.full(h.size, sf))
        return _csr(rows, cols, vals, (self.R, self.N))


class EmbeddedEnergy(_Energy):
    """Embedded deformation, Fig. 28 (Appendix A.2.1): every vertex carries a
    position and a full 3x3 matrix R (row-major, R[3r + c]) instead of Euler
    angles; soft constraints keep R a rotation.

    Unknowns: [dx, dy, dz, R00, R01, R02, R10, R11, R12, R20, R21, R22] (each
    V); the position is UrShape + (dx, dy, dz).  Residuals:
      * for every directed edge (a, b):
            s_w * ((O_a - O_b) - R_a (U_a - U_b))
        (Fig. 28 writes (O_b - O_a) - R_a (U_b - U_a), the negation of this
        residual: the same energy);
      * for every vertex, with the columns c_k = (R[k], R[3 + k], R[6 + k]):
            s_r * (c0 . c1), s_r * (c0 . c2), s_r * (c1 . c2),
            s_r * (c0 . c0 - 1), s_r * (c1 . c1 - 1), s_r * (c2 . c2 - 1);
      * for every handle h:  s_f * (O_h - C_h), C_h = UrShape_h + target.
    s_w = sqrt(w_reg), s_r = sqrt(w_rot), s_f = sqrt(w_fit).
    """

    PAIRS = ((0, 1), (0, 2), (1, 2), (0, 0), (1, 1), (2, 2))

    def __init__(self, prob):
        self.prob = prob
        self.V = self.n = prob.V
        self.N = 12 * self.V
        self.s_w = math.sqrt(prob.w_reg)
        self.s_r = math.sqrt(prob.w_rot)
        self.s_f = math.sqrt(prob.w_fit)
        self.U = prob.urshape.astype(np.float64)
        self.a = prob.v0.astype(np.int64)
        self.b = prob.v1.astype(np.int64)
        self.h = prob.handle_idx.astype(np.int64)
        self.C = self.U[:, self.h] + prob.handle_target.astype(np.float64).T
        self.R = 3 * self.a.size + 6 * self.V + 3 * self.h.size

    def split(self, x):
        x = np.asarray(x, np.float64).reshape(12, self.V)
        return x[0:3], x[3:12].reshape(3, 3, self.V)        # Rm[r, c, v] = R_v[3r + c]

    def residuals(self, x):
        d, Rm = self.split(x)
        O = self.U + d
        a, b = self.a, self.b
        v = self.U[:, a] - self.U[:, b]                       # (3, E)
        Rv = np.einsum('rce,ce->re', Rm[:, :, a], v)
        reg = self.s_w * ((O[:, a] - O[:, b]) - Rv)
        col = [Rm[:, k, :] for k in range(3)]                 # c_k as (3, V)
        rot = [self.s_r * (np.sum(col[i] * col[j], axis=0) - (1.0 if i == j else 0.0)) for i, j in self.PAIRS]
        fit = self.s_f * (O[:, self.h] - self.C)
        return np.concatenate([reg.reshape(-1), np.concatenate(rot), fit.reshape(-1)])

    def jacobian(self, x):
        d, Rm = self.split(x)
        V, a, b, h = self.V, self.a, self.b, self.h
        m = a.size
        sw, sr, sf = self.s_w, self.s_r, self.s_f
        v = self.U[:, a] - self.U[:, b]
        rows, cols, vals = [], [], []
        # edge rows: d/dO_a = s_w I, d/dO_b = -s_w I, d/dR_a[3i + c] = -s_w v_c (row i only)
        for i in range(3):
            rr = i * m + np.arange(m)
            rows += [rr, rr]
            cols += [i * V + a, i * V + b]
            vals += [np.full(m, sw), np.full(m, -sw)]
            for c in range(3):
                rows.append(rr)
                cols.append((3 + 3 * i + c) * V + a)
                vals.append(-sw * v[c])
        # rotation rows: d(c_i . c_j)/d c_i = c_j and d/d c_j = c_i (2 c_i when i == j);
        # column k entry r is the unknown R[3r + k]
        base = 3 * m
        vid = np.arange(V)
        for t, (i, j) in enumerate(self.PAIRS):
            rr = base + t * V + vid
            for r in range(3):
                if i == j:
                    rows.append(rr)
                    cols.append((3 + 3 * r + i) * V + vid)
                    vals.append(2.0 * sr * Rm[r, i])
                else:
                    rows += [rr, rr]
                    cols += [(3 + 3 * r + i) * V + vid, (3 + 3 * r + j) * V + vid]
                    vals += [sr * Rm[r, j], sr * Rm[r, i]]
        base += 6 * V
        for i in range(3):
            rows.append(base + i * h.size + np.arange(h.size))
            cols.append(i * V + h)
            vals.append(np.full(h.size, sf))
        return _csr(rows, cols, vals, (self.R, self.N))


def make_energy(prob):
    """Oracle energy object for a synth problem instance."""
    return {"warp": WarpEnergy, "poisson": PoissonEnergy, "mesh": MeshEnergy,
            "warp_graph": WarpGraphEnergy, "volume": VolumeEnergy,
            "embedded": EmbeddedEnergy}[prob.kind](prob)
