"""DUGKS step on a structured curvilinear mesh (oracle; test infrastructure only).

The cylinder configuration of Sec. 4 runs on an O-grid.  The steps are those of the
Cartesian step (`dugks.step`), written for a mesh of quadrilateral cells given by their
nodes; the paper states the scheme for general cells (Eq. explicit_update with face areas
and normals, Eq. reconstruction with the cell slope vector).

Readings (the same ones the CUDA library uses):
 * Nodes X[j][i], Y[j][i], j = 0..ny, i = 0..nx (on a side that is periodic the last node
   column repeats the first).  Cell (i, j) has the nodes A = (i, j), B = (i+1, j),
   C = (i+1, j+1), D = (i, j+1) in counter-clockwise order (positive area).
 * Face normals: the i-face between cells (i-1, j) and (i, j) runs from node (i, j) to
   (i, j+1), e = that edge, n = (e_y, -e_x)/|e| points towards cell (i, j); the j-face between
   (i, j-1) and (i, j) runs from (i, j) to (i+1, j), n = (-e_y, e_x)/|e| points towards (i, j).
   Area |S| = |e|, midpoint x_b = mean of the two nodes.
 * Cell area by the cross product of the diagonals, centroid of the two triangles ABC, ACD.
 * Slopes: van Leer limited differences along the index directions (unit spacing), turned
   into the physical gradient with J^{-T}, J = [[dx/di, dx/dj], [dy/di, dy/dj]] from the
   mean edge vectors of the cell.  On a Cartesian node grid this is the Cartesian slope.
 * Ghost cells (non-periodic sides): copies of the boundary cell's phi-bar-plus and J^{-T};
   the centroid of the first ghost is the boundary cell's centroid reflected through the
   boundary face's midpoint (so the offsets x_b - x_c match the Cartesian step).
 * dt = CFL * min over cells of |V| / max |S| (the cell's smallest width: min(dx, dy) on a
   Cartesian cell), over max_i |xi_i|_inf.
 * Boundary faces: walls and freestream as in `dugks` (incoming half replaced, outgoing half
   reconstructed), with the face normal in place of the axis direction.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .dugks import (FREE, PERIODIC, WALL, Options, _face_model_phi, _limited, bar_plus, cell_state,
                    model_at, tilde_plus)
from .kinetic import Gas, compat_correct4, maxwell_gh


@dataclass
class CurviMesh:
    """Structured curvilinear mesh of the cylinder case (Sec. 4.4): nodes, side kinds, wall and
    freestream states."""
    X: np.ndarray            # [ny+1][nx+1] node x
    Y: np.ndarray            # [ny+1][nx+1] node y
    bc: tuple                # x-low (i = 0), x-high (i = nx), y-low (j = 0), y-high (j = ny)
    wall: tuple = ((0.0, 0.0, 1.0),) * 4
    far: tuple = (1.0, 0.0, 0.0, 1.0)

    @property
    def nx(self):
        return self.X.shape[1] - 1

    @property
    def ny(self):
        return self.X.shape[0] - 1


def geometry(mesh: CurviMesh):
    """Cell areas, centroids and J^{-T}; face normals, lengths and midpoints.
    Face lengths and normals of Eq. explicit_update, offsets and J^{-T} of Eq. reconstruction."""
    X, Y = mesh.X, mesh.Y
    A = np.stack([X[:-1, :-1], Y[:-1, :-1]], -1)
    B = np.stack([X[:-1, 1:], Y[:-1, 1:]], -1)
    C = np.stack([X[1:, 1:], Y[1:, 1:]], -1)
    D = np.stack([X[1:, :-1], Y[1:, :-1]], -1)

    def cross(u, v):
        return u[..., 0] * v[..., 1] - u[..., 1] * v[..., 0]

    area = 0.5 * cross(C - A, D - B)
    a1 = 0.5 * cross(B - A, C - A)
    a2 = 0.5 * cross(C - A, D - A)
    cen = (a1[..., None] * (A + B + C) + a2[..., None] * (A + C + D)) / (3.0 * area[..., None])
    di = 0.5 * ((B - A) + (C - D))
    dj = 0.5 * ((D - A) + (C - B))
    # J = [[di_x, dj_x], [di_y, dj_y]];  J^{-T} = 1/det [[dj_y, -di_y], [-dj_x, di_x]]
    det = di[..., 0] * dj[..., 1] - dj[..., 0] * di[..., 1]
    Jt = np.stack([dj[..., 1], -di[..., 1], -dj[..., 0], di[..., 0]], -1) / det[..., None]
    # i-faces: [ny][nx+1], from node (i, j) to (i, j+1)
    P0 = np.stack([X[:-1, :], Y[:-1, :]], -1)
    P1 = np.stack([X[1:, :], Y[1:, :]], -1)
    e = P1 - P0
    li = np.hypot(e[..., 0], e[..., 1])
    ni = np.stack([e[..., 1], -e[..., 0]], -1) / li[..., None]
    bi = 0.5 * (P0 + P1)
    # j-faces: [ny+1][nx], from node (i, j) to (i+1, j)
    Q0 = np.stack([X[:, :-1], Y[:, :-1]], -1)
    Q1 = np.stack([X[:, 1:], Y[:, 1:]], -1)
    e = Q1 - Q0
    lj = np.hypot(e[..., 0], e[..., 1])
    nj = np.stack([-e[..., 1], e[..., 0]], -1) / lj[..., None]
    bj = 0.5 * (Q0 + Q1)
    return {"area": area, "cen": cen, "Jt": Jt, "ni": ni, "li": li, "bi": bi, "nj": nj, "lj": lj, "bj": bj}


def time_step(mesh: CurviMesh, xi, cfl):
    """Time step: the reading of 'CFL = 0.5' (Sec. 4) with the cell width area / longest face."""
    G = geometry(mesh)
    longest = np.maximum(np.maximum(G["li"][:, :-1], G["li"][:, 1:]), np.maximum(G["lj"][:-1, :], G["lj"][1:, :]))
    L = np.min(G["area"] / longest)
    return cfl * L / np.max(np.abs(xi))


def _pad_cells(a, mesh: CurviMesh):
    """Pad cell arrays [ny][nx][...] by two: wrap on periodic sides, copy otherwise."""
    xm = "wrap" if mesh.bc[0] == PERIODIC else "edge"
    ym = "wrap" if mesh.bc[2] == PERIODIC else "edge"
    extra = [(0, 0)] * (a.ndim - 2)
    a = np.pad(a, [(0, 0), (2, 2)] + extra, mode=xm)
    return np.pad(a, [(2, 2), (0, 0)] + extra, mode=ym)


def period_shifts(mesh: CurviMesh):
    """Translation of the periodic image across the x and the y sides (node column nx minus
    column 0, node row ny minus row 0, averaged; zero on an O-grid).
    Periodic images of Eq. reconstruction."""
    sx = np.array([np.mean(mesh.X[:, -1] - mesh.X[:, 0]), np.mean(mesh.Y[:, -1] - mesh.Y[:, 0])])
    sy = np.array([np.mean(mesh.X[-1, :] - mesh.X[0, :]), np.mean(mesh.Y[-1, :] - mesh.Y[0, :])])
    return sx, sy


def _ghost_centroids(G, mesh: CurviMesh):
    """Padded centroids: periodic images moved by the period; the first ghost of a
    non-periodic side is the boundary cell's centroid reflected through the midpoint of its
    boundary face."""
    c = _pad_cells(G["cen"], mesh)
    ny, nx = G["area"].shape
    sx, sy = period_shifts(mesh)
    if mesh.bc[0] == PERIODIC:
        c[:, :2] -= sx
        c[:, nx + 2:] += sx
    if mesh.bc[2] == PERIODIC:
        c[:2, :] -= sy
        c[ny + 2:, :] += sy
    if mesh.bc[0] != PERIODIC:
        c[2:-2, 1] = 2.0 * G["bi"][:, 0] - G["cen"][:, 0]
        c[2:-2, nx + 2] = 2.0 * G["bi"][:, nx] - G["cen"][:, nx - 1]
    if mesh.bc[2] != PERIODIC:
        c[1, 2:-2] = 2.0 * G["bj"][0, :] - G["cen"][0, :]
        c[ny + 2, 2:-2] = 2.0 * G["bj"][ny, :] - G["cen"][ny - 1, :]
    return c


def step(gt, ht, mesh: CurviMesh, xi, w, gas: Gas, dt: float, opt: Options = Options()):
    """Advance (g~, h~) [ny][nx][Nv] by one time step on the curvilinear mesh.
    Sec. 2.2 on curvilinear cells."""
    s = 0.5 * dt
    ny, nx, nv = gt.shape
    G = geometry(mesh)
    st = cell_state(gt, ht, xi, w, gas, dt)
    gS, hS = model_at(st, xi, w, gas, dt, opt.compat_cell, opt.compat_moments)
    tau = st["tau"][..., None]
    gbp, hbp = bar_plus(gt, gS, tau, dt), bar_plus(ht, hS, tau, dt)
    gtp, htp = tilde_plus(gbp, gt), tilde_plus(hbp, ht)
    P = [_pad_cells(gbp, mesh), _pad_cells(hbp, mesh)]
    Jt = _pad_cells(G["Jt"], mesh)
    cen = _ghost_centroids(G, mesh)
    # physical slopes on the padded arrays (valid away from the outermost ring)
    sx, sy = [], []
    for a in P:
        di = np.zeros_like(a)
        dj = np.zeros_like(a)
        c = a[:, 1:-1, :]
        di[:, 1:-1, :] = _limited(a[:, 2:, :] - c, c - a[:, :-2, :], 1.0, opt.limiter)
        c = a[1:-1, :, :]
        dj[1:-1, :, :] = _limited(a[2:, :, :] - c, c - a[:-2, :, :], 1.0, opt.limiter)
        sx.append(Jt[..., 0:1] * di + Jt[..., 1:2] * dj)
        sy.append(Jt[..., 2:3] * di + Jt[..., 3:4] * dj)

    def recon(k, jj, ii, xb):
        """phi-bar at face midpoints xb [..., 2] from padded cells (jj, ii)."""
        off = xb - cen[jj, ii]
        return (P[k][jj, ii, :] + (off[..., 0:1] - xi[:, 0] * s) * sx[k][jj, ii, :]
                + (off[..., 1:2] - xi[:, 1] * s) * sy[k][jj, ii, :])

    def far_phi(n):
        rho, ux, uy, T = mesh.far
        r, u, t = np.full(n, rho), np.repeat(np.array([[ux, uy]]), n, 0), np.full(n, T)
        gf, hf = maxwell_gh(r, u, t, xi, gas)
        if opt.compat_face:
            gf, hf = compat_correct4(gf, hf, r, u, t, xi, w, gas)
        return gf, hf

    def faces(nrm, xb, jL, iL, jR, iR, sides):
        """phi at a family of faces with normals nrm [..., 2]; sides: ((index tuple, side,
        inward sign), ...) of its boundary faces."""
        # xi.n: its sign picks the upwind side (a tangential velocity rounds to a tiny value
        # of either sign, so the form of the expression is part of the reading)
        xn = nrm[..., 0:1] * xi[:, 0] + nrm[..., 1:2] * xi[:, 1]          # [..., Nv]
        bars = []
        for k in range(2):
            vL, vR = recon(k, jL, iL, xb), recon(k, jR, iR, xb)
            bars.append(np.where(xn > 0, vL, np.where(xn < 0, vR, 0.5 * (vL + vR))))
        out = list(_face_model_phi(bars[0], bars[1], xi, w, gas, s, opt.compat_face, opt.compat_moments))
        for idx, side, inward in sides:
            xin = inward * xn[idx]
            n = xin.shape[0]
            if mesh.bc[side] == FREE:
                gf, hf = far_phi(n)
                in_m = xin > 0.0
                out[0][idx] = np.where(in_m, gf, bars[0][idx])
                out[1][idx] = np.where(in_m, hf, bars[1][idx])
            elif mesh.bc[side] == WALL:
                uw, vw, Tw = mesh.wall[side]
                gw, hw = maxwell_gh(np.ones(n), np.repeat(np.array([[uw, vw]]), n, 0), np.full(n, Tw), xi, gas)
                out_m, in_m = xin <= 0.0, xin > 0.0
                gbar = bars[0][idx]
                num = -np.sum(w * xin * np.where(out_m, gbar, 0.0), axis=-1)
                den = np.sum(w * xin * np.where(in_m, gw, 0.0), axis=-1)
                rw = (num / den)[:, None]
                out[0][idx] = np.where(in_m, rw * gw, gbar)
                out[1][idx] = np.where(in_m, rw * hw, bars[1][idx])
        return out, xn

    # i-faces (all nx+1 columns; with periodic x the last column is the first one again)
    J, I = np.meshgrid(np.arange(ny) + 2, np.arange(nx + 1) + 2, indexing="ij")
    sides_i = []
    if mesh.bc[0] != PERIODIC:
        sides_i = [((slice(None), 0), 0, 1.0), ((slice(None), nx), 1, -1.0)]
    Fi, xni = faces(G["ni"], G["bi"], J, I - 1, J, I, sides_i)
    J, I = np.meshgrid(np.arange(ny + 1) + 2, np.arange(nx) + 2, indexing="ij")
    sides_j = []
    if mesh.bc[2] != PERIODIC:
        sides_j = [((0, slice(None)), 2, 1.0), ((ny, slice(None)), 3, -1.0)]
    Fj, xnj = faces(G["nj"], G["bj"], J - 1, I, J, I, sides_j)
    new = []
    for k, tp in enumerate((gtp, htp)):
        fi = xni * G["li"][..., None] * Fi[k]
        fj = xnj * G["lj"][..., None] * Fj[k]
        div = (fi[:, 1:] - fi[:, :-1]) + (fj[1:, :] - fj[:-1, :])
        new.append(tp - dt * div / G["area"][..., None])
    return new[0], new[1], st


def ogrid(ntheta, nr, r_in=1.0, r_out=11.0):
    """O-grid nodes around a cylinder of radius r_in: ntheta cells around (periodic in i,
    i running clockwise so that cells are counter-clockwise with j outward), nr cells out to
    r_out with geometric stretching; the first cell height is r_in * 2 pi / ntheta (cells of
    aspect ratio one at the wall).  Returns X, Y of shape [nr+1][ntheta+1].
    The cylinder case of Sec. 4.4."""
    h0 = r_in * 2.0 * np.pi / ntheta
    # ratio q with h0 (q^nr - 1)/(q - 1) = r_out - r_in, by bisection
    lo, hi = 1.0 + 1e-12, 2.0
    for _ in range(200):
        q = 0.5 * (lo + hi)
        if h0 * (q ** nr - 1.0) / (q - 1.0) > r_out - r_in:
            hi = q
        else:
            lo = q
    q = 0.5 * (lo + hi)
    r = r_in + h0 * (q ** np.arange(nr + 1) - 1.0) / (q - 1.0)
    r[-1] = r_out
    th = -2.0 * np.pi * np.arange(ntheta + 1) / ntheta
    th[-1] = -2.0 * np.pi
    R, TH = np.meshgrid(r, th, indexing="ij")
    X, Y = R * np.cos(TH), R * np.sin(TH)
    X[:, -1], Y[:, -1] = X[:, 0], Y[:, 0]
    return X, Y
