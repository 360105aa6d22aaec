"""DUGKS step on an unstructured mesh of polygonal cells (oracle; test infrastructure only).

The two-cavity expansion of Sec. 4 runs on unstructured cells.  The steps are those of the
Cartesian step (`dugks.step`) written for general polygons: Eq. explicit_update with the face
lengths and outward normals, Eq. reconstruction with the cell's gradient vector.

Readings (the paper names the limiter family only, "Venkatakrishnan or van Leer"):
 * Cells are counter-clockwise node lists; a face is an edge shared by one or two cells.  Its
   normal points from its first cell L out of L (towards R, or out of the domain).
 * Area and centroid of a polygon by the shoelace formula.
 * Gradient of phi-bar-plus per cell and velocity by least squares over the cells across its
   faces (unit weights); a boundary face contributes a ghost copy of the cell placed at the
   centroid reflected through the face midpoint (a zero difference, which only enters the
   normal matrix).  On a uniform Cartesian grid this is the central difference.
 * Limiter "venkat": Venkatakrishnan's function of the face-midpoint increments against the
   neighbour extrema, eps^2 = (K h)^3 P_c^2 with K = 1, h = sqrt(area) and P_c the cell's own
   value at that velocity (the data are not normalised, and across the two-cavity case's
   density ratio of 1000 an eps set by the dense side would let the thin side's values
   undershoot below zero); "none": unlimited.
 * Walls: diffuse, as in `dugks` (outgoing half reconstructed from the cell, incoming half the
   wall Maxwellian scaled for zero net mass flux), with the face normal.
 * dt = CFL * min over cells of area / longest face, over max |xi|_inf (min(dx, dy) on a
   Cartesian cell, as in `dugks.time_step`).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .dugks import Options, _face_model_phi, bar_plus, cell_state, model_at, tilde_plus
from .kinetic import Gas, maxwell_gh


@dataclass
class UMesh:
    """Polygonal cells of the two-cavity case (Sec. 4.5) with wall indices and wall states."""
    nodes: np.ndarray                 # (Nn, 2)
    cells: list                       # counter-clockwise node index tuples
    wall_of: object = None            # boundary face midpoint (2,) -> wall index (default 0)
    wall: tuple = ((0.0, 0.0, 1.0),)  # (u_w, v_w, T_w) per wall index
    geo: dict = field(default=None, repr=False)

    @property
    def ncell(self):
        return len(self.cells)


def geometry(mesh: UMesh):
    """Areas, centroids, faces (L, R, unit normal out of L, length, midpoint, wall index) and
    every cell's faces with the sign of its outward normal.  Cached on the mesh.
    (face lengths and normals of Eq. explicit_update)."""
    if mesh.geo is not None:
        return mesh.geo
    X = mesh.nodes
    nc = mesh.ncell
    area = np.zeros(nc)
    cen = np.zeros((nc, 2))
    edges = {}
    for c, poly in enumerate(mesh.cells):
        P = X[list(poly)]
        Q = np.roll(P, -1, axis=0)
        cr = P[:, 0] * Q[:, 1] - Q[:, 0] * P[:, 1]
        a = 0.5 * np.sum(cr)
        area[c] = a
        cen[c] = np.sum((P + Q) * cr[:, None], axis=0) / (6.0 * a)
        for k in range(len(poly)):
            n0, n1 = poly[k], poly[(k + 1) % len(poly)]
            edges.setdefault((min(n0, n1), max(n0, n1)), []).append((c, n0, n1))
    fL, fR, fn, fl, fb, fw = [], [], [], [], [], []
    cell_faces = [[] for _ in range(nc)]
    for key in sorted(edges):
        owners = edges[key]
        c, n0, n1 = owners[0]
        e = X[n1] - X[n0]
        L = np.hypot(e[0], e[1])
        f = len(fL)
        fL.append(c)
        fn.append(np.array([e[1], -e[0]]) / L)          # outward for a counter-clockwise cell
        fl.append(L)
        mid = 0.5 * (X[n0] + X[n1])
        fb.append(mid)
        cell_faces[c].append((f, 1.0))
        if len(owners) == 2:
            fR.append(owners[1][0])
            fw.append(-1)
            cell_faces[owners[1][0]].append((f, -1.0))
        else:
            fR.append(-1)
            fw.append(0 if mesh.wall_of is None else int(mesh.wall_of(mid)))
    mesh.geo = {"area": area, "cen": cen, "fL": np.array(fL), "fR": np.array(fR), "fn": np.array(fn),
                "fl": np.array(fl), "fb": np.array(fb), "fw": np.array(fw), "cell_faces": cell_faces}
    return mesh.geo


def time_step(mesh: UMesh, xi, cfl):
    """Time step: the reading of 'CFL = 0.5' (Sec. 4) with the cell width area / longest face."""
    G = geometry(mesh)
    longest = np.zeros(mesh.ncell)
    for c, fs in enumerate(G["cell_faces"]):
        longest[c] = max(G["fl"][f] for f, _ in fs)
    return cfl * np.min(G["area"] / longest) / np.max(np.abs(xi))


def _offsets(G, c):
    """(face, cell across or -1, d) per face of cell c: d the offset of the centroid across
    the face, or on a boundary face of the centroid reflected through the face midpoint."""
    cen = G["cen"]
    out = []
    for f, sgn in G["cell_faces"][c]:
        o = G["fR"][f] if sgn > 0 else G["fL"][f]
        d = cen[o] - cen[c] if o >= 0 else 2.0 * (G["fb"][f] - cen[c])
        out.append((f, o, d))
    return out


def ls_normal_matrix(mesh: UMesh):
    """Normal matrices sum d d^T (Nc, 2, 2) of the least-squares gradients of Eq.
    reconstruction on polygons (the reading in the module header)."""
    G = geometry(mesh)
    M = np.zeros((mesh.ncell, 2, 2))
    for c in range(mesh.ncell):
        for _, _, d in _offsets(G, c):
            M[c] += np.outer(d, d)
    return M


def _gradients(P, mesh: UMesh, limiter: str):
    """Least-squares gradient (Nc, Nv, 2) of P (Nc, Nv), limited per velocity."""
    G = geometry(mesh)
    cen = G["cen"]
    nc, nv = P.shape
    grad = np.zeros((nc, nv, 2))
    Ms = ls_normal_matrix(mesh)
    for c, fs in enumerate(G["cell_faces"]):
        rhs = np.zeros((nv, 2))
        nb = []
        for f, o, d in _offsets(G, c):
            if o >= 0:                                       # a boundary ghost copies the cell: du = 0
                rhs += (P[o] - P[c])[:, None] * d[None, :]
                nb.append(P[o])
        g = np.linalg.solve(Ms[c], rhs.T).T                  # (Nv, 2)
        if limiter == "venkat":
            umax = np.max(np.stack(nb + [P[c]]), axis=0) - P[c]
            umin = np.min(np.stack(nb + [P[c]]), axis=0) - P[c]
            eps2 = (1.0 * np.sqrt(G["area"][c])) ** 3 * P[c] * P[c]
            phi = np.ones(nv)
            for f, _ in fs:
                d2 = g @ (G["fb"][f] - cen[c])
                d1 = np.where(d2 > 0, umax, umin)
                with np.errstate(divide="ignore", invalid="ignore"):
                    v = ((d1 * d1 + eps2) * d2 + 2.0 * d2 * d2 * d1) / (d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + eps2) / d2
                phi = np.minimum(phi, np.where(d2 == 0.0, 1.0, v))
            g = g * phi[:, None]
        grad[c] = g
    return grad


def step(gt, ht, mesh: UMesh, xi, w, gas: Gas, dt: float, opt: Options = Options(), limiter: str = "venkat"):
    """Advance (g~, h~) (Nc, Nv) by one time step on the unstructured mesh.
    Sec. 2.2 on polygonal cells."""
    s = 0.5 * dt
    G = geometry(mesh)
    st = cell_state(gt, ht, xi, w, gas, dt)
    gS, hS = model_at(st, xi, w, gas, dt, opt.compat_cell, opt.compat_moments)
    tau = st["tau"][..., None]
    gbp, hbp = bar_plus(gt, gS, tau, dt), bar_plus(ht, hS, tau, dt)
    gtp, htp = tilde_plus(gbp, gt), tilde_plus(hbp, ht)
    P = [gbp, hbp]
    grads = [_gradients(p, mesh, limiter) for p in P]
    fL, fR, fn, fb = G["fL"], G["fR"], G["fn"], G["fb"]
    cen = G["cen"]
    xn = fn[:, 0:1] * xi[:, 0] + fn[:, 1:2] * xi[:, 1]        # (Nf, Nv)
    inner = fR >= 0
    Rc = np.where(inner, fR, fL)                              # a boundary face's ghost is its cell

    def recon(k, cells, shift):
        off = fb - cen[cells] + shift                         # (Nf, 2)
        gr = grads[k][cells]
        return P[k][cells] + (off[:, 0:1] - xi[:, 0] * s) * gr[..., 0] + (off[:, 1:2] - xi[:, 1] * s) * gr[..., 1]

    ghost_shift = np.where(inner[:, None], 0.0, -2.0 * (fb - cen[fL]))   # reflected centroid offset
    bars = []
    for k in range(2):
        vL = recon(k, fL, 0.0)
        vR = recon(k, Rc, ghost_shift)
        bars.append(np.where(xn > 0, vL, np.where(xn < 0, vR, 0.5 * (vL + vR))))
    out = list(_face_model_phi(bars[0], bars[1], xi, w, gas, s, opt.compat_face, opt.compat_moments))
    for f in np.nonzero(~inner)[0]:
        uw, vw, Tw = mesh.wall[G["fw"][f]]
        gw, hw = maxwell_gh(np.array(1.0), np.array([uw, vw]), np.array(Tw), xi, gas)
        xin = -xn[f]                                          # along the inward normal
        num = -np.sum(w * xin * np.where(xin <= 0.0, bars[0][f], 0.0))
        den = np.sum(w * xin * np.where(xin > 0.0, gw, 0.0))
        rw = num / den
        out[0][f] = np.where(xin > 0.0, rw * gw, bars[0][f])
        out[1][f] = np.where(xin > 0.0, rw * hw, bars[1][f])
    new = []
    for k, tp in enumerate((gtp, htp)):
        F = xn * G["fl"][:, None] * out[k]                    # out of L
        div = np.zeros_like(tp)
        np.add.at(div, fL, F)
        np.subtract.at(div, fR[inner], F[inner])
        new.append(tp - dt * div / G["area"][:, None])
    return new[0], new[1], st
