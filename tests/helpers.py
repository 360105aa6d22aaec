"""Test-side adapters: a workload description -> oracle objects, and GPU availability."""
from __future__ import annotations

import numpy as np

from oracle import curvi, dugks, kinetic, vspace


def oracle_setup(desc, L=0, compat=True):
    d = desc
    D = d["dim"]
    base = vspace.make_base(d["n_base"], d["umin"], d["umax"], D=D, rule=d["rule"])
    sp = vspace.uniform_space(base, L)
    mu = d["mu_ref"] or kinetic.mu_ref_from_kn(d["Kn"], d["omega"], R=d["R"])
    gas = kinetic.Gas(D=D, K=d["K"], R=d["R"], Pr=d["Pr"], omega=d["omega"], mu_ref=mu)
    far = tuple(d.get("far", (1.0, 0.0, 0.0, 1.0)))
    curv = d.get("nodes") is not None
    if curv:
        xy = d["nodes"]
        mesh = curvi.CurviMesh(xy[..., 0], xy[..., 1], bc=d["bc"], wall=d["wall"], far=far)
    else:
        mesh = dugks.Mesh(d["nx"], d["ny"], d["Lx"] / d["nx"], d["Ly"] / d["ny"], bc=d["bc"], wall=d["wall"],
                          far=far)
    init = d["init"]
    rho = init[..., 0]
    u = init[..., 1:1 + D]
    T = init[..., 3]
    g, h = dugks.initial_tilde(rho, u, T, sp.xi, sp.w, gas, compat=compat)
    dt = curvi.time_step(mesh, sp.xi, d["cfl"]) if curv else dugks.time_step(mesh, sp.xi, d["cfl"], D)
    opt = dugks.Options(cfl=d["cfl"], compat_cell=compat, compat_face=compat, limiter=d["limiter"])
    return {"base": base, "sp": sp, "gas": gas, "mesh": mesh, "g": g, "h": h, "dt": dt, "opt": opt,
            "curvi": curv}


def oracle_run(o, nsteps):
    g, h = o["g"], o["h"]
    stepper = curvi.step if o.get("curvi") else dugks.step
    for _ in range(nsteps):
        g, h, _ = stepper(g, h, o["mesh"], o["sp"].xi, o["sp"].w, o["gas"], o["dt"], o["opt"])
    return g, h


def oracle_moments(o, g, h):
    """Cell moments of the oracle state in the library's output order (rho, u, v, T, qx, qy, rhoE)."""
    st = dugks.cell_state(g, h, o["sp"].xi, o["sp"].w, o["gas"], o["dt"])
    D = o["gas"].D
    ny, nx = g.shape[:2]
    out = np.zeros((7, ny * nx))
    out[0] = st["rho"].ravel()
    out[1] = st["u"][..., 0].ravel()
    if D == 2:
        out[2] = st["u"][..., 1].ravel()
    out[3] = st["T"].ravel()
    out[4] = st["q"][..., 0].ravel()
    if D == 2:
        out[5] = st["q"][..., 1].ravel()
    u2 = np.sum(st["u"] ** 2, axis=-1)
    out[6] = (st["rho"] * (0.5 * u2 + o["gas"].cv * st["T"])).ravel()
    return out


def have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
