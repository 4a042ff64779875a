"""Run-level physics of the FFT-LB method on the GPU path (arXiv:1011.3582,
Sec. 4): batches of independent runs relaxed together (fftlb_batch_*) with
time-averaged diagnostics of the equilibrium they approach.

  * planar slabs (Sec. 4.1, Fig. 9 / Fig. 13): bulk vapour and liquid
    densities and temperatures, to be compared with the Maxwell construction
    of the vdW equation of state at the measured temperature;
  * circular droplets (Sec. 4.2, Eqs. 55-56): the pressure difference
    Delta P = P^w(inside) - P^w(outside) with P^w of Eq. 18 at the bulk
    averages over r < R/2 and r > 3R/2 (reading A12 of the paper), to be
    fitted by the Laplace law Delta P = sigma / R;
  * every run: the largest speed max |u| (the spurious velocity u^s of
    Figs. 10-12, 17-19) and the total energy e_T of Eq. 17 (its drift).

The initial fields and the densities they start from come from the caller
(paper_1011_3582_gb300.workloads lays them out); nothing here computes a
reference value.  The acoustic oscillations that the initial profiles launch
in a periodic box decay on the viscous time L^2 / nu, long against the time
an affordable run covers, so bulk values are averaged over the second half
of a run (several acoustic periods) rather than read at its end.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np


def vdw_pressure(rho, T, a, b):
    """P^w = rho T / (1 - b rho) - a rho^2 (Eq. 18 with general a, b)."""
    return rho * T / (1.0 - b * rho) - a * rho * rho


def slab_masks(n):
    """Bulk regions of a slab laid out by workloads.slab with its default
    interfaces at n/4 and 3n/4 (liquid in the middle): vapour within n/8 of
    the box edge, liquid within n/8 of the centre (each a quarter of the box,
    more than n/8 away from either interface)."""
    c = np.arange(n)
    vap = (c < n // 8) | (c >= n - n // 8)
    liq = (c >= 3 * n // 8) & (c < 5 * n // 8)
    return vap, liq


def droplet_masks(nx, ny, R, center=None):
    """Inside r < R/2 and outside r > 3R/2 of a drop centred as by
    workloads.droplet (reading A12 of the paper)."""
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    cx, cy = (nx / 2.0, ny / 2.0) if center is None else center
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    return r < R / 2.0, r > 1.5 * R


@dataclasses.dataclass
class Run:
    """One run of a relaxation batch: its parameters (fftlb_params), its
    initial fields (rho, u_x, u_y, T) and how its state is summarised:
    kind 'slab' (axis 'x' or 'y') or 'droplet' (radius R)."""
    params: object
    fields: tuple
    kind: str = "slab"
    axis: str = "x"
    R: float = 0.0


def summarise(run, fields):
    """Bulk averages of one sampled state (rho, ux, uy, T arrays)."""
    rho, ux, uy, T = fields
    p = run.params
    out = {"umax": float(np.sqrt(ux * ux + uy * uy).max())}
    if run.kind == "slab":
        n = p.nx if run.axis == "x" else p.ny
        vap, liq = slab_masks(n)
        r1 = rho.mean(axis=0) if run.axis == "x" else rho.mean(axis=1)
        t1 = T.mean(axis=0) if run.axis == "x" else T.mean(axis=1)
        out.update(rho_v=float(r1[vap].mean()), rho_l=float(r1[liq].mean()),
                   T_v=float(t1[vap].mean()), T_l=float(t1[liq].mean()))
    else:
        inside, outside = droplet_masks(p.nx, p.ny, run.R)
        ri, ro = float(rho[inside].mean()), float(rho[outside].mean())
        Ti, To = float(T[inside].mean()), float(T[outside].mean())
        # equimolar radius (lattice units): the disc of density ri in density
        # ro that holds the same excess mass
        Re = float(np.sqrt(max((rho - ro).sum(), 0.0) / (np.pi * (ri - ro))))
        out.update(rho_in=ri, rho_out=ro, T_in=Ti, T_out=To, R_e=Re,
                   dP=float(vdw_pressure(ri, Ti, p.a, p.b) - vdw_pressure(ro, To, p.a, p.b)))
    return out


def relax(fl, runs, t_end, sample_dt, avg_from=0.5, autotune=True, log=None):
    """Advances the runs together as one fftlb batch (runs with identical
    parameters share one engine and its launches) to time t_end, samples
    every sample_dt (rounded to whole steps of each run's dt; all runs of one
    call must share dt) and averages every summary over the samples with
    t >= avg_from * t_end.  Returns, per run, {"samples": [(t, summary,
    invariants)], "mean": {key: mean}, "std": {key: std}, "steps": n,
    "seconds": wall time, "finite": whether every sample was finite}.  A run
    that goes non-finite does not stop the others (the runs of a batch are
    independent)."""
    dts = {float(r.params.dt) for r in runs}
    if len(dts) != 1:
        raise ValueError("relax: all runs of one call must use the same dt")
    dt = dts.pop()
    every = max(1, int(round(sample_dt / dt)))
    nsteps = int(round(t_end / dt))
    hist = [[] for _ in runs]
    t0 = time.time()
    with fl.Batch([r.params for r in runs], autotune=autotune) as b:
        for i, r in enumerate(runs):
            b.set_fields(i, *r.fields)
        done = 0
        while done < nsteps:
            n = min(every, nsteps - done)
            b.step(n)
            done += n
            for i, r in enumerate(runs):
                inv = b.invariants(i)
                hist[i].append((done * dt, summarise(r, b.fields(i)), inv))
            if log:
                log(done * dt, hist)
    secs = time.time() - t0
    out = []
    for h in hist:
        keep = [s for t, s, _ in h if t >= avg_from * t_end - 1e-12]
        keys = keep[0].keys() if keep else []
        finite = all(np.isfinite(list(s.values())).all() for _, s, _ in h)
        out.append({"samples": h, "steps": nsteps, "seconds": secs, "finite": finite,
                    "mean": {k: float(np.mean([s[k] for s in keep])) for k in keys},
                    "std": {k: float(np.std([s[k] for s in keep])) for k in keys}})
    return out
