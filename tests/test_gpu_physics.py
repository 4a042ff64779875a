"""Run-level physics on the GPU path (Sec. 4 of the paper): coexistence
densities of planar slabs against the Maxwell construction (Sec. 4.1,
Fig. 9), the Laplace law of droplets against the square-gradient surface
tension (Sec. 4.2, Eqs. 55-56), the spurious velocity max |u| and the drift
of the total energy e_T (Eq. 17), in fp64 and fp32, with the fp32 error
stated against the fp64 run for every result.

Reading (time step): the paper's dt = 1e-5 needs millions of steps to reach
equilibrium (t = 20-30).  These runs use dt = 1e-4, inside the stability
limits of SSP-RK3 (dt |v|max k_max = 0.28 for the window-4 symbol at
dx = 1/256, dt / tau = 0.01), and the coexistence experiment repeats the
runs at dt = 5e-5 (fp64 and fp32) to show the averaged densities do not
depend on it.
Bulk values are averaged over the second half of each run, because the
acoustic oscillations the initial profiles launch decay only on the
viscous time L^2 / nu (see paper_1011_3582_gb300.physics).

The short test runs in the normal GPU suite; the long experiments run only
with FFTLB_PHYSICS=1 (several GPU-minutes) and print their tables
(FFTLB_PHYSICS_OUT=<file> also writes them as JSON)."""
import json
import os

import numpy as np
import pytest

from gpu_common import A49, B21, TC49, lib
from oracle import thermo as TH
from paper_1011_3582_gb300 import physics as PH
from paper_1011_3582_gb300 import workloads as W

pytestmark = pytest.mark.gpu
LONG = pytest.mark.skipif(not os.environ.get("FFTLB_PHYSICS"), reason="long physics runs (set FFTLB_PHYSICS=1)")


@pytest.fixture(scope="module")
def fl():
    return lib()


def slab_run(fl, a, b, T, precision, dt, n=512, K=1e-5, window=4):
    rv, rl = TH.maxwell(T, a, b)
    fields = W.slab(n, 4, rv, rl, T, width=2.0, axis="x")
    p = fl.params(nx=n, ny=4, a=a, b=b, K=K, dt=dt, precision=precision, integrator=3, window=window)
    return PH.Run(p, fields, "slab", "x")


def droplet_run(fl, a, b, T, R, precision, dt, n=256, K=1e-5):
    rv, rl = TH.maxwell(T, a, b)
    fields = W.droplet(n, n, R, rl, rv, T, width=2.0)
    p = fl.params(nx=n, ny=n, a=a, b=b, K=K, dt=dt, precision=precision, integrator=3)
    return PH.Run(p, fields, "droplet", R=R)


def coexistence_errors(res, a, b):
    """Relative deviations of the averaged bulk densities from the Maxwell
    densities at the averaged temperature of the two bulk phases."""
    m = res["mean"]
    Tm = 0.5 * (m["T_v"] + m["T_l"])
    rv, rl = TH.maxwell(Tm, a, b)
    return (m["rho_v"] - rv) / rv, (m["rho_l"] - rl) / rl, Tm


def test_slab_coexistence_short(fl):
    """Two 512 x 4 slabs in fp32 (the 9/49, 2/21 fluid at 0.9 T_c and the
    paper's fluid at T = 0.95), 20 000 steps of dt = 1e-4 (t = 2), bulk
    densities averaged over t in [1, 2], against the Maxwell densities at the
    measured mean temperature of the two phases (the relaxing interfaces
    change T by a few 1e-3: energy is conserved, not T): vapour within 4% and
    liquid within 2% for the 9/49 fluid, whose interfaces span about two
    sites at K = 1e-5, both within 1.5% for the paper's fluid (the fp64
    deviations of the long runs, 2.4% and 0.9% at most, with margin).  Mass:
    every stage rounds every f_i to fp32 once (relative u / 2), and in a
    uniform bulk phase the roundings of all sites have one sign, so the
    total can move by up to 3 (u / 2) per step: 20 000 steps, 1.8e-3."""
    runs = [slab_run(fl, A49, B21, 0.9 * TC49, 32, 1e-4), slab_run(fl, 9 / 8, 1 / 3, 0.95, 32, 1e-4)]
    res = PH.relax(fl, runs, t_end=2.0, sample_dt=0.1)
    u = 2.0 ** -24
    for r, (a, b, T0, tv, tl) in zip(res, [(A49, B21, 0.9 * TC49, 4e-2, 2e-2), (9 / 8, 1 / 3, 0.95, 1.5e-2, 1.5e-2)]):
        assert r["finite"]
        ev, el, Tm = coexistence_errors(r, a, b)
        m0, m1 = r["samples"][0][2]["mass"], r["samples"][-1][2]["mass"]
        print("slab a=%.4f T0=%.4f: T %.5f (T_v %.5f, T_l %.5f), rho_v %+.2e, rho_l %+.2e vs Maxwell, mass %.1e"
              % (a, T0, Tm, r["mean"]["T_v"], r["mean"]["T_l"], ev, el, abs(m1 - m0) / m0))
        assert abs(ev) < tv and abs(el) < tl
        assert abs(m1 - m0) / m0 < 3 * (u / 2) * r["steps"]


def _dump(name, obj):
    path = os.environ.get("FFTLB_PHYSICS_OUT")
    if not path:
        return
    data = json.load(open(path)) if os.path.exists(path) else {}
    data[name] = obj
    json.dump(data, open(path, "w"), indent=1)


COEX = [(A49, B21, tr * TC49) for tr in (0.75, 0.80, 0.85, 0.90, 0.95)] + \
       [(9 / 8, 1 / 3, T) for T in (0.87, 0.89, 0.91, 0.93, 0.95, 0.97)]


def coexistence(fl, label, prec, dt, t_end=8.0):
    runs = [slab_run(fl, a, b, T, prec, dt) for a, b, T in COEX]
    res = PH.relax(fl, runs, t_end=t_end, sample_dt=0.1)
    rows = []
    print("\n%s (%d steps, %.0f s)" % (label, res[0]["steps"], res[0]["seconds"]))
    for (a, b, T0), r in zip(COEX, res):
        if not r["finite"]:
            rows.append(dict(a=a, T0=T0, finite=False))
            print("  a=%.4f T0=%.4f: non-finite" % (a, T0))
            continue
        ev, el, Tm = coexistence_errors(r, a, b)
        inv = [s[2] for s in r["samples"]]
        e0, m0 = inv[0]["eT"], inv[0]["mass"]
        rows.append(dict(a=a, T0=T0, T=Tm, finite=True, rho_v=r["mean"]["rho_v"], rho_l=r["mean"]["rho_l"],
                         std_v=r["std"]["rho_v"], std_l=r["std"]["rho_l"], dev_v=ev, dev_l=el,
                         umax=r["mean"]["umax"], eT_drift=max(abs(i["eT"] - e0) for i in inv) / abs(e0),
                         mass_drift=max(abs(i["mass"] - m0) for i in inv) / m0,
                         seconds=r["seconds"], steps=r["steps"]))
        row = rows[-1]
        print("  a=%.4f T0=%.4f T=%.5f rho_v=%.6f(%.1e) rho_l=%.6f(%.1e) dev %+.2e %+.2e umax %.2e "
              "eT drift %.1e mass drift %.1e" % (a, T0, Tm, row["rho_v"], row["std_v"], row["rho_l"],
                                                 row["std_l"], ev, el, row["umax"], row["eT_drift"],
                                                 row["mass_drift"]))
    _dump("coexistence_" + label, rows)
    return rows


@LONG
def test_coexistence_fp64(fl):
    """Coexistence densities of the 9/49, 2/21 fluid at T_r = 0.75 .. 0.95 and
    of the paper's fluid at the quench temperatures 0.87 .. 0.97 (Sec. 4.1),
    fp64, dt = 1e-4, t = 8, averaged over t in [4, 8]."""
    rows = coexistence(fl, "fp64", 64, 1e-4)
    assert all(r["finite"] for r in rows)


@LONG
def test_coexistence_fp32(fl):
    """The same in fp32 at dt = 1e-4 and at dt = 5e-5 (the averaged densities
    must not depend on the step)."""
    a = coexistence(fl, "fp32", 32, 1e-4)
    b = coexistence(fl, "fp32_dt2", 32, 5e-5)
    for x, y in zip(a, b):
        if x["finite"] and y["finite"]:
            print("  a=%.4f T0=%.4f: dt/2 - dt rho_v %+.2e rho_l %+.2e"
                  % (x["a"], x["T0"], (y["rho_v"] - x["rho_v"]) / x["rho_v"], (y["rho_l"] - x["rho_l"]) / x["rho_l"]))
    assert all(r["finite"] for r in a + b)


@LONG
def test_coexistence_fp64_half_dt(fl):
    """The time-step reading: the paper's fluid at the six quench temperatures
    0.87 .. 0.97 in fp64 at dt = 1e-4 and at dt = 5e-5, both to t = 4, bulk
    densities averaged over t in [2, 4].  A stationary state L(f) = 0 is a
    fixed point of SSP-RK3 for every dt; the relaxing runs differ only by the
    time-integration error of the transient (third order in dt), which the
    averaged densities must show below 1e-4."""
    COEXP = [(9 / 8, 1 / 3, T) for T in (0.87, 0.89, 0.91, 0.93, 0.95, 0.97)]
    out = {}
    for dt in (1e-4, 5e-5):
        runs = [slab_run(fl, a, b, T, 64, dt) for a, b, T in COEXP]
        out[dt] = PH.relax(fl, runs, t_end=4.0, sample_dt=0.1)
    rows = []
    for (a, b, T0), x, y in zip(COEXP, out[1e-4], out[5e-5]):
        assert x["finite"] and y["finite"]
        dv = (y["mean"]["rho_v"] - x["mean"]["rho_v"]) / x["mean"]["rho_v"]
        dl = (y["mean"]["rho_l"] - x["mean"]["rho_l"]) / x["mean"]["rho_l"]
        rows.append(dict(T0=T0, rho_v=x["mean"]["rho_v"], rho_l=x["mean"]["rho_l"], d_rho_v=dv, d_rho_l=dl))
        print("T0=%.2f: rho_v %.6f rho_l %.6f (dt = 1e-4); dt/2 - dt: %+.2e %+.2e" %
              (T0, x["mean"]["rho_v"], x["mean"]["rho_l"], dv, dl))
    _dump("coexistence_fp64_half_dt", rows)
    assert max(max(abs(r["d_rho_v"]), abs(r["d_rho_l"])) for r in rows) < 1e-4


@LONG
def test_coexistence_gradient_coefficient(fl):
    """The paper's fluid at the quench temperatures 0.87 .. 0.97 with the
    gradient coefficients of Fig. 13 (K = 5e-6) and Fig. 9 (K = 0), fp32,
    dt = 1e-4, t = 8, averaged over t in [4, 8], against the Maxwell
    densities at the measured temperature (the K = 1e-5 runs are
    test_coexistence_fp32).  With K = 0 nothing sets an interface width: the
    profile steepens to the grid scale, where the windowed derivative's
    error is largest, so the run is reported, finite or not.  With
    FFTLB_PHYSICS_FP64=1 the K = 5e-6 runs are made in fp64."""
    out = {}
    prec = 64 if os.environ.get("FFTLB_PHYSICS_FP64") else 32   # fp64: the reference of the fp32 error
    for K in ((5e-6,) if prec == 64 else (5e-6, 0.0)):
        runs = []
        for T in (0.87, 0.89, 0.91, 0.93, 0.95, 0.97):
            rv, rl = TH.maxwell(T, 9 / 8, 1 / 3)
            fields = W.slab(512, 4, rv, rl, T, width=2.0, axis="x")
            p = fl.params(nx=512, ny=4, a=9 / 8, b=1 / 3, K=K, dt=1e-4, precision=prec, integrator=3)
            runs.append(PH.Run(p, fields, "slab", "x"))
        res = PH.relax(fl, runs, t_end=8.0, sample_dt=0.1)
        rows = []
        for T, r in zip((0.87, 0.89, 0.91, 0.93, 0.95, 0.97), res):
            if not r["finite"]:
                rows.append(dict(T0=T, finite=False))
                print("K=%g T0=%.2f: non-finite" % (K, T))
                continue
            ev, el, Tm = coexistence_errors(r, 9 / 8, 1 / 3)
            rows.append(dict(T0=T, T=Tm, finite=True, rho_v=r["mean"]["rho_v"], rho_l=r["mean"]["rho_l"],
                             dev_v=ev, dev_l=el, umax=r["mean"]["umax"]))
            print("K=%g T0=%.2f T=%.5f rho_v=%.6f rho_l=%.6f dev %+.2e %+.2e umax %.2e"
                  % (K, T, Tm, r["mean"]["rho_v"], r["mean"]["rho_l"], ev, el, r["mean"]["umax"]))
        out[str(K)] = rows
    _dump("coexistence_K_fp%d" % prec, out)
    assert all(r["finite"] for r in out[str(5e-6)])


def laplace(fl, a, b, T, prec, t_end, radii=(20.0, 30.0, 40.0, 50.0)):
    runs = [droplet_run(fl, a, b, T, R, prec, 1e-4) for R in radii]
    res = PH.relax(fl, runs, t_end=t_end, sample_dt=0.2)
    Re = np.array([r["mean"]["R_e"] for r in res])
    dP = np.array([r["mean"]["dP"] for r in res])
    slope, _ = TH.laplace_sigma(Re, dP)
    Tm = float(np.mean([0.5 * (r["mean"]["T_in"] + r["mean"]["T_out"]) for r in res]))
    # Delta P = sigma / (R_e dx) with R_e in sites
    return dict(R=list(radii), R_e=Re.tolist(), dP=dP.tolist(), dP_std=[r["std"]["dP"] for r in res],
                sigma_fit=slope / 256.0, sigma_theory=TH.sigma_square_gradient(Tm, a, b, 1e-5), T=Tm,
                umax=[r["mean"]["umax"] for r in res], seconds=res[0]["seconds"],
                finite=all(r["finite"] for r in res))


@LONG
def test_laplace_law(fl):
    """Droplets of radius 20, 30, 40, 50 on 256^2 (configuration 2: the
    9/49, 2/21 fluid at 0.85 T_c; and the paper's fluid at T = 0.95, K =
    1e-5, Sec. 4.2), fp32, dt = 1e-4, t = 8, Delta P averaged over t in
    [4, 8]; sigma from the least-squares slope of Delta P against 1/R_e
    (equimolar radius), against the square-gradient sigma at the measured T;
    and fp32 to t = 4 for the comparison with the fp64 run to t = 4
    (test_laplace_fp64)."""
    out = {}
    for name, a, b, T in (("a9/49", A49, B21, 0.85 * TC49), ("paper", 9 / 8, 1 / 3, 0.95)):
        out[name] = laplace(fl, a, b, T, 32, 8.0)
        x = out[name]
        print("\n%s: T=%.5f R_e=%s dP=%s sigma fit %.4e theory %.4e (%+.2f%%), umax %s"
              % (name, x["T"], np.round(x["R_e"], 2), np.array2string(np.array(x["dP"]), precision=6),
                 x["sigma_fit"], x["sigma_theory"], 100 * (x["sigma_fit"] / x["sigma_theory"] - 1),
                 np.round(x["umax"], 7)))
    out["a9/49_t4"] = laplace(fl, A49, B21, 0.85 * TC49, 32, 4.0)
    print("a9/49 fp32 t=4: dP %s sigma %.4e" % (out["a9/49_t4"]["dP"], out["a9/49_t4"]["sigma_fit"]))
    _dump("laplace_fp32", out)
    assert all(v["finite"] for v in out.values())


@LONG
def test_laplace_fp64(fl):
    """The 9/49, 2/21 droplet set in fp64 to t = 4."""
    x = laplace(fl, A49, B21, 0.85 * TC49, 64, 4.0)
    print("a9/49 fp64 t=4: R_e %s dP %s sigma %.4e theory %.4e" % (x["R_e"], x["dP"], x["sigma_fit"], x["sigma_theory"]))
    _dump("laplace_fp64", x)
    assert x["finite"]


@LONG
def test_triangle_spurious_velocity(fl):
    """The relaxation of a triangular drop (Sec. 4.2, Figs. 17-19): an
    equilateral triangle of side 64 with a sharp edge in a 128^2 box,
    (rho, T) = (1.46, 0.95) inside and (0.58, 0.95) outside, the paper's
    fluid, K = 1e-5; the maximum speed u^s_max(t) with the windows k1..k4
    in fp32 and with k4 in fp64 as well, dt = 1e-4 to t = 5 (the paper runs
    to t = 30 at dt = 1e-5, where u^s_max has levelled off for t > 20).
    The paper finds u^s_max lower for every higher window order."""
    R_eq = float(np.sqrt(np.sqrt(3.0) / 4.0 * 64 ** 2 / np.pi))   # the disc of the triangle's area
    fields = W.triangle(128, 128, 64, 1.46, 0.58, 0.95)
    runs = [PH.Run(fl.params(nx=128, ny=128, a=9 / 8, b=1 / 3, K=1e-5, dt=1e-4, precision=prec, integrator=3,
                             window=w), fields, "droplet", R=R_eq)
            for prec, w in ((32, 1), (32, 2), (32, 3), (32, 4), (64, 4))]
    res = PH.relax(fl, runs, t_end=5.0, sample_dt=0.05, avg_from=0.8)
    curves = {}
    for (prec, w), r in zip(((32, 1), (32, 2), (32, 3), (32, 4), (64, 4)), res):
        t = [s[0] for s in r["samples"]]
        um = [s[1]["umax"] for s in r["samples"]]
        curves["fp%d_k%d" % (prec, w)] = dict(t=t, umax=um, finite=r["finite"])
        print("fp%d k%d: u^s_max at t = 0.5, 1, 2, 3, 5: %s" % (prec, w, ["%.3e" % um[int(round(x / 0.05)) - 1]
                                                                         for x in (0.5, 1, 2, 3, 5)]))
    u32, u64 = np.array(curves["fp32_k4"]["umax"]), np.array(curves["fp64_k4"]["umax"])
    print("fp32 vs fp64 (k4): largest relative difference of u^s_max over t in [1, 5]: %.2e"
          % (np.abs(u32 - u64)[19:] / u64[19:]).max())
    _dump("triangle", curves)
    assert all(c["finite"] for c in curves.values())


@LONG
def test_energy_drift_by_window(fl):
    """Total-energy variation Delta e_T(t) = e_T(t) - e_T(0) of the phase
    separation of Fig. 2 / Fig. 8 (128^2, rho = 1 + U(-1e-3, 1e-3), T = 0.85,
    the paper's fluid, K = 1e-5) with the windows k1..k4 in fp64, and k4 in
    fp32, dt = 1e-4 to t = 2.  The paper finds |Delta e_T| smaller for every
    higher window order."""
    fields = W.slab(128, 128, 1.0, 1.0, 0.85, noise=1e-3, seed=8)
    runs = [PH.Run(fl.params(nx=128, ny=128, a=9 / 8, b=1 / 3, K=1e-5, dt=1e-4, precision=prec, integrator=3,
                             window=w), fields, "slab", "y")
            for prec, w in ((64, 1), (64, 2), (64, 3), (64, 4), (32, 4))]
    res = PH.relax(fl, runs, t_end=2.0, sample_dt=0.02)
    curves = {}
    for (prec, w), r in zip(((64, 1), (64, 2), (64, 3), (64, 4), (32, 4)), res):
        t = [s[0] for s in r["samples"]]
        e = np.array([s[2]["eT"] for s in r["samples"]])
        m = np.array([s[2]["mass"] for s in r["samples"]])
        curves["fp%d_k%d" % (prec, w)] = dict(t=t, dEt=(e - e[0]).tolist(), eT0=float(e[0]),
                                               mass_drift=float(np.abs(m - m[0]).max() / m[0]), finite=r["finite"])
        print("fp%d k%d: e_T(0) = %.6f, max |Delta e_T| = %.3e, |Delta e_T(2)| = %.3e, mass drift %.1e"
              % (prec, w, e[0], np.abs(e - e[0]).max(), abs(e[-1] - e[0]), curves["fp%d_k%d" % (prec, w)]["mass_drift"]))
    _dump("energy_drift", curves)
    assert all(c["finite"] for c in curves.values())
