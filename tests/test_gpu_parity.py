"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
paper-shaped workloads.  Bar: FP64 path within 1e-9 relative per field after
100 steps; FP32 path within bounds derived in each test from the fp32
rounding of the state and of the transforms."""
import functools

import numpy as np
import pytest

from gpu_common import (A49, B21, TC49, RHOC49, droplet_ragged, fp32_force_bound, gpu_run, lib, oracle_params,
                        oracle_run, rel_err, slab64)
from oracle import fftlb_oracle as O
from paper_1011_3582_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fl():
    return lib()


def test_set_fields_builds_equilibrium(fl):
    fields, kw = slab64()
    p = fl.params(precision=64, **kw)
    with fl.Handle(p) as h:
        h.set_fields(*fields)
        f = h.get_f()
        r, ux, uy, T = h.fields()
    fo = O.feq(*fields)
    assert rel_err(f, fo) < 1e-14
    assert rel_err(r, fields[0]) < 1e-14 and rel_err(T, fields[3]) < 1e-14
    assert np.abs(ux).max() < 1e-14 and np.abs(uy).max() < 1e-14


@pytest.mark.parametrize("integrator", [1, 3])
def test_slab64_fp64_100_steps(fl, integrator):
    f_o, (r_o, ux_o, uy_o, T_o), inv_o = oracle_run("slab64", 100, integrator)
    f_g, (r_g, ux_g, uy_g, T_g), inv_g = gpu_run(fl, "slab64", 100, integrator, 64)
    assert rel_err(r_g, r_o) < 1e-9
    assert rel_err(ux_g, ux_o) < 1e-9
    assert rel_err(uy_g, uy_o) < 1e-9
    assert rel_err(T_g, T_o) < 1e-9
    assert rel_err(f_g, f_o) < 1e-9
    assert inv_g["mass"] == pytest.approx(inv_o["mass"], rel=1e-12)
    assert inv_g["eT"] == pytest.approx(inv_o["eT"], rel=1e-9)
    assert inv_g["umax"] == pytest.approx(inv_o["umax"], rel=1e-9)


def test_slab64_fp32_100_steps(fl):
    """FP32 state and transforms.  Bound: every one of the S = 300 stage
    updates rounds f to fp32 (unit roundoff u = 2^-24); with small,
    correlated increments these roundings add up, so |drho|/rho, |dT|/T
    <= S u / 2 ~ 1e-5.  Velocities are differences of O(rho |v|) sums, so
    their absolute error is <= S u <|v|> ~ 3e-5, i.e. < 5e-3 of max |u|
    (~ 8e-3 here), measured component-wise against max |u|."""
    S, u = 300, 2.0 ** -24
    f_o, (r_o, ux_o, uy_o, T_o), inv_o = oracle_run("slab64", 100, 3)
    f_g, (r_g, ux_g, uy_g, T_g), inv_g = gpu_run(fl, "slab64", 100, 3, 32)
    umax = np.hypot(ux_o, uy_o).max()
    errs = dict(rho=rel_err(r_g, r_o), T=rel_err(T_g, T_o),
                u=max(np.abs(ux_g - ux_o).max(), np.abs(uy_g - uy_o).max()) / umax,
                mass=abs(inv_g["mass"] - inv_o["mass"]) / inv_o["mass"])
    print("fp32 vs fp64 oracle after 100 RK3 steps:", errs)
    assert errs["rho"] < S * u / 2 and errs["T"] < S * u / 2
    assert errs["u"] < 5e-3
    assert errs["mass"] < S * u / 2


@pytest.mark.parametrize("window", [0, 1, 2, 3])
def test_windows_fp64(fl, window):
    f_o, mo, _ = oracle_run("slab64", 10, 1, window)
    f_g, mg, _ = gpu_run(fl, "slab64", 10, 1, 64, window)
    for a, b in zip(mg, mo):
        assert rel_err(a, b) < 1e-10


def test_ragged_radix3_grid_fp64(fl):
    f_o, mo, inv_o = oracle_run("droplet_ragged", 20, 3)
    f_g, mg, inv_g = gpu_run(fl, "droplet_ragged", 20, 3, 64)
    for a, b in zip(mg, mo):
        assert rel_err(a, b) < 1e-10
    assert rel_err(f_g, f_o) < 1e-10


@pytest.mark.parametrize("shape", [(4, 4), (8, 4), (4, 12), (6, 8)])
def test_tiny_grids(fl, shape):
    ny, nx = shape
    fields = W.smooth_random(nx, ny, seed=11, rho0=1.2, T0=0.9, amp=0.05, umax=0.02)
    kw = dict(nx=nx, ny=ny, dx=1 / 64, K=1e-4)
    p = oracle_params(kw, integrator=3)
    f_o = O.run(O.init_equilibrium(*fields, p), p, 5)
    with fl.Handle(fl.params(precision=64, integrator=3, **kw)) as h:
        h.set_fields(*fields)
        h.step(5)
        f_g = h.get_f()
    assert rel_err(f_g, f_o) < 1e-12


def test_conservation_and_invariants_fp64(fl):
    fields, kw = slab64()
    with fl.Handle(fl.params(precision=64, integrator=3, **kw)) as h:
        h.set_fields(*fields)
        i0 = h.invariants()
        h.step(50)
        i1 = h.invariants()
    assert abs(i1["mass"] - i0["mass"]) < 1e-13 * i0["mass"]
    assert abs(i1["px"]) < 1e-14 * i0["mass"] and abs(i1["py"]) < 1e-14 * i0["mass"]
    assert i1["time"] == pytest.approx(50 * 1e-5)


def test_checkpoint_resume_is_bit_identical(fl, tmp_path):
    fields, kw = slab64()
    p = fl.params(precision=64, integrator=3, **kw)
    path = str(tmp_path / "ckpt.bin")
    with fl.Handle(p) as h:
        h.set_fields(*fields)
        h.step(5)
        h.save(path)
        h.step(5)
        f_a = h.get_f()
    with fl.Handle(p) as h2:
        h2.load(path)
        assert h2.invariants()["time"] == pytest.approx(5e-5)
        h2.step(5)
        f_b = h2.get_f()
    assert np.array_equal(f_a, f_b)


def test_unstable_state_is_reported_not_trapped(fl):
    """Host-side failure detection: an unphysical initial temperature is
    reported as ERR_UNSTABLE with the step count."""
    fields, kw = slab64()
    rho, ux, uy, T = (x.copy() for x in fields)
    T[5, 7] = -0.3
    with fl.Handle(fl.params(precision=64, integrator=1, check_every=1, **kw)) as h:
        h.set_fields(rho, ux, uy, T)
        with pytest.raises(fl.FFTLBError) as ei:
            h.step(3)
        assert ei.value.status == fl.ERR_UNSTABLE
        assert ei.value.steps_done == 1


@pytest.mark.parametrize("extra", [dict(zeta=2e-3), dict(H=5e-5), dict(zeta=1e-3, H=-3e-5, q=0.0)])
def test_bulk_viscosity_and_temperature_dependent_M_fp64(fl, extra):
    """zeta (the bulk-viscosity terms of Eqs. 21-22) and H (M = K + H T in
    Eq. 19, which brings in the -rho T d rho . d(M/T) term) off their zero
    defaults, on smooth non-uniform rho, u and T: fp64 against the oracle
    after 10 RK3 steps, 1e-9."""
    n = 32
    fields = W.smooth_random(n, n, seed=17, rho0=1.2, T0=0.9, amp=0.05, umax=0.02)
    kw = dict(nx=n, ny=n, dx=1 / 64, K=1e-4, **extra)
    p = oracle_params(kw, integrator=3)
    f_o = O.run(O.init_equilibrium(*fields, p), p, 10)
    with fl.Handle(fl.params(precision=64, integrator=3, **kw)) as h:
        h.set_fields(*fields)
        h.step(10)
        f_g = h.get_f()
    assert rel_err(f_g, f_o) < 1e-9


# a velocity set other than the paper's (1, 1.9, 2.9, 4.3)
SPEEDS_B = (1.0, 2.0, 3.0, 4.5)


def test_custom_velocity_set_fp64(fl):
    """Speeds 1, 2, 3, 4.5 on the rings of Eq. 1: the weights (Eqs. 4-6), the
    equilibrium and every velocity-dependent term follow the speeds.  FP64
    against the oracle run with the same set, 20 RK3 steps, 1e-9."""
    fields, kw = slab64()
    p = oracle_params(kw, integrator=3, speeds=SPEEDS_B)
    f_o = O.run(O.init_equilibrium(*fields, p), p, 20)
    with fl.Handle(fl.params(precision=64, integrator=3, **kw), speeds=SPEEDS_B) as h:
        h.set_fields(*fields)
        h.step(20)
        f_g = h.get_f()
    assert rel_err(f_g, f_o) < 1e-9


def test_velocity_set_is_one_per_precision(fl):
    """The velocity set lives in constant memory shared by the handles of one
    precision: another set is refused while a handle of that precision is
    alive, accepted for the other precision and after the last one closed."""
    import gc
    gc.collect()
    kw = dict(nx=32, ny=32)
    with fl.Handle(fl.params(precision=64, **kw)):
        with pytest.raises(fl.FFTLBError) as ei:
            fl.Handle(fl.params(precision=64, **kw), speeds=SPEEDS_B)
        assert ei.value.status == fl.ERR_ARG
        with fl.Handle(fl.params(precision=32, **kw), speeds=SPEEDS_B):
            pass
        with fl.Handle(fl.params(precision=64, **kw)):
            pass
    with fl.Handle(fl.params(precision=64, **kw), speeds=SPEEDS_B):
        pass


@functools.lru_cache(maxsize=None)
def _spinodal_oracle(n, nsteps):
    kw = dict(nx=n, ny=n, a=A49, b=B21)
    fields = W.spinodal(n, n, RHOC49, 0.8 * TC49, amp=0.01, seed=n)
    p = oracle_params(kw, integrator=3)
    f = O.run(O.init_equilibrium(*fields, p), p, nsteps)
    return fields, kw, f


@pytest.mark.parametrize("n,nsteps", [(256, 3), (384, 3), (512, 1)])
@pytest.mark.parametrize("precision", [64, 32])
def test_spinodal_sweep_grids(fl, n, nsteps, precision):
    """The grid sizes of the batched sweep (radix-2 and radix-3 lengths,
    several column tiles and row chunks per block) on a spinodal quench at
    T = 0.8 T_c, compared element by element with the oracle.  FP64: the
    1e-9 bar.  FP32: fp32_force_bound."""
    fields, kw, f_o = _spinodal_oracle(n, nsteps)
    with fl.Handle(fl.params(integrator=3, precision=precision, **kw)) as h:
        h.set_fields(*fields)
        h.step(nsteps)
        f_g = h.get_f()
    if precision == 64:
        assert rel_err(f_g, f_o) < 1e-9
    else:
        bound = fp32_force_bound(n, nsteps, fields[0], fields[3])
        err = (np.abs(f_g - f_o) / np.abs(f_o)).max()
        print(f"fp32 {n}^2 after {nsteps} RK3 steps: max |df|/f = {err:.3e} (bound {bound:.3e})")
        assert err < bound


# one split-BF16 first pass: |x - x_hi - x_lo| <= 2^-16 |x| for each operand
# (x_hi = bf16(x), x_lo = bf16(x - x_hi), nearest even) and the dropped
# W_lo x_lo <= 2^-16 |W| |x|
U_SPLIT = 3 * 2.0 ** -16


@pytest.mark.parametrize("n,nsteps", [(256, 3), (512, 1)])
def test_bf16split_spinodal(fl, n, nsteps):
    """precision 32 | BF16SPLIT: the first radix-16 pass of every power-of-two
    row and column transform is the split-BF16 DFT product on the tensor
    cores.  Element by element against the oracle within fp32_force_bound
    with that pass's rounding, and visibly apart from the plain fp32 path
    (the tensor-core pass ran: its 2^-16 rounding shows in f)."""
    fields, kw, f_o = _spinodal_oracle(n, nsteps)
    out = {}
    for prec in (32, 32 | fl.BF16SPLIT):
        with fl.Handle(fl.params(integrator=3, precision=prec, **kw)) as h:
            h.set_fields(*fields)
            h.step(nsteps)
            out[prec] = h.get_f()
    e32 = (np.abs(out[32] - f_o) / np.abs(f_o)).max()
    es = (np.abs(out[32 | fl.BF16SPLIT] - f_o) / np.abs(f_o)).max()
    bound = fp32_force_bound(n, nsteps, fields[0], fields[3], u_split=U_SPLIT)
    print(f"{n}^2, {nsteps} RK3 steps: max |df|/f fp32 {e32:.3e}, split-BF16 {es:.3e} (bound {bound:.3e})")
    assert es < bound
    assert es > e32


def test_bf16split_leaves_other_lengths_unchanged(fl):
    """384 = 3 * 2^7 takes the mixed-radix passes in rows and columns, where
    the split mode changes nothing: identical to the fp32 path bit for bit."""
    fields, kw, _ = _spinodal_oracle(384, 3)
    out = []
    for prec in (32, 32 | fl.BF16SPLIT):
        with fl.Handle(fl.params(integrator=3, precision=prec, **kw)) as h:
            h.set_fields(*fields)
            h.step(1)
            out.append(h.get_f())
    assert np.array_equal(out[0], out[1])


def test_torch_cufft_reference_matches_oracle():
    """The PyTorch/cuFFT step that bench.py times beside the CUDA kernels
    computes the same method: fp32, same bound as the CUDA fp32 path."""
    import torch
    from paper_1011_3582_gb300 import torch_reference as TR
    fields, kw, f_o = _spinodal_oracle(256, 3)
    ts = TR.TorchStep(256, 256, a=A49, b=B21, integrator=3)
    ts.set_fields(*fields)
    ts.step(3)
    f_t = ts.f.double().cpu().numpy()
    bound = fp32_force_bound(256, 3, fields[0], fields[3])
    err = (np.abs(f_t - f_o) / np.abs(f_o)).max()
    print(f"torch/cuFFT fp32 256^2 after 3 RK3 steps: max |df|/f = {err:.3e} (bound {bound:.3e})")
    assert err < bound


@functools.lru_cache(maxsize=None)
def _droplet512_oracle():
    from oracle import thermo as TH
    n, T = 512, 0.8 * TC49
    rv, rl = TH.maxwell(T, A49, B21)
    kw = dict(nx=n, ny=n, a=A49, b=B21)
    fields = W.droplet(n, n, 80, rl, rv, T, width=2.0)
    p = oracle_params(kw, integrator=3)
    return fields, kw, O.run(O.init_equilibrium(*fields, p), p, 1)


@functools.lru_cache(maxsize=None)
def _bench_workload_oracle():
    """One SSP-RK3 step of the benchmark workload at full size: 1024^2
    spinodal quench, rho = rho_c (1 + 0.01 N(0, 1)) seed 7, u = 0,
    T = 0.7 T_c, a = 9/49, b = 2/21, window k4 (about 15 s of numpy)."""
    n = 1024
    fields = W.spinodal(n, n, RHOC49, 0.7 * TC49, amp=0.01, seed=7)
    kw = dict(nx=n, ny=n, a=A49, b=B21, window=4)
    p = oracle_params(kw, integrator=3)
    return fields, kw, O.run(O.init_equilibrium(*fields, p), p, 1)


@pytest.mark.parametrize("precision", [32, 64, 32 | 256])   # 256: FFTLB_BF16SPLIT
def test_bench_workload_1024_full_size(fl, precision):
    """The benchmarked configuration itself: 1024^2, the launch parameters
    chosen by fftlb_autotune (as bench.py times it), one SSP-RK3 step,
    every element of f against the oracle: fp64 within 1e-9, fp32 (and the
    split-BF16 first passes) within fp32_force_bound."""
    fields, kw, f_o = _bench_workload_oracle()
    with fl.Handle(fl.params(integrator=3, precision=precision, **kw)) as h:
        h.set_fields(*fields)
        h.autotune()
        h.step(1)
        f_g = h.get_f()
    if precision == 64:
        assert rel_err(f_g, f_o) < 1e-9
    else:
        split = precision & fl.BF16SPLIT
        bound = fp32_force_bound(1024, 1, fields[0], fields[3], u_split=U_SPLIT if split else 0.0)
        err = (np.abs(f_g - f_o) / np.abs(f_o)).max()
        print(f"{'split-BF16' if split else 'fp32'} 1024^2 bench workload, 1 RK3 step: max |df|/f = {err:.3e} "
              f"(bound {bound:.3e})")
        assert err < bound


def test_max_size_2048_fp32_properties(fl):
    """The largest fp32 grid (2048^2: eight sites per thread in the row
    kernels), one SSP-RK3 step with autotuned launch parameters, checked by
    properties that hold at any size: translation equivariance (a field
    shifted by (37, 1001) sites steps to the shifted result, within twice
    fp32_force_bound since both runs round independently) and conservation
    of mass (to fp32 rounding of the state)."""
    n = 2048
    fields = W.spinodal(n, n, RHOC49, 0.8 * TC49, amp=0.01, seed=5)
    kw = dict(nx=n, ny=n, a=A49, b=B21)
    shift = (37, 1001)
    out = []
    for fl_in in (fields, tuple(np.roll(x, shift, axis=(0, 1)) for x in fields)):
        with fl.Handle(fl.params(integrator=3, precision=32, **kw)) as h:
            h.set_fields(*fl_in)
            h.autotune()
            m0 = h.invariants()["mass"]
            h.step(1)
            out.append(h.get_f())
            m1 = h.invariants()["mass"]
        assert abs(m1 - m0) < 1e-6 * m0
    f_a = np.roll(out[0], shift, axis=(1, 2))
    err = (np.abs(out[1] - f_a) / np.abs(f_a)).max()
    bound = 2 * fp32_force_bound(n, 1, fields[0], fields[3])
    print(f"fp32 2048^2 shifted vs unshifted after 1 RK3 step: max |df|/f = {err:.3e} (bound {bound:.3e})")
    assert err < bound


@pytest.mark.parametrize("precision", [64, 32, 32 | 256])   # 256: FFTLB_BF16SPLIT
def test_droplet_512_precision_config(fl, precision):
    """The precision configuration's droplet (512^2, R = 80, Maxwell
    densities at T = 0.8 T_c, tanh width 2), one SSP-RK3 step, element by
    element against the oracle: fp64 within 1e-9, fp32 within
    fp32_force_bound, fp32 with the split-BF16 first passes within the same
    bound with their rounding."""
    fields, kw, f_o = _droplet512_oracle()
    with fl.Handle(fl.params(integrator=3, precision=precision, **kw)) as h:
        h.set_fields(*fields)
        h.step(1)
        f_g = h.get_f()
    if precision == 64:
        assert rel_err(f_g, f_o) < 1e-9
    else:
        split = precision & fl.BF16SPLIT
        bound = fp32_force_bound(512, 1, fields[0], fields[3], u_split=U_SPLIT if split else 0.0)
        err = (np.abs(f_g - f_o) / np.abs(f_o)).max()
        name = "split-BF16" if split else "fp32"
        print(f"{name} 512^2 droplet after 1 RK3 step: max |df|/f = {err:.3e} (bound {bound:.3e})")
        assert err < bound


@pytest.mark.parametrize("nx,ny", [(1024, 32), (512, 48), (512, 16), (1024, 96), (16, 1024), (32, 512), (64, 256),
                                   (48, 1024), (96, 512), (256, 16), (256, 48), (16, 128), (48, 128)])
def test_wide_rows_fp32(fl, nx, ny):
    """Row widths nx = 256, 512 and 1024 and column lengths ny = 128, 256,
    512 and 1024, where the fp32 path runs its warp-resident row and column
    kernels, on narrow grids (the other axis 16 to 96, the radix-3 lengths
    48 and 96 included) against the oracle after 3 SSP-RK3 steps of a
    spinodal quench at T = 0.8 T_c, element by element within
    fp32_force_bound."""
    kw = dict(nx=nx, ny=ny, a=A49, b=B21)
    fields = W.spinodal(nx, ny, RHOC49, 0.8 * TC49, amp=0.01, seed=nx + ny)
    p = oracle_params(kw, integrator=3)
    f_o = O.run(O.init_equilibrium(*fields, p), p, 3)
    with fl.Handle(fl.params(integrator=3, precision=32, **kw)) as h:
        h.set_fields(*fields)
        h.step(3)
        f_g = h.get_f()
    bound = fp32_force_bound((ny, nx), 3, fields[0], fields[3])
    err = (np.abs(f_g - f_o) / np.abs(f_o)).max()
    print("fp32 %dx%d vs oracle: %.2e (bound %.2e)" % (ny, nx, err, bound))
    assert err < bound
