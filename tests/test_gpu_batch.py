"""Batched sweep (fftlb_batch_*): every run of a mixed-shape batch against
the oracle, element by element; runs of uneven grids advanced together by
CUDA-graph replays give exactly the results of single handles; the
autotuner changes launch parameters but not results."""
import numpy as np
import pytest

from gpu_common import A49, B21, TC49, droplet_ragged, fp32_force_bound, lib, oracle_params, rel_err
from oracle import fftlb_oracle as O
from oracle import thermo as TH
from paper_1011_3582_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fl():
    return lib()


def slab_case(n, Tr, precision, seed):
    T = Tr * TC49
    rv, rl = TH.maxwell(T, A49, B21)
    fields = W.slab(n, n, rv, rl, T, width=2.0, noise=1e-4, seed=seed)
    return fields, dict(nx=n, ny=n, a=A49, b=B21, precision=precision, integrator=3)


def spinodal_case(n, Tr, precision, seed):
    fields = W.spinodal(n, n, 1 / (3 * B21), Tr * TC49, amp=0.01, seed=seed)
    return fields, dict(nx=n, ny=n, a=A49, b=B21, precision=precision, integrator=3)


def wide_case(nx, ny, Tr, seed):
    fields = W.spinodal(nx, ny, 1 / (3 * B21), Tr * TC49, amp=0.01, seed=seed)
    return fields, dict(nx=nx, ny=ny, a=A49, b=B21, precision=32, integrator=3)


def test_batch_matches_single_handles(fl):
    cases = [slab_case(64, 0.9, 64, 1), slab_case(48, 0.8, 64, 2), slab_case(128, 0.95, 32, 3),
             slab_case(96, 0.75, 32, 4), spinodal_case(256, 0.8, 32, 5), spinodal_case(384, 0.9, 32, 6),
             slab_case(128, 0.85, 32, 7), spinodal_case(256, 0.8, 32 | fl.BF16SPLIT, 8),
             slab_case(128, 0.85, 32 | fl.BF16SPLIT, 9)]
    with fl.Batch([fl.params(**kw) for _, kw in cases], autotune=True) as b:
        for r, (fields, _) in enumerate(cases):
            b.set_fields(r, *fields)
        b.step(7)
        got = [b.get_f(r) for r in range(len(cases))]
        inv = [b.invariants(r) for r in range(len(cases))]
        tun = [b.tuning(r) for r in range(len(cases))]
    for r, (fields, kw) in enumerate(cases):
        with fl.Handle(fl.params(**kw)) as h:
            h.tuning(tun[r])            # same launch parameters
            h.set_fields(*fields)
            h.step(7)
            want = h.get_f()
        assert np.array_equal(got[r], want), r
        assert inv[r]["time"] == pytest.approx(7e-5)


@pytest.mark.parametrize("integrator", [3, 1])
def test_autotune_keeps_results_and_state(fl, integrator):
    """For SSP-RK3 the candidates write the stage buffer, for Euler a
    temporary one: the state is never touched."""
    fields, kw = slab_case(64, 0.9, 32, 5)
    kw = dict(kw, integrator=integrator)
    with fl.Handle(fl.params(**kw)) as h:
        h.set_fields(*fields)
        f0 = h.get_f()
        ms = h.autotune()
        assert ms > 0
        assert np.array_equal(h.get_f(), f0)        # state restored
        h.step(5)
        f_tuned = h.get_f()
        tun = h.tuning()
    with fl.Handle(fl.params(**kw)) as h:
        h.set_fields(*fields)
        h.step(5)
        f_default = h.get_f()
    # tile widths / chunking reorder independent work only
    assert rel_err(f_tuned, f_default) < 1e-6, tun


def test_batch_rejects_bad_arguments(fl):
    with pytest.raises(fl.FFTLBError):
        fl.Batch([])
    with pytest.raises(fl.FFTLBError):
        fl.Batch([fl.params(nx=10, ny=16)])


def test_batch_of_euler_runs_matches_single_handles(fl):
    """Two Euler runs of one grid share one batched engine (no RK stage
    buffer; autotune times into a temporary buffer)."""
    cases = [slab_case(64, 0.9, 64, 8), slab_case(64, 0.8, 64, 9)]
    for _, kw in cases:
        kw["integrator"] = 1
    with fl.Batch([fl.params(**kw) for _, kw in cases], autotune=True) as b:
        for r, (fields, _) in enumerate(cases):
            b.set_fields(r, *fields)
        b.step(5)
        got = [b.get_f(r) for r in range(2)]
        tun = [b.tuning(r) for r in range(2)]
    for r, (fields, kw) in enumerate(cases):
        with fl.Handle(fl.params(**kw)) as h:
            h.tuning(tun[r])
            h.set_fields(*fields)
            h.step(5)
            assert np.array_equal(got[r], h.get_f()), r


def test_batch_runs_match_oracle(fl):
    """A batch of uneven grids and both precisions, autotuned per group,
    compared run by run with the FP64 oracle after 3 SSP-RK3 steps: two
    64^2 slabs at different temperatures share one group (one launch over
    both runs), a 48 x 96 droplet has radix-3 axes, and two 128^2 spinodal
    quenches share an fp32 group beside a 96^2 fp32 slab and two 32 x 512
    quenches and two 256 x 32 quenches (the warp-resident row and column
    kernels over two runs), and two 4 x 512 quenches, whose 4-row columns
    the autotuner tries at tile widths with sub-128-byte tiles.  FP64 runs: the
    1e-9 bar; FP32 runs: fp32_force_bound elementwise."""
    nsteps = 3
    drop_fields, drop_kw = droplet_ragged()
    cases = [slab_case(64, 0.9, 64, 21), slab_case(64, 0.8, 64, 22),
             (drop_fields, dict(drop_kw, precision=64, integrator=3)),
             spinodal_case(128, 0.8, 32, 23), spinodal_case(128, 0.75, 32, 24), slab_case(96, 0.85, 32, 25),
             wide_case(512, 32, 0.8, 26), wide_case(512, 32, 0.85, 27), wide_case(32, 256, 0.8, 28),
             wide_case(32, 256, 0.9, 29), wide_case(512, 4, 0.85, 30), wide_case(512, 4, 0.9, 31)]
    with fl.Batch([fl.params(**kw) for _, kw in cases], autotune=True) as b:
        for r, (fields, _) in enumerate(cases):
            b.set_fields(r, *fields)
        b.step(nsteps)
        got = [b.get_f(r) for r in range(len(cases))]
    for r, (fields, kw) in enumerate(cases):
        p = oracle_params(kw)
        f_o = O.run(O.init_equilibrium(*fields, p), p, nsteps)
        if kw["precision"] == 64:
            assert rel_err(got[r], f_o) < 1e-9, r
        else:
            n = (kw["ny"], kw["nx"])
            bound = fp32_force_bound(n, nsteps, fields[0], fields[3])
            err = (np.abs(got[r] - f_o) / np.abs(f_o)).max()
            print("batch run %d fp32 vs oracle: %.2e (bound %.2e)" % (r, err, bound))
            assert err < bound, r
