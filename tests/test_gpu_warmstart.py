"""The warm-start network's CUDA kernels (BF16 tensor-core convolutions,
FP32 accumulation) against the CPU oracle that applies the same bfloat16
roundings: forward output, parameter gradient, Adam step, training, and the
warm start applied to an FFT-LB handle.

Tolerances: the oracle sums in fp64 and the GPU in fp32 (288 products per
output), a relative difference ~1e-6 before any rounding.  Where that
difference straddles a bfloat16 rounding point, the stored activation (or
gradient) differs by one bfloat16 unit (2^-8 relative) on the two sides;
such flips are rare (probability ~ 1e-6 / 2^-8 per value) and each moves
downstream values by at most about one unit of their own, so the bound is
a few bfloat16 units on the maximum and far less on the mean."""
import numpy as np
import pytest

from gpu_common import A49, B21, TC49, lib
from oracle import cnn_oracle as C
from paper_1011_3582_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U = 2.0 ** -8   # bfloat16 unit roundoff scale


@pytest.fixture(scope="module")
def fl():
    return lib()


def case(seed, H=32, Wd=64, scale=1.0):
    rng = np.random.default_rng(seed)
    params = C.init_params(seed, scale=scale)
    params = [(Wl, rng.standard_normal(Wl.shape[0]) * 0.1) for Wl, _ in params]
    X = rng.standard_normal((3, H, Wd)).astype(np.float32)
    Xt = (X[:2] + 0.5 * rng.standard_normal((2, H, Wd))).astype(np.float32)
    return params, X, Xt


def bf16_params(fl, params):
    """The fp32 parameter vector as the GPU receives it (float32)."""
    return fl.unpack_params(fl.pack_params(params).astype(np.float64))


@pytest.mark.parametrize("shape", [(32, 64), (7, 128), (64, 192)])
def test_forward_matches_oracle(fl, shape):
    H, Wd = shape
    params, X, _ = case(1, H, Wd)
    p32 = bf16_params(fl, params)
    with fl.CNN(H, Wd) as net:
        net.set_params(fl.pack_params(params))
        Y = net.forward(X)
    Yr, _ = C.forward(p32, X, bf16=True)
    scale = np.abs(Yr).max()
    err = np.abs(Y - Yr)
    print(f"forward {shape}: max {err.max() / scale:.2e}, mean {err.mean() / scale:.2e} (of max |Y|)")
    assert err.max() <= 4 * U * scale
    assert err.mean() <= 0.05 * U * scale


def test_gradient_matches_oracle(fl):
    params, X, Xt = case(2)
    p32 = bf16_params(fl, params)
    with fl.CNN(32, 64) as net:
        net.set_params(fl.pack_params(params))
        loss, g = net.gradient(X, Xt)
    L_ref, grads = C.loss_and_grads(p32, X, Xt, bf16=True)
    g_ref = fl.pack_params(grads).astype(np.float64)
    assert loss == pytest.approx(L_ref, rel=1e-5)
    o = 0
    for (Wl, bl) in grads:
        for arr in (Wl, bl):
            n = arr.size
            a, b = g[o:o + n].astype(np.float64), g_ref[o:o + n]
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            print(f"gradient block of {n}: relative L2 difference {rel:.2e}")
            assert rel <= 2 * U
            o += n


def test_adam_step_matches_oracle(fl):
    params, X, Xt = case(3)
    with fl.CNN(32, 64) as net:
        net.set_params(fl.pack_params(params))
        _, g = net.gradient(X, Xt)
        before = net.get_params().astype(np.float64)
        net.train_step(X, Xt, lr=1e-3)
        after = net.get_params().astype(np.float64)
    st = {}
    want = fl.pack_params(C.adam_step(fl.unpack_params(before), fl.unpack_params(g.astype(np.float64)), st, 1e-3))
    # first step: every parameter moves by lr g / (|g| + eps); fp32 arithmetic
    assert np.abs(after - want.astype(np.float64)).max() <= 1e-6


def test_training_reduces_the_loss(fl):
    """A learnable target (a fixed 3x3 smoothing of the input) is fitted by
    the GPU training loop: the loss falls by more than 10x in 300 steps."""
    rng = np.random.default_rng(4)
    H, Wd = 32, 64
    with fl.CNN(H, Wd) as net:
        net.set_params(fl.pack_params(C.init_params(5)))
        losses = []
        for it in range(300):
            X = rng.standard_normal((3, H, Wd)).astype(np.float32)
            sm = sum(np.roll(X[:2], (dy, dx), axis=(1, 2)) for dy in (-1, 0, 1) for dx in (-1, 0, 1)) / 9.0
            Xt = (X[:2] + 0.5 * (sm - X[:2])).astype(np.float32)
            losses.append(net.train_step(X, Xt, lr=3e-3))
    print("loss", losses[0], "->", np.mean(losses[-20:]))
    assert np.mean(losses[-20:]) < 0.1 * losses[0]


def test_warm_start_sets_the_decoded_state(fl):
    """fftlb_cnn_warm_start = encode (fields of the handle) -> network ->
    decode -> f = f^eq(rho', 0, T')."""
    n = 64
    rho_c, Tc = 1 / (3 * B21), TC49
    T_run = 0.75 * Tc
    fields = W.spinodal(n, n, rho_c, T_run, amp=0.01, seed=9)
    params, _, _ = case(6, scale=0.3)
    p32 = bf16_params(fl, params)
    norm = fl.fftlb_cnn_norm(rho_c, Tc, 50.0, 50.0)
    with fl.Handle(fl.params(nx=n, ny=n, a=A49, b=B21, precision=64)) as h, fl.CNN(n, n) as net:
        net.set_params(fl.pack_params(params))
        h.set_fields(*fields)
        h.step(3)
        r0, _, _, T0 = h.fields()
        net.warm_start(h, T_run, norm)
        r1, ux, uy, T1 = h.fields()
        assert h.invariants()["time"] == pytest.approx(3e-5)
    X = C.encode(r0, T0, T_run, rho_c, Tc).astype(np.float32)
    Y, _ = C.forward(p32, X, bf16=True)
    rr, Tr = C.decode(X.astype(np.float64), Y, T_run, rho_c)
    assert np.abs(ux).max() < 1e-14 and np.abs(uy).max() < 1e-14
    # one-unit bfloat16 flips move Y by < 4 U max|Y|; rho' = rho_c (1 + .../50)
    assert np.abs(r1 - rr).max() <= rho_c * 4 * U * np.abs(Y).max() / 50 + 1e-12
    assert np.abs(T1 - Tr).max() <= T_run * 4 * U * np.abs(Y).max() / 50 + 1e-12


def test_rejects_bad_grids(fl):
    for H, Wd in ((0, 64), (16, 48), (16, 8192)):
        with pytest.raises(fl.FFTLBError) as ei:
            fl.CNN(H, Wd)
        assert ei.value.status == fl.ERR_ARG


def test_trained_warm_start_shortens_time_to_onset(fl):
    """The committed parameters (trained by paper_1011_3582_gb300.warmstart on
    512^2 snapshots at T_r = 0.6, 0.65, 0.7, 0.75) on an unseen seed and
    temperature at 256^2: the warm-started run reaches the onset contrast
    (std(rho) / rho_c >= 0.2) in fewer than 0.7 times the plain run's steps,
    and both runs end phase-separated."""
    import os
    from paper_1011_3582_gb300 import warmstart as WS
    params = np.load(os.path.join(os.path.dirname(fl.__file__), "warmstart_params.npy"))
    with fl.CNN(256, 256) as net:
        net.set_params(params)
        r = WS.compare(fl, net, 256, 0.65, 23, max_steps=80000)
    print(r)
    assert r["cold_steps"] is not None and r["warm_steps"] is not None
    assert r["warm_steps"] <= 0.7 * r["cold_steps"]
