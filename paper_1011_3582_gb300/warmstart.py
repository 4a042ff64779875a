"""Learned warm start of FFT-LB spinodal quenches (arXiv:1011.3582, Sec. 4):
snapshot generation with the method itself, training of the network on
the GPU (fftlb_cnn_* kernels), and the time-to-onset comparison of warm- and
cold-started runs.

Protocol (every number here is a choice of this project, stated once):
  run        fp32 FFT-LB on an n x n grid, a = 9/49, b = 2/21 (T_c = 4/7,
             rho_c = 3.5), paper defaults otherwise, SSP-RK3; initial state
             rho_c (1 + 0.01 N(0, 1)) at rest at T_r T_c (workloads.spinodal)
  contrast   c(t) = std(rho) / rho_c over the grid
  input      the state at step T_IN = 500
  target     the state at the first multiple of 1000 steps where c >= C_TGT
             (0.05, mid linear growth)
  onset      the first multiple of 1000 steps where c >= C_ONSET (0.2: the
             two phases have formed); time-to-onset is the comparison
  warm run   step T_IN, then fftlb_cnn_warm_start (f = f^eq of the network's
             rho', T' at rest), then plain steps to onset
The warm run's cost counts the network inference and its steps from T_IN;
the cold run's counts its steps from T_IN.
"""
import json
import time

import numpy as np

A, B = 9.0 / 49.0, 2.0 / 21.0
TC, RHOC = 8.0 * A / (27.0 * B), 1.0 / (3.0 * B)
T_IN, C_TGT, C_ONSET, CHECK = 500, 0.05, 0.2, 1000


def init_params(seed):
    """Seeded He-normal weights (the last layer at a tenth of that scale) and
    zero biases, as the flat fp32 parameter vector of the C ABI."""
    rng = np.random.default_rng(seed)
    parts = []
    for l, (ci, co) in enumerate(((3, 32), (32, 32), (32, 32), (32, 2))):
        std = np.sqrt(2.0 / (9 * ci)) * (0.1 if l == 3 else 1.0)
        parts += [rng.standard_normal(co * 9 * ci) * std, np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)


def _contrast(h):
    r = h.fields()[0]
    return float(r.std() / RHOC)


def run_params(fl, n, precision=32):
    return fl.params(nx=n, ny=n, a=A, b=B, precision=precision, integrator=3)


def start(fl, h, n, Tr, seed):
    from paper_1011_3582_gb300 import workloads as W
    h.set_fields(*W.spinodal(n, n, RHOC, Tr * TC, amp=0.01, seed=seed))
    h.step(T_IN)


def run_to(h, level, max_steps):
    """Plain steps, CHECK at a time, until the contrast reaches level;
    returns the steps taken (None if max_steps ran out)."""
    done = 0
    while done < max_steps:
        h.step(CHECK)
        done += CHECK
        if _contrast(h) >= level:
            return done
    return None


def norm(fl):
    return fl.fftlb_cnn_norm(RHOC, TC, 50.0, 50.0)


def generate(fl, net, n, temps, seeds, max_steps=200000, log=print):
    """[(X, Xt, Tr)] of device tensors: X [3][n][n] at T_IN and the target's
    first two channels, for every (Tr, seed)."""
    import torch
    data = []
    for Tr in temps:
        for seed in seeds:
            t0 = time.time()
            with fl.Handle(run_params(fl, n)) as h:
                start(fl, h, n, Tr, seed)
                X = torch.empty((3, n, n), dtype=torch.float32, device="cuda")
                net.encode(h, Tr * TC, norm(fl), X)
                steps = run_to(h, C_TGT, max_steps)
                if steps is None:
                    log(f"T_r = {Tr}: target contrast not reached in {max_steps} steps; skipped")
                    continue
                Xt = torch.empty((3, n, n), dtype=torch.float32, device="cuda")
                net.encode(h, Tr * TC, norm(fl), Xt)
                torch.cuda.synchronize()
            data.append((X, Xt[:2].contiguous(), Tr))
            log(json.dumps(dict(T_r=Tr, seed=seed, target_step=T_IN + steps, s=round(time.time() - t0, 1))))
    return data


def augment(X, Xt, k, flip):
    """A symmetry of the square periodic grid (rotation by k quarter turns,
    optional flip) applied to input and target alike.  The FFT-LB dynamics
    are invariant under these, so the pair stays a valid sample."""
    import torch
    X = torch.rot90(X, k, dims=(1, 2))
    Xt = torch.rot90(Xt, k, dims=(1, 2))
    if flip:
        X, Xt = torch.flip(X, dims=(2,)), torch.flip(Xt, dims=(2,))
    return X.contiguous(), Xt.contiguous()


def train(fl, net, data, steps=2000, lr=2e-3, seed=0, log=print):
    rng = np.random.default_rng(seed)
    hist = []
    for it in range(steps):
        X, Xt, _ = data[rng.integers(len(data))]
        Xa, Xta = augment(X, Xt, int(rng.integers(4)), bool(rng.integers(2)))
        lr_t = lr * (0.1 if it > 0.8 * steps else 1.0)
        loss = net.train_step(Xa, Xta, lr_t, on_device=True, want_loss=(it % 50 == 0 or it == steps - 1))
        if loss is not None:
            hist.append((it, loss))
            if it % 500 == 0 or it == steps - 1:
                log(json.dumps(dict(train_step=it, loss=loss)))
    return hist


def compare(fl, net, n, Tr, seed, max_steps=200000, cold_precision=32):
    """Cold and warm steps from T_IN to onset, and their wall times.  The
    warm run is the mixed path (fp32 method, bf16 network); the cold run
    uses the method in cold_precision (32 or 64)."""
    import torch
    out = dict(n=n, T_r=Tr, seed=seed, cold_precision=cold_precision)
    with fl.Handle(run_params(fl, n, cold_precision)) as h:
        start(fl, h, n, Tr, seed)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out["cold_steps"] = run_to(h, C_ONSET, max_steps)
        out["cold_s"] = time.perf_counter() - t0
    with fl.Handle(run_params(fl, n)) as h:
        start(fl, h, n, Tr, seed)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net.warm_start(h, Tr * TC, norm(fl))
        torch.cuda.synchronize()
        out["warm_start_s"] = time.perf_counter() - t0
        out["warm_contrast"] = _contrast(h)
        out["warm_steps"] = run_to(h, C_ONSET, max_steps)
        out["warm_s"] = time.perf_counter() - t0
    if out["cold_steps"] and out["warm_steps"]:
        out["step_ratio"] = out["cold_steps"] / out["warm_steps"]
        out["time_ratio"] = out["cold_s"] / out["warm_s"]
    return out


def main(argv=None):
    import argparse
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1011_3582_gb300 import fftlb as fl
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--temps", default="0.6,0.65,0.7,0.75")
    ap.add_argument("--seeds", default="11,12")
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--eval", default="512:0.6:21,512:0.7:22,512:0.675:23")
    ap.add_argument("--out", default="warmstart_out")
    ap.add_argument("--params", default=None, help="skip training: evaluate these parameters (.npy)")
    ap.add_argument("--cold-precision", type=int, default=32, choices=[32, 64])
    a = ap.parse_args(argv)
    os.makedirs(a.out, exist_ok=True)
    logf = open(os.path.join(a.out, "log.jsonl"), "w")

    def log(msg):
        print(msg, flush=True)
        logf.write(msg + "\n")
        logf.flush()

    if a.params:
        params = np.load(a.params)
    else:
        with fl.CNN(a.n, a.n) as net:
            net.set_params(init_params(0))
            data = generate(fl, net, a.n, [float(t) for t in a.temps.split(",")],
                            [int(s) for s in a.seeds.split(",")], log=log)
            t0 = time.time()
            train(fl, net, data, a.train_steps, a.lr, log=log)
            log(json.dumps(dict(train_s=round(time.time() - t0, 1))))
            params = net.get_params()
        np.save(os.path.join(a.out, "warmstart_params.npy"), params)
    results = []
    for spec in a.eval.split(","):
        n, Tr, seed = spec.split(":")
        n = int(n)
        with fl.CNN(n, n) as net:
            net.set_params(params)
            r = compare(fl, net, n, float(Tr), int(seed), cold_precision=a.cold_precision)
        results.append(r)
        log(json.dumps(r))
    json.dump(results, open(os.path.join(a.out, "results.json"), "w"), indent=1)


if __name__ == "__main__":
    main()
