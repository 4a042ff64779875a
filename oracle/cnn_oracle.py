"""CPU oracle of the learned warm start: a 4-layer 3x3 convolutional network
mapping an early-time (rho, T) field and the run temperature to a later
state of the same run, with its loss, gradients and Adam update.

TEST INFRASTRUCTURE ONLY.  Imported by tests/ and nothing else; the CUDA
path never calls it.  The network is not in the paper (arXiv:1011.3582):
it is the project's warm start for the FFT-LB runs of Sec. 4, so what it
computes is fixed here, in words, and every formula below is the plain
definition:

  input    X[0] = s_rho (rho / rho_c - 1),  X[1] = s_T (T / T_run - 1),
           X[2] = T_run / T_c - 0.75         (channels x H x W, periodic)
  layer l  Z_l[o, y, x] = b_l[o] + sum_{i, dy, dx} W_l[o, dy+1, dx+1, i]
                                   A_{l-1}[i, (y+dy) mod H, (x+dx) mod W]
           (cross-correlation, dy, dx in {-1, 0, 1}), A_l = max(Z_l, 0) for
           l = 1..3, A_0 = X; channels 3 -> 32 -> 32 -> 32 -> 2
  output   Y = Z_4, the predicted change of (X[0], X[1]):
           rho' = rho_c (1 + (X[0] + Y[0]) / s_rho),
           T'   = T_run (1 + (X[1] + Y[1]) / s_T)
  loss     L = mean over the 2 H W outputs of (Y - (X_target - X[0:2]))^2
           (X as given, before any rounding)
  Adam     m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
           w -= lr (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps)

Mixed precision (the points where the GPU path rounds to bfloat16, so that
a parity test can reproduce them exactly): W_l, A_0 and the stored A_l
(l = 1..3) are rounded to bfloat16 (round to nearest, ties to even) when
bf16=True; the sums are accumulated in float64 here (float32 on the GPU);
Y = Z_4 is not rounded.  In the backward pass the output gradients
G_l = dL/dZ_l are rounded to bfloat16 before they multiply W_l or A_{l-1};
bias gradients sum the rounded G_l.  With bf16=False everything is float64
(the finite-difference pins use that).

Pins (tests/test_oracle_cnn.py): the convolution against a brute-force
quadruple loop, shift equivariance on the periodic grid, zero weights give
Y = 0 (the state passes through), gradients of every parameter against
central finite differences in float64, the Adam step against its closed
form on a quadratic, and the bfloat16 rounding against the bit patterns of
chosen values.
"""
import numpy as np

LAYERS = ((3, 32), (32, 32), (32, 32), (32, 2))   # (in, out) channels


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as
    float32 (NaN and infinity are not expected here)."""
    x = np.asarray(a, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(x.shape)


def init_params(seed=0, scale=1.0):
    """He-normal weights W_l [out, 3, 3, in] and zero biases, seeded;
    the last layer starts at a tenth of that scale."""
    rng = np.random.default_rng(seed)
    params = []
    for l, (ci, co) in enumerate(LAYERS):
        std = scale * np.sqrt(2.0 / (9 * ci)) * (0.1 if l == len(LAYERS) - 1 else 1.0)
        params.append((rng.standard_normal((co, 3, 3, ci)) * std, np.zeros(co)))
    return params


def conv3x3(A, W, b):
    """Periodic 3x3 cross-correlation: A [ci, H, W], W [co, 3, 3, ci],
    b [co] -> Z [co, H, W] (float64), summed one tap at a time."""
    A = np.asarray(A, np.float64)
    Wt = np.asarray(W, np.float64)
    Z = np.zeros((Wt.shape[0],) + A.shape[1:]) + np.asarray(b, np.float64)[:, None, None]
    for ky in range(3):
        for kx in range(3):
            S = np.roll(A, shift=(-(ky - 1), -(kx - 1)), axis=(1, 2))   # S[i, y, x] = A[i, y+dy, x+dx]
            Z += np.einsum('oi,iyx->oyx', Wt[:, ky, kx, :], S)
    return Z


def conv3x3_transpose(G, W):
    """Adjoint of conv3x3 with respect to its input: dA[i, y, x] =
    sum_{o, dy, dx} W[o, dy+1, dx+1, i] G[o, y-dy, x-dx]."""
    G = np.asarray(G, np.float64)
    Wt = np.asarray(W, np.float64)
    dA = np.zeros((Wt.shape[3],) + G.shape[1:])
    for ky in range(3):
        for kx in range(3):
            S = np.roll(G, shift=(ky - 1, kx - 1), axis=(1, 2))          # S[o, y, x] = G[o, y-dy, x-dx]
            dA += np.einsum('oi,oyx->iyx', Wt[:, ky, kx, :], S)
    return dA


def conv3x3_wgrad(G, A):
    """Gradient of sum(G * conv3x3(A, W, b)) with respect to W:
    dW[o, dy+1, dx+1, i] = sum_{y, x} G[o, y, x] A[i, y+dy, x+dx]."""
    G = np.asarray(G, np.float64)
    A = np.asarray(A, np.float64)
    dW = np.zeros((G.shape[0], 3, 3, A.shape[0]))
    for ky in range(3):
        for kx in range(3):
            S = np.roll(A, shift=(-(ky - 1), -(kx - 1)), axis=(1, 2))
            dW[:, ky, kx, :] = np.einsum('oyx,iyx->oi', G, S)
    return dW


def _rw(W, bf16):
    return bf16_round(W).astype(np.float64) if bf16 else np.asarray(W, np.float64)


def forward(params, X, bf16=False):
    """Returns Y [2, H, W] and the cache of stored activations A_0..A_3."""
    A = bf16_round(X).astype(np.float64) if bf16 else np.asarray(X, np.float64)
    acts = [A]
    for l, (W, b) in enumerate(params):
        Z = conv3x3(A, _rw(W, bf16), b)
        if l == len(params) - 1:
            return Z, acts
        A = np.maximum(Z, 0.0)
        if bf16:
            A = bf16_round(A).astype(np.float64)
        acts.append(A)
    raise AssertionError


def loss_and_grads(params, X, Xt, bf16=False):
    """L and [(dL/dW_l, dL/db_l)] for input X [3, H, W] and target
    Xt [2, H, W] (the later state in input units)."""
    Y, acts = forward(params, X, bf16)
    R = Y - (np.asarray(Xt, np.float64) - np.asarray(X, np.float64)[:2])   # X unrounded
    n = R.size
    L = float(np.sum(R * R) / n)
    G = 2.0 * R / n                                   # dL/dZ_4
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        Gq = bf16_round(G).astype(np.float64) if bf16 else G
        grads[l] = (conv3x3_wgrad(Gq, acts[l]), Gq.sum(axis=(1, 2)))
        if l > 0:
            dA = conv3x3_transpose(Gq, _rw(W, bf16))
            G = dA * (acts[l] > 0)
    return L, grads


def adam_step(params, grads, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (fp64 here); state = {'k': step count, 'm': [...],
    'v': [...]} is updated in place and the new parameters returned."""
    if not state:
        state.update(k=0, m=[(np.zeros_like(W), np.zeros_like(b)) for W, b in params],
                     v=[(np.zeros_like(W), np.zeros_like(b)) for W, b in params])
    state['k'] += 1
    k = state['k']
    out = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for j, (p, g) in enumerate(((W, gW), (b, gb))):
            m = b1 * state['m'][l][j] + (1 - b1) * g
            v = b2 * state['v'][l][j] + (1 - b2) * g * g
            mh = m / (1 - b1 ** k)
            vh = v / (1 - b2 ** k)
            new.append(p - lr * mh / (np.sqrt(vh) + eps))
            ms, vs = list(state['m'][l]), list(state['v'][l])
            ms[j], vs[j] = m, v
            state['m'][l], state['v'][l] = tuple(ms), tuple(vs)
        out.append(tuple(new))
    return out


def encode(rho, T, T_run, rho_c, T_c, s_rho=50.0, s_T=50.0):
    """Network input [3, H, W] from fields and the run temperature."""
    rho = np.asarray(rho, np.float64)
    return np.stack([s_rho * (rho / rho_c - 1.0), s_T * (np.asarray(T, np.float64) / T_run - 1.0),
                     np.full(rho.shape, T_run / T_c - 0.75)])


def decode(X, Y, T_run, rho_c, s_rho=50.0, s_T=50.0):
    """(rho', T') from the input and the network output."""
    return rho_c * (1.0 + (X[0] + Y[0]) / s_rho), T_run * (1.0 + (X[1] + Y[1]) / s_T)
