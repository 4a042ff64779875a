"""The separable split of the derivative passes on the host (CPU, no GPU).

The windowed derivative multipliers factor into functions of k_x and of
k_y (Eqs. K1-K4), so a derivative in k_x alone needs no column transform:
the stage's level-1 column pass forms only the 8 outputs that involve k_y,
the row kernel K3 forms the other 7 in the row spectrum (k3_form_x in
kernels_pipe.cuh) and, for level 2, writes i k_x X / nx of Lambda_xx,
Lambda_xy, Phi_x for the column pass to add to its d_y terms; the
convection terms of the velocities with v_y = 0 skip the column pass the
same way.  This test
runs that data flow with numpy in the engine's layouts (one-sided row
spectra with the row-Nyquist value packed into bin 0, unnormalised column
transforms with the 1 / (nx ny) multiplier scale, unnormalised inverse rows)
and checks every derivative the stage uses against the oracle's composed
derivative D."""
import numpy as np
import pytest

from oracle import fftlb_oracle as O

ARCSIN = [1.0, 1.0 / 6.0, 3.0 / 40.0, 5.0 / 112.0]


def kappa_engine(n, N, dx, window):
    """k_m of bin n (the engine's table: the Nyquist bin set to zero)."""
    if 2 * abs(n) == N:
        return 0.0
    s = np.sin(np.pi * n / N)
    return sum(ARCSIN[j] * s ** (2 * j + 1) for j in range(window)) * 2.0 / dx


def row_spec(a):
    """Forward rows: [ny][nx] real -> [ny][h] one-sided, Nyquist packed into bin 0."""
    X = np.fft.rfft(a, axis=1)
    h = a.shape[1] // 2
    Z = X[:, :h].copy()
    Z[:, 0] = X[:, 0].real + 1j * X[:, h].real
    return Z


def row_inv(Z):
    """Inverse rows, unnormalised: [ny][h] packed -> [ny][2h] real."""
    ny, h = Z.shape
    X = np.zeros((ny, h + 1), complex)
    X[:, :h] = Z
    X[:, 0] = Z[:, 0].real
    X[:, h] = Z[:, 0].imag
    return np.fft.irfft(X, n=2 * h, axis=1) * (2 * h)


def col_pass(terms, kx, ky, scale):
    """One column-pass output: sum of M(k_x, k_y) X over the terms, M given
    by (c0..c4) as in GroupDesc; unnormalised inverse; packed column 0 takes
    the multiplier at k_x = 0."""
    ny = terms[0][1].shape[0]
    acc = 0
    for c, X in terms:
        ax, ay = kx[None, :X.shape[1]], ky[:, None]
        M = 1j * (c[0] * ax + c[1] * ay) + (c[2] * ax * ax + c[3] * ay * ay + c[4] * ax * ay)
        acc = acc + M * np.fft.fft(X, axis=0)
    return np.fft.ifft(acc * scale, axis=0) * ny


DY, DYY, DXY = (0, 1, 0, 0, 0), (0, 0, 0, -1, 0), (0, 0, 0, 0, -1)


@pytest.mark.parametrize("ny,nx,window", [(16, 32, 4), (32, 16, 1), (24, 20, 3)])
def test_split_derivatives_match_composed_D(ny, nx, window):
    rng = np.random.default_rng(ny * nx + window)
    dx = 1.0 / 64
    h = nx // 2
    kx = np.array([kappa_engine(j, nx, dx, window) for j in range(h + 1)])
    ky = np.array([kappa_engine(j if j < ny // 2 else j - ny, ny, dx, window) for j in range(ny)])
    scale, sx = 1.0 / (nx * ny), 1.0 / nx
    f = {k: rng.standard_normal((ny, nx)) for k in ("rho", "ux", "uy", "T", "Pi", "g",
                                                   "Lxx", "Lxy", "Lyy", "Phx", "Phy")}
    S = {k: row_spec(v) for k, v in f.items()}

    # level-1 column pass: the 8 outputs that involve k_y
    col = {"ry": col_pass([(DY, S["rho"])], kx, ky, scale),
           "lap": col_pass([(DYY, S["rho"])], kx, ky, scale),
           "uxy": col_pass([(DY, S["ux"])], kx, ky, scale),
           "uyy": col_pass([(DY, S["uy"])], kx, ky, scale),
           "divy": col_pass([(DXY, S["ux"]), (DYY, S["uy"])], kx, ky, scale),
           "Ty": col_pass([(DY, S["T"])], kx, ky, scale),
           "Piy": col_pass([(DY, S["Pi"])], kx, ky, scale),
           "gy": col_pass([(DY, S["g"])], kx, ky, scale)}
    # K3's pointwise forms in the row spectrum (k3_form_x)
    ax = kx[None, :h]
    m = ax * sx
    im = lambda mult, z: 1j * mult * z
    uxx = im(m, S["ux"])
    rows = {"rx": im(m, S["rho"]), "ry": col["ry"], "lap": col["lap"] - ax * m * S["rho"],
            "uxx": uxx, "uxy": col["uxy"], "uyx": im(m, S["uy"]), "uyy": col["uyy"],
            "divx": im(ax, uxx + col["uyy"]), "divy": col["divy"],
            "Tx": im(m, S["T"]), "Ty": col["Ty"], "Pix": im(m, S["Pi"]), "Piy": col["Piy"],
            "gx": im(m, S["g"]), "gy": col["gy"]}
    Dx = lambda a: O.D(a, 'x', dx, window)
    Dy = lambda a: O.D(a, 'y', dx, window)
    div = Dx(f["ux"]) + Dy(f["uy"])
    want = {"rx": Dx(f["rho"]), "ry": Dy(f["rho"]), "lap": Dx(Dx(f["rho"])) + Dy(Dy(f["rho"])),
            "uxx": Dx(f["ux"]), "uxy": Dy(f["ux"]), "uyx": Dx(f["uy"]), "uyy": Dy(f["uy"]),
            "divx": Dx(div), "divy": Dy(div), "Tx": Dx(f["T"]), "Ty": Dy(f["T"]),
            "Pix": Dx(f["Pi"]), "Piy": Dy(f["Pi"]), "gx": Dx(f["g"]), "gy": Dy(f["g"])}
    assert len(rows) == 15
    for k, Z in rows.items():
        got = row_inv(Z)
        assert np.abs(got - want[k]).max() < 1e-9 * max(1.0, np.abs(want[k]).max()), k

    # level 2: K3 writes i k_x X / nx of Lambda_xx, Lambda_xy, Phi_x; the
    # column pass adds them to d_y of Lambda_xy, Lambda_yy, Phi_y
    mul = lambda X: im(m, X)
    out = {"dLx": col_pass([(DY, S["Lxy"])], kx, ky, scale) + mul(S["Lxx"]),
           "dLy": col_pass([(DY, S["Lyy"])], kx, ky, scale) + mul(S["Lxy"]),
           "dPh": col_pass([(DY, S["Phy"])], kx, ky, scale) + mul(S["Phx"])}
    want2 = {"dLx": Dx(f["Lxx"]) + Dy(f["Lxy"]), "dLy": Dx(f["Lxy"]) + Dy(f["Lyy"]),
             "dPh": Dx(f["Phx"]) + Dy(f["Phy"])}
    for k, Z in out.items():
        got = row_inv(Z)
        assert np.abs(got - want2[k]).max() < 1e-9 * max(1.0, np.abs(want2[k]).max()), k


@pytest.mark.parametrize("ring_speed", [1.0, 2.7])
def test_convection_without_v_y_needs_no_column_pass(ring_speed):
    """Directions 0 and 4 of every ring have v_y = 0 (Eq. 1): the column pass
    of i (v_x k_x + v_y k_y) X leaves i v_x k_x X / nx, the form the row
    kernel K1 writes for them (k1_wr, k1_pipe); against the oracle's
    v_x D_x f as well."""
    ny, nx, window, dx = 16, 32, 4, 1.0 / 64
    rng = np.random.default_rng(2)
    f = rng.standard_normal((ny, nx))
    h = nx // 2
    kx = np.array([kappa_engine(j, nx, dx, window) for j in range(h + 1)])
    ky = np.array([kappa_engine(j if j < ny // 2 else j - ny, ny, dx, window) for j in range(ny)])
    S = row_spec(f)
    for vx in (ring_speed, -ring_speed):
        col = col_pass([((vx, 0, 0, 0, 0), S)], kx, ky, 1.0 / (nx * ny))
        k1 = 1j * (vx * kx[None, :h] / nx) * S
        assert np.abs(col - k1).max() < 1e-12 * np.abs(col).max()
        want = vx * O.D(f, 'x', dx, window)
        assert np.abs(row_inv(k1) - want).max() < 1e-9 * np.abs(want).max()


def test_gradient_energy_by_parseval():
    """The invariants' gradient energy (e_T of Eq. 17 holds K |grad rho|^2 /
    2) as k_invariant_rows forms it: from the row spectrum Z of rho and the
    column pass's Y = DFT_x(D_y rho) / nx, per row
        (1 / nx) sum_{0<k<h} 2 k_x^2 |Z_k|^2 + nx (Y_0.x^2 + Y_0.y^2 + sum_{0<k<h} 2 |Y_k|^2),
    against sum over the sites of (D_x rho)^2 + (D_y rho)^2 with the oracle's D."""
    ny, nx, window, dx = 24, 32, 4, 1.0 / 64
    rng = np.random.default_rng(5)
    rho = 3.5 + rng.standard_normal((ny, nx))
    h = nx // 2
    kx = np.array([kappa_engine(j, nx, dx, window) for j in range(h + 1)])
    ky = np.array([kappa_engine(j if j < ny // 2 else j - ny, ny, dx, window) for j in range(ny)])
    Z = row_spec(rho)
    Y = col_pass([(DY, Z)], kx, ky, 1.0 / (nx * ny))
    gx = (2.0 * (kx[None, 1:h] ** 2) * np.abs(Z[:, 1:h]) ** 2).sum(axis=1) / nx
    gy = nx * (Y[:, 0].real ** 2 + Y[:, 0].imag ** 2 + 2.0 * (np.abs(Y[:, 1:h]) ** 2).sum(axis=1))
    want = O.D(rho, 'x', dx, window) ** 2 + O.D(rho, 'y', dx, window) ** 2
    assert np.abs(gx + gy - want.sum(axis=1)).max() < 1e-9 * want.sum(axis=1).max()


def test_planted_mistake_is_caught():
    """The same check fails when K3's Laplacian drops its k_x^2 term."""
    ny, nx, window, dx = 16, 32, 4, 1.0 / 64
    rng = np.random.default_rng(1)
    rho = rng.standard_normal((ny, nx))
    h = nx // 2
    kx = np.array([kappa_engine(j, nx, dx, window) for j in range(h + 1)])
    ky = np.array([kappa_engine(j if j < ny // 2 else j - ny, ny, dx, window) for j in range(ny)])
    lap_wrong = row_inv(col_pass([(DYY, row_spec(rho))], kx, ky, 1.0 / (nx * ny)))
    want = O.D(O.D(rho, 'x', dx, window), 'x', dx, window) + O.D(O.D(rho, 'y', dx, window), 'y', dx, window)
    assert np.abs(lap_wrong - want).max() > 1e-3 * np.abs(want).max()
