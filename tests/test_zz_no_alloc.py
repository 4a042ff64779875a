"""fftlb_gradient_static: the allocation-free variant of the spectral
gradient, for callers that must not call cudaMalloc/cudaFree while they run
(a plug-in inside a framework whose caching allocator owns the GPU's memory,
or a loop that cannot afford an allocation's implicit synchronisation).  It
keeps its scratch in one fixed array in device global memory.

Its output must equal the handle-based fftlb_gradient's within the parity
tolerance of the spectral tests (1e-12 relative), on consecutive calls that
reuse the shared array with different grids.  This file is collected last so
that a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from gpu_common import lib, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def reference_gradient(fl, g, window, dx):
    ny, nx = g.shape
    with fl.Handle(fl.params(nx=nx, ny=ny, dx=dx, window=window, precision=64)) as h:
        gd = torch.from_numpy(g[None].copy()).cuda()
        out = torch.empty((2, ny, nx), dtype=torch.float64, device="cuda")
        h.gradient(gd, out, 1)
        torch.cuda.synchronize()
        return out.cpu().numpy()


def static_gradient(fl, g, window, dx):
    ny, nx = g.shape
    gd = torch.from_numpy(g.copy()).cuda()
    out = torch.full((2, ny, nx), float("nan"), dtype=torch.float64, device="cuda")
    fl.gradient_static(gd, out, nx, ny, dx, window, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_static_gradient_matches_handle_gradient_on_consecutive_calls():
    fl = lib()
    rng = np.random.default_rng(2024)
    # (ny, nx): the limits of the array (nx or ny = 1024 at nx ny = 65536,
    # 4-point axes) between ordinary grids, on consecutive calls
    cases = [((64, 64), 4, 1 / 256), ((48, 96), 2, 1 / 128), ((256, 256), 0, 1 / 256), ((64, 1024), 4, 1 / 256),
             ((1024, 64), 3, 1 / 256), ((4, 256), 4, 1 / 64), ((256, 4), 1, 1 / 64), ((64, 64), 4, 1 / 256)]
    for (ny, nx), window, dx in cases:
        g = rng.standard_normal((ny, nx))
        want = reference_gradient(fl, g, window, dx)
        got = static_gradient(fl, g, window, dx)
        assert np.isfinite(got).all()
        assert rel_err(got[0], want[0]) < 1e-12, ((ny, nx), window)
        assert rel_err(got[1], want[1]) < 1e-12, ((ny, nx), window)


def test_static_gradient_rejects_oversized_grid():
    fl = lib()
    g = torch.zeros((512, 512), dtype=torch.float64, device="cuda")
    out = torch.zeros((2, 512, 512), dtype=torch.float64, device="cuda")
    with pytest.raises(fl.FFTLBError) as ei:
        fl.gradient_static(g, out, 512, 512)
    assert ei.value.status == fl.ERR_ARG
    assert "65536" in str(ei.value)
