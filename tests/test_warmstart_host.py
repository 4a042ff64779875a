"""Host logic of the warm-start protocol (paper_1011_3582_gb300/warmstart.py),
on the CPU: the initial parameter vector matches the C ABI's layout, the
data augmentation applies one symmetry of the square periodic grid to input
and target alike, and the protocol's critical point is that of the vdW EOS
it runs."""
import os
import re

import numpy as np
import pytest

from oracle import cnn_oracle as CO
from oracle import thermo as TH
from paper_1011_3582_gb300 import warmstart as WS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_nparams():
    src = open(os.path.join(ROOT, "include", "fftlb_warmstart.h")).read()
    expr = re.search(r"#define FFTLB_CNN_NPARAMS \(([^\n]+)\)\n", src).group(1)
    return eval(expr, {"__builtins__": {}})


def test_init_params_layout():
    p = WS.init_params(0)
    assert p.dtype == np.float32 and p.size == header_nparams()
    off = 0
    for l, (ci, co) in enumerate(CO.LAYERS):
        w = p[off:off + co * 9 * ci]
        b = p[off + co * 9 * ci:off + co * 9 * ci + co]
        off += co * 9 * ci + co
        std = np.sqrt(2.0 / (9 * ci)) * (0.1 if l == len(CO.LAYERS) - 1 else 1.0)
        assert np.all(b == 0)
        assert w.std() == pytest.approx(std, rel=0.2)
    assert off == p.size
    assert np.array_equal(WS.init_params(0), p) and not np.array_equal(WS.init_params(1), p)


def test_augment_is_one_grid_symmetry_for_input_and_target():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    X = torch.tensor(rng.standard_normal((3, 8, 8)), dtype=torch.float32)
    seen = set()
    for k in range(4):
        for flip in (False, True):
            Xa, Xta = WS.augment(X, X[:2].clone(), k, flip)
            # the target channels follow the input channels exactly
            assert torch.equal(Xta, Xa[:2])
            # the same map as numpy's rotation and reflection of the grid axes
            want = np.rot90(X.numpy(), k, axes=(1, 2))
            if flip:
                want = want[:, :, ::-1]
            assert np.array_equal(Xa.numpy(), want)
            assert Xa.is_contiguous() and Xta.is_contiguous()
            seen.add(Xa.numpy().tobytes())
    assert len(seen) == 8   # the 8 elements of the square's symmetry group


def test_protocol_constants_are_the_eos_critical_point():
    Tc, rhoc, _ = TH.critical_point(WS.A, WS.B)
    assert WS.TC == pytest.approx(Tc, rel=1e-15) and WS.RHOC == pytest.approx(rhoc, rel=1e-15)
    assert WS.TC == pytest.approx(4 / 7) and WS.RHOC == pytest.approx(3.5)
    assert WS.C_TGT < WS.C_ONSET and WS.T_IN % 100 == 0
