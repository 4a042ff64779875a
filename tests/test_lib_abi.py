"""The C-ABI library builds, loads without a GPU, exports every entry point
include/fftlb.h declares, and rejects invalid arguments before touching
the device."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fl():
    from paper_1011_3582_gb300 import build
    build.build()
    from paper_1011_3582_gb300 import fftlb
    return fftlb


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fftlb_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(fl):
    names = declared_functions()
    assert "fftlb_create" in names and "fftlb_step" in names
    lib = ct.CDLL(fl.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(fl.EXPORTED) <= names


def test_params_struct_layout_matches_header(fl):
    # int nx, ny; 9 doubles; 4 ints  (x86-64 / aarch64 LP64 layout)
    assert ct.sizeof(fl.fftlb_params) == 8 + 9 * 8 + 4 * 4


@pytest.mark.parametrize("kw", [dict(nx=10), dict(ny=6 * 5), dict(nx=2), dict(tau=0.0), dict(window=5),
                                dict(integrator=2), dict(precision=16), dict(precision=256),
                                dict(precision=64 | 256)])
def test_create_rejects_bad_arguments_without_device_work(fl, kw):
    base = dict(nx=16, ny=16)
    base.update(kw)
    p = fl.params(**base)
    with pytest.raises(fl.FFTLBError) as ei:
        fl.Handle(p)
    assert ei.value.status == fl.ERR_ARG
    assert len(str(ei.value)) > 10


def test_bf16split_flag_matches_header(fl):
    src = open(os.path.join(ROOT, "include", "fftlb.h")).read()
    assert int(re.search(r"#define FFTLB_BF16SPLIT (\d+)", src).group(1)) == fl.BF16SPLIT


def test_null_handle_calls_return_arg_error(fl):
    lib = fl.lib()
    assert lib.fftlb_step(None, 1, None) == fl.ERR_ARG
    assert lib.fftlb_invariants(None, None) == fl.ERR_ARG
    assert lib.fftlb_destroy(None) == fl.OK


def test_binding_rejects_wrongly_sized_host_buffers(fl):
    """The binding checks dtype, layout and element count of host buffers
    before any pointer reaches the C calls."""
    import numpy as np
    fftlb = fl
    a = np.zeros(12)
    assert fftlb._addr(a, False, 12) == a.ctypes.data
    with pytest.raises(ValueError):
        fftlb._addr(np.zeros(12), False, 16)
    with pytest.raises(TypeError):
        fftlb._addr(np.zeros(16, dtype=np.float32), False, 16)
    with pytest.raises(TypeError):
        fftlb._addr(np.zeros((4, 8))[:, ::2], False, 16)


def test_cnn_create_rejects_bad_grids_without_device_work(fl):
    for H, W in ((0, 64), (16, 48), (16, 8192)):
        with pytest.raises(fl.FFTLBError) as ei:
            fl.CNN(H, W)
        assert ei.value.status == fl.ERR_ARG


def test_cnn_parameter_packing_round_trip(fl):
    import numpy as np
    from oracle import cnn_oracle as C
    params = C.init_params(3)
    vec = fl.pack_params(params)
    assert vec.size == fl.CNN_NPARAMS
    back = fl.unpack_params(vec.astype(np.float64))
    for (W1, b1), (W2, b2) in zip(params, back):
        assert np.allclose(W1, W2, rtol=1e-6, atol=1e-7) and np.allclose(b1, b2)


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "fftlb.h"
#include "fftlb_warmstart.h"

int main(void) {
    fftlb_params p;
    memset(&p, 0, sizeof p);
    p.nx = 10; p.ny = 16; p.dx = 1.0 / 256; p.dt = 1e-5; p.tau = 1e-2;
    p.a = 9.0 / 8; p.b = 1.0 / 3; p.K = 1e-5; p.q = -0.004;
    p.window = 4; p.integrator = 3; p.precision = 32 | FFTLB_BF16SPLIT;
    fftlb_t h = (fftlb_t)1;
    fftlb_status st = fftlb_create(&h, &p, NULL, NULL);
    const char *msg = fftlb_last_error(NULL);   /* valid until the next call */
    if (st != FFTLB_ERR_ARG || h != NULL || msg == NULL || strlen(msg) < 10) return 1;
    printf("%s\n", msg);
    fftlb_cnn_t c = (fftlb_cnn_t)1;
    if (fftlb_cnn_create(&c, 8, 100, NULL) != FFTLB_ERR_ARG) return 2;
    return 0;
}
"""


def test_plain_c_client_compiles_links_and_gets_argument_errors(fl, tmp_path):
    """The boundary is a C ABI: a C99 program includes both headers, links
    libfftlb.so and gets FFTLB_ERR_ARG with a message for an invalid grid
    (the checks come before any device work, so no GPU is needed)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(fl.LIB_PATH)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-lfftlb", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, (run.returncode, run.stdout, run.stderr)
    assert "nx" in run.stdout
