"""The C-ABI library loads without a GPU and exports every entry point that
include/*.h declares; host-side logic (argument checks, step sizes) works on
the CPU. No compute call needs a device here."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(pnp_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2511_00870_b300 import build
    build.build()
    from paper_2511_00870_b300 import _lib
    return _lib.load()


def test_header_declares_core_calls():
    names = declared_functions()
    for n in ("pnp_create_problem", "pnp_step", "pnp_run_chain", "pnp_get_moments",
              "pnp_create_denoiser", "pnp_denoise", "pnp_blur", "pnp_langevin_update"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_covers_every_symbol():
    from paper_2511_00870_b300 import _lib
    missing = [n for n in declared_functions() if n not in _lib.SIGNATURES]
    assert not missing, missing


def test_stepsizes_match_oracle(lib, orc):
    from paper_2511_00870_b300 import pnp_stepsizes
    for args in [(1.0, 0.01, 1.0, 0.01, 0.9), (0.5, 0.2, 2.0, 0.1, 3.0), (1.0, 0.05, 0.0, 1.0, 0.0)]:
        got = pnp_stepsizes(*args)
        ref = orc.stepsizes(*args)
        np.testing.assert_allclose(got, ref, rtol=1e-15)


def test_argument_errors_are_reported(lib):
    from paper_2511_00870_b300 import PnpError, pnp_stepsizes
    with pytest.raises(PnpError) as e:
        pnp_stepsizes(1.0, -1.0, 1.0, 0.1, 0.9)
    assert e.value.status == 1
    assert b"sigma" in lib.pnp_last_error()


def test_problem_rejects_bad_descriptors_without_gpu(lib):
    """Validation happens on the host before any device work."""
    from paper_2511_00870_b300 import PnpError, Problem
    y = np.zeros((16, 16), np.float32)
    h = np.ones((3, 3), np.float32) / 9
    with pytest.raises(PnpError):
        Problem(y, h, sigma=-1.0)                      # sigma <= 0
    with pytest.raises(PnpError):
        Problem(y, np.ones((4, 4), np.float32), 0.1)    # even kernel
    bad = y.copy()
    bad[3, 3] = np.nan
    with pytest.raises(PnpError):
        Problem(bad, h, 0.1)                            # NaN in y
    with pytest.raises(PnpError):
        Problem(y, h, 0.1, blocks=(17, 1))              # more blocks than rows
    with pytest.raises(PnpError):
        Problem(y, h, 0.1, gamma=10.0)                  # violates Eq. 10
    big = np.zeros((200, 200), np.float32)
    with pytest.raises(PnpError):
        Problem(big, np.ones((131, 131), np.float32) / 131 ** 2, 0.1)   # kernel above 129
    with pytest.raises(PnpError) as e:
        Problem(big, np.ones((33, 33), np.float32) / 33 ** 2, 0.0, noise_model="poisson",
                eta=250.0, rho1=10.0, rho2=1e-3)        # Poisson with a large kernel
    assert e.value.status == 7
    with pytest.raises(PnpError):
        Problem(y, h, 0.0, noise_model="poisson", eta=250.0, rho1=10.0, rho2=1e-3,
                kappa1=20.0)                            # kappa1 >= rho1
    neg = y.copy()
    neg[0, 0] = -1.0
    with pytest.raises(PnpError):
        Problem(neg, h, 0.0, noise_model="poisson", eta=250.0, rho1=10.0, rho2=1e-3)
    with pytest.raises(PnpError):
        Problem(y, None, 0.1, mask=np.full(y.shape, 0.5))   # mask entries not 0/1
    with pytest.raises(PnpError):
        Problem(y, h, 0.1, noise_model="poisson", eta=250.0, rho1=10.0, rho2=1e-3,
                mask=np.ones(y.shape))                  # inpainting is Gaussian
    from paper_2511_00870_b300 import Denoiser
    import synth
    dw = synth.ddfb_weights(4, 16, 1)
    den = Denoiser.ddfb(dw.filters, dw.gammas, dw.ht)       # host-only creation
    with pytest.raises(PnpError) as e:
        Problem(y, h, 0.1, den, precision="bf16")       # DDFB runs in FP32
    assert e.value.status == 7
    with pytest.raises(PnpError):
        Problem(y, h, 0.1, den, blocks=(2, 2), halo=8)  # DDFB uses the direct layout
    with pytest.raises(PnpError):
        Denoiser.ddfb(dw.filters, -dw.gammas, dw.ht)     # gamma_k <= 0
    dw64 = synth.ddfb_weights(4, 64, 1)
    den64 = Denoiser.ddfb(dw64.filters, dw64.gammas, dw64.ht)
    import ctypes as C
    st = lib.pnp_denoise_noalloc(den64.handle, 1, C.c_void_p(16), 8, 8, 1, C.c_void_p(16), None)
    assert st == 7                                      # BF16 on a DDFB denoiser: refused


def test_stencil_tile_override_is_validated_on_the_host(lib):
    from paper_2511_00870_b300 import PnpError, pnp_set_stencil_tile, pnp_stencil_tile_count
    n = pnp_stencil_tile_count()
    assert n >= 2
    for bad in (-2, n):
        with pytest.raises(PnpError) as e:
            pnp_set_stencil_tile(bad)
        assert e.value.status == 1
    pnp_set_stencil_tile(n - 1)
    pnp_set_stencil_tile(-1)
