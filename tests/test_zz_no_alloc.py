"""pnp_denoise_noalloc: the denoiser for callers that must not allocate device
memory (for example when another allocator already holds nearly all of HBM,
or in a loop that cannot let cudaMalloc/cudaFree synchronize the device).

It runs on the library's fixed scratch area and must give the same result as
pnp_denoise, which allocates its own scratch. Two calls in a row with
different image sizes and contents check that what the previous call left in
the shared area does not leak into the next result.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_00870_b300 as P
    return P


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_noalloc_matches_allocating_entry_point(P, prec):
    dw = synth.denoiser_weights(8, 64, seed=21)
    den = P.Denoiser.from_weights(dw)
    shapes = [(1, 96, 130), (2, 64, 64)] if prec == "fp32" else [(1, 300, 257), (2, 128, 72)]
    for k, shape in enumerate(shapes):            # two calls in a row
        x = torch.from_numpy(np.stack([synth.ground_truth(shape[1], shape[2], seed=40 + 3 * k + c)
                                       for c in range(shape[0])]).astype(np.float32)).cuda()
        ref = den.denoise(x, precision=prec)
        out = torch.full_like(x, float("nan"))
        den.denoise_noalloc(x, out, precision=prec)
        torch.cuda.synchronize()
        G = (x - ref).abs().max().item()
        tol = (1e-5 if prec == "fp32" else 3e-2) * G
        assert torch.isfinite(out).all()
        assert (out - ref).abs().max().item() <= tol


def test_noalloc_rejects_oversized_requests(P):
    dw = synth.denoiser_weights(8, 64, seed=21)
    den = P.Denoiser.from_weights(dw)
    x = torch.zeros((1, 1024, 1024), device="cuda")
    out = torch.zeros_like(x)
    with pytest.raises(P.PnpError) as e:
        den.denoise_noalloc(x, out, precision="bf16")
    assert e.value.status == 1 and "scratch" in str(e.value)
    assert out.abs().max().item() == 0.0          # nothing was launched
