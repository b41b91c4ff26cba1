"""pnp_denoise_noalloc: the denoiser for callers that must not allocate device
memory (for example when another allocator already holds nearly all of HBM,
or in a loop that cannot let cudaMalloc/cudaFree synchronize the device).

It runs the same kernels as pnp_denoise, which allocates its own scratch, on
the library's fixed scratch area, so the two results must be bitwise equal.
The calls come in a row on one shared area: an FP32 call first leaves the
area dirty, then a wide BF16 call, then a narrower BF16 image whose width is
not a multiple of 8 (its padding columns sit where the previous call left
data), so anything stale that leaked into a result would show. A repeated
call must leave the device's free memory unchanged.
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


def _images(shape, seed):
    n, ny, nx = shape
    return torch.from_numpy(np.stack([synth.ground_truth(ny, nx, seed=seed + c)
                                      for c in range(n)]).astype(np.float32)).cuda()


def test_noalloc_matches_allocating_entry_point_bitwise(P):
    den = P.Denoiser.from_weights(synth.denoiser_weights(8, 64, seed=21))
    calls = [("fp32", (1, 96, 130)), ("bf16", (1, 300, 257)), ("bf16", (2, 128, 75)),
             ("fp32", (2, 64, 61))]
    for k, (prec, shape) in enumerate(calls):          # one shared area, calls in a row
        x = _images(shape, 40 + 7 * k)
        ref = den.denoise(x, precision=prec)
        out = torch.full_like(x, float("nan"))
        den.denoise_noalloc(x, out, precision=prec)
        torch.cuda.synchronize()
        den.status()
        assert torch.equal(out, ref), (prec, shape, (out - ref).abs().max().item())


def test_noalloc_repeat_call_allocates_nothing(P):
    den = P.Denoiser.from_weights(synth.denoiser_weights(8, 64, seed=22))
    x = _images((1, 200, 203), 5)
    out = torch.empty_like(x)
    den.denoise_noalloc(x, out, precision="bf16")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    den.denoise_noalloc(x, out, precision="bf16")
    den.denoise_noalloc(x, out, precision="fp32")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_oversized_requests_and_fp8(P):
    den = P.Denoiser.from_weights(synth.denoiser_weights(8, 64, seed=21))
    x = torch.zeros((1, 1024, 1024), device="cuda")
    out = torch.zeros_like(x)
    with pytest.raises(P.PnpError) as e:
        den.denoise_noalloc(x, out, precision="bf16")
    assert e.value.status == 1 and "scratch" in str(e.value)
    with pytest.raises(P.PnpError) as e:
        den.denoise_noalloc(x[:, :64, :64].contiguous(), out[:, :64, :64].contiguous(),
                            precision="fp8")
    assert e.value.status == 7
    torch.cuda.synchronize()
    assert out.abs().max().item() == 0.0          # nothing was launched
    with pytest.raises(ValueError):
        den.denoise_noalloc(x.double(), out, precision="bf16")
