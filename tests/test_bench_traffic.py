"""roofline.traffic bookkeeping in bench.py (host only): a DRAM figure from
profiles/ncu_traffic.txt is reported only while the kernel's source file still
hashes to the value recorded with the capture, and a capture with a pixel
count is scaled to another workload's pixels per launch."""
import hashlib
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _sha(name):
    path = os.path.join(ROOT, "paper_2511_00870_b300", "csrc", name)
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:12]


def test_source_hash_maps_kernels_to_files(bench):
    assert bench._source_sha("k_conv_tc<0,0>") == _sha("k_conv_tc.cu")
    assert bench._source_sha("k_first_tc<0>") == _sha("k_conv_tc.cu")
    assert bench._source_sha("k_update_os") == _sha("k_update_os.cu")
    assert bench._source_sha("k_sp_cols") == _sha("k_spectral.cu")
    assert bench._source_sha("k_update<25,2,1>") == _sha("k_stencil.cu")


def _with_table(bench, tmp_path, lines, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.txt").write_text("\n".join(lines) + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the kernel sources are still read from the repository
    monkeypatch.setattr(bench, "_source_sha", lambda k: "cafe00000001")


def test_exact_line_is_reported_and_scaled(bench, tmp_path, monkeypatch):
    _with_table(bench, tmp_path, ["# comment",
                                  "k_conv_tc<0,0> deconv1024 bf16 100 50 cafe00000001 1000"],
                monkeypatch)
    b, note = bench.ncu_traffic("k_conv_tc<0,0>", "deconv1024", "bf16", npix=1000)
    assert b == 150 and "cafe00000001" in note
    b, note = bench.ncu_traffic("k_conv_tc<0,0>", "serve", "bf16", npix=4000)
    assert b == 600 and "scaled" in note
    b, note = bench.ncu_traffic("k_conv_tc<0,0>", "serve", "fp8", npix=4000)
    assert b is None


def test_stale_capture_is_not_reported(bench, tmp_path, monkeypatch):
    _with_table(bench, tmp_path, ["k_conv_tc<0,0> deconv1024 bf16 100 50 0123456789ab 1000",
                                  "k_conv_tc<0,0> deconv8192 bf16 100 50"], monkeypatch)
    b, note = bench.ncu_traffic("k_conv_tc<0,0>", "deconv1024", "bf16", npix=1000)
    assert b is None and "changed" in note
    b, note = bench.ncu_traffic("k_conv_tc<0,0>", "deconv8192", "bf16", npix=1000)
    assert b is None
    b, note = bench.ncu_traffic("k_conv_tc<0,0>", "serve", "bf16", npix=1000)
    assert b is None
