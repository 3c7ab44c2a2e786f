"""The benchmark's rule for the DRAM traffic it reports beside the roofline: a committed ncu
summary counts only while both the kernel's source file and the shared device header it
includes are byte-for-byte what the summary's hashes name (otherwise traffic is null), and
the committed summaries of the step's dominant kernels match the sources as they stand."""
import hashlib
import os

import pytest

import bench


def _sha(path):
    with open(path, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()


def _layout(tmp_path, text):
    csrc = tmp_path / "paper_2212_05159_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("// kernel\n")
    (csrc / "common.cuh").write_text("// header\n")
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_case.txt").write_text(text.format(src=_sha(csrc / "k.cu"),
                                                                  hdr=_sha(csrc / "common.cuh")))
    return csrc


def test_traffic_needs_both_hashes_to_match(tmp_path, monkeypatch):
    text = "dram_bytes_per_launch: 12345\nsource_sha256: {src}   (k.cu)\nheader_sha256: {hdr}   (common.cuh)\n"
    csrc = _layout(tmp_path, text)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("k_case", str(csrc / "k.cu")) == 12345.0
    (csrc / "common.cuh").write_text("// header, edited\n")
    assert bench.ncu_traffic("k_case", str(csrc / "k.cu")) is None
    (csrc / "common.cuh").write_text("// header\n")
    (csrc / "k.cu").write_text("// kernel, edited\n")
    assert bench.ncu_traffic("k_case", str(csrc / "k.cu")) is None


def test_traffic_needs_the_header_hash(tmp_path, monkeypatch):
    csrc = _layout(tmp_path, "dram_bytes_per_launch: 7\nsource_sha256: {src}   (k.cu)\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("k_case", str(csrc / "k.cu")) is None
    assert bench.ncu_traffic("missing_case", str(csrc / "k.cu")) is None


@pytest.mark.parametrize("tag,src", [("spmm_t_sddmm_kernel_powerlaw_k32", "backward.cu"),
                                     ("spmm_t_sddmm_kernel_powerlaw_k128", "backward.cu"),
                                     ("spmm_t_sddmm_kernel_poisson3d_128_k32", "backward.cu"),
                                     ("spmm_kernel_powerlaw_k32", "spmm.cu")])
def test_committed_dominant_kernel_summaries_match_the_sources(tag, src):
    path = os.path.join(bench.ROOT, "paper_2212_05159_gb300", "csrc", src)
    assert bench.ncu_traffic(tag, path) is not None, f"profiles/{tag}.txt does not match {src} / common.cuh"
