"""The byte figures quoted in the committed ncu summaries are the benchmark's own byte models
(bench.launch_bytes / bench.gather_bytes) evaluated on the workload each summary names, so
the traffic ratios written there and the roofline fractions the benchmark reports use one
definition of the algorithmic bytes."""
import os
import re

import pytest

import bench

PROFILES = os.path.join(bench.ROOT, "profiles")
POWERLAW_N = 1 << 20
POISSON_128 = (128 ** 3, 7 * 128 ** 3 - 6 * 128 ** 2)     # rows, entries of the 7-point stencil


def _text(name):
    with open(os.path.join(PROFILES, name)) as fh:
        return fh.read()


def _number(text, label):
    m = re.search(label + r"\s+([\d,]+) B", text)
    assert m, label
    return int(m.group(1).replace(",", ""))


def _powerlaw_nnz(text):
    m = re.search(r"nnz = ([\d,]+)", text)
    return int(m.group(1).replace(",", ""))


@pytest.mark.parametrize("name,kind,k,label", [
    ("spmm_kernel_powerlaw_k32.txt", "spmm", 32, "compulsory bytes per launch"),
    ("sddmm_powerlaw_k32.txt", "sddmm", 32, r"compulsory bytes per launch\s+4\(m\+1\) \+ 8 nnz \+ 4 m k \+ 4 n k ="),
    ("spmm_t_powerlaw_k32.txt", "spmm_t", 32, "compulsory bytes per launch"),
    ("spmm_merge_kernel_powerlaw_k128.txt", "spmm", 128, "compulsory bytes per launch"),
    ("spmm_t_sddmm_kernel_powerlaw_k32.txt", "backward", 32, "algorithmic bytes per launch"),
    ("spmm_t_sddmm_kernel_powerlaw_k128.txt", "backward", 128, "algorithmic bytes per launch"),
])
def test_powerlaw_summaries_quote_the_launch_model(name, kind, k, label):
    text = _text(name)
    nnz = _powerlaw_nnz(text)
    assert nnz == 16_779_795
    assert _number(text, label) == bench.launch_bytes(POWERLAW_N, POWERLAW_N, nnz, k)[kind]


@pytest.mark.parametrize("name,kind,label", [
    ("spmm_lean_kernel_poisson3d_128_k32.txt", "spmm", "compulsory bytes per launch"),
    ("spmm_t_sddmm_kernel_poisson3d_128_k32.txt", "backward", "algorithmic bytes per launch"),
])
def test_poisson_summaries_quote_the_launch_model(name, kind, label):
    text = _text(name)
    m, nnz = POISSON_128
    assert f"{nnz:,}" in text and f"{m:,}" in text
    assert _number(text, label) == bench.launch_bytes(m, m, nnz, 32)[kind]


@pytest.mark.parametrize("name,k,gb", [("spmm_t_sddmm_kernel_powerlaw_k32.txt", 32, "2.69"),
                                       ("spmm_t_sddmm_kernel_powerlaw_k128.txt", 128, "9.94")])
def test_fused_backward_summaries_quote_the_gather_model(name, k, gb):
    text = _text(name)
    g = bench.gather_bytes(POWERLAW_N, POWERLAW_N, _powerlaw_nnz(text), k)["backward"]
    assert f"{g / 1e9:.2f}" == gb
    assert f"gather model (G's {4 * k}-byte row per entry) {gb} GB" in text
