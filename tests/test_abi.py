"""The C ABI without a GPU: the library loads and exports every entry point of
include/pscl.h, and the binding declares exactly those."""
import os
import re
import subprocess

import pytest

from paper_1412_1947_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "pscl.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pscl_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_function():
    lib = binding.lib()
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pscl_\w+)", out))
    assert set(names) <= exported


def test_binding_covers_the_header():
    assert sorted(binding.SIGNATURES) == header_functions()


def test_errors_are_status_codes_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(binding.PsclError) as e:
        binding.pscl_ctx_create(0)
    assert e.value.code == binding.PSCL_ECUDA
    assert binding.lib().pscl_last_error()


def test_null_arguments_are_rejected():
    lib = binding.lib()
    assert lib.pscl_ctx_create(None, 0, 0, None) == binding.PSCL_EINVAL
    assert lib.pscl_job_sync(None) == binding.PSCL_EINVAL
    assert lib.pscl_scale_features(None) == binding.PSCL_EINVAL
    assert b"NULL" in lib.pscl_last_error()
    assert lib.pscl_measure_fp32_fma(0, None) == binding.PSCL_EINVAL


@pytest.mark.gpu
def test_measured_fma_rate_is_plausible():
    # 152 SMs x 128 lanes x 2 flop at 1-2.1 GHz: between about 39 and 81 TFLOP/s; the
    # bound is loose on both sides so that clocks under another load still pass
    t = binding.pscl_measure_fp32_fma(0)
    assert 20.0 < t < 100.0, t


def test_grid_barrier_measurement_rejects_null():
    lib = binding.lib()
    assert lib.pscl_measure_grid_barrier(0, None) == binding.PSCL_EINVAL


@pytest.mark.gpu
def test_measured_grid_barrier_is_plausible():
    us = binding.pscl_measure_grid_barrier(0)
    assert 0.05 < us < 100.0
