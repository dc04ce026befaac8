"""The Python binding's argument checks, which run before any call into the
library (no GPU): candidate widths (int32, or 16-bit for ops and off both) and
shapes of host buffers, and the device entry points failing loudly when there
is no CUDA device."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import paper_2602_23685_gb300 as vrp


def fake(n=4, m=2):
    return SimpleNamespace(n=n, m=m, handle=None)


def test_16bit_dtypes_recognised():
    assert vrp._is16(torch.int16) and vrp._is16(np.dtype(np.int16)) and vrp._is16(np.dtype(np.uint16))
    assert not vrp._is16(torch.int32) and not vrp._is16(np.dtype(np.int32)) and not vrp._is16(np.dtype(np.int64))


def test_host_path_rejects_mixed_or_wrong_widths():
    inst = fake()
    o32, f32 = np.zeros((3, 8), np.int32), np.zeros((3, 3), np.int32)
    with pytest.raises(TypeError):
        vrp.evaluate_host(inst, o32, f32.astype(np.int16))
    with pytest.raises(TypeError):
        vrp.evaluate_host(inst, o32.astype(np.int16), f32)
    with pytest.raises(TypeError):
        vrp.evaluate_host(inst, o32.astype(np.int64), f32.astype(np.int64))
    with pytest.raises(TypeError):
        vrp.evaluate_host(inst, torch.zeros((3, 8), dtype=torch.int16), torch.zeros((3, 3), dtype=torch.int32))


def test_host_path_rejects_bad_shapes():
    with pytest.raises(ValueError):
        vrp.evaluate_host(fake(), np.zeros((3, 7), np.int32), np.zeros((3, 3), np.int32))
    with pytest.raises(ValueError):
        vrp.evaluate_host(fake(), np.zeros((3, 8), np.int16), np.zeros((3, 4), np.int16))


def test_device_path_fails_loudly_without_a_gpu():
    # no CPU fallback: without a CUDA device the device entry points raise
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    inst = fake()
    with pytest.raises(RuntimeError):
        vrp.evaluate(inst, torch.zeros((3, 8), dtype=torch.int32), torch.zeros((3, 3), dtype=torch.int32))
    with pytest.raises(RuntimeError):
        vrp.evaluate_plain(inst, torch.zeros((3, 8), dtype=torch.int32), torch.zeros((3, 3), dtype=torch.int32))
