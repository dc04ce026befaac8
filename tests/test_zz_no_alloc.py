"""The allocation-free plain evaluation entry point.

Callers that may not let the library allocate device memory (while recording
a CUDA graph, under a fixed serving memory budget, or next to a caching
allocator that holds the free memory) use vrprpd_evaluate_plain_noalloc, which
works out of a fixed scratch array inside the library.  This file is collected
last; it calls the entry point through the C ABI twice in a row with different
batches and checks each result, candidate by candidate, against the oracle and
against the batched entry point vrprpd_evaluate.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def call_noalloc(vrp, inst, ops, off):
    import torch
    L = vrp.lib()
    fn = L.vrprpd_evaluate_plain_noalloc
    fn.argtypes = [C.c_void_p, C.POINTER(vrp.Batch), C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    B = ops.shape[0]
    z = torch.full((B,), -7, dtype=torch.int32, device="cuda")
    st = torch.full((B,), -7, dtype=torch.int32, device="cuda")
    b = vrp.Batch(B, ops.data_ptr(), off.data_ptr())
    rc = fn(inst.handle, C.byref(b), z.data_ptr(), st.data_ptr(),
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.vrprpd_last_error()
    torch.cuda.synchronize()
    return z, st


def test_noalloc_matches_batched_twice(vrp):
    import torch
    w = workloads.make_instance(100, 4, 10, 5, "2x", seed=11)
    inst = vrp.Instance.from_workload(w)
    oi = oracle.OracleInstance.from_workload(w)
    for call, seed in enumerate((1, 2)):
        o1, f1 = workloads.precedence_candidates(w.n, w.m, 3000, seed=seed)
        o2, f2 = workloads.random_candidates(w.n, w.m, 1000, seed=seed + 10)
        ho, hf = np.concatenate([o1, o2]), np.concatenate([f1, f2])
        ops = torch.from_numpy(ho).cuda()
        off = torch.from_numpy(hf).cuda()
        z, st = call_noalloc(vrp, inst, ops, off)
        zo, so = oracle.evaluate_batch(oi, ho, hf)
        assert np.array_equal(z.cpu().numpy(), zo), f"makespans differ from the oracle on call {call}"
        assert np.array_equal(st.cpu().numpy().astype(np.uint32), so), f"status differs from the oracle on call {call}"
        zr, sr = vrp.evaluate(inst, ops, off)
        torch.cuda.synchronize()
        assert torch.equal(z, zr), f"makespans differ on call {call}"
        assert torch.equal(st, sr), f"status differs on call {call}"
