"""The allocation-free norm entry point, for callers that cannot allocate
device memory (allocator callbacks, host applications that own every
allocation).  It must report the same residual norms as hhg_residual, on
consecutive calls that share its static scratch array.  This file is
collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

from gpu_helpers import curl_workload, lib_problem, oracle_hierarchy, random_vector

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_norms_match_residual_norms(prec):
    from paper_2010_13513_gb300 import hhg
    lib = hhg.load()
    L = 3
    pb = lib_problem((1, 2, 1), L, "P2P1", lc=1, solve="mixed", workload=curl_workload())
    hy = oracle_hierarchy((1, 2, 1), L, "P2P1", lc=1)
    info = pb.layout(L)
    n_u = 3 * info.groups * info.array_elems
    n_p = info.array_elems
    x = pb.to_device(L, random_vector(hy.lv[L], 11), prec=prec)
    b = pb.to_device(L, random_vector(hy.lv[L], 12), prec=prec)
    r = pb.new_vector(L, prec)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(pb.stream.cuda_stream)
    for call in range(2):
        ref = pb.residual(L, x, b, r, norms=True)
        rc = lib.hhg_block_norms_noalloc(C.c_void_p(r.data_ptr()), prec, n_u, n_p, C.c_void_p(out.data_ptr()), stream)
        assert rc == 0
        pb.stream.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-12, atol=0), (call, got, ref)
        x.mul_(1.5)          # different inputs for the second call


def test_noalloc_rejects_oversized_parts():
    from paper_2010_13513_gb300 import hhg
    lib = hhg.load()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = lib.hhg_block_norms_noalloc(C.c_void_p(x.data_ptr()), 0, 1 << 31, 8, C.c_void_p(out.data_ptr()), None)
    assert rc == -1
    buf = C.create_string_buffer(256)
    lib.hhg_last_error(buf, 256)
    assert b"2^31" in buf.value
