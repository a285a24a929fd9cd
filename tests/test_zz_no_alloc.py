"""The allocation-free MGS entry point (iga_mgs_noalloc) against the context
path (iga_mgs), called through the C ABI, twice in a row.

iga_mgs_noalloc exists for callers that cannot call cudaMalloc: it keeps its
reduction scratch in a static device array instead of a context.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it passes alone in a fresh process and after the others."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _basis(n, k, seed):
    rng = np.random.default_rng(seed)
    q = np.linalg.qr(rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k)))[0]
    return torch.from_numpy(np.ascontiguousarray(q.T)).cuda()          # rows = basis vectors


def test_mgs_noalloc_matches_context_path_twice():
    from paper_2010_10232_gb300.solver import from_problem
    from paper_2010_10232_gb300 import _ffi
    L = _ffi.lib()
    h = from_problem(W.small_2d(n_el=24, p=2, k=10.0))
    n = h.n
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (k, j, seed) in enumerate([(7, 5, 1), (4, 2, 2)]):
        V = _basis(n, k, seed)
        w0 = torch.from_numpy(W.seeded_complex_vector(n, 10 + seed)).cuda()
        w_ref = w0.clone()
        h_ref = h.mgs(V, j, w_ref)                                          # context path
        w_na = w0.clone()
        h_na = torch.zeros(j + 2, dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        reserved_before = torch.cuda.memory_reserved()
        rc = L.iga_mgs_noalloc(C.c_void_p(V.data_ptr()), n, n, j, C.c_void_p(w_na.data_ptr()),
                               C.c_void_p(h_na.data_ptr()), stream)
        assert rc == 0, f"call {call}: status {rc}"
        torch.cuda.synchronize()
        if call > 0:        # after the first call (module load, address lookup) nothing is allocated
            assert torch.cuda.mem_get_info()[0] == free_before
            assert torch.cuda.memory_reserved() == reserved_before
        np.testing.assert_allclose(h_na.cpu().numpy(), h_ref.cpu().numpy(), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(w_na.cpu().numpy(), w_ref.cpu().numpy(), rtol=1e-12, atol=1e-12)


def test_mgs_noalloc_rejects_bad_sizes():
    from paper_2010_10232_gb300 import _ffi
    L = _ffi.lib()
    buf = torch.zeros(64, dtype=torch.complex128, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.iga_mgs_noalloc(p, 8, 16, 0, p, p, s) == -1       # ldv < n
    assert L.iga_mgs_noalloc(p, 16, 0, 0, p, p, s) == -1       # n = 0
    assert L.iga_mgs_noalloc(p, 16, 16, -1, p, p, s) == -1     # j < 0
    assert L.iga_mgs_noalloc(C.c_void_p(buf.data_ptr() + 8), 16, 16, 0, p, p, s) == -1   # misaligned
