"""pkasp_pmis_noalloc: the PMIS C/F splitting for callers that cannot let a library
allocate device memory (a process that reserved all GPU memory for its own pool, or code
that must not synchronize the device, as cudaMalloc/cudaFree do). It keeps its scratch in
a fixed array inside the library. Checked through the C ABI against the allocating
pkasp_pmis on the same inputs, on two calls in a row: the splittings are integers and
must be identical. (This file is collected last on purpose.)"""
import ctypes as C

import numpy as np
import pytest

from paper_1204_2586_gb300.inputs import kappa_lognormal, kuhn_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_2586_gb300 import build

    build.build()
    return torch


def _strength_graph(oracle_mod, n, seed):
    xyz, t = kuhn_mesh(n, 0.2, seed)
    P = oracle_mod.Problem(xyz, t, 2, kappa_lognormal(t.shape[0], seed + 1))
    A = P.matrix(1)
    return A, oracle_mod.strength(A, 0.25)


def _run(torch, fn, A, strong, stream_id):
    from paper_1204_2586_gb300 import _lib as L

    ptr = torch.tensor(A.ptr, device="cuda")
    col = torch.tensor(A.col, device="cuda")
    st = torch.tensor(strong, device="cuda")
    n = A.shape[0]
    cf = torch.full((n,), 7, dtype=torch.int8, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(n, ptr.data_ptr(), col.data_ptr(), st.data_ptr(), stream_id, cf.data_ptr(), s)
    assert rc == L.PKASP_OK, L.last_error()
    torch.cuda.synchronize()
    return cf.cpu().numpy()


def test_noalloc_matches_allocating_pmis_twice(torch_cuda, oracle_mod):
    from paper_1204_2586_gb300 import _lib as L

    lib = L.load()
    for n, seed, stream_id in ((8, 0, 32), (20, 3, 33)):
        A, strong = _strength_graph(oracle_mod, n, seed)
        ref = _run(torch_cuda, lib.pkasp_pmis, A, strong, stream_id)
        assert set(np.unique(ref)) <= {-1, 1}
        first = _run(torch_cuda, lib.pkasp_pmis_noalloc, A, strong, stream_id)
        second = _run(torch_cuda, lib.pkasp_pmis_noalloc, A, strong, stream_id)
        assert np.array_equal(first, ref)
        assert np.array_equal(second, ref)


def test_noalloc_rejects_inputs_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    from paper_1204_2586_gb300 import _lib as L

    lib = L.load()
    tiny = torch.zeros(4, dtype=torch.int64, device="cuda")
    n = 262144 + 1  # PKASP_NOALLOC_MAX_ROWS + 1
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.pkasp_pmis_noalloc(n, tiny.data_ptr(), tiny.data_ptr(), tiny.data_ptr(), 0, tiny.data_ptr(), s)
    assert rc == L.PKASP_EINVAL
    assert "exceed" in L.last_error()


def _call(torch, ptr, col, n, strong=None):
    from paper_1204_2586_gb300 import _lib as L

    lib = L.load()
    p = torch.tensor(ptr, dtype=torch.int64, device="cuda")
    c = torch.tensor(col if len(col) else [0], dtype=torch.int32, device="cuda")
    st = torch.ones(max(len(col), 1), dtype=torch.uint8, device="cuda") if strong is None else strong
    cf = torch.zeros(max(n, 1), dtype=torch.int8, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.pkasp_pmis_noalloc(n, p.data_ptr(), c.data_ptr(), st.data_ptr(), 0, cf.data_ptr(), s)
    return rc, L.last_error() if rc else ""


def test_noalloc_rejects_entries_beyond_its_scratch(torch_cuda):
    """ptr[n] above PKASP_NOALLOC_MAX_NNZ is rejected before any kernel runs (only ptr[n]
    is read), so the fixed array is never written past its end."""
    from paper_1204_2586_gb300 import _lib as L

    rc, msg = _call(torch_cuda, [0, 0, 0, 4194304 + 1], [], 3)
    assert rc == L.PKASP_EINVAL and "exceed" in msg


@pytest.mark.parametrize("ptr,col,what", [
    ([0, 2, 3, 4], [0, 1, 1, 2], "symmetric"),   # (0, 1) without (1, 0)
    ([0, 2, 4, 5], [1, 0, 0, 1, 2], "ascending"),  # row 0 unsorted
    ([0, 2, 3, 4], [0, 5, 1, 2], "outside"),       # column 5 of 3 rows
    ([0, 2, 1, 3], [0, 1, 2], "decrease"),         # row pointers go back
])
def test_noalloc_rejects_malformed_patterns(torch_cuda, ptr, col, what):
    from paper_1204_2586_gb300 import _lib as L

    rc, msg = _call(torch_cuda, ptr, col, 3)
    assert rc == L.PKASP_EINVAL, (rc, msg)
    assert what in msg


def test_noalloc_allocates_no_device_memory(torch_cuda, oracle_mod):
    """Free device memory is the same before and after three calls (after a first call
    has loaded the module and its fixed array): the entry point allocates nothing."""
    torch = torch_cuda
    from paper_1204_2586_gb300 import _lib as L

    lib = L.load()
    A, strong = _strength_graph(oracle_mod, 8, 1)
    _run(torch, lib.pkasp_pmis_noalloc, A, strong, 40)
    ptr = torch.tensor(A.ptr, device="cuda")
    col = torch.tensor(A.col, device="cuda")
    st = torch.tensor(strong, device="cuda")
    cf = torch.empty(A.shape[0], dtype=torch.int8, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rc = lib.pkasp_pmis_noalloc(A.shape[0], ptr.data_ptr(), col.data_ptr(), st.data_ptr(), 40,
                                    cf.data_ptr(), s)
        assert rc == L.PKASP_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
