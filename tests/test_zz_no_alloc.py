"""The allocation-free entry point gsvd_solve_small_noalloc (GPU).

It serves callers that may not allocate device memory (their device memory is
owned by a pool allocator, or a cudaMalloc would synchronize the device at a
bad time): its kernel's scratch is a fixed array inside the library.  This
file is collected last on purpose.  Each test calls the entry point through
the C ABI twice in a row, on different problems, and checks every output
against the ordinary entry point (gsvd_solve) within the tolerance of the
other parity tests, so a second call cannot be influenced by what the first
left in the shared array.
"""
import ctypes

import numpy as np
import pytest

from paper_1909_00101_gb300.inputs import make_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00101_gb300.build import build
    build()
    import paper_1909_00101_gb300 as m
    m.load_library()
    return m


def _dev(a):
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def _batch(seed0):
    shapes = [(64, 48, 32, False), (40, 33, 33, True), (20, 17, 7, False), (9, 8, 2, True), (70, 70, 64, False),
              (5, 3, 1, False), (30, 25, 12, True)]
    return [make_pair(mf, mg, n, cplx=c, seed=seed0 + k) for k, (mf, mg, n, c) in enumerate(shapes)]


def _compare(hz, pairs, res):
    for p, r in zip(pairs, res):
        assert r.info["status"] == 0, r.info
        ref = hz.solve(_dev(p.F), _dev(p.G), path="pointwise")
        assert ref.status == 0
        sig, sref = r.sigma.cpu().numpy(), ref.sigma.cpu().numpy()
        assert np.max(np.abs(sig - sref) / sref) <= 1e-12
        for a, b in ((r.Z, ref.Z), (r.U, ref.U), (r.V, ref.V)):
            assert torch.allclose(a, b, rtol=1e-10, atol=1e-12)
        assert np.max(np.abs(r.sigma_f.cpu().numpy() - ref.sigma_f.cpu().numpy())) <= 1e-12


def test_noalloc_two_calls_match_the_ordinary_entry_point(hz):
    first = _batch(300)
    st, res = hz.solve_small_noalloc([(_dev(p.F), _dev(p.G)) for p in first])
    assert st == 0
    _compare(hz, first, res)
    second = _batch(400)[::-1]
    st, res = hz.solve_small_noalloc([(_dev(p.F), _dev(p.G)) for p in second])
    assert st == 0
    _compare(hz, second, res)


def test_noalloc_rejects_out_of_range_requests(hz):
    lib = hz.load_library()
    p = make_pair(70, 70, 65, seed=1)                 # n = 65 > 64: not a small problem
    st, _ = hz.solve_small_noalloc([(_dev(p.F), _dev(p.G))])
    assert st == hz.ETOOBIG
    arr = (hz.Problem * 1)()
    assert lib.gsvd_solve_small_noalloc(arr, hz.NOALLOC_MAX_PROBLEMS + 1, None, None, None) == hz.ETOOBIG
    q = make_pair(10, 10, 5, seed=2)                   # host (numpy) buffers are refused
    F = np.asfortranarray(q.F)
    G = np.asfortranarray(q.G)
    Z = np.zeros((5, 5), order="F")
    v = np.zeros(5)
    prob = hz._problem(F, G, Z, v, v, v, False)
    assert lib.gsvd_solve_small_noalloc(ctypes.byref(prob), 1, None, None, None) == hz.EINVAL
    # after the rejections a valid call still works
    st, res = hz.solve_small_noalloc([(_dev(q.F), _dev(q.G))])
    assert st == 0 and res[0].info["status"] == 0
