"""lms_fit_noalloc, the entry point for callers that cannot let the library
allocate device memory (real-time loops that forbid allocation once
running, frameworks that own every device byte through their own pools),
gives the same result as lms_fit's plain path and as the oracle.  Called
directly through the C ABI, twice in a row on different inputs, so the
second call reuses the shared fixed scratch array left by the first; the
capacity edge (n = 1024) and a non-default order statistic are compared with
the oracle, and n = 1025 is refused.  The call is also captured in a CUDA
graph and replayed on new points.  Kept in a file that pytest collects
last."""
import ctypes

import numpy as np
import pytest

from paper_1510_01041_gb300 import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_01041_gb300 import build, lms
    build.build()
    lib = lms.lib()
    lib.lms_fit_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_void_p, ctypes.c_void_p]
    lib.lms_fit_noalloc.restype = ctypes.c_int
    return lms


def _noalloc(L, xt, yt, h=0):
    out = torch.zeros(L.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=xt.device)
    rc = L.lib().lms_fit_noalloc(ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(yt.data_ptr()), xt.numel(),
                                 h, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == L.LMS_OK, L.status_str(rc)
    torch.cuda.synchronize()
    return L.decode(out)[0]


def _same(got, ref):
    return {k: v for k, v in got.items() if k != "algorithm"} == {k: v for k, v in ref.items() if k != "algorithm"}


def test_noalloc_matches_lms_fit_twice(L):
    for seed, n in ((31, 512), (32, 777)):
        x, y = datagen.line_with_outliers(n, seed)
        xt = torch.from_numpy(x).cuda()
        yt = torch.from_numpy(y).cuda()
        got = _noalloc(L, xt, yt)
        ref = L.decode(L.fit(xt, yt, 0, "plain"))[0]
        torch.cuda.synchronize()
        assert _same(got, ref)
        assert got["status"] == L.LMS_OK


@pytest.mark.parametrize("n,h,seed", [(1024, 0, 33), (700, 300, 34), (1024, 1000, 35)])
def test_noalloc_capacity_edge_and_h_vs_oracle(L, orc, n, h, seed):
    x, y = datagen.line_with_outliers(n, seed)
    xt = torch.from_numpy(x).cuda()
    yt = torch.from_numpy(y).cuda()
    for _ in range(2):
        got = _noalloc(L, xt, yt, h)
        o = orc.lms_i16(x, y, h, "sweep")
        assert L.exact_fields(got) == o.exact()
        assert (got["theta1"], got["theta2"], got["med_sq"]) == (o.theta1, o.theta2, o.med_sq)
        ref = L.decode(L.fit(xt, yt, h, "plain"))[0]
        torch.cuda.synchronize()
        assert _same(got, ref)


def test_noalloc_rejects_above_capacity(L):
    for n in (1025, 2000):
        x = torch.zeros(n, dtype=torch.int16, device="cuda")
        out = torch.zeros(L.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        rc = L.lib().lms_fit_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), n, 0,
                                     ctypes.c_void_p(out.data_ptr()), None)
        assert rc == L.LMS_ERR_TOO_LARGE and "capacity" in L.status_str(rc)


def test_noalloc_captured_in_a_cuda_graph(L, orc):
    """After one warm-up call, the call is captured in a CUDA graph on a side
    stream in torch's global capture mode, which refuses the allocation and
    synchronising calls a capture cannot hold.  The graph is replayed on new
    points copied into the same input buffers, and each replay equals the
    oracle.  The replays leave the device's free memory unchanged."""
    n = 900
    x, y = datagen.line_with_outliers(n, 41)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    out = torch.zeros(L.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")

    def call(stream):
        return L.lib().lms_fit_noalloc(ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(yt.data_ptr()), n, 0,
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))

    assert call(torch.cuda.current_stream()) == L.LMS_OK
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            rc = call(s)
    assert rc == L.LMS_OK, L.status_str(rc)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    rng = np.random.default_rng(42)
    for k in range(3):
        y2 = (y.astype(np.int64) + rng.integers(-3, 4, n)).clip(-32768, 32767).astype(np.int16)
        yt.copy_(torch.from_numpy(y2))
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        got = L.decode(out)[0]
        o = orc.lms_i16(x, y2, 0, "sweep")
        assert L.exact_fields(got) == o.exact(), k
        assert (got["theta1"], got["theta2"], got["med_sq"]) == (o.theta1, o.theta2, o.med_sq)
    assert torch.cuda.mem_get_info()[0] == free0
