"""The learned fit through host buffers (lms_fit_learned_host): repeated
calls with one size replay a CUDA graph that the library captures on the
second call; each result equals the plain sweep bit for bit, across a new
size (a new graph), a workspace that moves under it (a larger fit grows the
workspace, so the graph is captured again), calls with statistics (direct
calls) in between, and a caller stream of its own."""
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
    return lms


def _same(got, ref):
    return {k: v for k, v in got.items() if k != "algorithm"} == {k: v for k, v in ref.items() if k != "algorithm"}


def test_learned_host_fits_replay_a_cached_graph(L):
    net = L.pretrained()
    launches = []

    def check(n, seed, stats=False, stream=None):
        x, y, _ = datagen.sloped(n, seed, 0.45, phi_max=1.4)
        ref = L.decode(L.fit(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), 0, "sweep"))[0]
        torch.cuda.synchronize()
        l0 = L.launch_count()
        out, st = net.fit_host(x, y, 0, stats=stats, stream=stream)
        launches.append(L.launch_count() - l0)
        got = L.decode(out)[0]
        assert got["status"] == L.LMS_OK
        assert _same(got, ref), (n, seed)
        return st

    for k in range(4):                      # direct, (direct,) captured, replayed
        check(3000, 900 + k)
    for k in range(3):                      # another size: another key
        check(2500, 910 + k)
    L.fit(*(torch.from_numpy(a).cuda() for a in datagen.sloped(20000, 5, 0.45, phi_max=1.4)[:2]), 0, "sweep")
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    for k in range(4):                      # the workspace moved: captured again; a stream of its own
        check(3000, 920 + k, stream=side)
    st = check(3000, 930, stats=True)       # statistics: a direct call
    assert st is not None and st["events_swept"] > 0
    check(3000, 931)
    assert min(launches) > 0                # replays count the launches they hold
