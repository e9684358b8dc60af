"""What the trained proposal gains, measured on held-out instances of the
learned-proposal workload (n = 8192, random slope angle in (-1.4, 1.4), 45%
outliers), against the method without it.

* The trained network predicts the LMS angle far better than the untrained
  network and than a constant guess.
* Exactness: the learned-seeded branch-and-bound, the branch-and-bound seeded
  at sample quantiles (the method without the network) and the one seeded at
  evenly spaced angles (no look at the data) all return the plain sweep's
  result bit for bit.
* Measured relation: both data-driven seedings sweep a small fraction of the
  candidate pairs and far fewer than angle seeding; the learned seeding
  matches quantile seeding (their swept events agree within a factor of 1.5
  either way) but does not beat it: after the zoom rounds both upper bounds
  sit within about 10^-3 of the optimum.
"""
import os

import numpy as np
import pytest

from paper_1510_01041_gb300 import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

F = ("status", "w_num", "w_den", "s_num", "s_den", "t_num", "t_den", "i", "j", "theta1", "theta2", "med_sq")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_01041_gb300 import build, lms
    build.build()
    if not os.path.exists(lms.WEIGHTS):
        pytest.skip("no trained weights")
    return lms


def _timed(fn):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    out, st = fn()
    b.record()
    torch.cuda.synchronize()
    return out, st, a.elapsed_time(b)


def test_learned_seeding_against_the_method_without_it(L):
    trained = L.pretrained()
    untrained = L.SetNet(seed=123)
    err_t, err_u, err_c = [], [], []
    swept = {"learned": [], "quantiles": [], "angles": []}
    ms = {"learned": [], "quantiles": []}
    total = []
    L.reserve(8192, algorithm="bnb")
    for k in range(8):
        x, y, _ = datagen.sloped(8192, 77000 + k, 0.45, phi_max=1.4)
        xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        off = torch.tensor([0, x.size], dtype=torch.int64, device="cuda")
        ref = L.decode(L.fit(xt, yt, 0, "sweep"))[0]
        target = float(np.arctan(ref["theta1"]))
        err_t.append(abs(float(trained.forward(xt, yt, off)[0, 0]) - target))
        err_u.append(abs(float(untrained.forward(xt, yt, off)[0, 0]) - target))
        err_c.append(abs(target))
        for arm, fn in (("learned", lambda: trained.fit(xt, yt)),
                        ("quantiles", lambda: L.fit_bnb(xt, yt, 0, None, seed_mode="quantiles")),
                        ("angles", lambda: L.fit_bnb(xt, yt, 0, None, seed_mode="angles"))):
            fn()                                  # warm
            out, st, t = _timed(fn)
            r = L.decode(out)[0]
            assert {q: r[q] for q in F} == {q: ref[q] for q in F}, (k, arm, r, ref)
            swept[arm].append(st["events_swept"])
            if arm in ms:
                ms[arm].append(t)
            total.append(st["events_total"])
    assert np.mean(err_t) < 0.5 * np.mean(err_u)
    assert np.mean(err_t) < 0.5 * np.mean(err_c)
    sl, sq, sa = (float(np.sum(swept[a])) for a in ("learned", "quantiles", "angles"))
    info = dict(events_learned=sl, events_quantiles=sq, events_angles=sa, events_total=float(np.sum(total)) / 3,
                ms_learned=float(np.median(ms["learned"])), ms_quantiles=float(np.median(ms["quantiles"])),
                angle_err_trained=float(np.mean(err_t)))
    assert sl < 0.01 * info["events_total"] and sq < 0.01 * info["events_total"], info
    assert sl < sa and sq < sa, info
    assert sl <= 1.5 * sq and sq <= 1.5 * sl, info
