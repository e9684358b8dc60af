"""What the trained proposal gains.  On held-out sets of the learned-proposal
workload (random slope, 45% outliers): the trained network predicts the LMS
angle better than the untrained network and than a constant guess, and its
seeds let branch-and-bound sweep fewer candidate pairs than seeds that do
not look at the data (evenly spaced angles) -- with the exact answer
unchanged."""
import os

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
    if not os.path.exists(lms.WEIGHTS):
        pytest.skip("no trained weights")
    return lms


def test_trained_network_gains(L, orc):
    trained = L.pretrained()
    untrained = L.SetNet(seed=123)
    err_t, err_u, err_c = [], [], []
    swept_learned, swept_blind = 0, 0
    for k in range(10):
        x, y, _ = datagen.sloped(2048, 77000 + k, 0.45, phi_max=1.4)
        xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        off = torch.tensor([0, x.size], dtype=torch.int64, device="cuda")
        o = orc.lms_i16(x, y, 0, "sweep")
        target = float(np.arctan(o.theta1))
        err_t.append(abs(float(trained.forward(xt, yt, off)[0, 0]) - target))
        err_u.append(abs(float(untrained.forward(xt, yt, off)[0, 0]) - target))
        err_c.append(abs(target))
        out, st = trained.fit(xt, yt)
        r = L.decode(out)[0]
        assert (r["w_num"], r["s_num"], r["s_den"], r["t_num"], r["i"], r["j"]) == \
               (o.w_num, o.s_num, o.s_den, o.t_num, o.i, o.j)
        swept_learned += st["events_swept"]
        out2, st2 = L.fit_bnb(xt, yt, 0, None, seed_mode="angles")
        assert L.decode(out2)[0]["w_num"] == o.w_num
        swept_blind += st2["events_swept"]
    assert np.mean(err_t) < np.mean(err_u)
    assert np.mean(err_t) < np.mean(err_c)
    assert swept_learned < swept_blind
