"""Writes tests/golden/lms_small.json: small seeded inputs and the oracle's
exact LMS fits.  Calls only ``oracle`` (and the input generators).  The paper
prints no worked example (its Fig. 3 with n = 20 is an image that is not
available), so these fixtures pin the oracle against its own history: any
later change to its arithmetic shows up here.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1510_01041_gb300 import datagen  # noqa: E402


def cases():
    yield "line_n64_s1", *datagen.line_with_outliers(64, 1), 0
    yield "line_n128_s2", *datagen.line_with_outliers(128, 2), 0
    yield "line_n257_s3_h100", *datagen.line_with_outliers(257, 3), 100
    x, y, _ = datagen.sloped(200, 4, 0.45)
    yield "sloped_n200_s4", x, y, 0
    x, y, _ = datagen.sloped(96, 5, 0.0, noise=0)
    yield "sloped_exact_n96_s5", x, y, 0


def main():
    out = []
    for name, x, y, h in cases():
        r = oracle.lms_i16(x, y, h, "brute")
        r2 = oracle.lms_i16(x, y, h, "sweep")
        assert r.exact() == r2.exact()
        out.append(dict(name=name, h=h, x=x.tolist(), y=y.tolist(),
                        w_num=r.w_num, w_den=r.w_den, s_num=r.s_num, s_den=r.s_den,
                        t_num=r.t_num, t_den=r.t_den, i=r.i, j=r.j, status=r.status,
                        theta1=r.theta1, theta2=r.theta2, med_sq=r.med_sq))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lms_small.json")
    with open(path, "w") as f:
        json.dump(dict(source="oracle O1 brute force (checked equal to O2 sweep)",
                       cases=out), f, indent=0)
    print("wrote", path)


if __name__ == "__main__":
    main()
