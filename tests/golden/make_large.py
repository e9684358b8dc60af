"""Writes tests/golden/lms_large.json: the oracle's exact LMS fits of the
seeded workload instances at the largest sizes (n = 32768 int16 and float32,
n = 65536 int16), which take the oracle minutes on the host and are too slow
to recompute inside a GPU test run.  Calls only ``oracle`` (the O2 exact
sweep) and the input generators; the points are not stored, they are
regenerated from (generator, n, seed, outlier fraction) on any machine.

    python tests/golden/make_large.py [case-name ...]

With names, only those cases are (re)computed and merged into the file.
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1510_01041_gb300 import datagen  # noqa: E402

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lms_large.json")

# name -> (generator, n, seed, outlier fraction)
CASES = {
    # the single-instance scaling workload at its largest size (40% outliers)
    "line_n32768_s1": ("line_with_outliers", 32768, 1, 0.4),
    # the same workload's float variant (Gaussian inliers on a random line)
    "gauss_f32_n32768_s1": ("gaussian_f32", 32768, 1, 0.4),
    # the learned-proposal workload at its largest size (random slope, 45% outliers)
    "sloped_n65536_s65": ("sloped", 65536, 65, 0.45),
}


def points(gen, n, seed, frac):
    """The instance's coordinates, regenerated from its seed."""
    if gen == "line_with_outliers":
        return datagen.line_with_outliers(n, seed, frac)
    if gen == "sloped":
        x, y, _ = datagen.sloped(n, seed, frac)
        return x, y
    if gen == "gaussian_f32":
        return datagen.gaussian_f32(n, seed, frac)
    raise KeyError(gen)


def solve(name):
    gen, n, seed, frac = CASES[name]
    x, y = points(gen, n, seed, frac)
    t0 = time.perf_counter()
    if gen == "gaussian_f32":
        r = oracle.lms_f32(x, y, 0, "sweep")
    else:
        r = oracle.lms_i16(x, y, 0, "sweep")
    dt = time.perf_counter() - t0
    return dict(generator=gen, n=n, seed=seed, outlier_frac=frac, h=0,
                w_num=r.w_num, w_den=r.w_den, s_num=r.s_num, s_den=r.s_den,
                t_num=r.t_num, t_den=r.t_den, i=r.i, j=r.j, status=r.status,
                scale_exp=r.scale_exp, theta1=r.theta1, theta2=r.theta2, med_sq=r.med_sq,
                oracle="O2 exact sweep", oracle_seconds=round(dt, 1),
                oracle_threads=oracle.max_threads())


def main(names):
    doc = {"source": "oracle O2 exact sweep (tests/golden/make_large.py)", "cases": {}}
    if os.path.exists(PATH):
        with open(PATH) as f:
            doc = json.load(f)
    for name in names or list(CASES):
        doc["cases"][name] = solve(name)
        with open(PATH, "w") as f:
            json.dump(doc, f, indent=1, sort_keys=True)
        print(name, doc["cases"][name], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
