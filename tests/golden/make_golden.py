"""Write exact_tiny.json: exact-rational brute-force log-likelihoods of tiny
pulsars (no signal), from oracle/exact.py only.

The paper prints no worked example, so the stored values come from the
definition itself: the Gaussian density of the residual vector under the
integrated-random-walk covariance (paper, Functionality: linear SDE state-space
model with EFAC/EQUAD white noise), evaluated in exact rational arithmetic
(det C and r^T C^-1 r exact; only the final logarithm is rounded).

    python tests/golden/make_golden.py
"""
import json
import math
import os
import sys
from fractions import Fraction as Fr

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import exact  # noqa: E402

CASES = [
    dict(name="one_toa", t=[0.0], r=[2.5e-7], sigma=[1e-7], p0=[1e-14, 0.0, 1e-32],
         sig2=1e-40, efac=1.0, equad=0.0),
    dict(name="two_toa_equal_times", t=[0.0, 0.0], r=[1e-7, -1e-7], sigma=[1e-7, 2e-7],
         p0=[1e-14, 0.0, 1e-32], sig2=1e-40, efac=1.1, equad=0.0),
    dict(name="four_toa", t=[0.0, 1.0e6, 3.5e6, 2.0e7], r=[1e-7, 3e-7, -2e-7, 5e-8],
         sigma=[1e-7, 1e-7, 1.5e-7, 1e-7], p0=[1e-14, 1e-24, 1e-32], sig2=1e-38,
         efac=0.9, equad=5e-8),
    dict(name="six_toa_strong_red", t=[0.0, 2e6, 9e6, 1.1e7, 5e7, 3e8],
         r=[1e-7, 4e-7, 9e-7, 1.2e-6, 3e-6, 2e-5], sigma=[1e-7] * 6,
         p0=[1e-14, 0.0, 1e-30], sig2=1e-36, efac=1.2, equad=0.0),
]


def main():
    out = []
    for c in CASES:
        n = len(c["t"])
        R = [Fr(c["efac"]) ** 2 * Fr(s) ** 2 + Fr(c["equad"]) ** 2 for s in c["sigma"]]
        C = exact.covariance([Fr(x) for x in c["t"]], Fr(c["sig2"]), [Fr(x) for x in c["p0"]], R)
        det, quad = exact.det_and_quad(C, [Fr(x) for x in c["r"]])
        logdet = math.log(det.numerator) - math.log(det.denominator)
        ll = -0.5 * (float(quad) + logdet + n * math.log(2 * math.pi))
        out.append(dict(c, loglik=ll, logdet=logdet, quad=float(quad)))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "exact_tiny.json")
    with open(path, "w") as f:
        json.dump({"source": "oracle/exact.py (exact rational dense Gaussian)", "cases": out},
                  f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
