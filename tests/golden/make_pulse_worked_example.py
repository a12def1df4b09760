"""Write ``pulse_worked_example.json``: exact sample values of one voxel's pulse.

Source: the paper's Appendix A, "Uniform Spherical Source" closed form: outside a
uniform sphere of radius a0 and amplitude p0 the pressure is
p(r, t) = p0 (r - v_s t) / (2 r) for r - a0 <= v_s t <= r + a0, and 0 otherwise.

Each sample is that pressure averaged over its sample interval
[t_n - 1/(2 fs), t_n + 1/(2 fs)], t_n = t0 + n / fs.  With tau = v_s t the
integrand is linear in tau, so the average is evaluated here in exact rational
arithmetic (``fractions.Fraction``) by integrating (r - tau) / (2 r) between
the overlap of the sample interval and the support.  No code of the oracle or of
the CUDA library is involved.

Run:  python tests/golden/make_pulse_worked_example.py
"""
from __future__ import annotations

import json
import math
import os
from fractions import Fraction as Fr


def exact_sample(r, n, c, fs, a0, t0):
    h = c / fs
    tau_n = c * (t0 + Fr(n) / fs)
    lo = max(tau_n - h / 2, r - a0)
    hi = min(tau_n + h / 2, r + a0)
    if lo >= hi:
        return Fr(0)

    def prim(tau):  # antiderivative of (r - tau) / (2 r)
        return (r * tau - tau * tau / 2) / (2 * r)

    return (prim(hi) - prim(lo)) / h


CASES = [
    # (distance r in mm, c mm/us, fs MHz, a0 mm, t0 us)
    (Fr(5), Fr(3, 2), Fr(40), Fr(1, 10), Fr(0)),
    (Fr(73, 10), Fr(3, 2), Fr(40), Fr(1, 20), Fr(0)),
    (Fr(1213, 100), Fr(3, 2), Fr(40), Fr(1, 5), Fr(1, 4)),
    (Fr(9), Fr(3, 2), Fr(20), Fr(3, 40), Fr(0)),  # a0 = 2h: support length 4 samples
]


def main():
    out = {"source": "Appendix A, uniform spherical source closed form, averaged "
                     "over each sample interval (exact rational arithmetic)",
           "cases": []}
    for r, c, fs, a0, t0 in CASES:
        h = c / fs
        n_lo = math.floor((r - a0 - c * t0) / h) - 3
        n_hi = math.ceil((r + a0 - c * t0) / h) + 3
        vals = {}
        for n in range(n_lo, n_hi + 1):
            v = exact_sample(r, n, c, fs, a0, t0)
            vals[str(n)] = [f"{v.numerator}/{v.denominator}", float(v)]
        out["cases"].append({"r_mm": str(r), "c_mm_per_us": str(c), "fs_mhz": str(fs),
                             "a0_mm": str(a0), "t0_us": str(t0), "samples": vals})
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pulse_worked_example.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
