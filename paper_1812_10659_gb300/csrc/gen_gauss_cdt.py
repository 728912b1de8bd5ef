"""Writes gauss_cdt.h: the cumulative table of the discrete Gaussian sampler.

Discrete Gaussian over the integers with sigma = 3.2 truncated to |e| <= 19
(six sigma): rho(k) = exp(-k^2 / (2 sigma^2)).  The sampler draws |e| with
probability rho(0)/S for 0 and 2 rho(k)/S for k >= 1 (S normalises over
-19..19) by comparing a uniform 63-bit integer u against
CDT[k] = floor(2^63 * P(|e| <= k)); the last entry is pinned to 2^63.

Run from this directory:  python gen_gauss_cdt.py > gauss_cdt.h
"""
from decimal import Decimal, localcontext

SIGMA = Decimal(32) / Decimal(10)
BOUND = 19


def table():
    with localcontext() as ctx:
        ctx.prec = 100
        weights = []
        for k in range(BOUND + 1):
            w = (-(Decimal(k * k)) / (2 * SIGMA * SIGMA)).exp()
            weights.append(w if k == 0 else 2 * w)
        total = sum(weights)
        out, run = [], Decimal(0)
        for w in weights:
            run += w
            out.append(int((run / total * (Decimal(2) ** 63)).to_integral_value(rounding="ROUND_FLOOR")))
    out[-1] = 1 << 63
    return out


if __name__ == "__main__":
    vals = table()
    print("// Generated by gen_gauss_cdt.py: cumulative table of the discrete Gaussian")
    print("// (sigma = 3.2, |e| <= 19) scaled by 2^63.  Do not edit.")
    print("#pragma once")
    print("#include <stdint.h>")
    print("static const uint64_t kGaussCdt[%d] = {" % len(vals))
    for v in vals:
        print("    %dull," % v)
    print("};")
