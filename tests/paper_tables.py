"""Readers for the paper's printed values under tests/golden/ and the integrands
of its Section 5 tables, shared by the oracle pins and the GPU tests."""
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


def one_unit(printed: str) -> float:
    """One unit in the last printed digit of a value such as '7.7798e-3'."""
    mant, exp = printed.lower().split("e")
    decimals = len(mant.split(".")[1]) if "." in mant else 0
    return 10.0 ** (int(exp) - decimals)


def midpoint_case(integrand, d):
    """(family, c, w) of the Section 5 integrands in the product families:
    gauss = (2 pi)^(-1/2) exp(-|x|^2/2) (the constant cancels in relative errors),
    expalt = exp(sum_i (-1)^(i+1) x_i), peak = prod_i 1/(0.9^2 + (x_i - 0.6)^2),
    cos2 = cos(2 pi + 2 sum_i x_i)."""
    if integrand == "gauss":
        return "gauss", np.full(d, 1.0 / math.sqrt(2.0)), np.zeros(d)
    if integrand == "expalt":
        return "exp", np.array([(-1.0) ** i for i in range(d)]), np.zeros(d)
    if integrand == "peak":
        return "peak", np.full(d, 1.0 / 0.9), np.full(d, 0.6)
    if integrand == "cos2":
        w = np.zeros(d)
        w[0] = 1.0  # cos(2 pi u + ...) with u = 1
        return "osc", np.full(d, 2.0), w
    raise KeyError(integrand)
