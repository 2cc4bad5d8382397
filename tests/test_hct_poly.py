"""The far-pair polynomials of the FP32 kernels (cph_device.cuh) against the
exact series they replace, on the whole interval the kernels use them for
(x = s/r <= 0.35): relative error <= 2e-8 in FP64, and <= 4 ulp of FP32 when
evaluated by Horner in FP32 as the kernels do."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1809_07726_gb300", "csrc", "cph_device.cuh")
Y = 0.35 ** 2


def coeffs(name):
    src = open(SRC).read()
    body = re.search(r"T %s\(T y\) \{.*?\n\}" % name, src, re.S).group(0)
    vals = [float(v) for v in re.findall(r"([0-9]+\.[0-9]+)f", body)]
    return vals[::-1]  # Horner lists the highest power first


def exact(kind, y):
    k = np.arange(1, 80)[:, None]
    if kind == "h":
        c = 2 * k / (2 * k + 1)
    elif kind == "dr":
        c = 2 * k * (2 * k + 2) / (2 * k + 1)
    else:
        return 2.0 / (1.0 - y) ** 2
    return (c * y[None, :] ** (k - 1)).sum(0)


@pytest.mark.parametrize("kind", ["h", "dr", "ds"])
def test_far_polynomial_matches_series(kind):
    c = coeffs("hct_series_" + kind)
    assert len(c) == 6
    y = np.linspace(0.0, Y, 4001)
    ex = exact(kind, y)
    approx = np.polynomial.polynomial.polyval(y, c)
    assert np.max(np.abs(approx / ex - 1)) <= 2e-8
    y32 = y.astype(np.float32)
    p = np.float32(c[-1])
    for v in c[-2::-1]:
        p = (p * y32 + np.float32(v)).astype(np.float32)
    assert np.max(np.abs(p.astype(np.float64) / ex - 1)) <= 4 * 2.0 ** -24
