"""The subhalo deflection bound the render's tile cull and early exit use: a subhalo
deflects by 4 kappa_s r_s g(x)/x (x = r/r_s, App. A), and the kernels take
|alpha| <= SUB_ALPHA_PER_KR kappa_s r_s for every ray position.  Its premises, checked
with the oracle's projected-mass functions (no device needed): the NFW function h is
increasing, the truncated function lies below it for every truncation, and
sup h(x)/x is below 0.32 (the grid's spacing accounted for)."""
import math
import os
import re

import torch

from oracle import rtu_oracle as O

RATIO = 1.01
X = torch.tensor([1e-3 * RATIO ** k for k in range(int(round(math.log(1e7) / math.log(RATIO))) + 1)],
                 dtype=torch.float64)


def test_nfw_mass_function_is_increasing_and_its_ratio_bounded():
    h = O._nfw_mass_fn(X)
    assert bool((h[1:] > h[:-1]).all())
    # between grid points x_i < x < x_i RATIO: h(x)/x <= h(x_i RATIO)/x_i = RATIO h/x at x_{i+1}
    r = h / X
    assert float(r.max()) * RATIO <= 0.32
    assert abs(float(r.max()) - 0.3105) < 1e-3
    # beyond the grid: h(x)/x rises towards the grid's low end and falls past its high end
    assert bool((r[:200][1:] > r[:200][:-1]).all())
    assert float(r[-1]) < 1e-2


def test_truncated_mass_function_lies_below_the_nfw_one():
    h = O._nfw_mass_fn(X)
    for tau in (0.3, 1.0, 3.0, 10.0, 30.0, 100.0):
        g = O._tnfw_mass_fn(X, torch.tensor(tau, dtype=torch.float64))
        assert bool((g <= h * (1 + 1e-9) + 1e-15).all()), tau
        assert bool((g >= 0).all()), tau


def test_kernel_constant_covers_the_bound():
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2606_30620_b300", "csrc",
                            "rtu_internal.cuh")).read()
    c = float(re.search(r"constexpr double SUB_ALPHA_PER_KR = ([0-9.]+);", src).group(1))
    assert c >= 4 * 0.32


def test_deflection_magnitude_within_the_bound():
    # the oracle's deflection itself, at positions around one subhalo of each kind
    r = X * 0.02
    x, y = 0.3 + r * 0.6, -0.1 + r * 0.8
    for kind in (O.SUB_NFW, O.SUB_TNFW):
        ax, ay = O.deflection_nfw(x, y, torch.tensor(1.7, dtype=torch.float64), torch.tensor(0.02, dtype=torch.float64),
                                  torch.tensor(8.0, dtype=torch.float64), 0.3, -0.1, kind)
        mag = torch.sqrt(ax * ax + ay * ay)
        assert float(mag.max()) <= 1.28 * 1.7 * 0.02
