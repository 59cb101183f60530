"""The double-float type of the FP32 path's FP64-class islands (centre rays, near-edge
and near-core rays, GP source) against FP64 on the device, through the C ABI
(rtu_selftest_df), over the argument ranges the islands use.  Inputs are exactly
representable double-float pairs (hi = float(x), lo = float(x - hi)), so the error
is the arithmetic's alone.  The type keeps its precision for values above 2^-100
(there the low float is still normal): exp is tested on [-60, 60], far beyond the
islands' arguments (the softplus's exp(-|x|) stops at |x| = 30, the lens power's
exponent stays within a few units).  Bound: 2^-46 relative (for log: of max(1, |log a|),
i.e. absolute near a = 1; for the sum: of |a| + |b|)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

BOUND = 2.0 ** -46


@pytest.fixture(scope="module")
def rtu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_30620_b300 import rtu as mod
    return mod


def df_exact(x):
    hi = x.astype(np.float32).astype(np.float64)
    lo = (x - hi).astype(np.float32).astype(np.float64)
    return hi + lo


def run(rtu, op, x):
    return rtu.rtu_selftest_df(op, torch.tensor(x, device="cuda")).cpu().numpy()


def test_df_exp(rtu):
    rng = np.random.default_rng(1)
    x = df_exact(np.concatenate([rng.uniform(-1.0, 1.0, 200000), rng.uniform(-30.0, 30.0, 200000),
                                 rng.uniform(-60.0, 60.0, 50000)]))
    y = run(rtu, "exp", x)
    err = np.abs(y - np.exp(x)) / np.exp(x)
    assert err.max() < BOUND, (err.max(), np.log2(err.max()))


def test_df_log(rtu):
    rng = np.random.default_rng(2)
    x = df_exact(np.concatenate([10.0 ** rng.uniform(-8, 8, 200000), rng.uniform(0.5, 2.0, 200000)]))
    y = run(rtu, "log", x)
    ref = np.log(x)
    err = np.abs(y - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() < BOUND, (err.max(), np.log2(err.max()))


def test_df_sqrt(rtu):
    rng = np.random.default_rng(3)
    x = df_exact(10.0 ** rng.uniform(-10, 10, 300000))
    y = run(rtu, "sqrt", x)
    err = np.abs(y - np.sqrt(x)) / np.sqrt(x)
    assert err.max() < BOUND, (err.max(), np.log2(err.max()))


@pytest.mark.parametrize("op", ["div", "mul", "add"])
def test_df_arithmetic(rtu, op):
    rng = np.random.default_rng(4)
    n = 300000
    a = df_exact(rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-3, 3, n))
    b = df_exact(rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-3, 3, n))
    y = run(rtu, op, np.stack([a, b], axis=1))
    if op == "div":
        ref, scale = a / b, np.abs(a / b)
    elif op == "mul":
        ref, scale = a * b, np.abs(a * b)
    else:
        ref, scale = a + b, np.abs(a) + np.abs(b)
    err = np.abs(y - ref) / scale
    assert err.max() < BOUND, (err.max(), np.log2(err.max()))


def test_df_floor_and_edge_distance(rtu):
    """The near-edge pass decides a ray's cell from a double-float grid coordinate: its
    floor must see the low float when the high one has rounded up onto an integer (a
    value 7.6e-7 below 35 has hi = 35.0f), and its distance to the nearest integer
    (a cell edge) must hold to float rounding of that distance."""
    rng = np.random.default_rng(7)
    ints = rng.integers(0, 256, 40000).astype(np.float64)
    off = np.concatenate([-(10.0 ** rng.uniform(-12, -3, 20000)), 10.0 ** rng.uniform(-12, -3, 20000)])
    x = df_exact(np.concatenate([ints + off, rng.uniform(0.0, 255.0, 40000), [35.0 - 7.6e-7, 63.0 - 1e-9, 1e-9]]))
    fl = run(rtu, "floor", x)
    assert np.array_equal(fl, np.floor(x)), x[fl != np.floor(x)][:5]
    d = run(rtu, "edge_dist", x)
    ref = np.abs(x - np.rint(x))
    assert np.all(np.abs(d - ref) <= 2.0 ** -24 * ref + 1e-30), np.max(np.abs(d - ref) / np.maximum(ref, 1e-300))


def test_fixed_point_pair_is_exact(rtu):
    """The cell gather's exact integer corner sums become float pairs by an exact split
    and two-sum: hi + lo equals the integer times 2^-S exactly for |k| < 2^48."""
    rng = np.random.default_rng(8)
    k = np.concatenate([rng.integers(-2 ** 47, 2 ** 47, 50000), rng.integers(-2 ** 24, 2 ** 24, 50000),
                        [0, 1, -1, 2 ** 47 - 1, -(2 ** 47)]]).astype(np.float64)
    S = rng.integers(0, 123, k.size).astype(np.float64)
    y = run(rtu, "fix_pair", np.stack([k, S], axis=1))
    assert np.array_equal(y, k * np.ldexp(1.0, -S.astype(np.int64))), (y[:3], k[:3])
