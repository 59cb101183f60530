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
