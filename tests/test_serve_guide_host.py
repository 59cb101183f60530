"""The packed prior array a request carries: the same bytes as the ABI's rtu_prior
records built field by field (no device needed)."""
import ctypes

import numpy as np

from paper_2606_30620_b300 import inputs as I
from paper_2606_30620_b300 import rtu, serve


def test_pack_priors_matches_field_by_field_records():
    m = I.config_serving_system(5001)
    pr, ph, loc, rho = serve.guide_start(m)
    arr = rtu.pack_priors(pr)
    assert isinstance(arr, ctypes.Array) and arr._type_ is rtu.Prior and len(arr) == len(pr)
    for row, p in zip(pr, arr):
        assert (p.kind, p.space) == (int(row[0]), int(row[1]))
        assert (p.a, p.b, p.c, p.d) == tuple(float(v) for v in row[2:6])


def test_start_guide_holds_contiguous_float64_arrays():
    m = I.config_serving_system(5002)
    packed, fixed, loc, rho = serve.start_guide(m)
    pr, ph, loc0, rho0 = serve.guide_start(m)
    for a, b in ((fixed, ph), (loc, loc0), (rho, rho0)):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
        np.testing.assert_array_equal(a, np.asarray(b, dtype=np.float64))
    assert len(packed) == len(pr)
