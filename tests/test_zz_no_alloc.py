"""rtu_gp_source_static -- the GP source step for callers that cannot allocate
device memory (an application whose device memory is planned up front, or a
process that must not call cudaMalloc after start-up).  Its scratch is a
static device array inside the library.  Checked through the C ABI against
the workspace path (rtu_forward's source output) on two calls in a row, at
the FP32 tolerance of the parity tests."""
import numpy as np
import pytest
import torch

from paper_2606_30620_b300 import inputs as I

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5


def _workspace_source(rtu, m):
    s = rtu.System.from_mock(m, precision=rtu.RTU_F32)
    b = rtu.Binding(s, m.lens, m.latents, m.ps, want_source=True, grads=False)
    rtu.Batch([b]).forward()
    torch.cuda.synchronize()
    return b.source.cpu().numpy().astype(np.float64)


def test_static_scratch_source_matches_the_workspace_path():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_30620_b300 import rtu
    mocks = [I.config_c2(1100, n_img=64, s=2, n_src=64), I.config_c2(1101, n_img=64, s=2, n_src=96)]
    for m in mocks:                                  # two calls in a row, different sizes
        ref = _workspace_source(rtu, m)
        lat = torch.tensor(m.latents, dtype=torch.float32, device="cuda")
        ps = torch.tensor(m.ps, dtype=torch.float64, device="cuda")
        out = torch.empty_like(lat)
        rtu.rtu_gp_source_static(m.n_src, m.src_pitch, m.ps_family, lat, ps, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel < F32_TOL, (m.n_src, rel)


def test_static_scratch_rejects_sizes_beyond_its_maximum():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_30620_b300 import rtu
    lat = torch.zeros(256, 256, dtype=torch.float32, device="cuda")
    ps = torch.tensor([1.0, 2.0, 1.5], dtype=torch.float64, device="cuda")
    out = torch.empty_like(lat)
    with pytest.raises(rtu.RTUError, match="static scratch"):
        rtu.rtu_gp_source_static(256, 0.05, 1, lat, ps, out)
