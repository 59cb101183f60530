"""rtu_gp_source_static -- the GP source step for callers that cannot allocate
device memory: an application whose device memory is planned up front and that
hands this library no workspace, or a process that must not call cudaMalloc
after start-up.  Its scratch is a static device array inside the library.
Checked through the C ABI against the workspace path (rtu_forward's source
output) on two calls in a row, at the FP32 tolerance of the parity tests, and
against the oracle's source for every power-spectrum family and for a field
that sits mostly near f = 0 (where the softplus map is most sensitive)."""
import numpy as np
import pytest
import torch

from oracle import rtu_oracle as O
from paper_2606_30620_b300 import inputs as I
from tests import oracle_io

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5


def _workspace_source(rtu, m):
    s = rtu.System.from_mock(m, precision=rtu.RTU_F32)
    b = rtu.Binding(s, m.lens, m.latents, m.ps, want_source=True, grads=False)
    rtu.Batch([b]).forward()
    torch.cuda.synchronize()
    return b.source.cpu().numpy().astype(np.float64)


def _static_source(rtu, m):
    lat = torch.tensor(m.latents, dtype=torch.float32, device="cuda")
    ps = torch.tensor(m.ps, dtype=torch.float64, device="cuda")
    out = torch.empty_like(lat)
    rtu.rtu_gp_source_static(m.n_src, m.src_pitch, m.ps_family, lat, ps, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _oracle_source(m):
    # the oracle on the same float32-rounded latents the GPU reads
    s = oracle_io.system(m)
    lat = torch.tensor(m.latents.astype(np.float32).astype(np.float64))
    src, _ = O.gp_source(s, lat, torch.tensor(m.ps))
    return src.numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def rtu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_30620_b300 import rtu as mod
    return mod


def test_static_scratch_source_matches_the_workspace_path(rtu):
    mocks = [I.config_c2(1100, n_img=64, s=2, n_src=64), I.config_c2(1101, n_img=64, s=2, n_src=96)]
    for m in mocks:                                  # two calls in a row, different sizes
        ref = _workspace_source(rtu, m)
        got = _static_source(rtu, m)
        assert _rel(got, ref) < F32_TOL, (m.n_src, _rel(got, ref))


@pytest.mark.parametrize("family", [I.PS_POWER_LAW, I.PS_MATERN_LIKE, I.PS_MATERN])
def test_static_scratch_source_matches_the_oracle_for_every_family(rtu, family):
    m = I.config_tiny(seed=120 + family, n_img=16, n_src=48, family=family)
    for _ in range(2):
        assert _rel(_static_source(rtu, m), _oracle_source(m)) < F32_TOL


def test_static_scratch_source_near_zero_field(rtu):
    # a field of rms ~ 1e-3 = s0/10: the source is mostly the softplus near f = 0
    m = I.config_c2(1102, n_img=64, s=2, n_src=128)
    m.ps = m.ps.copy()
    m.ps[0] *= 1e-5
    got, ref = _static_source(rtu, m), _oracle_source(m)
    assert _rel(got, ref) < F32_TOL
    assert _rel(got, _workspace_source(rtu, m)) < F32_TOL


def test_static_scratch_rejects_sizes_beyond_its_maximum(rtu):
    lat = torch.zeros(256, 256, dtype=torch.float32, device="cuda")
    ps = torch.tensor([1.0, 2.0, 1.5], dtype=torch.float64, device="cuda")
    out = torch.empty_like(lat)
    with pytest.raises(rtu.RTUError, match="static scratch"):
        rtu.rtu_gp_source_static(256, 0.05, 1, lat, ps, out)


def test_static_scratch_binding_checks_buffer_sizes(rtu):
    lat = torch.zeros(64, 64, dtype=torch.float32, device="cuda")
    ps = torch.tensor([1.0, 2.0, 1.5], dtype=torch.float64, device="cuda")
    out = torch.empty_like(lat)
    with pytest.raises(ValueError, match="n_src"):
        rtu.rtu_gp_source_static(128, 0.05, 1, lat, ps, out)
    with pytest.raises(ValueError, match="ps must hold"):
        rtu.rtu_gp_source_static(64, 0.05, 2, lat, ps, out)
