"""Turn a seeded input (paper_2606_30620_b300.inputs.Mock) into oracle arguments."""
import torch

from oracle import rtu_oracle as O


def system(m):
    return O.System(data=torch.tensor(m.data), mask=torch.tensor(m.mask).bool(),
                    psf=torch.tensor(m.psf), sigma=m.sigma, pix=m.pix, s_super=m.s_super,
                    n_src=m.n_src, src_pitch=m.src_pitch, profile=m.profile,
                    ps_family=m.ps_family, sub_kind=m.sub_kind,
                    weights=None if m.weights is None else torch.tensor(m.weights.astype("int64")))


def params(m):
    subs = None if m.subs is None else torch.tensor(m.subs)
    return torch.tensor(m.lens), torch.tensor(m.latents), torch.tensor(m.ps), subs


def light(m):
    return None if m.light is None else torch.tensor(m.light)
