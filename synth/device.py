"""Seeded device-side field generator (torch) for the large batched and
served workloads, where host generation would dominate the run.  Same recipe
as ``fields.grf`` (|u_hat(k)| ~ k^slope, random phases, rescaled to [-1, 1])
with torch's generator, so the numbers differ from the numpy version."""
import math


def grf_torch(shape, seed, device="cuda", dtype=None, slope=None):
    import torch
    dtype = dtype or torch.float32
    nd = len(shape)
    if slope is None:
        slope = -11.0 / 6.0 if nd == 3 else -4.0 / 3.0
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    freqs = [torch.fft.fftfreq(s, device=device) * s for s in shape[:-1]]
    freqs.append(torch.fft.rfftfreq(shape[-1], device=device) * shape[-1])
    k2 = None
    for ax, f in enumerate(freqs):
        sh = [1] * nd
        sh[ax] = f.numel()
        t = (f.reshape(sh) ** 2).float()
        k2 = t if k2 is None else k2 + t
    k = torch.sqrt(k2)
    k.view(-1)[0] = 1.0
    amp = k.pow(slope)
    amp.view(-1)[0] = 0.0
    phase = torch.rand(amp.shape, generator=g, device=device) * (2 * math.pi)
    spec = torch.polar(amp, phase)
    del amp, phase, k, k2
    f = torch.fft.irfftn(spec, s=shape)
    del spec
    lo, hi = f.min(), f.max()
    f = (f - lo) * (2.0 / (hi - lo)) - 1.0
    return f.to(dtype).contiguous()
