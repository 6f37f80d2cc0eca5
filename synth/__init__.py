"""Seeded synthetic fields shaped like the paper's workloads (Table 1 shapes).

This module only draws inputs; it holds none of the compressor's arithmetic and is shared by
the oracle tests, the GPU tests, ``__graft_entry__.smoke()`` and ``bench.py``.

Recipe (one field): x = sum over m = 1..8 of sin(2*pi*sum_a f_ma * p_a / n_a + phi_m), with
integer frequencies f_ma uniform in 1..6 per axis, phases phi_m uniform in [0, 2*pi), amplitude
1, p_a the integer coordinate along axis a and n_a that axis' length; plus Gaussian noise of
standard deviation 1e-3. Optionally 1% of the points (chosen uniformly, duplicates merged) get
a heavy-tailed spike +-LogNormal(0, sigma=2). Everything is computed in float64 with numpy's
PCG64 generator and rounded to the requested dtype at the end.
"""

from __future__ import annotations

import numpy as np


def sinusoid_field(shape, seed: int, dtype=np.float32, noise: float = 1e-3, spikes: float = 0.0,
                   n_modes: int = 8) -> np.ndarray:
    shape = tuple(int(n) for n in shape)
    nd = len(shape)
    rng = np.random.default_rng(seed)
    freqs = rng.integers(1, 7, size=(n_modes, nd))
    phases = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    out = np.empty(shape, dtype=dtype)
    if out.size == 0:
        return out
    # angle along each axis for every mode
    ang = [[2.0 * np.pi * freqs[m, a] * np.arange(shape[a], dtype=np.float64) / shape[a] for a in range(nd)]
           for m in range(n_modes)]
    if nd == 1:
        acc = np.zeros(shape[0])
        for m in range(n_modes):
            acc += np.sin(ang[m][0] + phases[m])
        acc += noise * rng.standard_normal(shape[0])
        out[...] = acc
    else:
        # sin(a0 + rest) = sin(a0) cos(rest) + cos(a0) sin(rest); rest covers the faster axes
        rest_sin, rest_cos = [], []
        for m in range(n_modes):
            r = phases[m]
            grids = np.meshgrid(*ang[m][1:], indexing="ij")
            tot = np.full(shape[1:], r)
            for gax in grids:
                tot = tot + gax
            rest_sin.append(np.sin(tot))
            rest_cos.append(np.cos(tot))
        for i in range(shape[0]):
            acc = np.zeros(shape[1:])
            for m in range(n_modes):
                a0 = ang[m][0][i]
                acc += np.sin(a0) * rest_cos[m] + np.cos(a0) * rest_sin[m]
            acc += noise * rng.standard_normal(shape[1:])
            out[i] = acc
    if spikes > 0.0:
        n = out.size
        k = max(1, int(round(spikes * n)))
        idx = np.unique(rng.integers(0, n, size=k))
        sign = rng.integers(0, 2, size=idx.size) * 2 - 1
        mag = rng.lognormal(0.0, 2.0, size=idx.size)
        flat = out.reshape(-1)
        flat[idx] = (flat[idx].astype(np.float64) + sign * mag).astype(dtype)
    return out


def integer_field(shape, seed: int, lo: int = -50, hi: int = 50, dtype=np.float32) -> np.ndarray:
    """Uniform random small integers (exactly representable); used for exactness checks."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=shape).astype(dtype)


def device_field(shape, seed, dtype, device, spikes=0.0):
    """The same recipe as ``sinusoid_field`` (8 sinusoids with integer frequencies 1..6 per axis,
    random phases, Gaussian noise 1e-3, optional 1% lognormal spikes), computed in float64 on a
    torch device with torch's seeded generators, for fields too large to draw on the host. The
    values differ from ``sinusoid_field``'s for the same seed (other generators)."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    nd = len(shape)
    freqs = torch.randint(1, 7, (8, nd), generator=g)
    phases = torch.rand(8, generator=g, dtype=torch.float64) * 2 * np.pi
    axes = [torch.arange(n, device=device, dtype=torch.float64) / n for n in shape]
    acc = torch.zeros(shape, device=device, dtype=torch.float64)
    for m in range(8):
        ang = phases[m].item()
        grid = None
        for a in range(nd):
            t = 2 * np.pi * freqs[m, a].item() * axes[a]
            t = t.view(*([1] * a), -1, *([1] * (nd - a - 1)))
            grid = t if grid is None else grid + t
        acc += torch.sin(grid + ang)
    gd = torch.Generator(device=device).manual_seed(seed + 1)
    acc += 1e-3 * torch.randn(shape, device=device, dtype=torch.float64, generator=gd)
    if spikes > 0:
        n = acc.numel()
        k = max(1, int(spikes * n))
        idx = torch.randint(0, n, (k,), device=device, generator=gd)
        sign = torch.randint(0, 2, (k,), device=device, generator=gd).to(torch.float64) * 2 - 1
        mag = torch.exp(2.0 * torch.randn(k, device=device, dtype=torch.float64, generator=gd))
        acc.view(-1)[idx] += sign * mag
    return acc.to(dtype).contiguous()
