"""Seeded synthetic terrains shaped like the paper's test data.

This module is the only code shared by the CUDA path's tests/benchmark and the
CPU oracle: it draws elevation grids and holds none of the siting method's
arithmetic.  The paper's own datasets (DEM1000 and the NASADEM US East / US
West extracts, Sec. "Testing") are not available, so these generators stand in
for them with the same shapes and elevation ranges.

* ``spectral_fbm``  -- fractional Brownian surface by spectral synthesis:
  amplitude |f|^-(H+1) with uniformly random phases, inverse real FFT, affine
  rescale to [zmin, zmax], round to nearest, optional "lakes" (every post at or
  below a quantile flattened to zmin).
* ``ridged_multifractal`` -- octave value noise combined with the ridged
  multifractal rule of Musgrave (Texturing & Modeling, 1994): each octave's
  ridge signal (offset - |n|)^2 is weighted by the previous octave's signal,
  octave amplitudes fall as lacunarity^(-H*i).

Randomness is counter-based (SplitMix64 of the element index), so a terrain
depends only on its parameters and seed; the floating-point synthesis runs on
the device that is asked for, and whichever side consumes a terrain receives
the same int16 bytes.
"""
import math

import numpy as np
import torch

_M64 = (1 << 64) - 1


def _to_i64(c):
    """Reinterpret an unsigned 64-bit constant as a signed int64 value."""
    c &= _M64
    return c - (1 << 64) if c >= (1 << 63) else c


_GOLD = _to_i64(0x9E3779B97F4A7C15)
_C1 = _to_i64(0xBF58476D1CE4E5B9)
_C2 = _to_i64(0x94D049BB133111EB)


def _lsr(x, k):
    """Logical right shift of an int64 tensor holding uint64 bit patterns."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def splitmix64(seed, idx):
    """SplitMix64 outputs number idx (0-based) of a generator seeded with seed;
    idx is an int64 tensor, the result holds uint64 bit patterns in int64."""
    x = idx.to(torch.int64) + 1
    x = x * _GOLD + _to_i64(seed)
    x = (x ^ _lsr(x, 30)) * _C1
    x = (x ^ _lsr(x, 27)) * _C2
    return x ^ _lsr(x, 31)


def uniform01(seed, idx, dtype=torch.float64):
    """Uniform [0,1) values from the top 53 bits of SplitMix64 outputs."""
    u = _lsr(splitmix64(seed, idx), 11)
    return u.to(dtype) * (1.0 / float(1 << 53))


def _rescale_to_int16(f, zmin, zmax):
    lo = f.min()
    hi = f.max()
    scale = (zmax - zmin) / torch.clamp(hi - lo, min=1e-30)
    out = torch.round((f - lo) * scale + zmin)
    return torch.clamp(out, zmin, zmax).to(torch.int16)


def _lakes(z, frac, zfloor):
    """Flatten every post at or below the frac-quantile of elevations to zfloor."""
    if frac <= 0:
        return z
    zi = z.to(torch.int32) - int(zfloor)
    nb = int(zi.max().item()) + 1
    hist = torch.bincount(zi.reshape(-1), minlength=nb).to(torch.int64)
    cum = torch.cumsum(hist, 0)
    need = math.ceil(frac * z.numel())
    vq = int(torch.nonzero(cum >= need)[0].item()) + int(zfloor)
    return torch.where(z <= vq, torch.full_like(z, int(zfloor)), z)


def spectral_fbm(H, W, hurst, seed, zmin=0, zmax=1000, lake_frac=0.0, device="cpu"):
    """Spectral-synthesis fBm terrain, int16 tensor of shape (H, W)."""
    dev = torch.device(device)
    ftype = torch.float64 if dev.type == "cpu" else torch.float32
    fy = torch.fft.fftfreq(H, d=1.0 / H, device=dev).to(ftype)       # integer cycles
    fx = torch.fft.rfftfreq(W, d=1.0 / W, device=dev).to(ftype)
    # keep memory bounded: build the spectrum row block by row block
    Wf = fx.numel()
    spec = torch.empty((H, Wf), dtype=torch.complex64 if ftype == torch.float32 else torch.complex128,
                       device=dev)
    rows = max(1, (1 << 24) // max(Wf, 1))
    for r0 in range(0, H, rows):
        r1 = min(H, r0 + rows)
        ff = torch.sqrt(fy[r0:r1, None] ** 2 + fx[None, :] ** 2)
        amp = torch.where(ff > 0, ff.clamp(min=1e-12) ** (-(hurst + 1.0)), torch.zeros_like(ff))
        idx = (torch.arange(r0, r1, device=dev, dtype=torch.int64)[:, None] * Wf
               + torch.arange(Wf, device=dev, dtype=torch.int64)[None, :])
        ph = uniform01(seed, idx, ftype) * (2.0 * math.pi)
        spec[r0:r1] = torch.polar(amp, ph)
    f = torch.fft.irfft2(spec, s=(H, W))
    del spec
    z = _rescale_to_int16(f, zmin, zmax)
    return _lakes(z, lake_frac, zmin)


def _value_noise(H, W, wavelength, seed, octave, dev, ftype):
    """Smooth value noise in [-1,1]: SplitMix64 values on a lattice of the
    given wavelength, bicubically interpolated to H x W."""
    lh = int(math.ceil(H / wavelength)) + 3
    lw = int(math.ceil(W / wavelength)) + 3
    idx = torch.arange(lh * lw, device=dev, dtype=torch.int64).reshape(lh, lw)
    lat = uniform01(seed * 1315423911 + octave * 2654435761 + 17, idx, ftype) * 2.0 - 1.0
    up = torch.nn.functional.interpolate(lat[None, None], scale_factor=float(wavelength),
                                         mode="bicubic", align_corners=False)[0, 0]
    return up[wavelength:wavelength + H, wavelength:wavelength + W] if wavelength >= 1 else up[:H, :W]


def ridged_multifractal(H, W, seed, zmin=0, zmax=4000, lake_frac=0.0, octaves=10,
                        base_wavelength=None, lacunarity=2.0, hurst=0.8, gain=2.0,
                        offset=1.0, device="cpu", chunk_rows=None):
    """Ridged multifractal terrain from octave value noise, int16 (H, W)."""
    dev = torch.device(device)
    ftype = torch.float32
    if base_wavelength is None:
        base_wavelength = max(8, min(H, W) // 6)
    acc = None
    weight = None
    for i in range(octaves):
        wl = max(1, int(round(base_wavelength / (lacunarity ** i))))
        if wl < 2:
            break
        n = _value_noise(H, W, wl, seed, i, dev, ftype)
        sig = offset - n.abs_()
        sig.mul_(sig)
        if weight is not None:
            sig.mul_(weight)
        amp = lacunarity ** (-hurst * i)
        if acc is None:
            acc = sig * amp
        else:
            acc.add_(sig, alpha=amp)
        weight = torch.clamp(sig * gain, 0.0, 1.0)
        del n, sig
    z = _rescale_to_int16(acc, zmin, zmax)
    del acc, weight
    return _lakes(z, lake_frac, zmin)


def flat(H, W, value=0):
    return torch.full((H, W), int(value), dtype=torch.int16)


def cone(H, W, cx, cy, top, slope):
    """z = top - round(slope * dist) around (cx, cy): a concave-down cone
    (used by the oracle's closed-form checks)."""
    y = torch.arange(H, dtype=torch.float64)[:, None]
    x = torch.arange(W, dtype=torch.float64)[None, :]
    d = torch.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    return (top - torch.round(slope * d)).to(torch.int16)


def pad_pitch(z, multiple=8):
    """Copy an (H, W) int16 grid into storage whose row pitch is a multiple of
    ``multiple`` elements; returns (storage (H, pitch), pitch)."""
    H, W = z.shape
    pitch = (W + multiple - 1) // multiple * multiple
    if pitch == W:
        return z.contiguous(), pitch
    out = torch.zeros((H, pitch), dtype=z.dtype, device=z.device)
    out[:, :W] = z
    return out, pitch
