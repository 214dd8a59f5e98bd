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
    out = torch.empty(f.shape, dtype=torch.int16, device=f.device)
    rows = max(1, (1 << 27) // max(1, f.shape[-1]))
    for r0 in range(0, f.shape[0], rows):
        v = torch.round((f[r0:r0 + rows] - lo) * scale + zmin)
        out[r0:r0 + rows] = torch.clamp(v, zmin, zmax).to(torch.int16)
    return out


def _lakes(z, frac, zfloor):
    """Flatten every post at or below the frac-quantile of elevations to zfloor."""
    if frac <= 0:
        return z
    nb = int(z.max().item()) - int(zfloor) + 1
    hist = torch.zeros(nb, dtype=torch.int64, device=z.device)
    flat = z.reshape(-1)
    step = 1 << 28
    for i in range(0, flat.numel(), step):
        zi = flat[i:i + step].to(torch.int32) - int(zfloor)
        hist += torch.bincount(zi, minlength=nb).to(torch.int64)
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


def _lattice(H, W, wavelength, seed, octave, dev, ftype):
    lh = int(math.ceil(H / wavelength)) + 3
    lw = int(math.ceil(W / wavelength)) + 3
    idx = torch.arange(lh * lw, device=dev, dtype=torch.int64).reshape(lh, lw)
    return uniform01(seed * 1315423911 + octave * 2654435761 + 17, idx, ftype) * 2.0 - 1.0


def _cubic_taps(n0, n1, wl, lmax, dev, ftype):
    """Lattice indices and Catmull-Rom weights (4 each) for output samples
    n0..n1-1 at lattice coordinate (n + 0.5)/wl - 0.5 + 1; the cell and the
    fraction come from exact integer arithmetic, so a sample's value does
    not depend on how the output is chunked."""
    n = torch.arange(n0, n1, device=dev, dtype=torch.int64)
    t = 2 * n + 1 + wl                       # 2*wl * (coordinate + 1)
    cell = torch.div(t, 2 * wl, rounding_mode="floor")
    fr = (t - cell * 2 * wl).to(ftype) / float(2 * wl)
    f2, f3 = fr * fr, fr * fr * fr
    w = torch.stack([-0.5 * f3 + f2 - 0.5 * fr,
                     1.5 * f3 - 2.5 * f2 + 1.0,
                     -1.5 * f3 + 2.0 * f2 + 0.5 * fr,
                     0.5 * f3 - 0.5 * f2], dim=0)
    idx = torch.stack([cell - 1 + k for k in range(4)], dim=0).clamp_(0, lmax - 1)
    return idx, w


def _value_noise_rows(lat, wavelength, r0, r1, W):
    """Rows [r0, r1) (width W) of smooth value noise in [-1,1]: the lattice
    interpolated with the Catmull-Rom cubic, separably (rows, then columns)."""
    dev, ftype = lat.device, lat.dtype
    iy, wy = _cubic_taps(r0, r1, wavelength, lat.shape[0], dev, ftype)
    ix, wx = _cubic_taps(0, W, wavelength, lat.shape[1], dev, ftype)
    T = sum(wy[k][:, None] * lat[iy[k]] for k in range(4))      # (rows, lw)
    return sum(wx[k][None, :] * T[:, ix[k]] for k in range(4))  # (rows, W)


def ridged_multifractal(H, W, seed, zmin=0, zmax=4000, lake_frac=0.0, octaves=10,
                        base_wavelength=None, lacunarity=2.0, hurst=0.8, gain=2.0,
                        offset=1.0, device="cpu", chunk_rows=1024):
    """Ridged multifractal terrain from octave value noise, int16 (H, W);
    generated in row chunks so that any size fits the upsampling kernels."""
    dev = torch.device(device)
    ftype = torch.float32
    if base_wavelength is None:
        base_wavelength = max(8, min(H, W) // 6)
    wls = []
    for i in range(octaves):
        wl = max(1, int(round(base_wavelength / (lacunarity ** i))))
        if wl < 2:
            break
        wls.append(wl)
    lats = [_lattice(H, W, wl, seed, i, dev, ftype) for i, wl in enumerate(wls)]
    acc = torch.empty((H, W), dtype=ftype, device=dev)
    for r0 in range(0, H, chunk_rows):
        r1 = min(H, r0 + chunk_rows)
        a = None
        weight = None
        for i, wl in enumerate(wls):
            n = _value_noise_rows(lats[i], wl, r0, r1, W)
            sig = offset - n.abs()
            sig.mul_(sig)
            if weight is not None:
                sig.mul_(weight)
            amp = lacunarity ** (-hurst * i)
            if a is None:
                a = sig * amp
            else:
                a.add_(sig, alpha=amp)
            weight = torch.clamp(sig * gain, 0.0, 1.0)
            del n, sig
        acc[r0:r1] = a
        del a, weight
    del lats
    z = _rescale_to_int16(acc, zmin, zmax)
    del acc
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
