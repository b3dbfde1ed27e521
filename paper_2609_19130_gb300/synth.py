"""Seeded synthetic inputs for the pressure projection.

This module only draws numbers: it holds none of the projection's arithmetic
(no divergence, gradient, transform or solve), so that the CUDA path and the
FP64 oracle can be fed identical inputs without sharing any method code.

Counter-based generator (splitmix64, Steele, Lea & Flood, OOPSLA 2014):
    key = splitmix64(seed)
    x   = splitmix64(key ^ (array_id << 56) ^ linear_index)
    U[-1,1] = 2 * (x >> 11) * 2^-53 - 1
where splitmix64(s) applies the published finaliser to s + 0x9E3779B97F4A7C15.
The same generator is written twice, once in numpy (host) and once with torch
int64 tensor ops (runs on the device for the large grids); a test checks that
the two agree bit for bit.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN_GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
M64 = (1 << 64) - 1

# array ids used by the velocity generators
AID_U, AID_V, AID_W, AID_NOISE_U, AID_NOISE_V, AID_NOISE_W, AID_WEIGHT = 1, 2, 3, 4, 5, 6, 7


def _mix_np(z: np.ndarray) -> np.ndarray:
    z = (z + np.uint64(GOLDEN_GAMMA))
    z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
    return z ^ (z >> np.uint64(31))


def splitmix64_scalar(s: int) -> int:
    z = (s + GOLDEN_GAMMA) & M64
    z = ((z ^ (z >> 30)) * MIX1) & M64
    z = ((z ^ (z >> 27)) * MIX2) & M64
    return z ^ (z >> 31)


def bits_np(seed: int, array_id: int, n: int, start: int = 0) -> np.ndarray:
    key = splitmix64_scalar(seed & M64)
    idx = np.arange(start, start + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix_np(idx ^ np.uint64((key ^ (array_id << 56)) & M64))


def uniform_np(seed: int, array_id: int, shape, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    n = int(np.prod(shape))
    x = bits_np(seed, array_id, n)
    u01 = (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return (lo + (hi - lo) * u01).reshape(shape)


def normal_np(seed: int, array_id: int, shape) -> np.ndarray:
    """Box-Muller on two uniform streams (array ids array_id and array_id|0x80)."""
    n = int(np.prod(shape))
    u1 = (bits_np(seed, array_id, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    u2 = (bits_np(seed, array_id | 0x80, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    r = np.sqrt(-2.0 * np.log1p(-u1))          # 1-u1 in (0,1]
    return (r * np.cos(2.0 * np.pi * u2)).reshape(shape)


def _to_signed(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


def bits_torch(seed: int, array_id: int, n: int, device="cpu", start: int = 0):
    """Same stream as bits_np, as torch.int64 (two's complement of the uint64 value)."""
    import torch
    key = splitmix64_scalar(seed & M64)
    k = _to_signed((key ^ (array_id << 56)) & M64)
    z = torch.arange(start, start + n, dtype=torch.int64, device=device) ^ k
    z = z + _to_signed(GOLDEN_GAMMA)

    def lsr(t, s):  # logical shift right on int64
        return (t >> s) & ((1 << (64 - s)) - 1)

    z = (z ^ lsr(z, 30)) * _to_signed(MIX1)
    z = (z ^ lsr(z, 27)) * _to_signed(MIX2)
    return z ^ lsr(z, 31)


def uniform_torch(seed: int, array_id: int, shape, lo=-1.0, hi=1.0, device="cpu"):
    import torch
    n = int(np.prod(shape))
    x = bits_torch(seed, array_id, n, device=device)
    top = (x >> 11) & ((1 << 53) - 1)
    u01 = top.to(torch.float64) * (2.0 ** -53)
    return (lo + (hi - lo) * u01).reshape(tuple(shape))


def normal_torch(seed: int, array_id: int, shape, device="cpu"):
    """Same stream as normal_np (Box-Muller on two uniform streams), as torch float64."""
    import torch
    n = int(np.prod(shape))
    u1 = ((bits_torch(seed, array_id, n, device=device) >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
    u2 = ((bits_torch(seed, array_id | 0x80, n, device=device) >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
    r = torch.sqrt(-2.0 * torch.log1p(-u1))
    return (r * torch.cos(2.0 * np.pi * u2)).reshape(tuple(shape))


# ---------------------------------------------------------------------------
# staggered field shapes: u [nz][ny][nxu], v [nz][nyv][nx], w [nz+1][ny][nx]
# nxu = nx (periodic x) or nx+1 (wall x);  nyv likewise.
# ---------------------------------------------------------------------------

def field_shapes(nx, ny, nz, wall_x=False, wall_y=False):
    return ((nz, ny, nx + 1 if wall_x else nx), (nz, ny + 1 if wall_y else ny, nx), (nz + 1, ny, nx))


def uniform_velocity_np(seed, nx, ny, nz, wall_x=False, wall_y=False, zero_walls=True):
    """u*,v*,w* i.i.d. U[-1,1]; normal velocity on every wall set to zero if asked."""
    su, sv, sw = field_shapes(nx, ny, nz, wall_x, wall_y)
    u = uniform_np(seed, AID_U, su)
    v = uniform_np(seed, AID_V, sv)
    w = uniform_np(seed, AID_W, sw)
    if zero_walls:
        w[0] = 0.0
        w[-1] = 0.0
        if wall_x:
            u[:, :, 0] = 0.0
            u[:, :, -1] = 0.0
        if wall_y:
            v[:, 0, :] = 0.0
            v[:, -1, :] = 0.0
    return u, v, w


def uniform_velocity_torch(seed, nx, ny, nz, device, zero_walls=True):
    su, sv, sw = field_shapes(nx, ny, nz)
    u = uniform_torch(seed, AID_U, su, device=device)
    v = uniform_torch(seed, AID_V, sv, device=device)
    w = uniform_torch(seed, AID_W, sw, device=device)
    if zero_walls:
        w[0].zero_()
        w[-1].zero_()
    return u, v, w


def batch_grid_draws(seed: int, ngrids: int, nxy=(64, 96, 128, 192), nzs=(64, 128, 256),
                     beta_lo=1.0, beta_hi=3.0):
    """Sizes and tanh clustering factors for a batch of uneven grids.

    Returns a list of (nx, ny, nz, beta) drawn from splitmix64 with array ids
    11 (nx), 12 (ny), 13 (nz), 14 (beta)."""
    def pick(aid, choices):
        b = bits_np(seed, aid, ngrids)
        return [choices[int(x % np.uint64(len(choices)))] for x in b]
    nx = pick(11, nxy)
    ny = pick(12, nxy)
    nz = pick(13, nzs)
    u = (bits_np(seed, 14, ngrids) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    beta = beta_lo + (beta_hi - beta_lo) * u
    return [(int(a), int(b), int(c), float(d)) for a, b, c, d in zip(nx, ny, nz, beta)]


def kolmogorov_modes(seed: int, kmax: int = 32):
    """Random Fourier modes for a smooth velocity with E(k) ~ k^-5/3.

    Integer wavevectors (kx, ky, kz) with 0 < |k| <= kmax, kx,ky in [-kmax,kmax],
    kz in [0, kmax]; amplitude |k|^(-11/6) (so that the energy in a shell of
    radius k, ~k^2 * |k|^(-11/3), falls as k^-5/3); a uniform random phase per
    mode and velocity component.  Returns (kx, ky, kz, amp, phase[3, nmodes])."""
    r = np.arange(-kmax, kmax + 1)
    KX, KY, KZ = np.meshgrid(r, r, np.arange(0, kmax + 1), indexing="ij")
    K2 = KX ** 2 + KY ** 2 + KZ ** 2
    sel = (K2 > 0) & (K2 <= kmax * kmax)
    kx, ky, kz = KX[sel], KY[sel], KZ[sel]
    amp = np.sqrt(K2[sel].astype(np.float64)) ** (-11.0 / 6.0)
    n = kx.size
    ph = np.stack([uniform_np(seed, 21 + c, (n,), 0.0, 2.0 * np.pi) for c in range(3)])
    return kx, ky, kz, amp, ph


def kolmogorov_velocity_torch(seed, nx, ny, nz, device, kmax=32, noise=0.01, dtype=None):
    """Staggered u*,v*,w* made of Fourier modes with a k^-5/3 spectrum plus U[-noise,noise].

    Positions are taken in index space (x = 2*pi*i/nx, y = 2*pi*j/ny and
    s = k/nz in z) with the half-cell offsets of the staggered layout; u and v
    carry cos(pi*kz*s), w carries sin(pi*kz*s), so w vanishes on both walls.
    Built per kz with an inverse 2D FFT (torch.fft is used here only to
    synthesise inputs).  Noise comes from the splitmix64 stream."""
    import torch
    dtype = dtype or torch.float64
    kx, ky, kz, amp, ph = kolmogorov_modes(seed, kmax)
    kxs = min(kmax, nx // 2 - 1)
    kys = min(kmax, ny // 2 - 1)
    keep = (np.abs(kx) <= kxs) & (np.abs(ky) <= kys)
    kx, ky, kz, amp, ph = kx[keep], ky[keep], kz[keep], amp[keep], ph[:, keep]
    # normalise so the largest component is O(1)
    amp = amp / np.sqrt(np.sum(amp ** 2) / 3.0)
    out = []
    shapes = field_shapes(nx, ny, nz)
    # per component: x offset, y offset, z sample points, z basis
    zc = (np.arange(nz) + 0.5) / nz
    zfc = np.arange(nz + 1) / nz
    specs = [(0.0, 0.5, zc, np.cos), (0.5, 0.0, zc, np.cos), (0.5, 0.5, zfc, np.sin)]
    for c, (ox, oy, zs, zb) in enumerate(specs):
        f = torch.zeros(shapes[c], dtype=dtype, device=device)
        for q in range(kmax + 1):
            m = kz == q
            if not np.any(m) or (zb is np.sin and q == 0):
                continue
            # complex amplitudes on the (ny, nx//2+1) half plane; cos(kx x + ky y + p)
            S = np.zeros((ny, nx // 2 + 1), dtype=np.complex128)
            a = amp[m] * np.exp(1j * (ph[c, m] + 2 * np.pi * (kx[m] * ox / nx + ky[m] * oy / ny)))
            kxq, kyq = kx[m], ky[m]
            neg = kxq < 0
            a = np.where(neg, np.conj(a), a)
            kxq = np.where(neg, -kxq, kxq)
            kyq = np.where(neg, -kyq, kyq)
            wgt = np.where(kxq == 0, 1.0, 0.5)       # irfft doubles non-zero kx columns
            np.add.at(S, (kyq % ny, kxq), a * wgt * nx * ny)
            plane = torch.fft.irfft2(torch.from_numpy(S).to(device), s=(ny, nx)).to(dtype)
            prof = torch.from_numpy(zb(np.pi * q * zs)).to(device=device, dtype=dtype)
            f.add_(prof.view(-1, 1, 1) * plane.view(1, ny, nx))
        n = int(np.prod(shapes[c]))
        f.add_(uniform_torch(seed, AID_NOISE_U + c, shapes[c], -noise, noise, device=device).to(dtype))
        out.append(f)
    out[2][0].zero_()
    out[2][-1].zero_()
    return tuple(out)
