"""Seeded synthetic inputs shaped like the paper's workloads (arXiv:2301.06061, section 4).

The paper images LOFAR HBA data (Table 2: 8 h track, 120-170 MHz, core-dense
uneven (u,v) coverage, section 3.1).  That data is not available, so these
generators stand in for it.  This module holds geometry and random numbers only:
station layouts, earth-rotation (u,v,w) tracks, point-source sky catalogues and
noise.  It contains none of the imaging method's arithmetic (no gridding,
transform or phase screen) and is shared by the CUDA path's callers and by the
oracle's tests.

Workloads (seed = 230106061 + workload number):

1. ``tiny``     10,000 (u,v) uniform in a disk of radius 0.45 N/FoV, w ~ U(-200, 200),
                256^2, FoV 0.1 rad, 8 planes; 10 sources, flux U(0.1, 1)
2. ``array``    60 stations in a 20 km disk, declination +45, latitude 52.9, 8 h,
                16 channels over 120-168 MHz, 144 dumps (~4.08 M visibilities),
                4096^2, FoV 0.2 rad, 32 planes; 200 sources, dN/dS ~ S^-2 on [0.01, 1]
3. ``large``    300 stations, 64 channels, 35 dumps truncated to exactly 1e8
                visibilities, 16384^2, FoV 0.5 rad, 32 planes
4. ``batched``  64 channel images, counts log-uniform in [1e5, 2e6], 2048^2,
                FoV 0.09 rad, 16 planes each, tracks of workload 2 at the channel frequency
5. ``learned``  512^2 skies of 1-50 sources, 2e5 visibilities of the ``tiny`` kind
                scaled to N = 512, FoV 0.1 rad, 8 planes, support 8
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 230106061
C_LIGHT = 299_792_458.0


def rng_for(workload: int, extra: int = 0) -> np.random.Generator:
    return np.random.default_rng([SEED_BASE + workload, extra])


# ----------------------------------------------------------------------------------------
# (u, v, w) coverage
# ----------------------------------------------------------------------------------------

def disk_uvw(n_vis: int, radius: float, w_half: float, rng: np.random.Generator):
    """(u, v) uniform in a disk of the given radius (wavelengths), w ~ U(-w_half, w_half)."""
    r = radius * np.sqrt(rng.random(n_vis))
    th = 2.0 * np.pi * rng.random(n_vis)
    u = (r * np.cos(th)).astype(np.float32)
    v = (r * np.sin(th)).astype(np.float32)
    w = rng.uniform(-w_half, w_half, n_vis).astype(np.float32)
    return u, v, w


def station_layout(n_stations: int, diameter_m: float, rng: np.random.Generator) -> np.ndarray:
    """Stations uniform in a disk (east, north) in metres, all at zero height."""
    r = 0.5 * diameter_m * np.sqrt(rng.random(n_stations))
    th = 2.0 * np.pi * rng.random(n_stations)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def baselines_xyz(enu: np.ndarray, lat_deg: float) -> np.ndarray:
    """Baseline vectors (metres) in the equatorial frame for every station pair i < j."""
    lat = math.radians(lat_deg)
    east, north = enu[:, 0], enu[:, 1]
    up = np.zeros_like(east)
    x = -math.sin(lat) * north + math.cos(lat) * up
    y = east
    z = math.cos(lat) * north + math.sin(lat) * up
    xyz = np.stack([x, y, z], axis=1)
    i, j = np.triu_indices(len(enu), k=1)
    return xyz[j] - xyz[i]


def earth_rotation_uvw(bl_xyz: np.ndarray, dec_deg: float, hour_angles_rad: np.ndarray) -> np.ndarray:
    """Standard interferometer geometry: (u, v, w) in metres, shape (n_times, n_baselines, 3)."""
    dec = math.radians(dec_deg)
    h = hour_angles_rad[:, None]
    lx, ly, lz = bl_xyz[None, :, 0], bl_xyz[None, :, 1], bl_xyz[None, :, 2]
    u = np.sin(h) * lx + np.cos(h) * ly
    v = -math.sin(dec) * np.cos(h) * lx + math.sin(dec) * np.sin(h) * ly + math.cos(dec) * lz
    w = math.cos(dec) * np.cos(h) * lx - math.cos(dec) * np.sin(h) * ly + math.sin(dec) * lz
    return np.stack([u, v, w], axis=-1)


def array_rows(n_stations: int, diameter_m: float, n_dumps: int, freqs_hz: np.ndarray,
               rng: np.random.Generator, lat_deg: float = 52.9, dec_deg: float = 45.0,
               track_hours: float = 8.0):
    """Earth-rotation tracks by row: FP64 [n_dumps * n_baselines, 3] baseline coordinates
    in metres, ordered (time, baseline), and FP64 [n_chan] channel scales nu / c."""
    enu = station_layout(n_stations, diameter_m, rng)
    bl = baselines_xyz(enu, lat_deg)
    ha = np.linspace(-0.5, 0.5, n_dumps) * track_hours * (2.0 * np.pi / 24.0)
    uvw_m = earth_rotation_uvw(bl, dec_deg, ha).reshape(-1, 3)
    return np.ascontiguousarray(uvw_m, dtype=np.float64), np.asarray(freqs_hz, dtype=np.float64) / C_LIGHT


def array_uvw(n_stations: int, diameter_m: float, n_dumps: int, freqs_hz: np.ndarray,
              rng: np.random.Generator, lat_deg: float = 52.9, dec_deg: float = 45.0,
              track_hours: float = 8.0, n_vis: int | None = None):
    """Earth-rotation tracks, ordered (time, baseline, channel) like a measurement set.

    Returns float32 u, v, w in wavelengths, truncated to ``n_vis`` if given.
    """
    uvw_m, scale = array_rows(n_stations, diameter_m, n_dumps, freqs_hz, rng, lat_deg, dec_deg, track_hours)
    return expand_tracks(uvw_m, scale, n_vis)


def expand_tracks(uvw_m: np.ndarray, scale: np.ndarray, n_vis: int | None = None):
    """float32 u, v, w in wavelengths of the rows x channels, truncated to ``n_vis``."""
    total = uvw_m.shape[0] * len(scale)
    n_vis = total if n_vis is None else min(int(n_vis), total)
    out = []
    for comp in range(3):
        # (time*baseline, channel) outer product, built in float64 then rounded once
        col = np.multiply.outer(uvw_m[:, comp], scale)
        out.append(col.reshape(-1)[:n_vis].astype(np.float32))
    return out[0], out[1], out[2]


# ----------------------------------------------------------------------------------------
# Skies and visibility values
# ----------------------------------------------------------------------------------------

@dataclass
class PointSky:
    l: np.ndarray
    m: np.ndarray
    flux: np.ndarray


def uniform_sky(n_src: int, half_extent: float, flux_lo: float, flux_hi: float,
                rng: np.random.Generator) -> PointSky:
    l = rng.uniform(-half_extent, half_extent, n_src)
    m = rng.uniform(-half_extent, half_extent, n_src)
    s = rng.uniform(flux_lo, flux_hi, n_src)
    return PointSky(l, m, s)


def power_law_sky(n_src: int, half_extent: float, s_lo: float, s_hi: float,
                  rng: np.random.Generator) -> PointSky:
    """Fluxes with dN/dS ~ S^-2 on [s_lo, s_hi] (inverse-CDF sampling)."""
    x = rng.random(n_src)
    s = 1.0 / (1.0 / s_lo - x * (1.0 / s_lo - 1.0 / s_hi))
    l = rng.uniform(-half_extent, half_extent, n_src)
    m = rng.uniform(-half_extent, half_extent, n_src)
    return PointSky(l, m, s)


def complex_noise(n: int, sigma: float, rng: np.random.Generator) -> np.ndarray:
    """Independent N(0, sigma^2) on the real and imaginary parts."""
    return (rng.normal(0.0, sigma, n) + 1j * rng.normal(0.0, sigma, n)).astype(np.complex128)


def random_visibilities(n: int, rng: np.random.Generator) -> np.ndarray:
    """Unit-variance complex Gaussian values (complex64)."""
    re = rng.standard_normal(n, dtype=np.float32)
    im = rng.standard_normal(n, dtype=np.float32)
    out = np.empty(n, np.complex64)
    out.real = re
    out.imag = im
    return out


# ----------------------------------------------------------------------------------------
# Workload descriptions
# ----------------------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    n: int
    fov: float
    n_w: int
    support: int
    w_min: float
    w_max: float
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    sky: PointSky | None = None
    noise_sigma: float = 0.0
    batch_offsets: np.ndarray | None = None
    # the same coordinates by row and channel (u, v, w = rows_m[i // C] * chan_scale[i % C])
    rows_m: np.ndarray | None = None
    chan_scale: np.ndarray | None = None

    @property
    def n_vis(self) -> int:
        return int(self.u.size)


def tiny(n_vis: int = 10_000, n: int = 256, fov: float = 0.1, n_w: int = 8, seed_extra: int = 0):
    rng = rng_for(1, seed_extra)
    u, v, w = disk_uvw(n_vis, 0.45 * n / fov, 200.0, rng)
    sky = uniform_sky(10, 0.5 * fov, 0.1, 1.0, rng)  # l, m ~ U(-FoV/2, FoV/2)
    return Workload("tiny", n, fov, n_w, 7, -200.0, 200.0, u, v, w, sky=sky, noise_sigma=0.01)


def array(n_dumps: int = 144, seed_extra: int = 0):
    rng = rng_for(2, seed_extra)
    freqs = np.linspace(120e6, 168e6, 16)
    rows, scale = array_rows(60, 20_000.0, n_dumps, freqs, rng)
    u, v, w = expand_tracks(rows, scale)
    sky = power_law_sky(200, 0.1, 0.01, 1.0, rng)
    return Workload("array", 4096, 0.2, 32, 7, 0.0, 0.0, u, v, w, sky=sky, rows_m=rows, chan_scale=scale)


def large(n_vis: int = 100_000_000, seed_extra: int = 0):
    rng = rng_for(3, seed_extra)
    freqs = np.linspace(120e6, 168e6, 64)
    per_dump = 300 * 299 // 2 * 64
    n_dumps = -(-n_vis // per_dump)
    rows, scale = array_rows(300, 20_000.0, n_dumps, freqs, rng)
    u, v, w = expand_tracks(rows, scale, n_vis)
    return Workload("large", 16384, 0.5, 32, 7, 0.0, 0.0, u, v, w, rows_m=rows, chan_scale=scale)


def batched_counts(n_images: int = 64, lo: float = 1e5, hi: float = 2e6, seed_extra: int = 0):
    rng = rng_for(4, seed_extra)
    return np.floor(10.0 ** rng.uniform(math.log10(lo), math.log10(hi), n_images)).astype(np.int64)


def batched(n_images: int = 64, counts: np.ndarray | None = None, seed_extra: int = 0):
    """64 channel images; image c uses the workload-2 tracks at its channel frequency."""
    rng = rng_for(4, 1000 + seed_extra)
    counts = batched_counts(n_images, seed_extra=seed_extra) if counts is None else counts
    freqs = np.linspace(120e6, 168e6, n_images)
    enu = station_layout(60, 20_000.0, rng)
    bl = baselines_xyz(enu, 52.9)
    us, vs, ws = [], [], []
    for c in range(n_images):
        n_dumps = max(2, -(-int(counts[c]) // bl.shape[0]))
        ha = np.linspace(-0.5, 0.5, n_dumps) * 8.0 * (2.0 * np.pi / 24.0)
        uvw = earth_rotation_uvw(bl, 45.0, ha).reshape(-1, 3)[: int(counts[c])]
        scale = freqs[c] / C_LIGHT
        us.append((uvw[:, 0] * scale).astype(np.float32))
        vs.append((uvw[:, 1] * scale).astype(np.float32))
        ws.append((uvw[:, 2] * scale).astype(np.float32))
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return Workload("batched", 2048, 0.09, 16, 7, 0.0, 0.0, np.concatenate(us), np.concatenate(vs),
                    np.concatenate(ws), batch_offsets=offsets)


def learned_sky(index: int, n: int = 512, fov: float = 0.1, n_vis: int = 200_000,
                max_src: int = 50):
    """Sky ``index`` of the learned-kernel training set: 1..max_src sources, U(0.1, 1) Jy."""
    rng = rng_for(5, index)
    u, v, w = disk_uvw(n_vis, 0.45 * n / fov, 200.0, rng)
    n_src = int(rng.integers(1, max_src + 1))
    sky = uniform_sky(n_src, 0.5 * fov, 0.1, 1.0, rng)
    return Workload("learned", n, fov, 8, 8, -200.0, 200.0, u, v, w, sky=sky)
