"""Seeded synthetic confocal NLOS captures (inputs only).

This module renders transient measurements of hidden scenes made of point
reflectors and planar patches. It simulates the capture described in Sec. 3
(confocal set-up, relay wall at z = 0, third-bounce time of flight), adds
Poisson photon noise and a uniform background, and returns counts. It holds
none of the reconstruction arithmetic: the CUDA path's tests, the benchmark
and the FP64 oracle's tests all draw their inputs from here, and nothing here
is derived from either reconstruction.

Capture conventions
  * The relay wall lies in the plane z = 0 and is scanned on an nx x ny grid
    of cell centres: x_i = -W_x/2 + (i + 1/2) W_x / nx, likewise for y.
  * Confocal: illumination and detection share the wall point, so a hidden
    point at one-way distance r returns after 2 r / c and lands in time bin
    floor(2 r / (c dt)); bins at or beyond nt are dropped.
  * Point reflectors contribute albedo / r^4 (inverse-square falloff on both
    legs). Patch samples also carry the cosine at the patch (its normal
    against the direction to the wall point) and at the wall (the wall normal
    is +z), each once per leg, times the sample area.
  * The expected-count volume is scaled so its maximum equals the requested
    peak count, a background of `background` counts per bin is added, and the
    result is drawn as Poisson counts with numpy's PCG64 generator.

Seeds follow seed = workload_index * 1000 + capture_index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299_792_458.0  # m/s, speed of light used to bin path lengths


@dataclass
class Geometry:
    nx: int
    ny: int
    nt: int
    bin_width_s: float
    wall_w_m: float
    wall_h_m: float

    @property
    def bin_depth_m(self) -> float:
        """Depth covered by one time bin for a round trip (c dt / 2)."""
        return C_LIGHT * self.bin_width_s / 2.0


@dataclass
class Scene:
    points: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))
    # Each patch: dict(center=(3,), normal=(3,), axis_u=(3,), axis_v=(3,),
    # size=(w, h), albedo=float)
    patches: list = field(default_factory=list)


@dataclass
class Capture:
    geometry: Geometry
    scene: Scene
    counts: np.ndarray          # float64 [nx][ny][nt], integer-valued
    expected: np.ndarray        # float64 noiseless expected counts (scaled)
    seed: int


def wall_coords(n: int, width_m: float) -> np.ndarray:
    """Cell-centre coordinates of n wall samples spanning width_m."""
    return -width_m / 2.0 + (np.arange(n) + 0.5) * (width_m / n)


def _torch():
    try:
        import torch  # noqa: F401
        return torch
    except Exception:  # pragma: no cover - torch is present in this project
        return None


def _render_samples(geom: Geometry, pos: np.ndarray, weight_fn, device=None,
                    chunk_pairs: int = 1 << 25) -> np.ndarray:
    """Accumulate samples at positions `pos` [S,3] into an [nx,ny,nt] volume.

    weight_fn(dx, dy, z, r) -> per-pair weight, evaluated on torch float64
    tensors of shape [wall_chunk, S].
    """
    torch = _torch()
    dev = torch.device(device) if device is not None else torch.device("cpu")
    xs = torch.as_tensor(wall_coords(geom.nx, geom.wall_w_m), dtype=torch.float64, device=dev)
    ys = torch.as_tensor(wall_coords(geom.ny, geom.wall_h_m), dtype=torch.float64, device=dev)
    wx, wy = torch.meshgrid(xs, ys, indexing="ij")
    wx = wx.reshape(-1)
    wy = wy.reshape(-1)
    P = torch.as_tensor(pos, dtype=torch.float64, device=dev)
    nwall = wx.numel()
    vol = torch.zeros(nwall * geom.nt, dtype=torch.float64, device=dev)
    if P.shape[0] == 0:
        return vol.reshape(geom.nx, geom.ny, geom.nt).cpu().numpy()
    step = max(1, chunk_pairs // P.shape[0])
    inv_bin = 2.0 / (C_LIGHT * geom.bin_width_s)
    for w0 in range(0, nwall, step):
        w1 = min(nwall, w0 + step)
        dx = P[None, :, 0] - wx[w0:w1, None]
        dy = P[None, :, 1] - wy[w0:w1, None]
        z = P[None, :, 2].expand(w1 - w0, -1)
        r = torch.sqrt(dx * dx + dy * dy + z * z)
        b = torch.floor(r * inv_bin).to(torch.int64)
        wgt = weight_fn(dx, dy, z, r)
        keep = (b < geom.nt) & (wgt > 0)
        wall_idx = torch.arange(w0, w1, device=dev, dtype=torch.int64)[:, None].expand_as(b)
        flat = (wall_idx * geom.nt + b)[keep]
        vol.index_add_(0, flat, wgt[keep])
    return vol.reshape(geom.nx, geom.ny, geom.nt).cpu().numpy()


def render_points(geom: Geometry, points: np.ndarray, device=None) -> np.ndarray:
    """Expected (unscaled) response of point reflectors [k, 4] = (x, y, z, albedo)."""
    points = np.asarray(points, dtype=np.float64).reshape(-1, 4)
    alb = points[:, 3].copy()
    torch = _torch()

    def wfn(dx, dy, z, r):
        a = torch.as_tensor(alb, dtype=torch.float64, device=r.device)[None, :]
        return a / (r ** 4)

    return _render_samples(geom, points[:, :3], wfn, device=device)


def _patch_samples(patch: dict, spacing: float, max_side: int):
    w, h = patch["size"]
    nu = int(min(max_side, max(2, math.ceil(w / spacing))))
    nv = int(min(max_side, max(2, math.ceil(h / spacing))))
    uu = (np.arange(nu) + 0.5) / nu - 0.5
    vv = (np.arange(nv) + 0.5) / nv - 0.5
    c = np.asarray(patch["center"], dtype=np.float64)
    au = np.asarray(patch["axis_u"], dtype=np.float64)
    av = np.asarray(patch["axis_v"], dtype=np.float64)
    U, V = np.meshgrid(uu * w, vv * h, indexing="ij")
    pos = c[None, :] + U.reshape(-1, 1) * au[None, :] + V.reshape(-1, 1) * av[None, :]
    area = (w / nu) * (h / nv)
    return pos, area


def render_patches(geom: Geometry, patches: list, device=None,
                   max_side: int = 128) -> np.ndarray:
    """Expected (unscaled) response of planar patches.

    Patches are sampled on a regular grid with spacing at most a quarter of
    the lateral wall-sample pitch, capped at `max_side` samples per side.
    """
    torch = _torch()
    pitch = min(geom.wall_w_m / geom.nx, geom.wall_h_m / geom.ny)
    spacing = pitch / 4.0
    vol = np.zeros((geom.nx, geom.ny, geom.nt))
    for patch in patches:
        pos, area = _patch_samples(patch, spacing, max_side)
        nrm = np.asarray(patch["normal"], dtype=np.float64)
        alb = float(patch["albedo"])

        def wfn(dx, dy, z, r, nrm=nrm, area=area, alb=alb):
            # direction patch -> wall point is (-dx, -dy, -z) / r
            cos_p = (-(dx * nrm[0] + dy * nrm[1] + z * nrm[2])) / r
            cos_p = torch.clamp(cos_p, min=0.0)
            cos_w = z / r
            return alb * area * (cos_p * cos_w) ** 2 / (r ** 4)

        vol += _render_samples(geom, pos, wfn, device=device)
    return vol


def _random_patch(rng: np.random.Generator, geom: Geometry, zmin: float, zmax: float,
                  size_range=(0.2, 0.6), max_tilt_deg: float = 30.0) -> dict:
    w, h = rng.uniform(size_range[0], size_range[1], size=2)
    cx = rng.uniform(-0.4, 0.4) * geom.wall_w_m
    cy = rng.uniform(-0.4, 0.4) * geom.wall_h_m
    cz = rng.uniform(zmin, zmax)
    # normal within max_tilt of -z (facing the wall)
    tilt = math.radians(max_tilt_deg) * math.sqrt(rng.uniform(0.0, 1.0))
    az = rng.uniform(0.0, 2.0 * math.pi)
    n = np.array([math.sin(tilt) * math.cos(az), math.sin(tilt) * math.sin(az), -math.cos(tilt)])
    ref = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    au = np.cross(n, ref)
    au /= np.linalg.norm(au)
    av = np.cross(n, au)
    return dict(center=(cx, cy, cz), normal=n, axis_u=au, axis_v=av, size=(w, h),
                albedo=float(rng.uniform(0.3, 1.0)))


def random_scene(geom: Geometry, rng: np.random.Generator, n_points: int, n_patches: int,
                 zmin: float, zmax: float, patch_size=(0.2, 0.6)) -> Scene:
    """Points uniform over the wall span at depths in [zmin, zmax], plus patches."""
    pts = np.zeros((n_points, 4))
    if n_points:
        pts[:, 0] = rng.uniform(-geom.wall_w_m / 2, geom.wall_w_m / 2, n_points)
        pts[:, 1] = rng.uniform(-geom.wall_h_m / 2, geom.wall_h_m / 2, n_points)
        pts[:, 2] = rng.uniform(zmin, zmax, n_points)
        pts[:, 3] = rng.uniform(0.3, 1.0, n_points)
    patches = [_random_patch(rng, geom, zmin, zmax, patch_size) for _ in range(n_patches)]
    return Scene(points=pts, patches=patches)


def render(geom: Geometry, scene: Scene, *, peak: float, background: float, seed: int,
           device=None, noise: bool = True) -> Capture:
    """Render a scene to noisy counts (or to expected counts if noise=False)."""
    vol = render_points(geom, scene.points, device=device)
    if scene.patches:
        vol = vol + render_patches(geom, scene.patches, device=device)
    m = vol.max()
    if m > 0:
        vol = vol * (peak / m)
    lam = vol + background
    if noise:
        rng = np.random.Generator(np.random.PCG64(seed + 7919))
        counts = rng.poisson(lam).astype(np.float64)
    else:
        counts = lam
    return Capture(geometry=geom, scene=scene, counts=counts, expected=vol, seed=seed)


# ---------------------------------------------------------------------------
# Workloads (shapes, sizes and value distributions of the paper's captures)
# ---------------------------------------------------------------------------

WORKLOADS = {
    # index 0: confocal 32x32 over 1 m x 1 m, 256 bins of 32 ps, 3 points at
    # 0.4-1.2 m, ~1e3 peak counts + 0.5 background
    "fk_32x32x256": dict(index=0, geom=Geometry(32, 32, 256, 32e-12, 1.0, 1.0),
                         n_points=3, n_patches=0, zmin=0.4, zmax=1.2, peak=1e3),
    # index 1: confocal 128x128 over 2 m x 2 m, 1024 bins of 16 ps, 2 rectangles
    # (20-60 cm) + 5 points at 0.8-2.0 m
    "pf_128x128x1024": dict(index=1, geom=Geometry(128, 128, 1024, 16e-12, 2.0, 2.0),
                            n_points=5, n_patches=2, zmin=0.8, zmax=2.0, peak=1e3),
    # index 2: confocal 256x256 over 2 m x 2 m, 512 bins of 16 ps, 10 points +
    # 3 oriented patches at 0.3-1.1 m, peak log-uniform in [1e2, 1e4]
    "fk_256x256x512": dict(index=2, geom=Geometry(256, 256, 512, 16e-12, 2.0, 2.0),
                           n_points=10, n_patches=3, zmin=0.3, zmax=1.1, peak=None),
}


def make_capture(workload: str, capture_index: int = 0, *, device=None, noise: bool = True,
                 geom: Geometry | None = None) -> Capture:
    """Seeded capture for one of the named workloads.

    `geom` may override the grid (for scaled-down test cases of the same
    scene recipe).
    """
    spec = WORKLOADS[workload]
    seed = spec["index"] * 1000 + capture_index
    rng = np.random.Generator(np.random.PCG64(seed))
    g = geom if geom is not None else spec["geom"]
    scene = random_scene(g, rng, spec["n_points"], spec["n_patches"], spec["zmin"], spec["zmax"])
    peak = spec["peak"]
    if peak is None:
        peak = float(10.0 ** rng.uniform(2.0, 4.0))
    return render(g, scene, peak=peak, background=0.5, seed=seed, device=device, noise=noise)


def point_capture(geom: Geometry, points, *, peak: float = 1e3, background: float = 0.0,
                  seed: int = 0, noise: bool = False) -> Capture:
    """Capture of explicit point reflectors [(x, y, z, albedo), ...]."""
    scene = Scene(points=np.asarray(points, dtype=np.float64).reshape(-1, 4))
    return render(geom, scene, peak=peak, background=background, seed=seed, noise=noise)


# ---------------------------------------------------------------------------
# Photon streams: the SPAD records a photon binner consumes
# ---------------------------------------------------------------------------

@dataclass
class PhotonStream:
    pixel: np.ndarray        # uint32 wall index x * ny + y
    ticks: np.ndarray        # uint32 time of flight in integer ticks
    t0: int                  # tick of the start of bin 0
    ticks_per_bin: int


def photons_from_counts(counts: np.ndarray, *, ticks_per_bin: int = 16, t0: int = 1000, seed: int = 0,
                        order: str = "scan", stray: int = 0) -> PhotonStream:
    """One photon record per count of an integer [nx][ny][nt] histogram.

    Each photon gets a uniformly drawn tick inside its bin. order="scan" emits
    the wall points one after another (photons of a point in random time
    order, like a scanning capture); order="shuffled" interleaves all points.
    `stray` extra records fall outside the window (before t0, after the last
    bin, or on a wall index past the grid) and must be dropped by a binner.
    """
    c = np.asarray(counts)
    nx, ny, nt = c.shape
    flat = np.rint(c.reshape(-1)).astype(np.int64)
    idx = np.repeat(np.arange(flat.size, dtype=np.int64), flat)
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    pixel = idx // nt
    ticks = t0 + (idx % nt) * ticks_per_bin + rng.integers(0, ticks_per_bin, size=idx.size)
    if stray:
        k = np.arange(stray)
        sp = rng.integers(0, nx * ny, size=stray)
        st = np.where(k % 3 == 0, rng.integers(0, t0, size=stray),
                      t0 + nt * ticks_per_bin + rng.integers(0, 4 * ticks_per_bin, size=stray))
        sp = np.where(k % 3 == 2, nx * ny + rng.integers(0, 64, size=stray), sp)
        st = np.where(k % 3 == 2, t0 + rng.integers(0, nt * ticks_per_bin, size=stray), st)
        pixel = np.concatenate([pixel, sp])
        ticks = np.concatenate([ticks, st])
    if order == "shuffled":
        perm = rng.permutation(pixel.size)
    else:
        perm = np.lexsort((rng.random(pixel.size), pixel))
    return PhotonStream(pixel=pixel[perm].astype(np.uint32), ticks=ticks[perm].astype(np.uint32),
                        t0=int(t0), ticks_per_bin=int(ticks_per_bin))


def photon_frame(capture: Capture, n_photons: int, *, seed: int = 0, ticks_per_bin: int = 16,
                 order: str = "scan") -> PhotonStream:
    """About n_photons records drawn from a capture's expected counts (signal
    + the 0.5-count background, rescaled to the requested total)."""
    e = capture.expected
    e = e.cpu().numpy() if hasattr(e, "cpu") else e
    lam = np.asarray(e, dtype=np.float64) + 0.5
    lam = lam * (n_photons / lam.sum())
    rng = np.random.Generator(np.random.PCG64(seed + 15485863))
    return photons_from_counts(rng.poisson(lam), ticks_per_bin=ticks_per_bin, seed=seed, order=order)
