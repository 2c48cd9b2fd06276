"""Seeded synthetic inputs for standard synthesis (stand-ins for OSKAR SKA-Low
and LOFAR MeasurementSets, which are not available).

This module only draws the *data*: station layouts, Earth-rotated positions,
point-source skies, visibilities from the measurement model of Sec. 2.1
(V = sum_s sigma_s e_s e_s^H + noise, with e_{s,i} = exp(+j 2 pi <r_s, p_i>/wl),
a column of Psi^*), pixel grids and gains. It holds none of the imaging
method's arithmetic (no Gram matrix, eigensolve or synthesis) and imports
neither the GPU library nor the CPU oracle; both consume what it returns.

Every generator takes a ``numpy.random.Generator``; ``make_config(i)`` seeds
``default_rng(1000 + i)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

EARTH_RATE_DEG_PER_H = 15.0
LATITUDE_DEG = -30.0  # SKA-Low-like site


def pixel_grid(n_side: int, cap_deg: float) -> np.ndarray:
    """Orthographic grid on the unit-sphere cap around +z.

    l, m uniform on [-sin(cap), sin(cap)] (n_side points each, endpoints
    included), r = (l, m, sqrt(1 - l^2 - m^2)); pixel index = il + n_side*im.
    Returns (n_side^2, 3) float64.
    """
    s = math.sin(math.radians(cap_deg))
    ax = np.linspace(-s, s, n_side)
    m, l = np.meshgrid(ax, ax, indexing="ij")  # l fastest
    l = l.ravel()
    m = m.ravel()
    n = np.sqrt(np.clip(1.0 - l * l - m * m, 0.0, None))
    return np.stack([l, m, n], axis=1)


def _reject_min_sep(cands_fn, n: int, min_sep: float, rng: np.random.Generator) -> np.ndarray:
    pts: list[np.ndarray] = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > 200000:
            raise RuntimeError("could not place stations with the requested minimum separation")
        p = cands_fn(rng)
        if pts:
            arr = np.asarray(pts)
            if np.min(np.sum((arr[:, :2] - p[:2]) ** 2, axis=1)) < min_sep * min_sep:
                continue
        pts.append(p)
    return np.asarray(pts)


def layout_disk(n: int, radius_m: float, z_sigma_m: float, min_sep_m: float,
                rng: np.random.Generator) -> np.ndarray:
    """n stations uniform in a disk of the given radius, z ~ N(0, z_sigma)."""
    def cand(r):
        rad = radius_m * math.sqrt(r.uniform())
        ang = r.uniform(0, 2 * math.pi)
        return np.array([rad * math.cos(ang), rad * math.sin(ang), r.normal(0, z_sigma_m)])
    return _reject_min_sep(cand, n, min_sep_m, rng)


def layout_lognormal(n: int, median_m: float, sigma: float, r_min_m: float, r_max_m: float,
                     z_sigma_m: float, min_sep_m: float, rng: np.random.Generator) -> np.ndarray:
    """SKA-Low-like layout: radius ~ lognormal(ln median, sigma) truncated to
    [r_min, r_max], uniform angle, z ~ N(0, z_sigma)."""
    def cand(r):
        while True:
            rad = math.exp(r.normal(math.log(median_m), sigma))
            if r_min_m <= rad <= r_max_m:
                break
        ang = r.uniform(0, 2 * math.pi)
        return np.array([rad * math.cos(ang), rad * math.sin(ang), r.normal(0, z_sigma_m)])
    return _reject_min_sep(cand, n, min_sep_m, rng)


def earth_rotate(p0: np.ndarray, t_s: float, lat_deg: float = LATITUDE_DEG) -> np.ndarray:
    """Rotate positions (n, 3) by the Earth-rotation angle 15 deg/h * t about
    the axis a = (0, cos(lat), sin(lat)) (Rodrigues' formula); the sky is
    fixed and +z is the cap centre."""
    th = math.radians(EARTH_RATE_DEG_PER_H * t_s / 3600.0)
    phi = math.radians(lat_deg)
    a = np.array([0.0, math.cos(phi), math.sin(phi)])
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    R = np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * (K @ K)
    return p0 @ R.T


def sources_in_cap(n_src: int, cap_deg: float, rng: np.random.Generator) -> np.ndarray:
    """Directions uniform on the spherical cap: cos(theta) ~ U[cos cap, 1]."""
    ct = rng.uniform(math.cos(math.radians(cap_deg)), 1.0, n_src)
    st = np.sqrt(1 - ct * ct)
    ph = rng.uniform(0, 2 * math.pi, n_src)
    return np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)


def flux_lognormal(n_src: int, rng: np.random.Generator, mu: float = 0.0, sigma: float = 1.0) -> np.ndarray:
    return np.exp(rng.normal(mu, sigma, n_src))


def flux_powerlaw(n_src: int, rng: np.random.Generator, index: float = -1.8,
                  s_min: float = 0.1, s_max: float = 100.0) -> np.ndarray:
    """dN/dS ~ S^index on [s_min, s_max], by inverse CDF."""
    a = index + 1.0  # CDF ~ S^a
    u = rng.uniform(0, 1, n_src)
    return (s_min ** a + u * (s_max ** a - s_min ** a)) ** (1.0 / a)


def visibilities(st_xyz: np.ndarray, wl: float, src_dir: np.ndarray, src_flux: np.ndarray,
                 snr: float | None, rng: np.random.Generator) -> np.ndarray:
    """Measurement model of Sec. 2.1: V = E diag(sigma) E^H + N with
    E_{i,s} = exp(+j 2 pi <r_s, p_i> / wl) and Hermitian complex Gaussian
    noise N = (X + X^H)/2, X_ij ~ CN(0, 1), scaled to ||V_sig||_F/||N||_F = snr.
    Returns (n_st, n_st) complex128, Hermitian."""
    ph = 2.0 * math.pi * (st_xyz @ src_dir.T) / wl
    E = np.exp(1j * ph)
    Vs = (E * src_flux[None, :]) @ E.conj().T
    Vs = 0.5 * (Vs + Vs.conj().T)
    if snr is None:
        return Vs
    n = st_xyz.shape[0]
    X = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) / math.sqrt(2.0)
    N = 0.5 * (X + X.conj().T)
    N *= np.linalg.norm(Vs) / (snr * np.linalg.norm(N))
    return Vs + N


def gains(n_st: int, sigma: float, rng: np.random.Generator) -> np.ndarray:
    """Complex station gains 1 + N(0, sigma) + j N(0, sigma)."""
    return 1.0 + rng.normal(0, sigma, n_st) + 1j * rng.normal(0, sigma, n_st)


@dataclass
class SSInput:
    """One standard-synthesis problem set: T steps at one wavelength."""
    name: str
    wl: float
    pix: np.ndarray                 # (n_pix, 3)
    st_xyz: list                    # T arrays (n_st_t, 3)
    vis: list                       # T arrays (n_st_t, n_st_t) complex
    n_eig: int
    n_level: int
    src_dir: np.ndarray = field(default=None)
    src_flux: np.ndarray = field(default=None)
    extra: dict = field(default_factory=dict)

    @property
    def n_pix(self) -> int:
        return self.pix.shape[0]

    @property
    def n_t(self) -> int:
        return len(self.vis)


def make_steps(p0: np.ndarray, n_t: int, dt_s: float, wl: float, src_dir, src_flux, snr, rng,
               vis_dtype=np.complex128):
    st, vis = [], []
    for t in range(n_t):
        p = earth_rotate(p0, t * dt_s)
        st.append(p)
        vis.append(visibilities(p, wl, src_dir, src_flux, snr, rng).astype(vis_dtype).astype(np.complex128))
    return st, vis


def make_config(i: int, *, n_t: int | None = None, n_side: int | None = None, seed: int | None = None) -> SSInput:
    """Synthetic problem shaped like configuration i of the benchmark table:

    0: 24 stations in a 2 km-diameter disk, wl 2 m, 10 steps, 20 lognormal
       sources in a 10 deg cap, SNR 20, N_eig 12, 4 levels, 64^2 px, FP64.
    1: 512 SKA-Low-like stations (lognormal radius to 65 km), wl 2 m, 100 steps,
       500 power-law sources, SNR 20, N_eig 64, 4 levels, 1024^2 px in a 20 deg
       cap, visibilities rounded to complex64.
    2: same inputs as 1 (precision variant).
    4: 256 stations (subset of the 512 layout), 512^2 px, 16 steps, N_eig 32.
    (Configuration 3, the multi-channel batch, is ``make_batch_config``.)
    ``n_t`` / ``n_side`` shrink the problem for tests without changing the
    layout or the sky.
    """
    rng = np.random.default_rng(1000 + i if seed is None else seed)
    if i == 0:
        p0 = layout_disk(24, 1000.0, 5.0, 10.0, rng)
        wl, T, cap, side, n_eig = 2.0, 10, 10.0, 64, 12
        src = sources_in_cap(20, cap, rng)
        flux = flux_lognormal(20, rng)
        vdt = np.complex128
    elif i in (1, 2):
        p0 = layout_lognormal(512, 1000.0, 1.0, 20.0, 65000.0, 5.0, 35.0, rng)
        wl, T, cap, side, n_eig = 2.0, 100, 20.0, 1024, 64
        src = sources_in_cap(500, cap, rng)
        flux = flux_powerlaw(500, rng)
        vdt = np.complex64
    elif i == 4:
        rng1 = np.random.default_rng(1001)
        full = layout_lognormal(512, 1000.0, 1.0, 20.0, 65000.0, 5.0, 35.0, rng1)
        p0 = full[np.sort(rng.choice(512, 256, replace=False))]
        wl, T, cap, side, n_eig = 2.0, 16, 10.0, 512, 32
        src = sources_in_cap(500, cap, rng)
        flux = flux_powerlaw(500, rng)
        vdt = np.complex64
    else:
        raise ValueError(f"no single-channel configuration {i}")
    T = T if n_t is None else n_t
    side = side if n_side is None else n_side
    st, vis = make_steps(p0, T, 60.0, wl, src, flux, 20.0, rng, vdt)
    return SSInput(name=f"config{i}", wl=wl, pix=pixel_grid(side, cap), st_xyz=st, vis=vis,
                   n_eig=n_eig, n_level=4, src_dir=src, src_flux=flux,
                   extra={"cap_deg": cap, "n_side": side, "p0": p0})


def make_nufft_config(*, n_t: int = 50, n_side: int = 1024, pix_arcsec: float = 4.0, hours: float = 6.0,
                      n_st: int = 512, seed: int = 1005) -> SSInput:
    """Workload of the NUFFT-synthesis comparison (Sec. 5: 512 SKA-Low-like
    stations, 50 steps spread over 6 hours, pixels of 4 arcsec, so that the
    field of view grows with the image size): the 512-station layout of
    configuration 1 (its first n_st stations), wl 2 m, 500 power-law sources
    within the field, SNR 20, N_eig 64, 4 levels; n_side^2 pixels spaced
    pix_arcsec apart in l and m around +z; visibilities rounded to complex64."""
    rng1 = np.random.default_rng(1001)
    p0 = layout_lognormal(512, 1000.0, 1.0, 20.0, 65000.0, 5.0, 35.0, rng1)[:n_st]
    rng = np.random.default_rng(seed)
    half = 0.5 * (n_side - 1) * math.radians(pix_arcsec / 3600.0)  # half-width in l, m
    cap = math.degrees(math.asin(half))
    src = sources_in_cap(500, cap, rng)
    flux = flux_powerlaw(500, rng)
    st, vis = make_steps(p0, n_t, hours * 3600.0 / n_t, 2.0, src, flux, 20.0, rng, np.complex64)
    return SSInput(name="nufft", wl=2.0, pix=pixel_grid(n_side, cap), st_xyz=st, vis=vis, n_eig=64, n_level=4,
                   src_dir=src, src_flux=flux,
                   extra={"cap_deg": cap, "n_side": n_side, "p0": p0, "pix_arcsec": pix_arcsec})


def make_batch_config(n_chan: int = 64, n_t: int = 20, n_side: int = 512, seed: int = 1003,
                      wl_lo: float = 1.5, wl_hi: float = 3.0, n_st_lo: int = 48, n_st_hi: int = 512,
                      n_eig_lo: int = 8, n_eig_hi: int = 64, sizes=None):
    """Batched multi-channel workload: n_chan channels (wl linear on
    [wl_lo, wl_hi]) x n_t steps; per problem a random flagging of the
    512-station layout keeps n_st ~ U{n_st_lo..n_st_hi} stations and asks for
    n_eig ~ U{n_eig_lo..min(n_eig_hi, n_st)} eigenpairs. sizes: optional
    [n_chan][n_t] list of (n_st, n_eig) that replaces those draws (the
    flagging itself stays random). Returns a list of per-channel dicts with
    keys wl, st_xyz (list), vis (list), n_eig (list)."""
    rng = np.random.default_rng(seed)
    rng1 = np.random.default_rng(1001)
    full = layout_lognormal(512, 1000.0, 1.0, 20.0, 65000.0, 5.0, 35.0, rng1)
    cap = 10.0
    src = sources_in_cap(500, 20.0, rng)
    flux = flux_powerlaw(500, rng)
    chans = []
    for c in range(n_chan):
        wl = wl_lo + (wl_hi - wl_lo) * (c / max(1, n_chan - 1))
        sts, viss, neigs = [], [], []
        for t in range(n_t):
            n_st = int(rng.integers(n_st_lo, n_st_hi + 1))
            if sizes is not None:
                n_st = int(sizes[c][t][0])
            keep = np.sort(rng.choice(512, n_st, replace=False))
            p = earth_rotate(full[keep], t * 60.0)
            sts.append(p)
            viss.append(visibilities(p, wl, src, flux, 20.0, rng).astype(np.complex64).astype(np.complex128))
            k = int(rng.integers(n_eig_lo, min(n_eig_hi, n_st) + 1))
            neigs.append(int(sizes[c][t][1]) if sizes is not None else k)
        chans.append({"wl": wl, "st_xyz": sts, "vis": viss, "n_eig": neigs})
    return {"pix": pixel_grid(n_side, cap), "channels": chans, "n_level": 4, "cap_deg": cap}
