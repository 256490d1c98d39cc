"""Seeded field generators (host, numpy).  No compressor arithmetic lives here."""
import numpy as np

try:  # scipy's FFT is multithreaded; numpy's is the fallback
    import scipy.fft as _fft
    _FFT_KW = {"workers": -1}
except Exception:  # pragma: no cover
    import numpy.fft as _fft
    _FFT_KW = {}


def _rescale(f, lo=-1.0, hi=1.0):
    fmin, fmax = float(f.min()), float(f.max())
    if fmax == fmin:
        return np.zeros_like(f)
    return (f - fmin) * ((hi - lo) / (fmax - fmin)) + lo


def gaussians(shape, seed, n_blobs=8, amp=(0.5, 2.0), width=(4.0, 16.0),
              noise=1e-3, dtype=np.float32):
    """Sum of ``n_blobs`` random Gaussians plus N(0, noise) white noise."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = tuple(int(s) for s in shape)
    grids = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape],
                        indexing="ij", sparse=True)
    f = np.zeros(shape, dtype=np.float64)
    for _ in range(n_blobs):
        centre = [rng.uniform(0, s) for s in shape]
        a = rng.uniform(*amp)
        sigma = rng.uniform(*width)
        r2 = sum((g - c) ** 2 for g, c in zip(grids, centre))
        f += a * np.exp(-r2 / (2.0 * sigma * sigma))
    f += rng.normal(0.0, noise, size=shape)
    return f.astype(dtype)


def grf(shape, seed, dtype=np.float32, slope=None):
    """Spectral Gaussian random field, |u_hat(k)| = k^slope, random phases.

    Default slope: -11/6 in 3-D and -4/3 in 2-D, both giving a shell energy
    spectrum E(k) ~ k^-5/3.  u_hat(0) = 0; the real field comes from an inverse
    real FFT of the half spectrum; the result is rescaled to [-1, 1].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    if slope is None:
        slope = -11.0 / 6.0 if nd == 3 else -4.0 / 3.0
    freqs = [np.fft.fftfreq(s) * s for s in shape[:-1]]
    freqs.append(np.fft.rfftfreq(shape[-1]) * shape[-1])
    half = tuple(len(f) for f in freqs)
    k2 = np.zeros(half, dtype=np.float64)
    for ax, f in enumerate(freqs):
        sh = [1] * nd
        sh[ax] = len(f)
        k2 = k2 + (f.reshape(sh) ** 2)
    k = np.sqrt(k2, out=k2)
    k[(0,) * nd] = 1.0
    amp = np.power(k, slope, out=k)
    amp[(0,) * nd] = 0.0
    phase = rng.random(half) * (2.0 * np.pi)
    spec = amp * np.exp(1j * phase)
    del amp, phase
    f = _fft.irfftn(spec, s=shape, **_FFT_KW)
    del spec
    return _rescale(f).astype(dtype)


def climate(shape, seed, dtype=np.float64, sigma_noise=0.3, smooth=1.5):
    """Zonal bands times lognormal small-scale noise (Miranda-shaped stand-in).

    Axes: (level z, latitude in [-pi/2, pi/2], longitude in [0, 2 pi)).
    f = sum_{k in 3,7,15} a_k cos(lat) sin(k lon + phi_k) (1 + 0.2 z / (nz-1))
        * exp(sigma_noise * g),  a = 1, 0.5, 0.25,
    g = white noise smoothed by a Gaussian of ``smooth`` cells, renormalised to
    unit variance.
    """
    from scipy.ndimage import gaussian_filter
    rng = np.random.Generator(np.random.PCG64(seed))
    nz, nlat, nlon = (int(s) for s in shape)
    z = np.arange(nz, dtype=np.float64).reshape(nz, 1, 1)
    lat = np.linspace(-np.pi / 2, np.pi / 2, nlat).reshape(1, nlat, 1)
    lon = (np.arange(nlon, dtype=np.float64) * (2 * np.pi / nlon)).reshape(1, 1, nlon)
    base = np.zeros((1, nlat, nlon))
    for k, a in ((3, 1.0), (7, 0.5), (15, 0.25)):
        phi = rng.uniform(0, 2 * np.pi)
        base = base + a * np.cos(lat) * np.sin(k * lon + phi)
    f = base * (1.0 + 0.2 * z / max(nz - 1, 1))
    g = gaussian_filter(rng.standard_normal((nz, nlat, nlon)), smooth)
    g /= g.std()
    f = f * np.exp(sigma_noise * g)
    return f.astype(dtype)


def polynomial(shape, seed, degree, dtype=np.float64):
    """Random separable-and-mixed polynomial of total degree <= ``degree``
    evaluated on integer coordinates scaled to [0, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    coords = np.meshgrid(*[np.arange(s, dtype=np.float64) / max(s - 1, 1)
                           for s in shape], indexing="ij")
    f = np.zeros(shape)
    import itertools
    for powers in itertools.product(range(degree + 1), repeat=nd):
        if sum(powers) > degree:
            continue
        term = rng.uniform(-1, 1)
        for c, p in zip(coords, powers):
            term = term * c ** p
        f = f + term
    return f.astype(dtype)


def random_field(shape, seed, dtype=np.float32, kind="grf"):
    if kind == "grf":
        return grf(shape, seed, dtype)
    if kind == "gaussians":
        return gaussians(shape, seed, dtype=dtype)
    if kind == "climate":
        return climate(shape, seed, dtype=dtype)
    if kind == "uniform":
        rng = np.random.Generator(np.random.PCG64(seed))
        return rng.uniform(-1, 1, size=shape).astype(dtype)
    raise ValueError(kind)


# The five evaluation workloads (synthetic stand-ins; see module docstring).
CONFIGS = {
    "c1_gaussians_64": dict(shape=(64, 64, 64), dtype="f32", kind="gaussians", seed=1),
    "c2_grf_512": dict(shape=(512, 512, 512), dtype="f32", kind="grf", seed=2),
    "c3_climate_256x384x384": dict(shape=(256, 384, 384), dtype="f64", kind="climate", seed=3),
    "c4_batch": dict(shapes=[(100, 500, 500)] * 32 + [(64, 256, 1024)] * 32
                     + [(1800, 3600)] * 32, dtype="f32", kind="grf", seed=1000),
    "c5_serving": dict(shapes=[(512, 512, 512)] * 48 + [(256, 256, 256)] * 192,
                       dtype="f32", kind="grf", seed=2000),
}


def config_field(name, index=0):
    cfg = CONFIGS[name]
    dt = np.float32 if cfg["dtype"] == "f32" else np.float64
    if "shape" in cfg:
        return random_field(cfg["shape"], cfg["seed"], dt, cfg["kind"])
    return random_field(cfg["shapes"][index], cfg["seed"] + index, dt, cfg["kind"])
