"""Seeded synthetic inputs shared by the tests, the oracle runs and the benchmark.

This module only draws and describes inputs: instrument and sky parameters,
beam transfer functions, prior spectra, mixing scalars, smooth noise-depth
patterns, masks and Gaussian draws.  It holds none of the solver's
arithmetic (no transforms, no operators, no preconditioner) and imports
neither the oracle nor the CUDA library.  Pixel positions and quadrature
weights, where a recipe needs them, are passed in by the caller.

The recipes stand in for the paper's Planck inputs (RMS maps, beams, C_l),
which are not available: Gaussian beams with the FWHMs of the workloads, power-law
spectra, power-law mixing (q = (nu/nu_0)^beta, flat for the CMB) and a
smooth scan-depth pattern sigma(n) = sigma_nu * contrast^s(n), s in [0, 1] a
band-limited field (a random polynomial of degree <= 8 in the Cartesian
coordinates of n, hence band-limited at l <= 8).  Prior amplitudes are set
so that S^-1 crosses the approximate diagonal of P^T N^-1 P at a fixed
fraction of L_k, the rule the paper uses when it downgrades its inputs
(Sec. 5).
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED_BASE = 1710_00621
ARCMIN = np.pi / (180.0 * 60.0)


def ell_of_index(lmax):
    """l of each packed real coefficient (m = 0 block, then cos/sin blocks per m)."""
    out = [np.arange(lmax + 1)]
    for m in range(1, lmax + 1):
        l = np.arange(m, lmax + 1)
        out += [l, l]
    return np.concatenate(out)


def beam_gaussian(fwhm_arcmin, lmax):
    """Gaussian beam transfer b_l = exp(-l(l+1) sigma_b^2 / 2), sigma_b = FWHM / sqrt(8 ln 2)."""
    sb = fwhm_arcmin * ARCMIN / np.sqrt(8.0 * np.log(2.0))
    l = np.arange(lmax + 1, dtype=np.float64)
    return np.exp(-0.5 * l * (l + 1.0) * sb * sb)


def cl_shape(kind, lmax):
    """Unnormalised prior spectrum C_l for l = 0..lmax."""
    l = np.arange(lmax + 1, dtype=np.float64)
    c = np.empty(lmax + 1)
    if kind == "cmb":                      # ~ 1/(l(l+1)), C_0 = C_1 = C_2
        c[2:] = 1.0 / (l[2:] * (l[2:] + 1.0))
        c[:2] = c[2] if lmax >= 2 else 1.0
    elif kind == "dust":                   # ~ l^-2.4, C_0 = C_1
        c[1:] = l[1:] ** -2.4
        c[0] = c[1] if lmax >= 1 else 1.0
    elif kind == "synch":                  # ~ l^-2.7, C_0 = C_1
        c[1:] = l[1:] ** -2.7
        c[0] = c[1] if lmax >= 1 else 1.0
    elif kind == "freefree":               # ~ l^-2.0, C_0 = C_1
        c[1:] = l[1:] ** -2.0
        c[0] = c[1] if lmax >= 1 else 1.0
    else:
        raise ValueError(kind)
    return c


def mixing_scalar(freq, beta, nu0):
    """q = (nu / nu0)^beta; beta None means a flat SED (q = 1, the CMB)."""
    if beta is None:
        return 1.0
    return (freq / nu0) ** beta


def smooth_field(z, phi, rng, degree=8, nterm=24):
    """Random band-limited (l <= degree) field in [0, 1] at positions (z = cos theta, phi)."""
    st = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    x, y = st * np.cos(phi), st * np.sin(phi)
    f = np.zeros_like(z)
    for _ in range(nterm):
        a, b, c = rng.integers(0, degree + 1, size=3)
        while a + b + c > degree:
            a, b, c = rng.integers(0, degree + 1, size=3)
        f += rng.normal() * x ** a * y ** b * z ** c
    lo, hi = f.min(), f.max()
    return (f - lo) / (hi - lo) if hi > lo else np.zeros_like(f)


def draw_alm(rng, cl, lmax):
    """Gaussian real coefficients with variance C_l (packed layout)."""
    ell = ell_of_index(lmax)
    return rng.standard_normal(ell.size) * np.sqrt(np.asarray(cl, dtype=np.float64)[ell])


@dataclass
class Band:
    freq: float
    grid: str              # "gl" or "healpix"
    n: int                 # GL: lmax (rings = lmax + 1); HEALPix: Nside
    lmax: int
    fwhm: float            # arcmin
    sigma: float           # noise rms per pixel (arbitrary units)
    contrast: float = 1.0  # max/min ratio of sigma over the sky
    nphi: Optional[int] = None


@dataclass
class Comp:
    name: str
    lmax: int
    cl_kind: Optional[str]     # None = no prior
    beta: Optional[float]
    nu0: float
    crossover: float = 0.4     # S^-1 meets diag(P^T N^-1 P) at l = crossover * L_k


@dataclass
class Workload:
    name: str
    seed: int
    bands: List[Band]
    comps: List[Comp]
    tol: float = 1e-6

    def q(self):
        return np.array([[mixing_scalar(b.freq, c.beta, c.nu0) for c in self.comps]
                         for b in self.bands])

    def beams(self):
        return [beam_gaussian(b.fwhm, b.lmax) for b in self.bands]

    def rng(self, stream=0):
        return np.random.default_rng([self.seed, stream])


def tiny_plain():
    """Ncomp = 2 (CMB, dust beta 1.6), Nobs = 3 (30/100/353 GHz), GL lmax 63 (64 x 127 px),
    FWHM 60/40/30 arcmin, sigma = 10 per pixel, full sky, scalar mixing, tol 1e-8."""
    bands = [Band(f, "gl", 63, 63, fw, 10.0) for f, fw in ((30.0, 60.0), (100.0, 40.0), (353.0, 30.0))]
    comps = [Comp("cmb", 63, "cmb", None, 1.0, 0.40), Comp("dust", 63, "dust", 1.6, 353.0, 0.75)]
    return Workload("tiny_gl63_2comp_3band", SEED_BASE + 0, bands, comps, tol=1e-8)


PLANCK_FREQS = (30.0, 44.0, 70.0, 100.0, 143.0, 217.0, 353.0, 545.0, 857.0)


def multires_fullsky(scale=1):
    """Ncomp = 3 (CMB L 2000, synch beta -3.0 L 500, dust beta 1.6 L 3000), Nobs = 9 HEALPix bands
    at Nside 256/512/1024 (L_nu = 3 Nside - 1), FWHM 33 -> 5 arcmin, sigma varying x3 over the sky.

    ``scale`` divides every Nside and band-limit (scale = 8 gives Nside 32/64/128)."""
    nsides = (256, 256, 256, 512, 512, 512, 1024, 1024, 1024)
    bands = []
    for i, (f, ns) in enumerate(zip(PLANCK_FREQS, nsides)):
        ns = ns // scale
        fw = 33.0 * (5.0 / 33.0) ** (i / 8.0) * scale
        bands.append(Band(f, "healpix", ns, 3 * ns - 1, fw, 1.0, contrast=3.0))
    comps = [Comp("cmb", 2000 // scale, "cmb", None, 1.0, 0.40),
             Comp("synch", 500 // scale, "synch", -3.0, 30.0, 0.35),
             Comp("dust", 3000 // scale, "dust", 1.6, 353.0, 0.75)]
    return Workload(f"multires_fullsky_nside{256 // scale}-{1024 // scale}", SEED_BASE + 1, bands, comps)


def differentiable(lmax=511):
    """Ncomp = 3 (CMB, synch beta -3.0, dust beta 1.6), Nobs = 5 (30/70/143/353/857 GHz), all
    on Gauss-Legendre grids at L = lmax (lmax + 1 rings x 2 lmax + 1 px), FWHM 40/30/20/15/10
    arcmin, sigma varying x3 over the sky, full sky, scalar mixing."""
    bands = [Band(f, "gl", lmax, lmax, fw, 10.0, contrast=3.0)
             for f, fw in ((30.0, 40.0), (70.0, 30.0), (143.0, 20.0), (353.0, 15.0), (857.0, 10.0))]
    comps = [Comp("cmb", lmax, "cmb", None, 1.0, 0.40),
             Comp("synch", lmax, "synch", -3.0, 30.0, 0.35),
             Comp("dust", lmax, "dust", 1.6, 353.0, 0.75)]
    return Workload(f"differentiable_gl{lmax}_3comp_5band", SEED_BASE + 5, bands, comps)


def harmonic_weight(lmax_comp, seed=SEED_BASE + 5):
    """Diagonal harmonic weight w_lm ~ U[0, 1] over a stacked component vector."""
    n = sum((L + 1) ** 2 for L in lmax_comp)
    return np.random.default_rng([seed, 7]).uniform(0.0, 1.0, n)


def sigma_map(band, z, phi, rng):
    """Per-pixel noise rms: sigma_nu * contrast^s(n) with s a smooth field in [0, 1]."""
    if band.contrast == 1.0:
        return np.full(z.shape, band.sigma)
    s = smooth_field(z, phi, rng)
    return band.sigma * band.contrast ** s


def prior_amplitudes(work, taus, weights):
    """C_{k,l} = amp_k * shape_k(l), amp_k set so that 1/C_{k,l_x} equals
    sum_nu q_{nu,k}^2 b_{nu,l_x}^2 <tau/w>_nu at l_x = crossover * L_k."""
    q = work.q()
    beams = work.beams()
    cls = []
    for k, c in enumerate(work.comps):
        if c.cl_kind is None:
            cls.append(None)
            continue
        shape = cl_shape(c.cl_kind, c.lmax)
        lx = max(2, int(round(c.crossover * c.lmax)))
        dsum = 0.0
        for nu, b in enumerate(work.bands):
            if lx <= b.lmax:
                dsum += q[nu, k] ** 2 * beams[nu][lx] ** 2 * float(np.mean(taus[nu] / weights[nu]))
        amp = 1.0 / (dsum * shape[lx]) if dsum > 0 else 1.0
        cls.append(amp * shape)
    return cls


def make_inputs(work, pixel_coords, pixel_weights, with_noise=True):
    """Draw every random input of a workload.

    pixel_coords[nu] = (z, phi) arrays and pixel_weights[nu] the quadrature weight of
    each pixel of band nu, supplied by the caller.  Returns a dict with tau (inverse
    noise variance maps), cl, q, beams, x_true (stacked), noise maps and sigma maps.
    Draw order: noise pattern, C_l, x_true, noise realisation.
    """
    taus, sigmas = [], []
    for nu, b in enumerate(work.bands):
        z, ph = pixel_coords[nu]
        s = sigma_map(b, z, ph, work.rng(100 + nu))
        sigmas.append(s)
        taus.append(1.0 / (s * s))
    cls = prior_amplitudes(work, taus, pixel_weights)
    rng = work.rng(1)
    x_parts = []
    for k, c in enumerate(work.comps):
        cl = cls[k] if cls[k] is not None else np.ones(c.lmax + 1)
        x_parts.append(draw_alm(rng, cl, c.lmax))
    noise = None
    if with_noise:
        rng_n = work.rng(2)
        noise = [sigmas[nu] * rng_n.standard_normal(sigmas[nu].size) for nu in range(len(work.bands))]
    return dict(tau=taus, sigma=sigmas, cl=cls, q=work.q(), beams=work.beams(),
                x_true=np.concatenate(x_parts), noise=noise)


def batched_uneven(nprob=64, lmin=128, lmax=1024, fmax=0.3, seed_offset=0):
    """Independent problems (Ncomp = 2: CMB + dust beta 1.6; Nobs = 3: 30/100/353 GHz) with
    band-limits L_p ~ U{lmin..lmax} on Gauss-Legendre grids and a galactic-band mask
    |b| < b0, sin b0 = f_p ~ U[0, fmax] (sky fraction f_p), applied through the mixing maps.
    Beams follow the resolution, as for maps downgraded to L_p: sigma_b = c_nu / L_p with
    c = 2.0 / 1.6 / 1.3, so the inverse-noise term has decayed by ~0.1 where the dust prior
    takes over (0.75 L_p).  Returns [(workload, f_p)]."""
    rng = np.random.default_rng([SEED_BASE + 3, seed_offset])
    out = []
    fwhm_per_sigma = np.sqrt(8.0 * np.log(2.0)) / ARCMIN
    for p in range(nprob):
        L = int(rng.integers(lmin, lmax + 1))
        f = float(rng.uniform(0.0, fmax))
        bands = [Band(fr, "gl", L, L, c / L * fwhm_per_sigma, 10.0)
                 for fr, c in ((30.0, 2.0), (100.0, 1.6), (353.0, 1.3))]
        comps = [Comp("cmb", L, "cmb", None, 1.0, 0.40), Comp("dust", L, "dust", 1.6, 353.0, 0.75)]
        w = Workload(f"batched_p{p}_gl{L}_f{f:.3f}", SEED_BASE + 3 + 1000 * (p + 1) + seed_offset,
                     bands, comps)
        out.append((w, f))
    return out


def galactic_mask(z, f):
    """1 outside the band |b| < b0 with sin b0 = f (b = 90 deg - theta, so sin b = z), 0 inside."""
    return (np.abs(z) >= f).astype(np.float64)


def masked_cr(scale=1):
    """Planck-shaped masked constrained realization at reduced resolution: Ncomp = 4 (CMB,
    synchrotron beta -3.0, dust beta 1.6, free-free beta -2.1 at nu_0 = 30 GHz), L_k = 511 / scale;
    Nobs = 9 HEALPix bands (30/44/70 GHz at Nside 128 / scale, 100-857 GHz at 256 / scale,
    L_nu = 3 Nside - 1), FWHM 33' -> 5' scaled by 4 scale (the downgrade), noise rms x3 smooth
    pattern.  The mask (``planck_like_mask``) enters through every mixing map."""
    nsides = (128, 128, 128, 256, 256, 256, 256, 256, 256)
    bands = []
    for i, (f, ns) in enumerate(zip(PLANCK_FREQS, nsides)):
        ns = ns // scale
        fw = 33.0 * (5.0 / 33.0) ** (i / 8.0) * 4 * scale
        bands.append(Band(f, "healpix", ns, 3 * ns - 1, fw, 1.0, contrast=3.0))
    L = 511 // scale
    comps = [Comp("cmb", L, "cmb", None, 1.0, 0.40),
             Comp("synch", L, "synch", -3.0, 30.0, 0.35),
             Comp("dust", L, "dust", 1.6, 353.0, 0.75),
             Comp("freefree", L, "freefree", -2.1, 30.0, 0.35)]
    return Workload(f"masked_cr_4comp_nside{128 // scale}-{256 // scale}", SEED_BASE + 3, bands, comps)


def planck_like_mask(z, phi, seed=SEED_BASE + 3, ndisk=200, band_deg=20.0):
    """1 inside the mask: the galactic band |b| < band_deg (sin b = z) and ndisk disks with
    centres uniform on the sphere and radii U[0.5, 3] degrees."""
    rng = np.random.default_rng([seed, 11])
    inside = np.abs(z) < np.sin(np.radians(band_deg))
    st = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    v = np.stack([st * np.cos(phi), st * np.sin(phi), z], axis=-1)
    cz = rng.uniform(-1.0, 1.0, ndisk)
    cp = rng.uniform(0.0, 2 * np.pi, ndisk)
    cs = np.sqrt(1.0 - cz * cz)
    c = np.stack([cs * np.cos(cp), cs * np.sin(cp), cz], axis=-1)
    rad = np.radians(rng.uniform(0.5, 3.0, ndisk))
    for k in range(ndisk):
        inside |= (v @ c[k]) >= np.cos(rad[k])
    return inside.astype(np.float64)

