"""Seeded synthetic initial conditions for the SPH hot path.

This module is shared by the tests, the benchmark and the smoke check, for both
the CUDA library and the oracle.  It draws particle sets only; it holds none of
the method's arithmetic (no kernel, density, force or time-step formula).

Every generator returns a dict with
  pos  float64 [N, 3] in the periodic unit box [0, 1)^3
  vel  float64 [N, 3]
  m    float64 [N]      equal masses 1/N
  u    float64 [N]      specific internal energy
  h0   float64 [N]      initial smoothing-length guess eta * n_est^-1/3
  meta dict             the recipe and the realised statistics

The paper measures on EAGLE snapshots (clustered, deep time-bin hierarchy,
Fig. 1), which are not available; the clustered and Zel'dovich sets below stand
in for them.
"""
from __future__ import annotations

import math

import numpy as np

ETA = 1.2348


def _h_guess(n_est):
    return ETA * np.asarray(n_est, dtype=np.float64) ** (-1.0 / 3.0)


def lattice(nside: int, jitter: float = 0.1, seed: int = 1, u: float = 1.0):
    """nside^3 cubic lattice at cell centres, each coordinate jittered by
    U(-jitter, jitter) lattice spacings; equal masses, uniform u, v = 0."""
    rng = np.random.default_rng(seed)
    d = 1.0 / nside
    g = (np.arange(nside) + 0.5) * d
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    if jitter:
        pos = pos + rng.uniform(-jitter, jitter, size=pos.shape) * d
    pos %= 1.0
    n = pos.shape[0]
    return dict(pos=pos, vel=np.zeros((n, 3)), m=np.full(n, 1.0 / n), u=np.full(n, float(u)),
                h0=np.full(n, ETA * d),
                meta=dict(kind="lattice", nside=nside, jitter=jitter, seed=seed))


def sedov(nside: int = 64, seed: int = 2, n_hot: int = 32, energy: float = 1.0,
          u_background: float = 1e-5):
    """Sedov blast: jittered lattice, background u, and `energy` shared equally
    as internal energy by the n_hot particles nearest the box centre."""
    ic = lattice(nside, 0.1, seed, u_background)
    pos, m = ic["pos"], ic["m"]
    r2 = ((pos - 0.5) ** 2).sum(axis=1)
    hot = np.argsort(r2, kind="stable")[:n_hot]
    ic["u"][hot] = energy / (n_hot * m[hot])
    ic["meta"] = dict(kind="sedov", nside=nside, seed=seed, n_hot=n_hot, energy=energy,
                      u_background=u_background, hot_index=hot)
    return ic


def _plummer_radii(rng, a, count, rmax_over_a=10.0):
    """Radii of a Plummer sphere with scale radius a, truncated at rmax_over_a * a
    (inverse of the enclosed-mass fraction X = r^3 / (r^2 + a^2)^(3/2))."""
    out = np.empty(0)
    while out.size < count:
        X = rng.uniform(0.0, 1.0, size=2 * (count - out.size) + 16)
        X = X[X > 0]
        r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        out = np.concatenate([out, r[r <= rmax_over_a * a]])
    return out[:count]


def _unit_vectors(rng, count):
    v = rng.normal(size=(count, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _plummer_number_density(pos, centres, radii, per_sphere, chunk=1 << 18):
    """Sum over spheres of the analytic Plummer number density at pos
    (minimum-image distance in the unit box)."""
    out = np.zeros(pos.shape[0])
    norm = 3.0 * per_sphere / (4.0 * math.pi * radii ** 3)
    for s in range(0, pos.shape[0], chunk):
        p = pos[s:s + chunk]
        acc = np.zeros(p.shape[0])
        for c, a, nrm in zip(centres, radii, norm):
            d = p - c
            d -= np.round(d)
            r2 = (d * d).sum(axis=1)
            acc += nrm * (1.0 + r2 / (a * a)) ** -2.5
        out[s:s + chunk] = acc
    return out


def clustered(n_background: int = 1 << 20, n_spheres: int = 64, per_sphere: int = 1 << 14,
              a_min: float = 1e-3, a_max: float = 3e-2, seed: int = 3,
              bin_span: float = 13.0):
    """Uniform background plus Plummer spheres (scale radii log-uniform in
    [a_min, a_max], centres uniform).  u = 1 in the background and
    u = (n_est / n_bg)^beta in the spheres, beta chosen so that the CFL
    estimate dt ~ n^-1/3 u^-1/2 spans 2^bin_span between the densest particle
    and the background.  v = 0."""
    rng = np.random.default_rng(seed)
    bg = rng.uniform(0.0, 1.0, size=(n_background, 3))
    centres = rng.uniform(0.0, 1.0, size=(n_spheres, 3))
    radii = np.exp(rng.uniform(math.log(a_min), math.log(a_max), size=n_spheres))
    parts = [bg]
    for c, a in zip(centres, radii):
        r = _plummer_radii(rng, a, per_sphere)
        parts.append(c + r[:, None] * _unit_vectors(rng, per_sphere))
    pos = np.concatenate(parts) % 1.0
    n = pos.shape[0]
    n_bg = float(n_background)
    n_est = n_bg + _plummer_number_density(pos, centres, radii, per_sphere)
    contrast = n_est / n_bg
    # dt ratio between the densest particle and the background:
    # contrast_max^(1/3 + beta/2) = 2^bin_span
    cmax = float(contrast.max())
    beta = max(0.0, 2.0 * (bin_span * math.log(2.0) / math.log(cmax) - 1.0 / 3.0))
    u = np.ones(n)
    u[n_background:] = contrast[n_background:] ** beta
    return dict(pos=pos, vel=np.zeros((n, 3)), m=np.full(n, 1.0 / n), u=u, h0=_h_guess(n_est),
                meta=dict(kind="clustered", n_background=n_background, n_spheres=n_spheres,
                          per_sphere=per_sphere, a_min=a_min, a_max=a_max, seed=seed,
                          beta=beta, contrast_max=cmax, radii=radii, centres=centres))


def clumpy_lattice(nside: int = 32, n_clumps: int = 8, per_clump: int = 512,
                   a_min: float = 1e-3, a_max: float = 3e-2, seed: int = 4, u: float = 1.0):
    """Jittered lattice in which n_clumps * per_clump randomly chosen particles
    are moved into Plummer clumps (scale radii log-uniform)."""
    rng = np.random.default_rng(seed)
    ic = lattice(nside, 0.1, seed, u)
    pos = ic["pos"]
    n = pos.shape[0]
    moved = rng.choice(n, size=n_clumps * per_clump, replace=False)
    centres = rng.uniform(0.0, 1.0, size=(n_clumps, 3))
    radii = np.exp(rng.uniform(math.log(a_min), math.log(a_max), size=n_clumps))
    for k, (c, a) in enumerate(zip(centres, radii)):
        idx = moved[k * per_clump:(k + 1) * per_clump]
        r = _plummer_radii(rng, a, per_clump)
        pos[idx] = c + r[:, None] * _unit_vectors(rng, per_clump)
    pos %= 1.0
    n_bg = float(n - n_clumps * per_clump)
    n_est = n_bg + _plummer_number_density(pos, centres, radii, per_clump)
    ic.update(pos=pos, h0=_h_guess(n_est))
    ic["meta"] = dict(kind="clumpy_lattice", nside=nside, n_clumps=n_clumps,
                      per_clump=per_clump, seed=seed, radii=radii, centres=centres)
    return ic


def zeldovich(nside: int = 256, spectral_index: float = -2.5, rms_cells: float = 0.3,
              seed: int = 5, u: float = 1.0):
    """Zel'dovich-displaced lattice: Gaussian density contrast with
    P(k) ~ k^spectral_index up to the Nyquist frequency, displacement
    psi(k) = i k delta(k) / k^2, rescaled to an rms |psi| of rms_cells lattice
    spacings; v = 0, uniform u."""
    rng = np.random.default_rng(seed)
    n = nside
    d = 1.0 / n
    k1 = np.fft.fftfreq(n, d=d) * 2.0 * math.pi
    kz1 = np.fft.rfftfreq(n, d=d) * 2.0 * math.pi
    kx, ky, kz = np.meshgrid(k1, k1, kz1, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    knyq = math.pi * n
    amp = np.zeros_like(k2)
    ok = (k2 > 0) & (k2 <= knyq * knyq)
    amp[ok] = np.sqrt(k2[ok] ** (0.5 * spectral_index))
    noise = rng.normal(size=(n, n, n))
    delta_k = np.fft.rfftn(noise) * amp
    disp = []
    inv_k2 = np.zeros_like(k2)
    inv_k2[ok] = 1.0 / k2[ok]
    for kk in (kx, ky, kz):
        psi_k = 1j * kk * delta_k * inv_k2
        disp.append(np.fft.irfftn(psi_k, s=(n, n, n)).astype(np.float64))
    del delta_k, noise
    psi = np.stack([p.reshape(-1) for p in disp], axis=1)
    rms = float(np.sqrt((psi ** 2).sum(axis=1).mean()))
    psi *= rms_cells * d / rms
    g = (np.arange(n) + 0.5) * d
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    pos = (pos + psi) % 1.0
    N = pos.shape[0]
    return dict(pos=pos, vel=np.zeros((N, 3)), m=np.full(N, 1.0 / N), u=np.full(N, float(u)),
                h0=np.full(N, ETA * d),
                meta=dict(kind="zeldovich", nside=n, spectral_index=spectral_index,
                          rms_cells=rms_cells, seed=seed))


def subsample_active(n: int, count: int, seed: int = 0):
    """A seeded mask of `count` distinct particles out of n."""
    rng = np.random.default_rng(seed)
    mask = np.zeros(n, dtype=np.uint8)
    mask[rng.choice(n, size=min(count, n), replace=False)] = 1
    return mask
