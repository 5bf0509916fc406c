"""Seeded synthetic inputs for the porosity-wave PT solver.

This module is shared by the CPU oracle (tests, CPU baseline) and the CUDA path. It only builds
*inputs*: parameter sets and initial fields. It holds none of the method's arithmetic: no
rheology, no PT update, no derived coefficient (background density, pseudo-time steps and
initial viscosities are computed by each implementation on its own side).

Array convention: every field is a C-ordered ``numpy.float64`` array of shape
``(nz_s, ny_s, nx_s)`` (x fastest), where ``(nx_s, ny_s, nz_s)`` is the staggered size of the
field (``nx`` cells in x for cell-centred fields, ``nx + 1`` for x-faces, and so on).

Workloads (thesis Art. 1, Sections 2.1-2.2, Table 2; nondimensional units):

* ``c1_params`` — the 32^3 single-step case: phi0 = 0.01, one centred Gaussian anomaly of added
  amplitude 2*phi0 and width 0.1, k0 = 1, mu0 = 1, eta0 = 1, weakening multiplier 0.01 where
  Pf > Pt, power-law exponent 3 with tau0 = 0.04 (Table 2), Biot alpha = 0.9 and Skempton
  B = 0.89 (Table 2), compressibilities beta_phi = 1e-2, beta_d = 1.3 beta_phi and shear modulus
  G = 0.5 / beta_phi (ratios of the appendix two-phase script), rho_f g = 1, rho_s g = 2.
* ``large_params`` — the same model at any n (511^3 is the benchmark grid) with a seeded
  anomaly position (centre + U(-0.05, 0.05)^3).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "c1_params", "large_params", "gaussian_porosity", "perturbed_centre",
    "field_shapes", "random_state", "ensemble", "PARAM_KEYS", "shear_params", "ellipsoid_porosity",
    "rx_params", "rx_initial",
]

# Parameter names as used at both boundaries (C ABI struct members and the oracle's struct).
PARAM_KEYS = (
    # grid
    "nx", "ny", "nz", "lx", "ly", "lz",
    # physics
    "phi0", "k0", "mu0", "eta0", "R_weak", "n_pow", "tau0", "alpha", "B", "beta_d", "beta_phi",
    "G", "rhof_g", "rhos_g", "powerlaw_on", "compaction_on", "tau_bg",
    # numerics
    "dt", "tol", "max_iter", "nup", "damp_x", "damp_y", "damp_z", "rho_i", "beta_n",
    "rel_mu", "rel_eta", "cfl_v", "cfl_pf", "dtpt_scale", "xsi_w",
)


def c1_params(nx: int = 32, ny: int | None = None, nz: int | None = None) -> dict:
    """Parameter set of the single-step 32^3 workload (any grid size may be passed)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    beta_phi = 1e-2
    return dict(
        nx=nx, ny=ny, nz=nz, lx=1.0, ly=1.0, lz=1.0,
        phi0=0.01, k0=1.0, mu0=1.0, eta0=1.0, R_weak=0.01, n_pow=3.0, tau0=0.04,
        alpha=0.9, B=0.89, beta_d=1.3 * beta_phi, beta_phi=beta_phi, G=0.5 / beta_phi,
        rhof_g=1.0, rhos_g=2.0, powerlaw_on=1, compaction_on=1, tau_bg=0.0,
        dt=1e-4 * (32.0 / max(nx, ny, nz)) ** 2, tol=1e-8, max_iter=20000, nup=15,
        damp_x=1.0 - 1.0 / nx, damp_y=1.0 - 1.0 / ny, damp_z=1.0 - 1.0 / nz,
        rho_i=1.0, beta_n=0.0, rel_mu=0.1, rel_eta=0.5,
        cfl_v=1.0 / 6.1, cfl_pf=1.0 / 6.1, dtpt_scale=1.0, xsi_w=1.0,
    )


def large_params(n: int = 511, max_iter: int = 20000) -> dict:
    """Same model and parameters on an n^3 grid (the benchmark uses n = 511)."""
    p = c1_params(n)
    p["max_iter"] = max_iter
    return p


def field_shapes(nx: int, ny: int, nz: int) -> dict:
    """Staggered (z, y, x) shapes of every field (thesis Art. 1, Fig. 1 placement)."""
    return dict(
        centre=(nz, ny, nx),
        Vx=(nz, ny, nx + 1), Vy=(nz, ny + 1, nx), Vz=(nz + 1, ny, nx),
        txy=(nz, ny + 1, nx + 1), txz=(nz + 1, ny, nx + 1), tyz=(nz + 1, ny + 1, nx),
    )


def perturbed_centre(seed: int, base=(0.5, 0.5, 0.5), half_width: float = 0.05) -> tuple:
    """Anomaly centre = base + U(-half_width, half_width)^3 from numpy's PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.uniform(-half_width, half_width, size=3)
    return tuple(float(b + x) for b, x in zip(base, d))


def gaussian_porosity(p: dict, centres=((0.5, 0.5, 0.5),), amp: float | None = None,
                      width: float = 0.1) -> np.ndarray:
    """Initial porosity at cell centres: phi0 + sum_a amp * exp(-(|x - x_a| / width)^2).

    Cell-centred grid on [0, lx] x [0, ly] x [0, lz] with dx = lx / nx; centres are given as
    fractions of the box lengths. ``amp`` defaults to 2 * phi0 (added amplitude).
    """
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    lx, ly, lz = p["lx"], p["ly"], p["lz"]
    phi0 = p["phi0"]
    amp = 2.0 * phi0 if amp is None else amp
    x = (np.arange(nx) + 0.5) * (lx / nx)
    y = (np.arange(ny) + 0.5) * (ly / ny)
    z = (np.arange(nz) + 0.5) * (lz / nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    phi = np.full((nz, ny, nx), phi0, dtype=np.float64)
    for (cx, cy, cz) in centres:
        r2 = (X - cx * lx) ** 2 + (Y - cy * ly) ** 2 + (Z - cz * lz) ** 2
        phi += amp * np.exp(-r2 / width ** 2)
    return phi


def random_state(p: dict, seed: int, scale: float = 1e-3) -> dict:
    """A seeded, smooth-ish random mid-solve state (for parity tests that start off-rest).

    Velocities on interior faces, pressures, stresses and old-step fields are uniform random of
    the given scale; porosity is phi0 * (1 + 0.5 U(0,1)); boundary-normal velocities and
    boundary-edge shear stresses are zero (free-slip). Viscosities are *not* produced: each
    implementation initialises them from the porosity itself.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    sh = field_shapes(nx, ny, nz)
    out = {}
    for name in ("Vx", "Vy", "Vz"):
        out[name] = scale * rng.standard_normal(sh[name])
    out["Vx"][:, :, 0] = 0.0; out["Vx"][:, :, -1] = 0.0
    out["Vy"][:, 0, :] = 0.0; out["Vy"][:, -1, :] = 0.0
    out["Vz"][0, :, :] = 0.0; out["Vz"][-1, :, :] = 0.0
    for name in ("Pt", "Pf"):
        out[name] = scale * rng.standard_normal(sh["centre"])
    out["phi"] = p["phi0"] * (1.0 + 0.5 * rng.uniform(size=sh["centre"]))
    for name in ("txx", "tyy", "tzz"):
        out[name] = scale * rng.standard_normal(sh["centre"])
    out["txy"] = scale * rng.standard_normal(sh["txy"])
    out["txy"][:, 0, :] = 0; out["txy"][:, -1, :] = 0; out["txy"][:, :, 0] = 0; out["txy"][:, :, -1] = 0
    out["txz"] = scale * rng.standard_normal(sh["txz"])
    out["txz"][0, :, :] = 0; out["txz"][-1, :, :] = 0; out["txz"][:, :, 0] = 0; out["txz"][:, :, -1] = 0
    out["tyz"] = scale * rng.standard_normal(sh["tyz"])
    out["tyz"][0, :, :] = 0; out["tyz"][-1, :, :] = 0; out["tyz"][:, 0, :] = 0; out["tyz"][:, -1, :] = 0
    return out


def ensemble(seed: int = 0, n_inst: int = 64, sizes=(32, 48, 64, 96, 127), max_iter: int = 40000):
    """Seeded ensemble of independent instances: [(params, phi), ...].

    Instance i draws (numpy PCG64(seed), in order) its grid size n ~ U{sizes} (n^3 cells), the
    weakening multiplier R_weak ~ U[0.01, 0.2], the background porosity phi0 ~ U[0.005, 0.02]
    and 1-3 Gaussian anomalies (added amplitude 2 phi0, width 0.1) centred at U[0.2, 0.8]^3;
    every other parameter is that of the 32^3 workload at grid size n.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n_inst):
        n = int(rng.choice(np.asarray(sizes)))
        R = float(rng.uniform(0.01, 0.2))
        phi0 = float(rng.uniform(0.005, 0.02))
        na = int(rng.integers(1, 4))
        centres = [tuple(float(x) for x in rng.uniform(0.2, 0.8, size=3)) for _ in range(na)]
        p = c1_params(n)
        p.update(R_weak=R, phi0=phi0, max_iter=max_iter)
        out.append((p, gaussian_porosity(p, centres=centres)))
    return out


def gaussian_random_field(shape, seed: int, corr_len: float = 0.1, std: float = 0.5) -> np.ndarray:
    """Seeded Gaussian random field on the unit box (cell-centred, shape (nz, ny, nx)): white
    noise filtered in Fourier space by a Gaussian of correlation length `corr_len`, rescaled to
    standard deviation `std` (log-permeability prefactor fields for the adjoint's inputs)."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape)
    ks = [np.fft.fftfreq(n, d=1.0 / n) for n in shape]
    kz, ky, kx = np.meshgrid(*ks, indexing="ij")
    filt = np.exp(-0.5 * (2 * np.pi * corr_len) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    f = np.real(np.fft.ifftn(np.fft.fftn(w) * filt))
    f -= f.mean()
    sd = f.std()
    return f * (std / sd) if sd > 0 else f


def shear_params(nx: int = 64, ny: int | None = None, nz: int | None = None, dt: float = 1e-5) -> dict:
    """The background-shear workload of thesis Art. 1 Section 3.1 (Table 2), scaled down: a
    30 x 30 x 60 box sheared by tau_bg = 1, K_phi = 333.33 (beta_phi = 3e-3), G = 166.66,
    decompaction weakening factor R0 = 2000 (bulk viscosity / 2000 where Pf > Pt), n = 3,
    tau0 = 0.04; drained compressibility 1.3 beta_phi and phi0 = 1e-2 as in the appendix script."""
    ny = nx if ny is None else ny
    nz = 2 * nx if nz is None else nz
    p = c1_params(nx, ny, nz)
    beta_phi = 1.0 / 333.33
    p.update(lx=30.0, ly=30.0, lz=60.0, R_weak=1.0 / 2000.0, beta_phi=beta_phi, beta_d=1.3 * beta_phi,
             G=166.66, tau_bg=1.0, dt=dt)
    return p


def ellipsoid_porosity(p: dict, centre=(0.5, 0.5, 0.2), axes=(14.0, 14.0, 3.5), factor: float = 2.0):
    """Porosity phi0 with an ellipsoid of `factor` phi0 (Table 2: axis lengths 14 x 14 x 3.5,
    twice the background porosity), centred at `centre` in fractions of the box (one fifth of
    the height), sampled at the cell centres; shape (nz, ny, nx)."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    x = (np.arange(nx) + 0.5) * p["lx"] / nx - centre[0] * p["lx"]
    y = (np.arange(ny) + 0.5) * p["ly"] / ny - centre[1] * p["ly"]
    z = (np.arange(nz) + 0.5) * p["lz"] / nz - centre[2] * p["lz"]
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    r2 = (xx / (0.5 * axes[0])) ** 2 + (yy / (0.5 * axes[1])) ** 2 + (zz / (0.5 * axes[2])) ** 2
    return np.where(r2 <= 1.0, factor * p["phi0"], p["phi0"])


def rx_params(nx: int = 32, ny: int | None = None, nz: int | None = None, Da: float = 100.0,
              dt: float = 1e-6) -> dict:
    """Reactive porosity-wave workload of thesis Art. 3 (appendix A.6 values, nondimensional in
    the compaction length, compaction pressure and viscous time): box lz = 50, lx = ly = lz / 4
    (nz = 4 nx by default), Deborah number 1e-3 (beta_d = 1e-3), beta_s = 11/12 beta_d,
    beta_f = 6 beta_d, rho_s = 1.5, rho_f = 0.5, g = 1, Clapeyron slope -1 (d Xs_eq / d Pf = -0.2),
    Delta X = 3, Xs_max = 0.05, phi0 = 0.01, Damkoehler number Da (reaction time 1 / Da)."""
    ny = nx if ny is None else ny
    nz = 4 * nx if nz is None else nz
    beta_d = 1e-3
    return dict(nx=nx, ny=ny, nz=nz, lx=12.5, ly=12.5, lz=50.0, phi0=0.01, k0=1.0, eta=1.0,
                rhof=0.5, rhos=1.5, g=1.0, beta_d=beta_d, beta_s=beta_d * 11.0 / 12.0, beta_f=6.0 * beta_d,
                beta_x=-0.2, dX=3.0, xs_max=0.05, tau=1.0 / Da, dt=dt, tol=2e-8, cfl_div=16.1,
                pf_scale=10.0, max_iter=20000, nup=10)


def rx_initial(p: dict):
    """Two vertically stacked Gaussian porosity anomalies (amplitudes 1.5 phi0 at 0.1 lz and
    0.75 phi0 at 0.23 lz, widths 0.12 lx horizontally and 0.03 lz vertically) on phi0, Xs at
    half its maximum, zero fluid pressure: (Pf, phi, Xs), each (nz, ny, nx)."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    x = (np.arange(nx) + 0.5) * p["lx"] / nx - 0.5 * p["lx"]
    y = (np.arange(ny) + 0.5) * p["ly"] / ny - 0.5 * p["ly"]
    z = (np.arange(nz) + 0.5) * p["lz"] / nz
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    rh, rv = 0.12 * p["lx"], 0.03 * p["lz"]
    g = lambda zc: np.exp(-(xx / rh) ** 2 - (yy / rh) ** 2 - ((zz - zc * p["lz"]) / rv) ** 2)
    phi = p["phi0"] + 1.5 * p["phi0"] * g(0.1) + 0.75 * p["phi0"] * g(0.23)
    return np.zeros_like(phi), phi, np.full_like(phi, 0.5 * p["xs_max"])
