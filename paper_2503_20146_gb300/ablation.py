"""Ablations of the PWF settings on a synthetic tomographic series.

The paper's supplementary Figs. S3-S5 compare tomograms retrieved without the
preconditioner (the phase is underestimated), with other oversampling ratios
gamma of the regularization window (Eq. (15); gamma = 0 switches the
regularizer off) and with other regularization weights alpha (alpha = 0 is no
regularization; a wrong alpha blurs delta or enhances edges). Here each
setting runs Algorithm S1 on every projection of a seeded phantom series
(``pwf_solve``), reconstructs delta and beta by filtered back projection
(``pwf_fbp``), and is scored against the phantom:

* ``delta_rel_err`` / ``beta_rel_err``: RMS error over the reconstruction disc
  of the scored slices, relative to the RMS of the true values;
* ``delta_ratio``: mean retrieved delta over mean true delta inside the
  objects (below 1 when the phase is underestimated);
* ``rmse_image_pct``: the RMSE image |y - f(x)| of the paper's Methods, averaged
  over pixels and projections, in per cent of the mean reference intensity
  (the detector intensity without the sample).

Every step of the path runs in the library's kernels; the scoring reductions
are plain PyTorch on the device.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

from . import pwf as P
from . import synth as S


@dataclass(frozen=True)
class Setting:
    name: str
    gamma: float = 1.0
    alpha: complex = 0.1 + 0.01j
    flags: int = 0


SETTINGS = (
    Setting("paper"),
    Setting("no_precond", flags=P.FLAG_NO_PRECOND),
    Setting("gamma_0", gamma=0.0),
    Setting("gamma_0.5", gamma=0.5),
    Setting("gamma_2", gamma=2.0),
    Setting("alpha_0", alpha=0j),
    Setting("alpha_0.01+0.001i", alpha=0.01 + 0.001j),
    Setting("alpha_1+0.1i", alpha=1.0 + 0.1j),
)


@dataclass
class Series:
    """A synthetic tomographic series and what the scores need."""
    w: S.Workload
    angles: np.ndarray
    psi_true: object       # torch complex64 [A][n][n]
    t: object              # torch complex64 [n][n]
    y: object              # torch float32 [A][n][n]
    delta_true: object     # torch float64 [rows][n][n]
    beta_true: object
    rows: tuple
    ref_mean: float        # mean detector intensity without the sample


def _rasterise(ph: S.EllipsoidPhantom, rows, n, torch, dev):
    c = torch.arange(n, dtype=torch.float64, device=dev) - n / 2 + 0.5
    Z, X = torch.meshgrid(c, c, indexing="ij")
    d = torch.zeros((len(rows), n, n), dtype=torch.float64, device=dev)
    b = torch.zeros_like(d)
    for k, row in enumerate(rows):
        yv = row - n / 2 + 0.5
        for i in range(len(ph.delta)):
            R = ph.rotations[i]
            A = torch.from_numpy(R @ np.diag(1.0 / ph.semi_axes[i] ** 2) @ R.T).to(dev)
            m = torch.stack([X - ph.centres[i][0], torch.full_like(X, yv - ph.centres[i][1]),
                             Z - ph.centres[i][2]], -1)
            inside = torch.einsum("...i,ij,...j->...", m, A, m) <= 1.0
            d[k] += float(ph.delta[i]) * inside
            b[k] += float(ph.beta[i]) * inside
    return d, b


def make_series(n_angles: int = 48, n: int = 256, delta_max: float = 2e-7, photons: float = 1e4,
                rows=None, seed: int = 0, device: str = "cuda") -> Series:
    """Phantom projections (exact ellipsoid chords), shared diffuser, and
    Poisson-noisy detector images from the library's forward model."""
    import torch
    base = S.WORKLOADS["tomo180x1024_iotf"]
    w = replace(base, name=f"tomo{n_angles}x{n}_iotf", batch=n_angles, ny=n, nx=n)
    ph = S.ellipsoid_phantom(S.rng_for(base.config, 900 + seed), size=n, n_ellipsoids=12,
                             axis_range=(60.0, 200.0), delta_range=(0.3 * delta_max, delta_max))
    angles = S.tomo_angles(n_angles)
    xd, yd = S.detector_grid(n, n, xp=torch)
    xd, yd = xd.to(device), yd.to(device)
    psi = torch.empty((n_angles, n, n), dtype=torch.complex64, device=device)
    for a in range(n_angles):
        re, im = S.ellipsoid_projection(ph, float(angles[a]), xd, yd, w.wavelength_m, w.pixel_m)
        psi[a] = torch.complex(re.float(), im.float())
    t = torch.from_numpy(S.diffuser(n, n, S.rng_for(base.config, 99)).astype(np.complex64)).to(device)
    with P.Plan(plan_desc(w, Setting("paper"))) as plan:
        f = plan.forward(psi, t)
        f0 = plan.forward(torch.zeros_like(psi), t)
    gen = torch.Generator(device=device).manual_seed(20146000 + seed)
    y = torch.poisson(torch.clamp(f, min=0) * photons, generator=gen) / photons
    rows = tuple(rows) if rows is not None else (n // 2 - n // 8, n // 2, n // 2 + n // 8)
    d, b = _rasterise(ph, rows, n, torch, device)
    return Series(w, angles, psi, t, y.float().contiguous(), d, b, rows, float(f0.mean()))


def plan_desc(w: S.Workload, s: Setting) -> P.PlanDesc:
    # every setting on the untuned column shapes: settings differ only in what they switch
    return P.PlanDesc(w.batch, w.ny, w.nx, w.pixel_m, w.wavelength_m, w.L1_m, w.L2_m, w.xcoh_m, w.ycoh_m,
                      s.gamma, s.alpha.real, s.alpha.imag, w.eta, s.flags | P.FLAG_NO_TUNE)


def run_setting(series: Series, s: Setting, iters: int):
    """Retrieve, reconstruct and score one setting; returns (scores, psi, vol)."""
    import torch
    w = series.w
    with P.Plan(plan_desc(w, s)) as plan:
        psi = torch.zeros_like(series.psi_true)
        plan.solve(series.y, series.t, psi, iters)
        f = plan.forward(psi, series.t)
    vol = P.pwf_fbp(psi, series.angles, w.wavelength_m, w.pixel_m)
    rows = list(series.rows)
    delta = vol[rows].imag.double()
    beta = vol[rows].real.double()
    n = w.nx
    c = torch.arange(n, dtype=torch.float64, device=psi.device) - n / 2 + 0.5
    disc = (c[None, :] ** 2 + c[:, None] ** 2) < (0.45 * n) ** 2
    inside = (series.delta_true > 0) & disc
    dt, bt = series.delta_true, series.beta_true
    scores = {
        "setting": s.name, "gamma": s.gamma, "alpha": [s.alpha.real, s.alpha.imag],
        "preconditioner": not (s.flags & P.FLAG_NO_PRECOND),
        "delta_rel_err": float(torch.sqrt(((delta - dt)[:, disc] ** 2).mean() / (dt[:, disc] ** 2).mean())),
        "beta_rel_err": float(torch.sqrt(((beta - bt)[:, disc] ** 2).mean() / (bt[:, disc] ** 2).mean())),
        "delta_ratio": float(delta[inside].mean() / dt[inside].mean()),
        "rmse_image_pct": float((series.y - f).abs().mean() / series.ref_mean * 100.0),
    }
    return scores, psi, vol


def run_ablation(series: Series, iters: int = 200, settings=SETTINGS):
    return [run_setting(series, s, iters)[0] for s in settings]


def summary_table(rows) -> str:
    head = f"{'setting':20s} {'delta err':>10s} {'beta err':>10s} {'delta ratio':>12s} {'RMSE img %':>11s}"
    lines = [head]
    for r in rows:
        lines.append(f"{r['setting']:20s} {r['delta_rel_err']:10.3f} {r['beta_rel_err']:10.3f} "
                     f"{r['delta_ratio']:12.3f} {r['rmse_image_pct']:11.3f}")
    return "\n".join(lines)


__all__ = ["Setting", "SETTINGS", "Series", "make_series", "run_setting", "run_ablation", "summary_table",
           "plan_desc"]
