"""Shared helpers of the GPU parity tests: parameter conversion between the
library binding and the oracle (two independent dataclasses), error metrics
and patch extraction for sampled full-size checks."""
from __future__ import annotations

import numpy as np

import oracle as O
import paper_2208_01525_gb300 as U


def to_oracle(p: U.Params) -> O.Params:
    return O.Params(p.nx, p.ny, p.nz, dx=p.dx, deta=p.deta, eta0=p.eta0, m=p.m, eta_ref=p.eta_ref,
                    beta=p.beta, alpha=p.alpha, lam=(p.lambda_p, p.lambda_q), e=(p.e_p, p.e_q),
                    sigma=(p.sigma_p, p.sigma_q), kappa=p.kappa, seed=p.seed)


def field_maxrel(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Per field array: max_x |a - b| / max_x |b| (b the reference)."""
    a = a.reshape(a.shape[0], -1).astype(np.float64)
    b = b.reshape(b.shape[0], -1).astype(np.float64)
    num = np.abs(a - b).max(axis=1)
    den = np.abs(b).max(axis=1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def host_state(lat: U.Lattice) -> np.ndarray:
    return lat.state().double().cpu().numpy()


def patches(fields, shape, sites, radius=2):
    """Gather (2r+1)^3 periodic patches of the 20 fields around each site
    (z, y, x); ``fields`` is the list of 20 flat device tensors of a lattice
    (no full-state copy is made).  Returns float64 numpy
    (nsites, 20, 2r+1, 2r+1, 2r+1)."""
    import torch
    nz, ny, nx = shape
    dev = fields[0].device
    off = torch.arange(-radius, radius + 1, device=dev)
    s = torch.as_tensor(sites, device=dev)
    z = (s[:, 0, None] + off[None, :]) % nz
    y = (s[:, 1, None] + off[None, :]) % ny
    x = (s[:, 2, None] + off[None, :]) % nx
    idx = (x[:, None, None, :] + nx * (y[:, None, :, None] + ny * z[:, :, None, None])).reshape(-1)
    out = torch.stack([f[idx] for f in fields]).reshape(len(fields), len(sites), 2 * radius + 1,
                                                      2 * radius + 1, 2 * radius + 1)
    return out.permute(1, 0, 2, 3, 4).double().cpu().numpy()


def gather_sites(fields, shape, sites):
    """Values of the 20 fields at the given sites: (nsites, 20) float64."""
    import torch
    nz, ny, nx = shape
    s = torch.as_tensor(sites, device=fields[0].device)
    idx = s[:, 2] + nx * (s[:, 1] + ny * s[:, 0])
    return torch.stack([f[idx] for f in fields]).T.double().cpu().numpy()
