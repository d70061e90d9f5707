"""Synthetic MLMC workloads (plain parameter dictionaries).

Keys:
  dim        2 or 3
  n0         cells per side of mesh 0; mesh l has n0 * 2^l cells per side
  levels     number of levels L + 1
  sigma2     variance of the Gaussian log-field
  corr_len   correlation length of the separable exponential covariance
  m          KLE modes per axis (M = m^dim tensor modes)
  qoi        'domain' (mean of u over the domain) or 'box' (mean over box^dim)
  box        (lo, hi) of the QoI box
  solver     'jacobi' or 'gmg' preconditioned CG
  rtol       ||r||_2 <= rtol ||b||_2 stopping rule
  seed, stream_id   Philox key and request id
  eps        target RMSE for the adaptive run
  pilot      pilot samples per level
  N          fixed sample counts (None -> adaptive)
"""
import copy
import math

import numpy as np

WORKLOADS = {
    # 2D plain FP64, 16^2..64^2, Jacobi-PCG, fixed N = (200, 50, 20).
    "2d-small": dict(dim=2, n0=16, levels=3, sigma2=1.0, corr_len=0.3, m=4,
                     qoi='domain', box=(0.25, 0.75), solver='jacobi', rtol=1e-11,
                     seed=0, stream_id=0, eps=None, pilot=0, N=(200, 50, 20)),
    # 2D plain FP64 at scale: 6 levels 32^2..1024^2, corr 0.1, M = 64,
    # GMG-PCG rtol 1e-10, adaptive to RMSE 1e-3 after 100 pilot samples.
    "2d-scale": dict(dim=2, n0=32, levels=6, sigma2=1.0, corr_len=0.1, m=8,
                     qoi='domain', box=(0.25, 0.75), solver='gmg', rtol=1e-10,
                     seed=0, stream_id=0, eps=1e-3, pilot=100, N=None),
    # 3D, 5 levels 8^3..128^3, corr 0.2, M = 125, box QoI, FP64, eps 5e-4.
    "3d-batched": dict(dim=3, n0=8, levels=5, sigma2=1.0, corr_len=0.2, m=5,
                       qoi='box', box=(0.25, 0.75), solver='gmg', rtol=1e-10,
                       seed=0, stream_id=0, eps=5e-4, pilot=100, N=None),
    # 3D mixed precision: 5 levels 16^3..256^3, corr 0.1, M = 343.
    # No target RMSE or sample counts are given for it: a fixed-N run with
    # N_l halving per level (64 .. 4) is used.
    "3d-mixed": dict(dim=3, n0=16, levels=5, sigma2=1.0, corr_len=0.1, m=7,
                     qoi='box', box=(0.25, 0.75), solver='gmg', rtol=1e-10,
                     seed=0, stream_id=0, eps=None, pilot=0, N=(64, 32, 16, 8, 4),
                     precision='mixed'),
    # The paper-shaped sample mix: 3 levels 16^3..64^3 (the grids of the
    # paper's 3D Poisson example), N = C (1024, 64, 4) with C = 1 (Table 1),
    # the example's field (correlation length 0.25, standard deviation 0.25,
    # 16 eigenfunctions per axis under a total-order truncation: 680 modes
    # with 0-based orders summing to at most 14), box-mean QoI, mixed form.
    "3d-paper-mix": dict(dim=3, n0=16, levels=3, sigma2=0.0625, corr_len=0.25, m=16,
                         total_order=14, qoi='box', box=(0.25, 0.75), solver='gmg',
                         rtol=1e-10, seed=0, stream_id=0, eps=None, pilot=0,
                         N=(1024, 64, 4), precision='mixed'),
}


def workload(name, **overrides):
    """A copy of a named workload with optional overrides."""
    cfg = copy.deepcopy(WORKLOADS[name])
    cfg.update(overrides)
    return cfg


def small_case(dim=2, **overrides):
    """A tiny workload for oracle-speed tests (spans several tiles + a ragged tail)."""
    base = dict(dim=dim, n0=4 if dim == 2 else 2, levels=3, sigma2=1.0,
                corr_len=0.3, m=4 if dim == 2 else 3, qoi='domain',
                box=(0.25, 0.75), solver='jacobi', rtol=1e-11, seed=0,
                stream_id=0, eps=None, pilot=0, N=(8, 4, 2))
    base.update(overrides)
    return base


def serving_request(dim, sigma2, corr_len, stream_id):
    """One request of the serving stream: 32^2..1024^2 (2D, domain-mean QoI)
    or 8^3..128^3 (3D, box QoI) elements, GMG-PCG rtol 1e-10, mixed form,
    m = ceil(1.5 / corr_len) modes per axis capped at 8 (2D) or 7 (3D); the
    request index is the Philox stream word."""
    m = min(int(math.ceil(1.5 / corr_len)), 8 if dim == 2 else 7)
    if dim == 2:
        return dict(dim=2, n0=32, levels=6, sigma2=sigma2, corr_len=corr_len, m=m,
                    qoi='domain', box=(0.25, 0.75), solver='gmg', rtol=1e-10, seed=0,
                    stream_id=stream_id, eps=None, pilot=0, N=None, precision='mixed')
    return dict(dim=3, n0=8, levels=5, sigma2=sigma2, corr_len=corr_len, m=m,
                qoi='box', box=(0.25, 0.75), solver='gmg', rtol=1e-10, seed=0,
                stream_id=stream_id, eps=None, pilot=0, N=None, precision='mixed')


def serving_stream(n_requests, rate=20.0, seed=1):
    """Poisson arrivals at `rate` per second: a list of (arrival time in s,
    workload, eps) with eps ~ U[5e-4, 5e-3], dim 2 or 3 with probability 1/2,
    sigma2 ~ U[0.5, 2], corr_len ~ U[0.05, 0.3]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += rng.exponential(1.0 / rate)
        eps = rng.uniform(5e-4, 5e-3)
        dim = 2 if rng.random() < 0.5 else 3
        sigma2 = rng.uniform(0.5, 2.0)
        corr = rng.uniform(0.05, 0.3)
        out.append((t, serving_request(dim, sigma2, corr, k), eps))
    return out
