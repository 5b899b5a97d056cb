"""Seeded synthetic inputs: coefficient fields and right-hand sides.

This module is the only code shared by the CUDA path's tests/bench and the
CPU oracle.  It draws random numbers and shapes them into coefficient fields
of the kinds the workloads use; it holds none of the solver's arithmetic (no
discretisation, no network, no iteration).  Importing it does not load the
CUDA library.

Grid convention: an n x n interior grid on the unit square with h = 1/(n+1);
nodal fields that include the Dirichlet boundary ring have shape
(n+2, n+2) and are indexed [j, i] with x = i*h, y = j*h.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "block_board_k",
    "gaussian_random_field",
    "lognormal_k",
    "random_blocks_k",
    "checkerboard_k",
    "channelised_k",
    "paper_white_noise_mu",
    "multilevel_noise",
    "paper_coefficient",
    "paper_mldata_mu",
    "paper_mldata_k",
    "normal_rhs",
    "unit_rhs",
]


def block_board_k(n: int, rng: np.random.Generator, nblocks: int = 8, cell: int = 4,
                  log10_lo: float = -1.0, log10_hi: float = 1.0) -> np.ndarray:
    """Piecewise-constant nodal k on an nblocks x nblocks board of cell x cell blocks.

    Draws nblocks^2 uniforms for log10 k (block-row major: block j then block i)
    and assigns node (j, i), 0 <= i, j <= n+1, to block
    (min(j // cell, nblocks-1), min(i // cell, nblocks-1)).
    """
    logk = rng.uniform(log10_lo, log10_hi, size=(nblocks, nblocks))
    idx = np.minimum(np.arange(n + 2) // cell, nblocks - 1)
    return 10.0 ** logk[idx[:, None], idx[None, :]]


def gaussian_random_field(m: int, corr_len: float, h: float, rng: np.random.Generator) -> np.ndarray:
    """Stationary Gaussian field on an m x m node lattice of spacing h.

    Covariance sigma^2 exp(-r^2 / (2 l^2)) with sigma = 1, made by filtering
    white noise with a Gaussian of standard deviation l/sqrt(2) (the
    self-convolution of that Gaussian has the target correlation), through an
    FFT on a grid padded by 4 l on each side so the periodic wrap does not
    correlate opposite edges, and normalised so the field has unit variance.
    """
    s = corr_len / np.sqrt(2.0)
    pad = int(np.ceil(4.0 * corr_len / h)) + 1
    M = m + 2 * pad
    noise = rng.standard_normal((M, M))
    d = np.minimum(np.arange(M), M - np.arange(M)) * h
    g1 = np.exp(-d * d / (2.0 * s * s))
    kern = g1[:, None] * g1[None, :]
    kern /= np.sqrt(np.sum(kern * kern))
    field = np.fft.irfft2(np.fft.rfft2(noise) * np.fft.rfft2(kern), s=(M, M))
    return np.ascontiguousarray(field[pad:pad + m, pad:pad + m])


def lognormal_k(n: int, corr_len: float, rng: np.random.Generator, sigma: float = 1.0) -> np.ndarray:
    """Nodal k = exp(sigma * g) on (n+2)^2 nodes, g a unit-variance GRF."""
    h = 1.0 / (n + 1)
    return np.exp(sigma * gaussian_random_field(n + 2, corr_len, h, rng))


def random_blocks_k(n: int, rng: np.random.Generator, board: int = 16,
                    log10_lo: float = -2.0, log10_hi: float = 2.0) -> np.ndarray:
    """Piecewise-constant nodal k on a board x board partition of the unit square,
    log10 k ~ U(log10_lo, log10_hi) per block (contrast up to 1e4)."""
    logk = rng.uniform(log10_lo, log10_hi, size=(board, board))
    idx = np.minimum((np.arange(n + 2) * board) // (n + 2), board - 1)
    return 10.0 ** logk[idx[:, None], idx[None, :]]


def checkerboard_k(n: int, board: int = 16, k_lo: float = 1.0, k_hi: float = 100.0) -> np.ndarray:
    """Nodal k on a board x board checkerboard with values {k_lo, k_hi}."""
    idx = np.minimum((np.arange(n + 2) * board) // (n + 2), board - 1)
    par = (idx[:, None] + idx[None, :]) % 2
    return np.where(par == 0, k_lo, k_hi).astype(np.float64)


def channelised_k(n: int, rng: np.random.Generator, corr_len: float = 0.02,
                  quantile: float = 0.70, k_lo: float = 1.0, k_hi: float = 1e3) -> np.ndarray:
    """Binary channelised nodal k: k_hi where a GRF exceeds its `quantile`, else k_lo."""
    h = 1.0 / (n + 1)
    g = gaussian_random_field(n + 2, corr_len, h, rng)
    thr = np.quantile(g, quantile)
    return np.where(g > thr, k_hi, k_lo).astype(np.float64)


def paper_white_noise_mu(n: int, rng: np.random.Generator, Re: float = 1000.0) -> np.ndarray:
    """The paper's white-noise coefficient (Sec. 4.1) as the diffusion mu of the
    non-divergence operator on the n x n interior nodes.  The paper draws
    coef = 1/Re in [1/Re, 1] (white noise mapped linearly to a power in
    [0, log10 Re], then 10^(-power)) and its stencil is
    (1/h){coef [0 -1 0; -1 4 -1; 0 -1 0] + v . K_upwind} (Sec. 2.5), i.e.
    coef = mu / h: so mu = coef h, and Re is the mesh Reynolds number."""
    w = rng.uniform(0.0, 1.0, size=(n, n))
    power = w * np.log10(Re)
    return 10.0 ** (-power) / (n + 1)


def _resize_linear(a: np.ndarray, size: int) -> np.ndarray:
    """Separable linear interpolation of a square array to size x size, corner
    samples kept (sample positions spread evenly from the first to the last)."""
    m = a.shape[0]
    src = np.arange(m, dtype=np.float64)
    dst = np.linspace(0.0, m - 1.0, size)
    rows = np.stack([np.interp(dst, src, a[j]) for j in range(m)])        # m x size
    return np.stack([np.interp(dst, src, rows[:, i]) for i in range(size)], axis=1)


def multilevel_noise(size: int, levels: int, rng: np.random.Generator, init_size: int = 5) -> np.ndarray:
    """The paper's multi-level data (Appendix, Algorithm "Generate Multi-Level
    Data"): white noise on init_size^2, then `levels` times doubled in size by
    interpolation with white noise of weight 2^-i added, finally interpolated to
    size^2.  White noise is uniform on [0, 1) and interpolation is linear (the
    paper names neither)."""
    data = rng.uniform(0.0, 1.0, size=(init_size, init_size))
    for i in range(1, levels + 1):
        data = _resize_linear(data, 2 * data.shape[0])
        data = data + 2.0 ** (-i) * rng.uniform(0.0, 1.0, size=data.shape)
    return _resize_linear(data, size)


def paper_coefficient(x: np.ndarray, Re: float = 1000.0) -> np.ndarray:
    """The paper's map of a random tensor to a coefficient (Sec. 4.1): linearly to a
    power in [0, log10 Re] (the tensor's minimum to 0, its maximum to log10 Re),
    then coef = 10^(-power) in [1/Re, 1]."""
    lo, hi = float(x.min()), float(x.max())
    power = (x - lo) / (hi - lo) * np.log10(Re)
    return 10.0 ** (-power)


def _mldata_levels(size: int, init_size: int) -> int:
    """Doublings of init_size that stay within the goal size (the paper does not say)."""
    levels = 0
    while init_size * 2 ** (levels + 1) <= size:
        levels += 1
    return levels


def paper_mldata_mu(n: int, rng: np.random.Generator, Re: float = 1000.0, init_size: int = 5) -> np.ndarray:
    """Non-divergence mu on the n x n interior nodes from multi-level data: the
    paper's coef in [1/Re, 1] times h (coef = mu / h, as for the white noise)."""
    return paper_coefficient(multilevel_noise(n, _mldata_levels(n, init_size), rng, init_size), Re) / (n + 1)


def paper_mldata_k(n: int, rng: np.random.Generator, Re: float = 1000.0, init_size: int = 5) -> np.ndarray:
    """Divergence-form nodal k on the (n+2)^2 nodes (boundary ring included) from
    multi-level data, mapped to [1/Re, 1] as the paper maps its coefficient."""
    m = n + 2
    return paper_coefficient(multilevel_noise(m, _mldata_levels(m, init_size), rng, init_size), Re)


def normal_rhs(n: int, rng: np.random.Generator) -> np.ndarray:
    """f iid N(0, 1) on the n x n interior nodes."""
    return rng.standard_normal((n, n))


def unit_rhs(n: int) -> np.ndarray:
    """The paper's test right-hand side, constant 1 (Sec. 4.1)."""
    return np.ones((n, n))
