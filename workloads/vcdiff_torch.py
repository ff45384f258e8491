"""The variable-coefficient operator of ``stencils.make_vcdiff`` assembled with
torch operations, so that its stored values are a differentiable function of
the per-cell log-diffusivity theta (same pattern and value order as the numpy
assembly: per row the stored entries south, west, centre, east, north)."""
import numpy as np
import torch

from .stencils import make_vcdiff


def vcdiff_pattern(n: int):
    """(rowptr, col) of the n x n operator (int32 numpy arrays)."""
    A = make_vcdiff(n, np.zeros(n * n))
    return A.rowptr, A.col


def vcdiff_values(n: int, theta: torch.Tensor, conv=(10.0, 10.0)) -> torch.Tensor:
    """Stored values of A(theta) in CSR order (float64, differentiable in theta)."""
    h = 1.0 / (n + 1)
    k = torch.exp(theta.reshape(n, n))  # [iy, ix]
    kx = torch.cat([k[:, :1], 0.5 * (k[:, :-1] + k[:, 1:]), k[:, -1:]], dim=1)  # n x (n+1)
    ky = torch.cat([k[:1, :], 0.5 * (k[:-1, :] + k[1:, :]), k[-1:, :]], dim=0)  # (n+1) x n
    cx, cy = float(conv[0]), float(conv[1])
    west = -kx[:, :n] / h**2 - max(cx, 0.0) / h
    east = -kx[:, 1:] / h**2 + min(cx, 0.0) / h
    south = -ky[:n, :] / h**2 - max(cy, 0.0) / h
    north = -ky[1:, :] / h**2 + min(cy, 0.0) / h
    diag = (kx[:, :n] + kx[:, 1:] + ky[:n, :] + ky[1:, :]) / h**2 + (abs(cx) + abs(cy)) / h
    p = torch.arange(n * n, device=theta.device)
    ix, iy = p % n, p // n
    ok = torch.stack([iy > 0, ix > 0, torch.ones_like(ix, dtype=torch.bool), ix < n - 1, iy < n - 1], dim=1)
    vals = torch.stack([south.reshape(-1), west.reshape(-1), diag.reshape(-1), east.reshape(-1),
                        north.reshape(-1)], dim=1)
    return vals[ok]
