"""Invariants of an HT reduction evaluated on the GPU in genuine FP64.

Harness code (used by bench.py and the GPU tests), not part of the
reduction: it checks the structure and the two O(u) bounds the paper's
Sec. 4 and Appendix A fix,
  * H(i, j) == 0 for i > j+1 and T(i, j) == 0 for i > j (exact zeros),
  * ||Q^T Q - I||_F, ||Z^T Z - I||_F,
  * ||Q H Z^T - A||_F / ||A||_F and ||Q T Z^T - B||_F / ||B||_F,
either exactly (FP64 matrix products) or, for large n, as Frobenius-norm
estimates from Gaussian probe vectors (E ||M g||^2 = ||M||_F^2).
"""
from __future__ import annotations

import math

import torch

EPS64 = 2.0 ** -52


def structure_violations(H: torch.Tensor, T: torch.Tensor) -> tuple[int, int]:
    n = H.shape[0]
    r = torch.arange(n, device=H.device)
    below_h = r[:, None] > r[None, :] + 1
    below_t = r[:, None] > r[None, :]
    return int(torch.count_nonzero(H[below_h]).item()), int(torch.count_nonzero(T[below_t]).item())


@torch.no_grad()
def invariants(A0, B0, H, T, Q, Z, probes: int = 0, seed: int = 0) -> dict:
    """A0, B0: original inputs (B0 upper triangle used).  probes = 0: exact
    products; probes > 0: that many Gaussian probe vectors."""
    n = H.shape[0]
    B0u = torch.triu(B0)
    sh, st = structure_violations(H, T)
    na = torch.linalg.norm(A0).item()
    nbv = torch.linalg.norm(B0u).item()
    if probes <= 0:
        I = torch.eye(n, dtype=torch.float64, device=H.device)
        oq = torch.linalg.norm(Q.T @ Q - I).item()
        oz = torch.linalg.norm(Z.T @ Z - I).item()
        ra = torch.linalg.norm(Q @ H @ Z.T - A0).item() / max(na, 1e-300)
        rb = torch.linalg.norm(Q @ T @ Z.T - B0u).item() / max(nbv, 1e-300)
    else:
        g = torch.Generator(device=H.device).manual_seed(seed)
        G = torch.randn((n, probes), dtype=torch.float64, device=H.device, generator=g)
        scale = math.sqrt(probes)
        oq = torch.linalg.norm(Q.T @ (Q @ G) - G).item() / scale
        oz = torch.linalg.norm(Z.T @ (Z @ G) - G).item() / scale
        ra = torch.linalg.norm(Q @ (H @ (Z.T @ G)) - A0 @ G).item() / scale / max(na, 1e-300)
        rb = torch.linalg.norm(Q @ (T @ (Z.T @ G)) - B0u @ G).item() / scale / max(nbv, 1e-300)
    qe1 = torch.linalg.norm(Q[:, 0] - torch.eye(n, 1, dtype=torch.float64, device=H.device)[:, 0]).item()
    return {"n": n, "h_nonzeros_below_subdiag": sh, "t_nonzeros_below_diag": st, "orth_q": oq, "orth_z": oz,
            "bwd_a": ra, "bwd_b": rb, "q_e1": qe1, "tol": 20.0 * n * EPS64, "probes": probes}


def passes(rep: dict, bwd_tol: float | None = None, factor: float = 1.0) -> bool:
    tol = rep["tol"] if bwd_tol is None else bwd_tol
    return (rep["h_nonzeros_below_subdiag"] == 0 and rep["t_nonzeros_below_diag"] == 0
            and rep["orth_q"] <= factor * rep["tol"] and rep["orth_z"] <= factor * rep["tol"]
            and rep["bwd_a"] <= factor * tol and rep["bwd_b"] <= factor * tol and rep["q_e1"] == 0.0)
