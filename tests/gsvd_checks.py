"""Invariant checks shared by the oracle pins and the GPU parity tests (test-side only)."""
import numpy as np


def rel_sigma_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / np.abs(b))) if a.size else 0.0


def invariants(F, G, U, V, Z, sf, sg, sigma):
    """Return the residuals the paper and the mathematics fix for a GSVD."""
    n = F.shape[1]
    In = np.eye(n)
    res = {}
    res["FZ"] = np.linalg.norm(F @ Z - U * sf[None, :]) / np.linalg.norm(F)
    res["GZ"] = np.linalg.norm(G @ Z - V * sg[None, :]) / np.linalg.norm(G)
    res["UU"] = np.linalg.norm(U.conj().T @ U - In)
    res["VV"] = np.linalg.norm(V.conj().T @ V - In)
    res["scale"] = float(np.max(np.abs(sf * sf + sg * sg - 1.0))) if n else 0.0
    res["ratio"] = rel_sigma_err(sf / sg, sigma) if n else 0.0
    res["sorted"] = bool(np.all(np.diff(sigma) <= 0))
    # the paper's normwise errors (Sec. 5) with X = Z^{-1}
    X = np.linalg.solve(Z, In)
    res["F_USX"] = np.linalg.norm(F - (U * sf[None, :]) @ X) / np.linalg.norm(F)
    res["G_VSX"] = np.linalg.norm(G - (V * sg[None, :]) @ X) / np.linalg.norm(G)
    return res
