"""Helpers shared by the GPU tests: parity metrics against the oracle."""
import numpy as np

EIG_RTOL = 1e-10      # |E_gpu - E_oracle| <= 1e-10 * max(1, |E_oracle|)
VEC_TOL = 1e-9        # || a/|a| - a_ora/|a_ora| ||_2 <= 1e-9 per column


def unit_cols(A):
    A = np.asarray(A)
    return A / np.linalg.norm(A, axis=0)


def eig_err(E, Eo):
    E, Eo = np.asarray(E), np.asarray(Eo)
    return float(np.max(np.abs(E - Eo) / np.maximum(1.0, np.abs(Eo))))


def vec_err(A, Ao):
    return float(np.max(np.linalg.norm(unit_cols(A) - unit_cols(Ao), axis=0)))


def to_np(x):
    try:
        import torch
        if isinstance(x, torch.Tensor):
            return x.detach().cpu().numpy()
    except ImportError:
        pass
    return np.asarray(x)
