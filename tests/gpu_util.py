"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

# Tolerances on the relative L2 error against the FP64 oracle: FP32 paths
# 1e-5, FP64 paths 1e-12.
TOL32 = 1e-5
TOL64 = 1e-12


def rel_l2(got, want) -> float:
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    den = np.linalg.norm(want.ravel())
    num = np.linalg.norm((got - want).ravel())
    return float(num / den) if den > 0 else float(num)


def rounded(x, dt):
    """The values the GPU sees, as FP64 arrays for the oracle."""
    return np.asarray(x, dtype=np.float32 if dt == torch.float32 else np.float64).astype(np.float64)


def dev(x, dt):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def tol(dt):
    return TOL32 if dt == torch.float32 else TOL64


def roundoff_spread(orc, m, g, r, v, s, n_it, n_cg, nu0, dt):
    """How far round-off alone moves the oracle's own reconstruction.

    The oracle is rerun with a dense copy of A (its entries from the oracle's
    pair term; A x then sums in another order) and with the data moved by one
    unit in the last place; for FP32 every operator application is further
    perturbed by relative noise of FP32 size (6e-8).  CG iterates on
    (A^T A + nu I) are not continuous at round-off level once the Krylov
    basis loses orthogonality, so this spread, not 1e-12, is the floor of any
    comparison of whole reconstructions at these settings."""
    ny, nx = g["ny"], g["nx"]
    n = nx * ny
    A = np.stack([orc.forward(m, g, r, v, np.eye(n)[k].reshape(ny, nx)).reshape(-1)
                  for k in range(n)], 1)
    rng = np.random.default_rng(99)
    eps = 6e-8 if dt == torch.float32 else 0.0

    def noisy(y):
        return y * (1.0 + eps * rng.standard_normal(y.shape)) if eps else y
    op = lambda x: noisy((A @ x.reshape(-1)).reshape(s.shape))  # noqa: E731
    opT = lambda y: noisy((A.T @ y.reshape(-1)).reshape(ny, nx))  # noqa: E731
    base = orc.pnp(op, opT, s, (ny, nx), n_it, n_cg, nu0)
    ulp = rng.choice([-1.0, 1.0], size=s.shape) * np.spacing(np.abs(s))
    pert = orc.pnp(op, opT, s + ulp, (ny, nx), n_it, n_cg, nu0)
    ref = orc.pnp(lambda x: orc.forward(m, g, r, v, x), lambda y: orc.adjoint(m, g, r, v, y), s,
                  (ny, nx), n_it, n_cg, nu0)
    return max(rel_l2(pert, base), rel_l2(base, ref))
