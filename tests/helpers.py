"""Test helpers: run the CUDA path (through the C ABI binding) and the CPU
oracle on the same seeded inputs."""
import numpy as np


def gpu_solver(prob_or_st, **params):
    import torch
    import paper_2006_16465_gb300 as hj
    st = getattr(prob_or_st, "st", prob_or_st)
    sig = None
    if st.sigma is not None:
        sig = hj.grid_from(st.sigma, st.dim, torch.float64)
    coef = None
    if getattr(st, "coef", None) is not None and "coef" not in params:
        # per-point neighbour coefficients, padded to the solver's ld
        dtype = torch.float32 if params.get("precision") == "f32" else torch.float64
        ld = hj.padded_ld(st.nx, dtype)
        c = np.asarray(st.coef)
        coef = torch.zeros((c.shape[0], c.shape[1], ld), dtype=torch.float64, device="cuda")
        coef[:, :, :st.nx + 2] = torch.as_tensor(c)
    if coef is not None:
        params["coef"] = coef
    return hj.Solver(st, sigma=sig, **params)


def to_dev(a, dim, dtype):
    import paper_2006_16465_gb300 as hj
    return hj.grid_from(a, dim, dtype)


def to_host(t, nx):
    return t[..., :nx + 2].double().cpu().numpy()


def rel_max(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
