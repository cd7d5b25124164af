"""Helpers of the GPU parity tests: run the CUDA path through the C ABI."""
import numpy as np
import pytest

from paper_1111_0716_gb300 import synth  # noqa: F401

FP32_TOL = 1e-5     # max|dV_x c| <= 1e-5 max|V_x c|, |dE_x| <= 1e-5 |E_x| (mixed precision)
FP64_TOL = 1e-11    # the all-FP64 path

# Achieved errors against the FP64 oracle (or a closed form), one entry per
# checked result: (workload, precision, quantity, error, tolerance).  The
# conftest prints them after the run, and writes them as JSON to the path in
# XX_PARITY_JSON when that is set.
PARITY = []


def record(workload, prec, quantity, err, tol):
    """Note an achieved error and return it (for the assertion that follows)."""
    name = {0: "fp32-mixed", 1: "fp64"}.get(prec, str(prec))
    PARITY.append((str(workload), name, str(quantity), float(err), float(tol)))
    return float(err)


def rel_err(x, ref):
    """|x - ref| / |ref| for scalars."""
    return abs(x - ref) / abs(ref)


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_0716_gb300 import xx
    xx.load()
    return torch, xx


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(wl, precision, shared=True, c_occ=None, w_occ=None, c_tgt=None, w_tgt=None, batch=None,
        mu=None):
    """(vx [nk][n_tgt][npw_max] numpy, E_x (re, im)) from the CUDA path."""
    import torch
    from paper_1111_0716_gb300 import xx
    plan = xx.Plan.from_workload(wl, precision=precision, mu=mu)
    if batch:
        plan.set_batch(*batch)
    ct = dev(wl.c_tgt if c_tgt is None else c_tgt)
    wt = dev(wl.w_tgt if w_tgt is None else w_tgt)
    if shared and c_occ is None:
        wo = dev(wl.w_occ if w_occ is None else w_occ)
        vx = torch.empty_like(ct)
        ex = torch.empty(2, dtype=torch.float64, device="cuda")
        xx.xx_energy(plan.handle, ct, ct.shape[1], wo, wo.shape[1], ct, wt, ct.shape[1], vx, ex)
    else:
        co = dev(wl.c_occ if c_occ is None else c_occ)
        wo = dev(wl.w_occ if w_occ is None else w_occ)
        ex, vx = plan.energy(co, wo, ct, wt)
    plan.sync(timeout_s=600.0)
    out = vx.cpu().numpy(), (float(ex[0].item()), float(ex[1].item()))
    info = plan.info()
    plan.close()
    return out[0], out[1], info


def rel_max(a, ref):
    return float(np.abs(a - ref).max() / np.abs(ref).max())


def hermitian_defect(c, vx):
    H = np.einsum("kag,kbg->kab", c.conj(), vx)
    return float(np.abs(H - np.conj(np.transpose(H, (0, 2, 1)))).max() / np.abs(H).max())
