"""The no-allocation E_x reduction (xx_energy_from_vx_noalloc).

It serves callers that cannot allocate device memory (their memory manager
already owns it, or they must avoid cudaFree's device-wide synchronisation).
Its result must match the plan-based xx_energy_from_vx and the FP64 oracle's
reduction on the same inputs, on two calls in a row (the shared fixed scratch
keeps the previous call's contents: the smaller workload runs first, so stale
rows of the first call would be left in the scratch the second call reads),
it must clamp a basis size past npw_max, and it must reject sizes beyond its
fixed scratch.  This file is
collected last so that a run stopping at its first failure has already run
every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1111_0716_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-13         # same FP64 fixed-order reduction on both sides
ORACLE_TOL = 1e-12  # FP64 on both sides, different summation order


def _inputs(torch, wl):
    rng = np.random.default_rng(7)
    vx = rng.standard_normal(wl.c_tgt.shape) + 1j * rng.standard_normal(wl.c_tgt.shape)
    for k in range(wl.nk):
        vx[k, :, wl.npw[k]:] = 0
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    return dev(wl.c_tgt), dev(wl.w_tgt), dev(vx), dev(wl.npw.astype(np.int32))


def test_noalloc_matches_plan_reduction_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_0716_gb300 import xx

    from oracle import oracle

    results = []
    # the tiny cell (8 rows) first, the 8 k-point cell (48 rows) second
    for wl in (synth.tiny_cubic(),
               synth.make_workload("noalloc-a", synth.rhombohedral_lattice(7.5, 65.0), (24,) * 3,
                                   synth.monkhorst_pack(2), 2.4, 4, 6, [1.0, 1.0, 0.75, 0.3], 21)):
        c, w, vx, npw = _inputs(torch, wl)
        plan = xx.Plan.from_workload(wl, precision=xx.XX_FP64)
        ref = torch.empty(2, dtype=torch.float64, device="cuda")
        xx.xx_energy_from_vx(plan.handle, c, w, wl.n_tgt, vx, ref)
        got = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        xx.xx_energy_from_vx_noalloc(wl.nk, wl.n_tgt, wl.npw_max, npw, c, w, vx, got)
        torch.cuda.synchronize()
        plan.close()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert abs(g[0] - r[0]) <= TOL * abs(r[0])
        assert abs(g[1] - r[1]) <= TOL * max(abs(r[0]), 1e-300)
        o_re, o_im = oracle.energy_from_vx(wl, vx.cpu().numpy())
        assert abs(g[0] - o_re) <= ORACLE_TOL * abs(o_re)
        assert abs(g[1] - o_im) <= ORACLE_TOL * abs(o_re)
        results.append(g[0])
    # the two workloads give different energies: the second call did not reuse the first's sums
    assert results[0] != results[1]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_0716_gb300 import xx
    L = xx.load()
    nk = 2
    n_tgt = xx.XX_NOALLOC_MAX_ROWS // nk + 1
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    st = L.xx_energy_from_vx_noalloc(nk, n_tgt, 1, p, p, p, p, p, None)
    assert st == -9
    assert "XX_NOALLOC_MAX_ROWS" in xx.xx_status_string(st)


def test_noalloc_clamps_a_basis_size_past_npw_max():
    """npw lives on the device, so the kernel clamps it: npw[k] = npw_max + 5 gives
    the sum over the whole padded row (padding filled with nonzero values here, so
    the clamp is visible), and never a read past the last row."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from oracle import oracle
    from paper_1111_0716_gb300 import xx

    wl = synth.make_workload("noalloc-a", synth.rhombohedral_lattice(7.5, 65.0), (24,) * 3,
                             synth.monkhorst_pack(2), 2.4, 4, 6, [1.0, 1.0, 0.75, 0.3], 21)
    assert int(wl.npw.min()) < wl.npw_max
    rng = np.random.default_rng(11)
    shape = wl.c_tgt.shape
    c_pad = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    vx = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    npw_bad = torch.full((wl.nk,), wl.npw_max + 5, dtype=torch.int32, device="cuda")
    got = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    xx.xx_energy_from_vx_noalloc(wl.nk, wl.n_tgt, wl.npw_max, npw_bad, dev(c_pad), dev(wl.w_tgt),
                                 dev(vx), got)
    torch.cuda.synchronize()
    g = got.cpu().numpy()
    # the oracle with every basis size set to npw_max sums the same whole rows
    full = wl.replace(npw=np.full(wl.nk, wl.npw_max, dtype=wl.npw.dtype))
    o_re, o_im = oracle.energy_from_vx(full, vx, c_tgt=c_pad)
    assert abs(g[0] - o_re) <= ORACLE_TOL * abs(o_re)
    assert abs(g[1] - o_im) <= ORACLE_TOL * abs(o_re)
