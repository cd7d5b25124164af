"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances: mixed precision max|dV_x c| <= 1e-5 max|V_x c| and |dE_x| <= 1e-5
|E_x| (the two precision settings of the method agree to 1e-3 %); all-FP64
path 1e-11.
"""
import math

import numpy as np
import pytest

from paper_1111_0716_gb300 import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def rhombo24(kernel=synth.KERNEL_HSE, seed=21):
    """Rhombohedral cell with a 2x2x2 MP mesh, targets beyond the occupied set."""
    wl = synth.make_workload("rhombo24", synth.rhombohedral_lattice(7.5, 65.0), (24,) * 3,
                             synth.monkhorst_pack(2), 2.4, 4, 6, [1.0, 1.0, 0.75, 0.3], seed,
                             kernel=kernel)
    assert np.all(4 * wl.n_max() + 1 <= 24)
    return wl


@pytest.fixture(scope="module")
def gpu():
    return gu.need_gpu()


@pytest.fixture(scope="module")
def oracle_cache(oracle_mod):
    cache = {}

    def get(key, fn):
        if key not in cache:
            cache[key] = fn()
        return cache[key]
    return get


@pytest.mark.parametrize("prec,tol", [(0, gu.FP32_TOL), (1, gu.FP64_TOL)])
def test_tiny_cubic(gpu, oracle_mod, oracle_cache, prec, tol):
    wl = synth.tiny_cubic()
    ref = oracle_cache("tiny", lambda: oracle_mod.apply(wl))
    e_ref, _ = oracle_mod.energy_from_vx(wl, ref)
    vx, (e, e_im), _ = gu.run(wl, prec)
    w = "tiny cubic 24^3 (8/8, Gamma)"
    assert gu.record(w, prec, "max|dVx|/max|Vx|", gu.rel_max(vx, ref), tol) <= tol
    assert gu.record(w, prec, "|dE_x|/|E_x|", gu.rel_err(e, e_ref), tol) <= tol
    assert abs(e_im) <= tol * abs(e_ref)


@pytest.mark.parametrize("kernel", [synth.KERNEL_HSE, synth.KERNEL_COULOMB])
@pytest.mark.parametrize("prec,tol", [(0, gu.FP32_TOL), (1, gu.FP64_TOL)])
def test_k_mesh_targets_beyond_occupied(gpu, oracle_mod, oracle_cache, kernel, prec, tol):
    wl = rhombo24(kernel)
    ref = oracle_cache(("rh", kernel), lambda: oracle_mod.apply(wl))
    e_ref, _ = oracle_mod.energy_from_vx(wl, ref)
    # separate occupied array (no grid sharing)
    vx, (e, _), _ = gu.run(wl, prec, shared=False)
    w = "rhombo 24^3 MP2x2x2 " + ("screened" if kernel == synth.KERNEL_HSE else "Coulomb")
    assert gu.record(w, prec, "max|dVx|/max|Vx|", gu.rel_max(vx, ref), tol) <= tol
    assert gu.record(w, prec, "|dE_x|/|E_x|", gu.rel_err(e, e_ref), tol) <= tol
    # shared grids: occupied = leading bands of the target array
    vx2, (e2, _), _ = gu.run(wl, prec, shared=True)
    assert gu.record(w + " shared", prec, "max|dVx|/max|Vx|", gu.rel_max(vx2, ref), tol) <= tol
    assert gu.record(w + " shared", prec, "|dE_x|/|E_x|", gu.rel_err(e2, e_ref), tol) <= tol


def test_ragged_batches_match(gpu, oracle_mod, oracle_cache):
    wl = rhombo24()
    base, (e0, _), _ = gu.run(wl, 1)
    for batch in [(1, 1), (5, 3), (4, 4), (6, 4)]:
        vx, (e, _), info = gu.run(wl, 1, batch=batch)
        assert info["targets_per_batch"] == batch[0] and info["occupied_per_batch"] == batch[1]
        assert gu.rel_max(vx, base) <= 1e-13
        assert abs(e - e0) <= 1e-13 * abs(e0)


def test_deterministic(gpu):
    wl = rhombo24()
    a, ea, _ = gu.run(wl, 0)
    b, eb, _ = gu.run(wl, 0)
    assert np.array_equal(a, b) and ea == eb


def test_edge_cases(gpu, oracle_mod):
    torch, xx = gpu
    wl = rhombo24()
    plan = xx.Plan.from_workload(wl, precision=1)
    ct = gu.dev(wl.c_tgt)
    # no occupied bands: V_x c = 0
    vx = torch.full_like(ct, 7.0)
    xx.xx_apply(plan.handle, ct, 0, gu.dev(wl.w_occ), 0, ct, ct.shape[1], vx)
    assert float(vx.abs().max()) == 0.0
    # no targets: nothing to do
    xx.xx_apply(plan.handle, ct, 0, gu.dev(wl.w_occ), 4, ct, 0, vx)
    # zero-weight occupied bands contribute nothing
    w0 = wl.w_occ.copy()
    w0[:, 2:] = 0.0
    ref = oracle_mod.apply(wl, c_occ=wl.c_occ[:, :2], w_occ=w0[:, :2])
    vx1, _, _ = gu.run(wl, 1, shared=False, w_occ=w0)
    assert gu.rel_max(vx1, ref) <= gu.FP64_TOL
    # a single target band and a single occupied band
    ref1 = oracle_mod.apply(wl, c_occ=wl.c_occ[:, :1], w_occ=wl.w_occ[:, :1], c_tgt=wl.c_tgt[:, :1])
    vx2, _, _ = gu.run(wl, 1, shared=False, c_occ=wl.c_occ[:, :1], w_occ=wl.w_occ[:, :1],
                       c_tgt=wl.c_tgt[:, :1], w_tgt=wl.w_tgt[:, :1])
    assert gu.rel_max(vx2, ref1) <= gu.FP64_TOL
    plan.close()


def test_k_range_shards_sum_to_full(gpu, oracle_mod):
    """Disjoint target k-ranges (the multi-GPU decomposition) reproduce the full result."""
    torch, xx = gpu
    wl = rhombo24()
    full, (e_full, _), _ = gu.run(wl, 1, shared=False)
    plan = xx.Plan.from_workload(wl, precision=1)
    co, wo = gu.dev(wl.c_occ), gu.dev(wl.w_occ)
    parts, e_sum = [], 0.0
    for k0, kn in [(0, 3), (3, 1), (4, 4)]:
        ct = gu.dev(wl.c_tgt[k0:k0 + kn])
        wt = gu.dev(wl.w_tgt[k0:k0 + kn])
        ex, vx = plan.energy_range(k0, kn, co, wo, ct, wt)
        parts.append(vx.cpu().numpy())
        e_sum += float(ex[0].item())
    plan.close()
    assert gu.rel_max(np.concatenate(parts), full) <= 1e-13
    assert abs(e_sum - e_full) <= 1e-13 * abs(e_full)


@pytest.mark.parametrize("prec,tol", [(0, gu.FP32_TOL), (1, gu.FP64_TOL)])
def test_differentiation_cell_48(gpu, oracle_mod, oracle_cache, prec, tol):
    wl = synth.differentiation_cell()
    ref = oracle_cache("cfg4", lambda: oracle_mod.apply(wl))
    e_ref, _ = oracle_mod.energy_from_vx(wl, ref)
    vx, (e, _), _ = gu.run(wl, prec)
    w = "differentiation cell 48^3 (32/32)"
    assert gu.record(w, prec, "max|dVx|/max|Vx|", gu.rel_max(vx, ref), tol) <= tol
    assert gu.record(w, prec, "|dE_x|/|E_x|", gu.rel_err(e, e_ref), tol) <= tol


@pytest.mark.parametrize("shell", synth.PW_SHELLS)
def test_plane_wave_cells_exact_lattice_sum(gpu, shell):
    """Single-plane-wave orbitals: V_x c_a = lam_a c_a with the exact lattice sum."""
    from tests.test_oracle_pins import pw_closed_form
    wl = synth.plane_wave_cell(shell)
    lam, ex = pw_closed_form(wl)
    ref = lam[:, None] * wl.c_tgt[0]
    vx, (e, _), _ = gu.run(wl, 0)
    w = "plane-wave 32^3 |m|^2<=%d (%d orb)" % (shell, wl.npw[0])
    q = "(closed-form lattice sum)"
    assert gu.record(w, 0, "max|dVx|/max|Vx| " + q, gu.rel_max(vx[0], ref), gu.FP32_TOL) <= gu.FP32_TOL
    assert gu.record(w, 0, "|dE_x|/|E_x| " + q, gu.rel_err(e, ex), gu.FP32_TOL) <= gu.FP32_TOL
    # Dirac exchange of the homogeneous gas after the q -> 0 correction
    omega = abs(np.linalg.det(wl.lattice))
    n_e = 2 * wl.npw[0]
    kf = (3 * math.pi ** 2 * n_e / omega) ** (1 / 3)
    qc = (6 * math.pi ** 2 / omega) ** (1 / 3)
    corr = -wl.npw[0] * 16 * math.pi ** 2 * qc / (2 * math.pi) ** 3
    dirac = abs((e + corr) / n_e / (-3 * kf / (4 * math.pi)) - 1)
    assert gu.record(w, 0, "|E_x/N_e / Dirac - 1| (q->0 corr.)", dirac, 0.03) <= 0.03
    if shell <= 5:
        vx64, (e64, _), _ = gu.run(wl, 1)
        assert gu.record(w, 1, "max|dVx|/max|Vx| " + q, gu.rel_max(vx64[0], ref),
                         gu.FP64_TOL) <= gu.FP64_TOL
        assert gu.record(w, 1, "|dE_x|/|E_x| " + q, gu.rel_err(e64, ex), gu.FP64_TOL) <= gu.FP64_TOL


@pytest.mark.parametrize("i", range(len(synth.SWEEP_GRIDS)))
@pytest.mark.parametrize("kernel", [synth.KERNEL_HSE, synth.KERNEL_COULOMB])
def test_precision_sweep_cells(gpu, oracle_mod, i, kernel):
    """Uneven sweep: each cell in mixed precision, sampled targets vs the oracle,
    Hermiticity on every target, and an FP64 slice."""
    wl = synth.sweep_cell(i, kernel)
    vx, (e, e_im), _ = gu.run(wl, 0)
    sel = [(0, 0), (0, wl.n_tgt - 1)]
    ref = oracle_mod.apply(wl, sel=sel)
    got = np.stack([vx[k, a] for k, a in sel])
    w = "sweep %d^3 (%d bands) %s" % (wl.grid[0], wl.n_occ,
                                     "screened" if kernel == synth.KERNEL_HSE else "Coulomb")
    t32 = gu.FP32_TOL
    assert gu.record(w, 0, "max|dVx|/max|Vx| (2 targets)", gu.rel_max(got, ref), t32) <= t32
    assert gu.record(w, 0, "Hermiticity defect", gu.hermitian_defect(wl.c_tgt, vx), t32) <= t32
    # per-target energy contributions of the sampled targets
    for (k, a), r in zip(sel, ref):
        d_gpu = np.vdot(wl.c_tgt[k, a], vx[k, a]).real
        d_ref = np.vdot(wl.c_tgt[k, a], r).real
        assert gu.record(w, 0, "<c|Vx c> rel, target %d" % a, gu.rel_err(d_gpu, d_ref), t32) <= t32
    # FP64 on two target bands, all occupied bands
    vx64, _, _ = gu.run(wl, 1, shared=False, c_tgt=wl.c_tgt[:, [0, wl.n_tgt - 1]],
                        w_tgt=wl.w_tgt[:, [0, wl.n_tgt - 1]])
    assert gu.record(w, 1, "max|dVx|/max|Vx| (2 targets)", gu.rel_max(vx64[0], ref),
                     gu.FP64_TOL) <= gu.FP64_TOL


def test_run_many_sweep_cells_match_single_runs(gpu):
    """The six sweep cells as one xx_run_many call (concurrent streams) equal separate runs."""
    torch, xx = gpu
    cells = [synth.sweep_cell(i) for i in range(len(synth.SWEEP_GRIDS))]
    plans, jobs = [], []
    for wl in cells:
        plan = xx.Plan.from_workload(wl, precision=0)
        c = gu.dev(wl.c_tgt)
        jobs.append({"plan": plan, "c_occ": c, "ld_occ": c.shape[1], "w_occ": gu.dev(wl.w_occ),
                     "c_tgt": c, "w_tgt": gu.dev(wl.w_tgt), "vx_out": torch.empty_like(c),
                     "ex_out": torch.empty(2, dtype=torch.float64, device="cuda")})
        plans.append(plan)
    xx.xx_run_many(jobs)
    torch.cuda.synchronize()
    for wl, job, plan in zip(cells, jobs, plans):
        vx, (e, _), _ = gu.run(wl, 0)
        assert np.array_equal(job["vx_out"].cpu().numpy(), vx)
        assert float(job["ex_out"][0].item()) == e
        plan.close()
    with pytest.raises(xx.XXError):
        xx.xx_run_many([jobs[0], dict(jobs[0])])


@pytest.mark.parametrize("make,prec,tol", [(synth.tiny_cubic, 1, 1e-12),
                                           (synth.differentiation_cell, 0, gu.FP32_TOL),
                                           (lambda: synth.sweep_cell(1), 1, 1e-12),
                                           (lambda: rhombo24(), 1, 1e-12)])
def test_pair_symmetry_matches_direct_pairs(gpu, make, prec, tol):
    """Pair symmetry (default; k = q tiles and, on k-meshes, blocks q > k) against
    transforming every pair (option off)."""
    torch, xx = gpu
    wl = make()
    out = []
    for on in (True, False):
        plan = xx.Plan.from_workload(wl, precision=prec)
        plan.set_batch(3, 3)                     # several tiles, ragged edges
        plan.set_pair_symmetry(on)
        c = gu.dev(wl.c_tgt)
        ex, vx = plan.energy(c, gu.dev(wl.w_occ), c, gu.dev(wl.w_tgt), shared=True)
        plan.sync(timeout_s=600.0)
        out.append((vx.cpu().numpy(), float(ex[0].item())))
        plan.close()
    assert gu.rel_max(out[0][0], out[1][0]) <= tol
    assert abs(out[0][1] - out[1][1]) <= tol * abs(out[1][1])


def expected_transforms(nk, n_occ, n_tgt, TA, TJ, sym):
    """Band pairs the host loop sends through the codensity transform."""
    if not sym:
        return nk * nk * n_tgt * n_occ
    T = min(TA, TJ)
    tiles = [min(T, n_occ - i) for i in range(0, n_occ, T)]
    diag = sum(tiles[i] * tiles[j] for i in range(len(tiles)) for j in range(i, len(tiles)))
    rest = (n_tgt - n_occ) * n_occ            # targets past the occupied set meet every j
    upper = nk * (nk - 1) // 2                # blocks q > k: the whole occupied square
    return nk * (diag + rest) + upper * (n_occ * n_occ + rest) + (nk * nk - nk - upper) * rest


def test_pair_symmetry_transform_count(gpu):
    """The k != q symmetry transforms each occupied pair of blocks (k, q), (q, k) once."""
    torch, xx = gpu
    wl = rhombo24()
    logical = wl.nk * wl.n_tgt * wl.nk * wl.n_occ
    for on in (True, False):
        plan = xx.Plan.from_workload(wl, precision=0)
        plan.set_batch(3, 3)
        plan.set_pair_symmetry(on)
        c = gu.dev(wl.c_tgt)
        plan.energy(c, gu.dev(wl.w_occ), c, gu.dev(wl.w_tgt), shared=True)
        plan.sync(timeout_s=600.0)
        n = plan.info()["pairs_transformed"]
        plan.close()
        assert n == expected_transforms(wl.nk, wl.n_occ, wl.n_tgt, 3, 3, on)
    assert expected_transforms(wl.nk, wl.n_occ, wl.n_tgt, 3, 3, True) < logical


@pytest.mark.parametrize("make", [synth.tiny_cubic, rhombo24] +
                         [lambda i=i: synth.sweep_cell(i) for i in range(len(synth.SWEEP_GRIDS))])
def test_staged_passes_match_unstaged(gpu, make):
    """FP32 pass B staged by bulk tensor copies and pass A fed by bulk copies of the
    occupied planes (both forced on) against the one-row-per-block pass B and the
    global-load pass A, on every grid length the sweep uses; ragged batches."""
    torch, xx = gpu
    wl = make()
    out = []
    for tma, stage in ((2, True), (0, False)):
        plan = xx.Plan.from_workload(wl, precision=0)
        plan.set_batch(5, 3)
        plan.set_tma_pass_b(tma)
        plan.set_stage_pass_a(2 if stage else 0)
        c = gu.dev(wl.c_tgt)
        ex, vx = plan.energy(c, gu.dev(wl.w_occ), c, gu.dev(wl.w_tgt), shared=True)
        plan.sync(timeout_s=600.0)
        out.append((vx.cpu().numpy(), float(ex[0].item())))
        plan.close()
    assert gu.rel_max(out[0][0], out[1][0]) <= 1e-6
    assert abs(out[0][1] - out[1][1]) <= 1e-6 * abs(out[1][1])
    plan = xx.Plan.from_workload(wl, precision=0)
    with pytest.raises(xx.XXError):
        plan.set_tma_pass_b(3)
    with pytest.raises(xx.XXError):
        plan.set_stage_pass_a(-1)
    plan.close()


def test_accumulator_limit_falls_back_to_per_k_accumulators(gpu):
    """With no room for the accumulators of every k-point (XX_OPT_ACC_LIMIT_MB = 0)
    the k != q blocks run in both orders and only the k = q tiles use the symmetry;
    the result matches the default path and the one without symmetry (FP64)."""
    torch, xx = gpu
    wl = rhombo24()
    out = []
    for limit, sym in ((None, True), (0, True), (None, False)):
        plan = xx.Plan.from_workload(wl, precision=1)
        plan.set_batch(3, 3)
        plan.set_pair_symmetry(sym)
        if limit is not None:
            xx.xx_set_option(plan.handle, xx.XX_OPT_ACC_LIMIT_MB, limit)
        c = gu.dev(wl.c_tgt)
        ex, vx = plan.energy(c, gu.dev(wl.w_occ), c, gu.dev(wl.w_tgt), shared=True)
        plan.sync(timeout_s=600.0)
        out.append((vx.cpu().numpy(), float(ex[0].item()), plan.info()["pairs_transformed"]))
        plan.close()
    for vx, e, _ in out[1:]:
        assert gu.rel_max(vx, out[0][0]) <= 1e-12
        assert abs(e - out[0][1]) <= 1e-12 * abs(out[0][1])
    nk, no, nt = wl.nk, wl.n_occ, wl.n_tgt
    diag = expected_transforms(1, no, nt, 3, 3, True)           # one k = q block
    assert out[1][2] == nk * diag + (nk * nk - nk) * nt * no       # k != q in both orders
    assert out[0][2] == expected_transforms(nk, no, nt, 3, 3, True)
    assert out[2][2] == nk * nk * nt * no
    plan = xx.Plan.from_workload(wl, precision=1)
    with pytest.raises(xx.XXError):
        xx.xx_set_option(plan.handle, xx.XX_OPT_ACC_LIMIT_MB, -1)
    plan.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_kept_kernel_tables_change_nothing(gpu, prec):
    """The kernel tables of every (k, q), built once and kept (XX_OPT_TABLE_CACHE,
    default), against tables built per band-pair batch: the same values, so the
    same V_x c and E_x bit for bit, with one table launch per plan instead of one
    per (k, q) and batch; the apply and the backward (which builds its dv/dmu
    tables per batch) still agree after the option is switched back and forth."""
    torch, xx = gpu
    wl = rhombo24()
    out = []
    for cache in (True, False, True):
        plan = xx.Plan.from_workload(wl, precision=prec)
        plan.set_batch(3, 3)
        plan.set_table_cache(cache)
        c = gu.dev(wl.c_tgt)
        plan.profile(True)
        ex, vx = plan.energy(c, gu.dev(wl.w_occ), c, gu.dev(wl.w_tgt), shared=True)
        tables = plan.profile_read(reset=True)["kernel_table"][1]
        dc, dmu = plan.backward(c, gu.dev(wl.w_tgt))
        ex2, vx2 = plan.energy(c, gu.dev(wl.w_occ), c, gu.dev(wl.w_tgt), shared=True)
        plan.sync(timeout_s=600.0)
        out.append((vx.cpu().numpy(), ex.cpu().numpy(), vx2.cpu().numpy(), dc.cpu().numpy(),
                    float(dmu.item()), tables))
        plan.close()
    for o in out[1:]:
        assert np.array_equal(o[0], out[0][0]) and np.array_equal(o[1], out[0][1])
        assert np.array_equal(o[2], out[0][0]) and np.array_equal(o[3], out[0][3])
        assert o[4] == out[0][4]
    assert out[0][5] == 1 and out[2][5] == 1
    assert out[1][5] > wl.nk
    # a workspace cap whose eighth cannot hold the nk^2 tables: built per batch
    plan = xx.Plan.from_workload(wl, precision=prec, workspace_cap=1 << 20)
    plan.set_batch(3, 3)
    c = gu.dev(wl.c_tgt)
    plan.profile(True)
    ex, vx = plan.energy(c, gu.dev(wl.w_occ), c, gu.dev(wl.w_tgt), shared=True)
    tables = plan.profile_read(reset=True)["kernel_table"][1]
    plan.sync(timeout_s=600.0)
    assert tables > wl.nk
    assert np.array_equal(vx.cpu().numpy(), out[0][0])
    plan.close()


@pytest.mark.parametrize("prec,tol", [(0, gu.FP32_TOL), (1, gu.FP64_TOL)])
def test_grid_64_k_mesh(gpu, oracle_mod, prec, tol):
    """The one supported FFT length no other workload uses (64 = 8 x 8): a cubic
    cell with a 2x2x2 MP mesh and targets past the occupied set, sampled targets
    against the oracle and Hermiticity on every k-point."""
    wl = synth.make_workload("cubic64", synth.cubic_lattice(10.0 * 64 / 24), (64,) * 3,
                             synth.monkhorst_pack(2), math.pi, 6, 8,
                             [1.0, 1.0, 1.0, 1.0, 0.5, 0.25], 64)
    assert np.all(4 * wl.n_max() + 1 <= 64)
    vx, (e, e_im), _ = gu.run(wl, prec)
    sel = [(0, 0), (wl.nk - 1, wl.n_tgt - 1), (3, 5)]
    ref = oracle_mod.apply(wl, sel=sel)
    got = np.stack([vx[k, a] for k, a in sel])
    assert gu.record("cubic 64^3 MP2x2x2 (6/8)", prec, "max|dVx|/max|Vx| (3 targets)",
                     gu.rel_max(got, ref), tol) <= tol
    assert gu.hermitian_defect(wl.c_tgt, vx) <= max(tol, 1e-12)
    assert abs(e_im) <= max(tol, 1e-12) * abs(e)


@pytest.mark.parametrize("shared", [True, False])
def test_q_point_segments_match_single_q_batches(gpu, shared):
    """Occupied sets of several k-points in one batch (default: 4 bands per k-point
    and a batch up to 160 wide) against one k-point per batch (occupied width 4), FP64,
    with the pair symmetry (shared grids, split layout) and without (separate
    occupied array)."""
    torch, xx = gpu
    wl = rhombo24()
    out = []
    for batch in (None, (6, 4)):
        plan = xx.Plan.from_workload(wl, precision=1)
        if batch:
            plan.set_batch(*batch)
        if shared:
            c = gu.dev(wl.c_tgt)
            ex, vx = plan.energy(c, gu.dev(wl.w_occ), c, gu.dev(wl.w_tgt), shared=True)
        else:
            ex, vx = plan.energy(gu.dev(wl.c_occ), gu.dev(wl.w_occ), gu.dev(wl.c_tgt),
                                 gu.dev(wl.w_tgt))
        plan.sync(timeout_s=600.0)
        info = plan.info()
        out.append((vx.cpu().numpy(), float(ex[0].item()), info["q_per_batch"]))
        plan.close()
    assert out[0][2] == wl.nk and out[1][2] == 1
    assert gu.rel_max(out[0][0], out[1][0]) <= 1e-12
    assert abs(out[0][1] - out[1][1]) <= 1e-12 * abs(out[1][1])
