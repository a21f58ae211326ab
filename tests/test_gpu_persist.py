"""Persistent batched solve (one kernel launch, one (crossbar, input vector) item per CTA at
a time): its tensor-core preconditioner against the oracle's eigenbasis inverse of eq. (P),
and its solves against the oracle's residual of eq. (F) and direct Newton solution, over
mixed and ragged shapes, several maps per shape, slot reuse across shapes, GMRES(1), the
Yakopcic-form device, zero inputs and the statistical-characterisation mix."""
import numpy as np
import pytest

import mca_inputs as mi
from oracle import mca_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_07929_gb300 as mca  # noqa: E402

DEV = torch.device("cuda", 0)


def _params(p, **kw):
    base = dict(g_wire_top=p.g_wire_top, g_wire_bot=p.g_wire_bot, g_src=p.g_src,
                g_term_top_right=p.g_term_top_right, g_term_bot_top=p.g_term_bot_top,
                g_sense=p.g_sense, b=p.b, neg_ratio=p.neg_ratio,
                device_model=mca.DEVICE_YAKOPCIC if p.neg_ratio != 1.0 else mca.DEVICE_SINH,
                precision=mca.PREC_BF16_SPLIT, max_batch=1, newton_rtol=1e-10)
    base.update(kw)
    return mca.default_params(p.rows, p.cols, **base)


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _check_item(p, gmap, vin, vt, vb, io, st, tol, vtol=1e-7):
    assert st["status"] == 0, st
    Ft, Fb = O.residual(p, gmap, vin, vt.ravel(), vb.ravel())
    Yt, _ = O.source_vector(p, vin)
    rel = np.linalg.norm(np.concatenate([Ft, Fb])) / np.linalg.norm(Yt)
    assert rel <= tol * 1.01, rel
    np.testing.assert_allclose(st["rel_residual"], rel, rtol=1e-3, atol=tol * 1e-3)
    ref = O.newton_solve(p, gmap, vin, tol=1e-13, linear="direct")
    scale = max(np.abs(ref.Vt).max(), np.abs(ref.Vb).max())
    assert np.abs(vt - ref.Vt).max() <= vtol * scale
    assert np.abs(vb - ref.Vb).max() <= vtol * scale
    np.testing.assert_allclose(io, p.g_sense * vb[-1], rtol=1e-15)
    assert st["kcl_rel_error"] <= 1e-6


@pytest.mark.parametrize("shapes", [[(1, 1), (33, 47), (130, 70)], [(256, 384), (64, 512)]],
                         ids=["small", "large"])
def test_persistent_preconditioner_matches_oracle(shapes):
    cbs = [mi.make_crossbar(m, n, 4, g_wire_bot=0.5) for m, n in shapes]
    solvers = [mca.Solver(_params(cb.params), cb.gmap) for cb in cbs]
    rng = np.random.default_rng(8)
    a = np.array([2.1e-5, 7.0e-5, 3.3e-4])
    try:
        with mca.Batch(solvers) as b:
            hs, rs, tops, bots, avals = [], [], [], [], []
            for k, cb in enumerate(cbs):
                m, n = cb.params.rows, cb.params.cols
                for v in range(3):
                    r = rng.standard_normal(2 * m * n)
                    rs.append(r)
                    tops.append(_t(r[:m * n]))
                    bots.append(_t(r[m * n:]))
                    hs.append(k)
                    avals.append(a[v])
            items = mca.Batch.items(hs, [0] * len(hs), [None] * len(hs), tops, bots)
            b.precond(items, avals)
            torch.cuda.synchronize()
            for q, k in enumerate(hs):
                p = cbs[k].params
                m, n = p.rows, p.cols
                eig = O.eig_setup(p)
                zt, zb = O.precond_apply_modes(eig, avals[q], avals[q], rs[q][:m * n],
                                               rs[q][m * n:], (m, n))
                ref = np.concatenate([zt, zb])
                z = np.concatenate([tops[q].cpu().numpy(), bots[q].cpu().numpy()])
                err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
                assert err < 3e-2, (shapes[k], q, err)
                # the batched kernels' split preconditioner: same operands, other tiling
                zh = torch.empty(1, 2 * m * n, dtype=torch.float64, device=DEV)
                solvers[k].precond_apply(np.array([avals[q]]), _t(rs[q][None]), zh)
                zh = zh.cpu().numpy()[0]
                assert np.linalg.norm(z - zh) / np.linalg.norm(zh) < 1e-2
    finally:
        for s in solvers:
            s.close()


def _run_batch(cbs, per_maps, tol, max_ctas=0, **kw):
    """cbs: list of lists of crossbars sharing a shape (maps of one handle).  Solves every
    input vector of every crossbar in one persistent launch; returns per item
    (p, gmap, vin, vt, vb, io, stats)."""
    solvers = []
    for group in cbs:
        p = group[0].params
        solvers.append(mca.Solver(_params(p, newton_rtol=tol, **kw),
                                  np.stack([cb.gmap for cb in group])))
    try:
        hs, maps, vins, vts, vbs, ios, meta = [], [], [], [], [], [], []
        for k, group in enumerate(cbs):
            for mp_, cb in enumerate(group):
                m, n = cb.params.rows, cb.params.cols
                for v in range(min(per_maps, len(cb.vin))):
                    hs.append(k)
                    maps.append(mp_)
                    vins.append(_t(cb.vin[v]))
                    vts.append(torch.empty(m, n, dtype=torch.float64, device=DEV))
                    vbs.append(torch.empty(m, n, dtype=torch.float64, device=DEV))
                    ios.append(torch.empty(n, dtype=torch.float64, device=DEV))
                    meta.append((cb, v))
        with mca.Batch(solvers, max_ctas=max_ctas) as b:
            items = mca.Batch.items(hs, maps, vins, vts, vbs, ios)
            st = b.solve_items(items)
        torch.cuda.synchronize()
        out = []
        for q, (cb, v) in enumerate(meta):
            out.append((cb.params, cb.gmap, cb.vin[v], vts[q].cpu().numpy(),
                        vbs[q].cpu().numpy(), ios[q].cpu().numpy(), st[q], hs[q]))
        return out, solvers
    except Exception:
        for s in solvers:
            s.close()
        raise


def test_persistent_solve_mixed_ragged_shapes():
    shapes = [(1, 1), (1, 17), (5, 1), (33, 47), (130, 70), (64, 128), (128, 64)]
    cbs = [[mi.make_crossbar(m, n, 11 + k, nvec=3, g_wire_bot=0.5)] for k, (m, n) in
           enumerate(shapes)]
    out, solvers = _run_batch(cbs, 3, 1e-11)
    try:
        for p, gmap, vin, vt, vb, io, st, k in out:
            _check_item(p, gmap, vin, vt, vb, io, st, 1e-11)
        # the same vectors through the handles' batched kernels
        for k, group in enumerate(cbs):
            vt1, vb1, io1, _ = solvers[k].solve(group[0].vin)
            mine = [o for o in out if o[7] == k]
            for v, o in enumerate(mine):
                scale = np.abs(vt1[v]).max()
                assert np.abs(o[3] - vt1[v]).max() <= 1e-8 * scale
    finally:
        for s in solvers:
            s.close()


def test_persistent_solve_several_maps_and_slot_reuse():
    """Two shapes with three maps each, all items through a single CTA (each slot reused
    across shapes and maps)."""
    groups = [[mi.make_crossbar(48, 40, 100 + c, nvec=2, sigma=0.1) for c in range(3)],
              [mi.make_crossbar(96, 160, 200 + c, nvec=2, sigma=0.1) for c in range(3)]]
    out, solvers = _run_batch(groups, 2, 1e-10, max_ctas=1)
    try:
        assert len(out) == 12
        for p, gmap, vin, vt, vb, io, st, k in out:
            _check_item(p, gmap, vin, vt, vb, io, st, 1e-10)
    finally:
        for s in solvers:
            s.close()


def test_persistent_gmres_restart_1_and_30():
    cb = mi.make_crossbar(24, 40, 13, nvec=2)
    for restart in (1, 30):
        out, solvers = _run_batch([[cb]], 2, 1e-9, gmres_restart=restart)
        try:
            for p, gmap, vin, vt, vb, io, st, k in out:
                _check_item(p, gmap, vin, vt, vb, io, st, 1e-9)
                if restart == 1:
                    assert st["gmres_iters"] == st["newton_iters"]
        finally:
            for s in solvers:
                s.close()


@pytest.mark.parametrize("m,n", [(24, 40), (130, 70)])
def test_persistent_yakopcic_signed_inputs(m, n):
    """Yakopcic-form devices (a2/a1 = 0.5) with inputs of both signs."""
    cb = mi.make_crossbar(m, n, 19, nvec=3, vmin=-0.3, neg_ratio=0.5)
    assert (cb.vin < 0).any()
    out, solvers = _run_batch([[cb]], 3, 1e-10)
    try:
        for p, gmap, vin, vt, vb, io, st, k in out:
            _check_item(p, gmap, vin, vt, vb, io, st, 1e-10)
    finally:
        for s in solvers:
            s.close()


def test_persistent_zero_input_and_rejections():
    cb = mi.make_crossbar(16, 24, 3, nvec=2)
    cb.vin[1] = 0.0
    out, solvers = _run_batch([[cb]], 2, 1e-10)
    try:
        assert out[1][6]["status"] == 0 and out[1][6]["newton_iters"] == 0
        assert np.all(out[1][3] == 0.0) and np.all(out[1][4] == 0.0)
        with mca.Batch(solvers) as b:
            vin = _t(cb.vin[0])
            for hs, maps in (([1], [0]), ([0], [1]), ([-1], [0])):
                with pytest.raises(mca.MCAError) as e:
                    b.solve_items(mca.Batch.items(hs, maps, [vin]))
                assert e.value.code == mca.ERR_INVALID_ARG
            with pytest.raises(mca.MCAError) as e:
                b.solve_items(mca.Batch.items([0], [0], [None]))
            assert e.value.code == mca.ERR_INVALID_ARG
            assert b.solve_items(mca.Batch.items([], [], [])) == []
    finally:
        for s in solvers:
            s.close()
    with mca.Solver(_params(cb.params, precision=mca.PREC_FP64), cb.gmap) as s64:
        with pytest.raises(mca.MCAError) as e:
            mca.Batch([s64])
        assert e.value.code == mca.ERR_UNSUPPORTED


def test_persistent_statistical_mix_sample():
    """A sample of the statistical-characterisation workload: crossbars with rows and
    columns from {64, 128, 256, 512}, two input vectors each, Newton to 1e-8, restart 16;
    oracle residual on every item, oracle solution on one item per shape."""
    cbs = mi.config_batched(count=10, nvec=2)
    groups = {}
    for cb in cbs:
        groups.setdefault((cb.params.rows, cb.params.cols), []).append(cb)
    keys = sorted(groups)
    out, solvers = _run_batch([groups[k] for k in keys], 2, 1e-8, gmres_restart=16)
    try:
        seen = set()
        for p, gmap, vin, vt, vb, io, st, k in out:
            assert st["status"] == 0
            Ft, Fb = O.residual(p, gmap, vin, vt.ravel(), vb.ravel())
            Yt, _ = O.source_vector(p, vin)
            rel = np.linalg.norm(np.concatenate([Ft, Fb])) / np.linalg.norm(Yt)
            assert rel <= 1e-8 * 1.01
            if k not in seen and p.rows * p.cols <= 128 * 256:
                seen.add(k)
                _check_item(p, gmap, vin, vt, vb, io, st, 1e-8, vtol=1e-6)
    finally:
        for s in solvers:
            s.close()


def test_persistent_long_cycles_and_per_handle_settings():
    """The paper's normalised regime (wires and terminations 1 S, linear devices with g in
    [0, 0.4]; the oracle's exact-P GMRES needs 21 iterations to 5e-12 on it) with a tiny
    first forcing term: the linear solve runs long GMRES cycles (basis widths past 16, the
    widest Gram-Schmidt passes).  A second handle in the same launch keeps the default
    forcing terms and its own tolerance.  Every item against the oracle, and against the
    handle path with the same settings."""
    cb_long = mi.make_crossbar(40, 56, 31, nvec=2, gdist="uniform_paper", g_src=1.0,
                               g_term_top_right=1.0, g_term_bot_top=1.0, g_sense=1.0, b=0.0)
    cb_loose = mi.make_crossbar(72, 24, 32, nvec=2, sigma=0.1)
    s_long = mca.Solver(_params(cb_long.params, newton_rtol=1e-11, eta0=1e-12, eta_max=1e-12,
                                gmres_restart=30), cb_long.gmap)
    s_loose = mca.Solver(_params(cb_loose.params, newton_rtol=1e-8), cb_loose.gmap)
    try:
        items_in = []
        for k, (s, cb) in enumerate(((s_long, cb_long), (s_loose, cb_loose))):
            m, n = cb.params.rows, cb.params.cols
            for v in range(2):
                items_in.append((k, cb, v, torch.empty(m, n, dtype=torch.float64, device=DEV),
                                 torch.empty(m, n, dtype=torch.float64, device=DEV),
                                 torch.empty(n, dtype=torch.float64, device=DEV)))
        vins = [_t(cb.vin[v]) for _, cb, v, *_ in items_in]
        with mca.Batch([s_long, s_loose]) as b:
            items = mca.Batch.items([x[0] for x in items_in], [0] * len(items_in), vins,
                                    [x[3] for x in items_in], [x[4] for x in items_in],
                                    [x[5] for x in items_in])
            st = b.solve_items(items)
        torch.cuda.synchronize()
        for (k, cb, v, vt, vb, io), sq in zip(items_in, st):
            tol = 1e-11 if k == 0 else 1e-8
            _check_item(cb.params, cb.gmap, cb.vin[v], vt.cpu().numpy(), vb.cpu().numpy(),
                        io.cpu().numpy(), sq, tol, vtol=1e-7 if k == 0 else 1e-6)
        long_iters = [sq["gmres_iters"] for (k, *_), sq in zip(items_in, st) if k == 0]
        assert min(long_iters) > 16, long_iters
        # the handle path with the same settings reaches the same solution
        vt1, vb1, _, st1 = s_long.solve(cb_long.vin[:2])
        for v in range(2):
            vt = items_in[v][3].cpu().numpy()
            assert np.abs(vt - vt1[v]).max() <= 1e-9 * np.abs(vt1[v]).max()
    finally:
        s_long.close()
        s_loose.close()
