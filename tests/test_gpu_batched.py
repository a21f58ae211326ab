"""Batched statistical-characterisation path: several crossbars per handle (one shape,
per-vector conductance map), CUDA-graph replay of the GMRES iterations, the tile
autotuner, and concurrent solves of many handles; every result is checked against the
single-crossbar solve and the CPU oracle."""
import numpy as np
import pytest

import mca_inputs as mi
from oracle import mca_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_07929_gb300 as mca  # noqa: E402


def _params(p, **kw):
    base = dict(g_wire_top=p.g_wire_top, g_wire_bot=p.g_wire_bot, g_src=p.g_src,
                g_term_top_right=p.g_term_top_right, g_term_bot_top=p.g_term_bot_top,
                g_sense=p.g_sense, b=p.b, newton_rtol=1e-11)
    base.update(kw)
    return mca.default_params(p.rows, p.cols, **base)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_multi_map_matches_single_maps():
    cbs = [mi.make_crossbar(48, 40, 100 + k, nvec=2, sigma=0.1) for k in range(3)]
    p = cbs[0].params
    gmaps = np.stack([cb.gmap for cb in cbs])
    order = [0, 1, 2, 2, 1, 0]
    vin = np.stack([cbs[k].vin[i % 2] for i, k in enumerate(order)])
    with mca.Solver(_params(p, max_batch=4), gmaps) as s:
        vt, vb, io, st = s.solve(vin, map_index=order)
    for v, k in enumerate(order):
        assert st[v]["status"] == 0
        with mca.Solver(_params(p, max_batch=1), cbs[k].gmap) as s1:
            vt1, vb1, _, _ = s1.solve(vin[v:v + 1])
        assert _rel(vt[v], vt1[0]) < 1e-9 and _rel(vb[v], vb1[0]) < 1e-8
        ref = O.newton_solve(p, cbs[k].gmap, vin[v], tol=1e-13, linear="direct")
        assert _rel(vt[v], ref.Vt) < 1e-7 and _rel(vb[v], ref.Vb) < 1e-7


def test_map_index_out_of_range_rejected():
    cb = mi.make_crossbar(8, 8, 1)
    with mca.Solver(_params(cb.params, max_batch=1), np.stack([cb.gmap, cb.gmap])) as s:
        with pytest.raises(mca.MCAError) as e:
            s.solve(cb.vin, map_index=[2])
        assert e.value.code == mca.ERR_INVALID_ARG


@pytest.mark.parametrize("prec", [mca.PREC_FP64, mca.PREC_BF16_SPLIT], ids=["fp64", "bf16split"])
def test_graph_replay_and_autotune_match_direct_launches(prec):
    cb = mi.make_crossbar(96, 160, 7, nvec=5)
    p = cb.params
    res = []
    for flags in (0, mca.FLAG_GRAPHS, mca.FLAG_GRAPHS | mca.FLAG_AUTOTUNE):
        with mca.Solver(_params(p, precision=prec, max_batch=3, flags=flags), cb.gmap) as s:
            res.append(s.solve(cb.vin))
            res.append(s.solve(cb.vin))          # replays the captured graphs
    for r in res[1:]:
        np.testing.assert_allclose(r[0], res[0][0], rtol=1e-13, atol=0)
        np.testing.assert_allclose(r[1], res[0][1], rtol=1e-13, atol=1e-18)
        assert [x["gmres_iters"] for x in r[3]] == [x["gmres_iters"] for x in res[0][3]]


def test_solve_many_mixed_shapes():
    shapes = [(64, 128), (128, 64), (96, 96), (33, 47), (200, 130)]
    cbs = [mi.make_crossbar(m, n, 300 + k, nvec=3, sigma=0.1) for k, (m, n) in enumerate(shapes)]
    solvers = [mca.Solver(_params(cb.params, max_batch=3), cb.gmap) for cb in cbs]
    try:
        out = mca.solve_many(solvers, [cb.vin for cb in cbs], n_threads=3)
        for s, cb, (vt, vb, io, st) in zip(solvers, cbs, out):
            assert all(x["status"] == 0 for x in st)
            vt1, vb1, io1, _ = s.solve(cb.vin)
            assert _rel(vt, vt1) < 1e-12 and _rel(io, io1) < 1e-12
            ref = O.newton_solve(cb.params, cb.gmap, cb.vin[0], tol=1e-13, linear="direct")
            assert _rel(vt[0], ref.Vt) < 1e-7
    finally:
        for s in solvers:
            s.close()


def test_statistical_characterisation_sample():
    """A sample of the 128-crossbar workload (sizes from {64,128,256,512}, 16 vectors
    each): grouped by shape into multi-map handles and solved concurrently; every
    solve meets 1e-8 and the oracle's residual of the returned voltages agrees."""
    cbs = mi.config_batched(count=6, nvec=4)
    groups = {}
    for k, cb in enumerate(cbs):
        groups.setdefault((cb.params.rows, cb.params.cols), []).append(k)
    solvers, vins, maps = [], [], []
    for (m, n), ks in groups.items():
        p = cbs[ks[0]].params
        solvers.append(mca.Solver(_params(p, newton_rtol=1e-8, max_batch=8),
                                  np.stack([cbs[k].gmap for k in ks])))
        vins.append(np.concatenate([cbs[k].vin for k in ks]))
        maps.append(np.repeat(np.arange(len(ks)), 4))
    try:
        out = mca.solve_many(solvers, vins, map_indices=maps, n_threads=4)
        for ((m, n), ks), (vt, vb, io, st), vin in zip(groups.items(), out, vins):
            for v in range(vin.shape[0]):
                cb = cbs[ks[v // 4]]
                assert st[v]["status"] == 0 and st[v]["rel_residual"] <= 1e-8
                Ft, Fb = O.residual(cb.params, cb.gmap, vin[v], vt[v].ravel(), vb[v].ravel())
                Yt, _ = O.source_vector(cb.params, vin[v])
                rel = np.linalg.norm(np.concatenate([Ft, Fb])) / np.linalg.norm(Yt)
                assert rel <= 1.01e-8
    finally:
        for s in solvers:
            s.close()


def test_concurrent_handles_device_buffers():
    """The bench's pattern: two handles of one crossbar solved concurrently from two host
    threads with device-resident inputs and outputs (graph capture in both threads at once).
    Each handle's results equal a later solve of the same vectors on its own, and the oracle
    recomputes the KCL residual of some of them."""
    cb = mi.make_crossbar(256, 256, 21, nvec=32)
    p = cb.params
    prm = _params(p, precision=mca.PREC_BF16_SPLIT, max_batch=16, newton_rtol=1e-8)
    hs = [mca.Solver(prm, cb.gmap) for _ in range(2)]
    try:
        dev = "cuda:0"
        vin = torch.as_tensor(cb.vin, device=dev)
        outs = [(torch.empty(16, 256, 256, dtype=torch.float64, device=dev),
                 torch.empty(16, 256, 256, dtype=torch.float64, device=dev),
                 torch.empty(16, 256, dtype=torch.float64, device=dev)) for _ in range(2)]
        res = mca.solve_many(hs, [vin[:16], vin[16:]], n_threads=2, outs=outs)
        for k in range(2):
            assert all(x["status"] == 0 for x in res[k][3])
            vt1, vb1, io1, _ = hs[k].solve(cb.vin[16 * k:16 * (k + 1)])
            assert _rel(outs[k][0].cpu().numpy(), vt1) < 1e-12
            assert _rel(outs[k][2].cpu().numpy(), io1) < 1e-12
        for v in (0, 17, 31):
            k, j = divmod(v, 16)
            vt = outs[k][0][j].cpu().numpy().ravel()
            vb = outs[k][1][j].cpu().numpy().ravel()
            Ft, Fb = O.residual(p, cb.gmap, cb.vin[v], vt, vb)
            Yt, _ = O.source_vector(p, cb.vin[v])
            assert np.linalg.norm(np.concatenate([Ft, Fb])) / np.linalg.norm(Yt) <= 1e-8 * 1.01
    finally:
        for h in hs:
            h.close()
