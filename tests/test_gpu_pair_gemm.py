"""Two-SM form of the persistent preconditioner GEMM (CTA pairs, cta_group::2 MMAs over
256 x 256 tiles) against the one-SM kernel and the CPU FP64 oracle, through the C ABI.

The pair form multiplies the same BF16 operands in the same K order as the one-SM kernel,
so the two agree to FP32 rounding of the accumulators (1e-6 in relative 2-norm covers a
different summation order; a misplaced half tile, a transposed or missing B half, or a
skipped stage gives O(1) differences).  Against the oracle the tolerance is the one of
the tensor-core preconditioner, 3e-2 in relative 2-norm (BF16 operands).
"""
import numpy as np
import pytest

import mca_inputs as mi
from oracle import mca_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_07929_gb300 as mca  # noqa: E402

DEV = "cuda:0"
PAIR = mca.FLAG_GRAPHS | mca.FLAG_PAIR_GEMM
SINGLE = mca.FLAG_GRAPHS


def _params(p, **kw):
    base = dict(g_wire_top=p.g_wire_top, g_wire_bot=p.g_wire_bot, g_src=p.g_src,
                g_term_top_right=p.g_term_top_right, g_term_bot_top=p.g_term_bot_top,
                g_sense=p.g_sense, b=p.b)
    base.update(kw)
    return mca.default_params(p.rows, p.cols, **base)


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _apply(cb, prec, flags, a, r):
    B = r.shape[0]
    m, n = cb.params.rows, cb.params.cols
    with mca.Solver(_params(cb.params, precision=prec, max_batch=B, flags=flags), cb.gmap) as s:
        z = torch.empty(B, 2 * m * n, dtype=torch.float64, device=DEV)
        s.precond_apply(a, _t(r), z)
        return z.cpu().numpy(), s.tile_config()


@pytest.mark.parametrize("prec", [mca.PREC_BF16, mca.PREC_BF16_SPLIT], ids=["bf16", "bf16split"])
@pytest.mark.parametrize("m,n,B", [(256, 256, 3), (512, 768, 2), (1024, 1024, 33)])
def test_pair_precond_matches_single_sm_and_oracle(m, n, B, prec):
    cb = mi.make_crossbar(m, n, 4, g_wire_bot=0.5)
    rng = np.random.default_rng(11)
    r = rng.standard_normal((B, 2 * m * n))
    a = rng.uniform(1e-5, 4e-4, B)
    zp, cfg = _apply(cb, prec, PAIR, a, r)
    # transforms 1, 3 and 4 in the two-SM form, the modes transform in the one-SM form
    assert [c[0] for c in cfg] == [2, 1, 2, 2], cfg
    assert [c[1] for c in cfg[0:1] + cfg[2:]] == [256, 256, 256], cfg
    zs, cfg1 = _apply(cb, prec, SINGLE, a, r)
    assert all(c[0] != 2 for c in cfg1), cfg1
    for v in range(B):
        d = np.linalg.norm(zp[v] - zs[v]) / np.linalg.norm(zs[v])
        assert d < 1e-6, (v, d)
    eig = O.eig_setup(cb.params)
    for v in sorted({0, B // 2, B - 1}):
        zt, zb = O.precond_apply_modes(eig, a[v], a[v], r[v, :m * n], r[v, m * n:], (m, n))
        ref = np.concatenate([zt, zb])
        err = np.linalg.norm(zp[v] - ref) / np.linalg.norm(ref)
        assert err < 3e-2, (v, err)


@pytest.mark.parametrize("m,n", [(256, 384), (130, 70), (384, 256)])
def test_pair_not_used_where_the_tile_does_not_fit(m, n):
    """Rows or columns not a multiple of 256: the transform keeps the one-SM form."""
    cb = mi.make_crossbar(m, n, 5, g_wire_bot=0.5)
    rng = np.random.default_rng(12)
    r = rng.standard_normal((2, 2 * m * n))
    a = np.array([3e-5, 1e-4])
    zp, cfg = _apply(cb, mca.PREC_BF16_SPLIT, PAIR, a, r)
    mp, np_ = (m + 127) // 128 * 128, (n + 127) // 128 * 128
    fits = mp % 256 == 0 and np_ % 256 == 0
    assert all((c[0] == 2) == (fits and s != 1) for s, c in enumerate(cfg)), cfg
    zs, _ = _apply(cb, mca.PREC_BF16_SPLIT, SINGLE, a, r)
    np.testing.assert_allclose(zp, zs, rtol=0, atol=1e-6 * np.abs(zs).max())


@pytest.mark.parametrize("flags", [PAIR, PAIR | mca.FLAG_AUTOTUNE], ids=["forced", "autotuned"])
def test_pair_solve_against_oracle(flags):
    """Whole solves (Newton + FGMRES, BF16-split) with the two-SM GEMMs forced or offered to
    the autotuner: relative KCL residual recomputed by the oracle within the tolerance,
    voltages as the one-SM solver's."""
    m = n = 512
    cb = mi.make_crossbar(m, n, 7, nvec=4)
    p = _params(cb.params, precision=mca.PREC_BF16_SPLIT, max_batch=4, flags=flags)
    with mca.Solver(p, cb.gmap) as s:
        vt, vb, io, st = s.solve(cb.vin)
        cfg = s.tile_config()
    if not (flags & mca.FLAG_AUTOTUNE):
        assert cfg[0][0] == 2 and cfg[2][0] == 2 and cfg[3][0] == 2, cfg
    p1 = _params(cb.params, precision=mca.PREC_BF16_SPLIT, max_batch=4, flags=SINGLE)
    with mca.Solver(p1, cb.gmap) as s1:
        vt1, vb1, _, _ = s1.solve(cb.vin)
    ops = O.layer_operators(cb.params)
    for v in range(4):
        assert st[v]["status"] == 0, st[v]
        Ft, Fb = O.residual(cb.params, cb.gmap, cb.vin[v], vt[v].ravel(), vb[v].ravel(), ops)
        Yt, _ = O.source_vector(cb.params, cb.vin[v])
        rel = np.linalg.norm(np.concatenate([Ft, Fb])) / np.linalg.norm(Yt)
        assert rel <= 1.01 * p.newton_rtol, (v, rel)
        scale = max(np.abs(vt1[v]).max(), np.abs(vb1[v]).max())
        assert np.abs(vt[v] - vt1[v]).max() / scale < 1e-6
        assert np.abs(vb[v] - vb1[v]).max() / scale < 1e-6
