"""The allocation-free residual entry point gives the same results as the handle-based
one (mca_residual), on two calls in a row through the C ABI.  Kept in a file collected
last so a stop-at-first-failure run has already run every other test."""
import numpy as np
import pytest

import mca_inputs as mi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_07929_gb300 as mca  # noqa: E402


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")


@pytest.mark.parametrize("m,n,nvec", [(33, 47, 3), (256, 256, 8)])
def test_noalloc_residual_matches_handle_residual(m, n, nvec):
    cb = mi.make_crossbar(m, n, 31, nvec=nvec)
    p = cb.params
    params = mca.default_params(m, n, g_wire_top=p.g_wire_top, g_wire_bot=p.g_wire_bot,
                                g_src=p.g_src, g_term_top_right=p.g_term_top_right,
                                g_term_bot_top=p.g_term_bot_top, g_sense=p.g_sense, b=p.b,
                                precision=mca.PREC_FP64, max_batch=nvec)
    g = _dev(cb.gmap)
    vin = _dev(cb.vin)
    rng = np.random.default_rng(2)
    with mca.Solver(params, cb.gmap) as s:
        for call in range(2):   # two calls in a row share the fixed scratch array
            x = _dev(rng.uniform(-0.1, 0.35, size=(nvec, 2 * m * n)))
            F0 = torch.empty(nvec, 2 * m * n, dtype=torch.float64, device="cuda:0")
            D0 = torch.empty(nvec, m * n, dtype=torch.float64, device="cuda:0")
            fn0, dm0 = s.residual(x, vin, F0, D0)
            F1 = torch.full_like(F0, float("nan"))
            D1 = torch.full_like(D0, float("nan"))
            fn1 = torch.full((nvec,), float("nan"), dtype=torch.float64, device="cuda:0")
            dm1 = torch.full_like(fn1, float("nan"))
            torch.cuda.synchronize()
            used0 = torch.cuda.memory_allocated()
            free0 = torch.cuda.mem_get_info()[0]
            mca.residual_noalloc(params, g, x, vin, F1, D1, fn1, dm1)
            torch.cuda.synchronize()
            if call == 1:
                # after the first call (which loads the kernels and looks up the scratch
                # address) a call leaves the device allocator and free memory untouched
                assert torch.cuda.memory_allocated() == used0
                assert torch.cuda.mem_get_info()[0] == free0
            assert torch.equal(F0, F1) and torch.equal(D0, D1)
            np.testing.assert_allclose(fn1.cpu().numpy(), fn0, rtol=1e-12)
            np.testing.assert_allclose(dm1.cpu().numpy(), dm0, rtol=1e-12)


def test_noalloc_rejects_too_many_vectors():
    params = mca.default_params(4, 4)
    x = torch.zeros(9, 32, dtype=torch.float64, device="cuda:0")
    with pytest.raises(mca.MCAError) as e:
        mca.residual_noalloc(params, torch.ones(16, dtype=torch.float64, device="cuda:0"), x,
                             torch.zeros(9, 4, dtype=torch.float64, device="cuda:0"),
                             torch.empty_like(x), torch.empty(9, 16, dtype=torch.float64,
                                                              device="cuda:0"))
    assert e.value.code == mca.ERR_INVALID_ARG


@pytest.mark.parametrize("field,value", [("g_wire_top", 0.0), ("b", float("nan")),
                                         ("device_model", 7), ("g_sense", -1.0)])
def test_noalloc_rejects_bad_circuit_parameters(field, value):
    params = mca.default_params(4, 4)
    setattr(params, field, value)
    x = torch.zeros(1, 32, dtype=torch.float64, device="cuda:0")
    with pytest.raises(mca.MCAError) as e:
        mca.residual_noalloc(params, torch.ones(16, dtype=torch.float64, device="cuda:0"), x,
                             torch.zeros(1, 4, dtype=torch.float64, device="cuda:0"),
                             torch.empty_like(x), torch.empty(1, 16, dtype=torch.float64,
                                                              device="cuda:0"))
    assert e.value.code == mca.ERR_INVALID_ARG
