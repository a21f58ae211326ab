"""The precision split of the tensor-core preconditioner (which transform operands carry a
hi + lo BF16 pair), checked on the NumPy model of its arithmetic in precision_model.py.

The model's BF16 rounding is pinned to PyTorch's float32 -> bfloat16 conversion (round to
nearest even).  Then Newton + GMRES(30) with the solver's forcing terms is run on the
log-uniform crossbar (wires 1 S / 0.5 S, sinh devices b = 2) to 1e-8, and the GMRES
iterations per solve of each arithmetic are compared with the exact preconditioner's:

    1024^2 (seed 0):  fp64 6, fp16 9, bf16 32, split3 6, split2 6

The split forms must match the exact preconditioner's count (the back transforms' rounding
of the eigenvectors would otherwise leak the amplified low modes into the high ones), and
the one-word forms must not.  split2 (transform 3 with Y_hat as one word, two products)
is the form the library runs.
"""
import numpy as np
import pytest

import mca_inputs as mi
import precision_model as PM

torch = pytest.importorskip("torch")


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32) *
                        np.float32(10.0) ** rng.integers(-30, 30, 20000).astype(np.float32),
                        np.array([0.0, -0.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8,
                                  1.0 + 2.0 ** -9, -(1.0 + 2.0 ** -8)], np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(PM.bf16(x), ref)
    hi, lo = PM.split(x)
    # hi + lo carries 16 significant bits: within 2^-16 of x (relative)
    assert np.all(np.abs(hi.astype(np.float64) + lo - x) <= 2.0 ** -16 * np.abs(x) + 1e-300)


def _iters(n, variant, seed=0):
    cb = mi.config_large(n, seed, nvec=1)
    steps, its, rel = PM.newton_gmres(cb.params, cb.gmap, cb.vin[0], variant)
    assert rel <= 1e-8, (variant, rel)
    return steps, sum(its)


@pytest.mark.parametrize("n", [256, 1024])
def test_split_back_transforms_keep_the_exact_iteration_count(n):
    steps64, it64 = _iters(n, "fp64")
    assert steps64 == 2
    for v in ("split3", "split2"):
        steps, it = _iters(n, v)
        assert steps == 2 and it <= it64, (v, it, it64)
    _, it_bf16 = _iters(n, "bf16")
    assert it_bf16 >= 2 * it64 + 2
    if n == 1024:
        _, it_fp16 = _iters(n, "fp16")
        assert it64 < it_fp16 < it_bf16
