"""Multi-right-hand-side (block) Krylov for the first Newton step of the statistical-
characterisation workload: what it would save, measured on the CPU model in
block_krylov_model.py.

All 16 input vectors of one crossbar share J(0), so their first Newton systems could be
solved as one block.  With the exact Kronecker preconditioner each GMRES iteration already
cuts every column's residual by a factor of 30-100, and the block space does not converge
in fewer block iterations than the single solves take per vector: at the solver's first
forcing term eta0 = 1e-3 both take 2 preconditioner applies per vector (measured on the
64^2 .. 512^2 shapes of the workload; at 1e-4 the block form takes more, 48 against 38
applies at 256^2).  So a block solve saves no tensor-core or Jacobian work, and its block
orthogonalisation costs more dot products; the library solves the vectors as a batch of
independent systems that share every kernel launch and the GEMM operands instead.
"""
import numpy as np
import pytest

import mca_inputs as mi
import block_krylov_model as BK


def test_block_gmres_solves_the_block_system():
    cb = mi.make_crossbar(6, 9, 3, nvec=4, g_wire_bot=0.5)
    J, pc, B = BK.first_step_systems(cb.params, cb.gmap, cb.vin)
    kb, applies, res = BK.block_gmres_applies(J, pc, B, 1e-11)
    assert res <= 1e-10 and applies == 4 * kb


def _workload_crossbar(m, n):
    cbs = mi.config_batched(count=128, nvec=16)
    return next(cb for cb in cbs if (cb.params.rows, cb.params.cols) == (m, n))


@pytest.mark.parametrize("m,n", [(64, 64), (128, 256)])
def test_block_first_step_saves_no_applies(m, n):
    cb = _workload_crossbar(m, n)
    J, pc, B = BK.first_step_systems(cb.params, cb.gmap, cb.vin)
    eta0 = 1e-3
    single = BK.single_gmres_applies(J, pc, B, eta0)
    kb, block, res = BK.block_gmres_applies(J, pc, B, eta0)
    assert res <= eta0
    assert sum(single) == 32 and block == 32      # 2 applies per vector either way
