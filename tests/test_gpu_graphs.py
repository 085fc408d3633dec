"""CUDA-graph replay of the natural-gradient iteration reproduces the eager
launches bit for bit (same kernels, same order, the random stream position
kept on the device), for the float32 and mixed paths."""

import numpy as np
import pytest

from gpu_common import host, need_gpu
from paper_2103_08804_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _run(prec, graphs, Lx=16, M=32, B=2048, nm=5):
    from paper_2103_08804_gb300 import api, driver
    E0, a = synth.safe_rescaling(Lx, 1)
    cfg = driver.SeqConfig(Lx=Lx, Ly=1, M=M, q=(np.pi / 2, 0.0), n_moments=nm, n_iter=6,
                           E0=E0, a=a, n_therm=2, solver=api.SOLVE_CG, cg_maxit=20, cg_tol=1e-5)
    ctx = api.Context(Lx, 1, M, B, prec=prec)
    seq = driver.Sequence(ctx, cfg, synth.rbm_params(7, Lx, M, 0.05), synth.sz0_spins(8, B, Lx),
                          synth.sz0_spins(9, B, Lx), graphs=graphs)
    seq.run()
    ctx.sync_status()
    return seq


@pytest.mark.parametrize("prec", [1, 2])
def test_graph_replay_equals_eager(prec):
    a = _run(prec, False)
    b = _run(prec, True)
    assert b.graph_launches > 0
    assert np.array_equal(host(a.spins), host(b.spins))
    assert np.array_equal(host(a.params), host(b.params))
    assert np.array_equal(host(a.mu), host(b.mu))
    assert np.array_equal(host(a.betas), host(b.betas))
    assert np.array_equal(host(a.stats), host(b.stats))
    assert a.counter() == b.counter()
