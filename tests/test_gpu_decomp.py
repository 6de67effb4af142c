"""Block decomposition (Sec. III-A) on one GPU: 2, 4 and 8 blocks, each its
own context, three ghost layers per shared side exchanged once per RK stage
through device memory, dt from the wave speed reduced over the blocks.

The decomposed FP64 run must equal the serial oracle's undecomposed run bit
for bit (state and time advanced): the full 32^3 x 100-step shock-droplet
run with 2 and 4 blocks, periodic random states split along every dimension
(including two blocks along a periodic dimension, which share both sides),
and single right-hand sides.  The FP32 forms must equal their own
undecomposed runs bit for bit (same kernels, same ghost values)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2409_10729_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_10729_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


_ORACLE = {}


def _oracle_run(key, p, w, steps):
    if key not in _ORACLE:
        _ORACLE[key] = O.run_cfl(p, O.prim_to_cons(p, w), 0.4, steps)
    return _ORACLE[key]


@pytest.mark.parametrize("counts", [(2, 1, 1), (2, 2, 1)], ids=["2 blocks", "4 blocks"])
def test_droplet_run_decomposed_is_the_oracle_run(counts):
    from paper_2409_10729_gb300 import decomp as D
    p, w = I.shock_droplets(32)
    qo, to = _oracle_run("droplets32", p, w, 100)
    s = D.DecomposedSolver(p, counts, "fp64")
    s.set_state_prim(w)
    t = s.step_rk3(0.4, 100)
    q = s.get_state()
    s.close()
    assert np.array_equal(q, qo), "decomposed run differs from the oracle"
    assert t == to


@pytest.mark.parametrize("ndim,n,counts", [(3, [20, 18, 16], (2, 2, 2)), (2, [30, 21], (3, 2)),
                                           (1, [40], (4,)), (3, [18, 12, 15], (1, 3, 2))])
def test_periodic_runs_decomposed_are_the_oracle_runs(ndim, n, counts):
    from paper_2409_10729_gb300 import decomp as D
    p, w = I.random_periodic(ndim, n, seed=17)
    qo, to = O.run_cfl(p, O.prim_to_cons(p, w), 0.4, 8)
    s = D.DecomposedSolver(p, counts, "fp64")
    s.set_state_prim(w)
    t = s.step_rk3(0.4, 8)
    assert np.array_equal(s.get_state(), qo)
    assert t == to
    # the right-hand side of the advanced state, ghosts from the blocks' halos
    assert np.array_equal(s.rhs(), O.rhs(p, qo))
    s.close()


@pytest.mark.parametrize("form", ["fp64_fast", "mixed", "gated"])
def test_fp32_and_fast_forms_decomposed_equal_their_undecomposed_runs(form):
    from paper_2409_10729_gb300 import decomp as D
    from paper_2409_10729_gb300 import mfc
    p, w = I.shock_droplets(32)
    weights = np.load(os.path.join(ROOT, "paper_2409_10729_gb300", "gate_weights.npy")) if form == "gated" else None
    u = mfc.Solver(p, form)
    s = D.DecomposedSolver(p, (2, 2, 1), form)
    if weights is not None:
        u.set_mlp_weights(weights)
        s.set_mlp_weights(weights)
    u.set_state_prim(w)
    s.set_state_prim(w)
    dts_u = [u.step_rk3(0.4, 1) for _ in range(30)]
    dts_s = [s.step_rk3(0.4, 1) for _ in range(30)]
    assert dts_u == dts_s
    assert np.array_equal(s.get_state(), u.get_state())
    u.close()
    s.close()


def test_block_contexts_refuse_whole_step_calls_and_bad_blocks():
    import torch
    from paper_2409_10729_gb300 import mfc
    p, w = I.random_periodic(2, [16, 12], seed=3)
    b = mfc.Solver(p, "fp64", block=([0, 0], [8, 12]))
    b.set_state_prim(np.ascontiguousarray(w[:, :, :, :8]))
    with pytest.raises(mfc.MfcError) as e:
        b.step_rk3(0.4, 1)
    assert e.value.status == mfc.MFC_ESTATE
    with pytest.raises(mfc.MfcError) as e:
        b.rhs()
    assert e.value.status == mfc.MFC_ESTATE
    off, tot, el = b.halo_layout()
    assert el == 8 and off[0] == 0 and off[1] == 6 * 3 * 12 and off[2:] == [-1] * 4 and tot == 2 * 6 * 3 * 12
    b.close()
    for blk in (([0, 0], [2, 12]), ([10, 0], [8, 12]), ([-1, 0], [8, 12])):   # too thin, outside, negative
        with pytest.raises(mfc.MfcError) as e:
            mfc.Solver(p, "fp64", block=blk)
        assert e.value.status == mfc.MFC_EINVAL
    # a block spanning the whole grid has no neighbours and behaves as a plain context
    whole = mfc.Solver(p, "fp64", block=([0, 0], [16, 12]))
    whole.set_state_prim(w)
    assert np.array_equal(whole.rhs(), O.rhs(p, O.prim_to_cons(p, w)))
    assert whole.halo_layout()[1] == 0
    whole.close()
    torch.cuda.synchronize()


def test_nonphysical_block_is_reported():
    from paper_2409_10729_gb300 import decomp as D
    from paper_2409_10729_gb300 import mfc
    p, w = I.random_periodic(2, [16, 12], seed=0)
    bad = w.copy()
    bad[0, 0, 5, 13] = -1.0          # in the second block along x
    bad[1, 0, 5, 13] = 0.0
    s = D.DecomposedSolver(p, (2, 1), "fp64")
    s.set_state_prim(bad)
    with pytest.raises(mfc.MfcError) as e:
        s.step_rk3(0.4, 1)
    assert e.value.status == mfc.MFC_ENONPHYSICAL
    s.close()
