"""Host arrays in and out of a context: page-locked (copied by the SMs through
the device mapping), page-locked but not 16-byte aligned, odd sizes and
pageable memory (cudaMemcpyAsync) all give the same bits."""
import numpy as np
import pytest

from paper_2409_10729_gb300 import inputs as I
from paper_2409_10729_gb300 import mfc

pytestmark = pytest.mark.gpu


def pinned(shape, offset=0):
    import torch
    n = int(np.prod(shape))
    buf = torch.empty(n + offset, dtype=torch.float64).pin_memory().numpy()
    return buf[offset:].reshape(shape)


@pytest.mark.parametrize("ndim,n", [(3, [24, 20, 18]), (2, [5, 3]), (1, [33])])
@pytest.mark.parametrize("offset", [0, 1])
def test_state_round_trip_through_host_buffers(ndim, n, offset):
    import torch
    p, w = I.random_periodic(ndim, n, seed=7)
    s = mfc.Solver(p, "fp64")
    s.set_state_prim(w)
    ref = s.get_state()                       # pageable
    q_in = pinned(s.shape, offset)
    q_in[...] = ref
    s2 = mfc.Solver(p, "fp64")
    s2.set_state(q_in)
    out = pinned(s.shape, offset)
    out[...] = np.nan
    s2.get_state(out)
    torch.cuda.synchronize()
    assert np.array_equal(out, ref)
    assert np.array_equal(s2.get_state(), ref)
    # the RHS into page-locked and pageable host arrays
    L_pin = pinned(s.shape, offset)
    s2.rhs(L_pin)
    L_page = np.empty(s.shape)
    s2.rhs(L_page)
    assert np.array_equal(L_pin, L_page)
    s.close()
    s2.close()


def test_full_size_state_copy_is_exact():
    """A 256^3 droplet state (0.94 GB) through page-locked buffers both ways."""
    p, w = I.shock_droplets(256)
    s = mfc.Solver(p, "fp64")
    s.set_state_prim(w)
    q = pinned(s.shape)
    s.get_state(q)
    rng = np.random.default_rng(3)
    idx = tuple(rng.integers(0, m, 4096) for m in q.shape)
    probe = q[idx].copy()
    s.set_state(q)
    back = pinned(s.shape)
    back[...] = 0.0
    s.get_state(back)
    assert np.array_equal(back[idx], probe)
    assert np.array_equal(back, q)
    s.close()
