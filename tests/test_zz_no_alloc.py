"""heat_run_noalloc, the allocation-free stepper, against heat_run.

Callers that cannot allocate device memory (graph capture, real-time loops,
foreign memory pools) use heat_run_noalloc, whose ping-pong buffer is a fixed
device array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2307_01117_gb300 import heat as H
from paper_2307_01117_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_01117_gb300 import build
    build.build()


def reference(u0, nt, k, arith):
    """The existing entry point: a context, heat_set, heat_run, heat_get."""
    with H.Heat(len(u0), 1, k, 1.0, 1.0, form="plain", arith=arith) as h:
        h.set(u0).run(nt)
        return h.get()


@pytest.mark.parametrize("arith", [H.HEAT_ARITH_EXACT, H.HEAT_ARITH_FMA])
def test_two_calls_in_a_row_match_heat_run(arith):
    import torch
    cases = [(100003, 37, 0.3, 1), (1 << 20, 12, 0.25, 2)]   # odd and even step counts, max size second
    stream = torch.cuda.Stream()
    for n, nt, k, seed in cases:
        u0 = workloads.uniform(n, seed, -1, 1)
        d_in = torch.from_numpy(u0).cuda()
        d_out = torch.full_like(d_in, float("nan"))
        torch.cuda.synchronize()
        H.heat_run_noalloc(d_in, d_out, n, k, 1.0, 1.0, nt, arith, stream)
        stream.synchronize()
        got = d_out.cpu().numpy()
        ref = reference(u0, nt, k, arith)
        # same arithmetic, same rounding: the tolerance of these tests is bitwise equality
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), (n, nt)
        assert np.array_equal(d_in.cpu().numpy(), u0)   # the input is only read


def test_zero_steps_copies_and_limits_are_enforced():
    import torch
    n = 4096
    u0 = workloads.uniform(n, 5, -1, 1)
    d_in = torch.from_numpy(u0).cuda()
    d_out = torch.zeros_like(d_in)
    H.heat_run_noalloc(d_in, d_out, n, 0.25, 1.0, 1.0, 0)
    torch.cuda.synchronize()
    assert np.array_equal(d_out.cpu().numpy(), u0)
    big = torch.zeros((1 << 20) + 1, dtype=torch.float64, device="cuda")
    big_out = torch.zeros_like(big)
    with pytest.raises(H.HeatError) as e:
        H.heat_run_noalloc(big, big_out, big.numel(), 0.25, 1.0, 1.0, 3)
    assert e.value.code == H.HEAT_EINVAL
    with pytest.raises(H.HeatError) as e:                      # overlapping input and output
        H.heat_run_noalloc(d_in, d_in, n, 0.25, 1.0, 1.0, 3)
    assert e.value.code == H.HEAT_EINVAL
