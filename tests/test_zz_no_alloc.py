"""heat_run_noalloc, the allocation-free stepper, against the oracle and heat_run.

Some callers cannot allocate device memory: code recorded into a CUDA graph,
real-time loops kept off the allocator, and hosts whose device memory belongs
to another framework's pool.  heat_run_noalloc serves them: the caller passes
input and output, and the ping-pong buffer of a multi-step run is a fixed
device array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_2307_01117_gb300 import heat as H
from paper_2307_01117_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_01117_gb300 import build
    build.build()


def same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint64), np.asarray(b).view(np.uint64))


def with_heat_run(u0, nt, k, dt, dx, arith):
    """The existing entry point: a context, heat_set, heat_run, heat_get."""
    with H.Heat(len(u0), 1, k, dt, dx, form="plain", arith=arith) as h:
        h.set(u0).run(nt)
        return h.get()


@pytest.mark.parametrize("arith", [H.HEAT_ARITH_EXACT, H.HEAT_ARITH_FMA])
def test_two_calls_in_a_row_match_the_oracle_and_heat_run(arith):
    import torch
    # odd and even step counts, dt, dx != 1 in one case, the maximum size last
    cases = [(100003, 37, (0.3, 1.0, 1.0), 1), (30001, 11, (0.44845565991743563, 0.6130994749175215, 1.3), 3),
             (1 << 20, 12, (0.25, 1.0, 1.0), 2)]
    stream = torch.cuda.Stream()
    for n, nt, (k, dt, dx), seed in cases:
        u0 = workloads.uniform(n, seed, -1, 1)
        d_in = torch.from_numpy(u0).cuda()
        d_out = torch.full_like(d_in, float("nan"))
        torch.cuda.synchronize()
        H.heat_run_noalloc(d_in, d_out, n, k, dt, dx, nt, arith, stream)
        stream.synchronize()
        got = d_out.cpu().numpy()
        # same arithmetic, same rounding: the tolerance of these tests is bitwise equality
        want = oracle.run(u0, oracle.coef(k, dt, dx), nt, fma=arith == H.HEAT_ARITH_FMA)
        assert same_bits(got, want), (n, nt)
        assert same_bits(got, with_heat_run(u0, nt, k, dt, dx, arith)), (n, nt)
        assert np.array_equal(d_in.cpu().numpy(), u0)   # the input is only read


def test_calls_allocate_no_device_memory():
    """After the first call on the device, calls in either reading change
    neither the free device memory nor torch's allocated bytes."""
    import torch
    n = 50000
    u0 = workloads.uniform(n, 6, -1, 1)
    d_in = torch.from_numpy(u0).cuda()
    d_out = torch.empty_like(d_in)
    H.heat_run_noalloc(d_in, d_out, n, 0.3, 1.0, 1.0, 3)
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for arith in (H.HEAT_ARITH_FMA, H.HEAT_ARITH_EXACT):
        H.heat_run_noalloc(d_in, d_out, n, 0.3, 1.0, 1.0, 5, arith)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert same_bits(d_out.cpu().numpy(), oracle.run(u0, 0.3, 5))


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
