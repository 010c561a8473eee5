"""GPU parity: every kernel form against the CPU oracle, element by element,
through the C ABI (binding in paper_2307_01117_gb300.heat).

Bar: bitwise equality for binary64 with the exact reading of Eq. 2 and for the
fused reading against the oracle's fused reading; the fused reading is also
within 1e-12 * max|u0| of the exact one; binary32-compensated state bitwise
against the oracle's compensated form with the same block length.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2307_01117_gb300 import heat as H
from paper_2307_01117_gb300 import workloads

pytestmark = pytest.mark.gpu

FORMS_F64 = [("plain", 0), ("persist", 0), ("persist", 1), ("persist", 5), ("persist", 64), ("tblock", 1), ("tblock", 4), ("tblock", 7), ("tblock", 64),
             ("persist_tb", 1), ("persist_tb", 4), ("persist_tb", 13)]
FORMS_F32C = [("plain", 0), ("persist", 0), ("persist", 1), ("persist", 13), ("tblock", 1), ("tblock", 8), ("tblock", 13), ("tblock", 64),
              ("persist_tb", 8), ("persist_tb", 32)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_01117_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def run_gpu(u0, np_, r, nt, form="plain", T=0, dtype="f64", arith=H.HEAT_ARITH_EXACT, chunks=None):
    n = len(u0)
    assert n % np_ == 0
    with H.Heat(n // np_, np_, r, 1.0, 1.0, dtype=dtype, form=form, T=T, arith=arith) as h:
        h.set(u0)
        for c in (chunks or [nt]):
            h.run(c)
        out = h.get()
        assert h.steps == nt
    return out


def same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint64), np.asarray(b).view(np.uint64))


SIZES = [(1, 1), (2, 1), (3, 1), (5, 1), (7, 1), (64, 1), (65, 1), (127, 1), (128, 1), (129, 1),
         (1000, 4), (4000, 4), (65537, 1), (3 * (7 * 1024 + 5), 3), (16 * 4099, 16)]


@pytest.mark.parametrize("form,T", FORMS_F64)
@pytest.mark.parametrize("n,np_", SIZES)
def test_f64_exact_bitwise(form, T, n, np_):
    u0 = workloads.uniform(n, 1000 + n, -1, 1)
    for nt, r in [(0, 0.25), (1, 0.5), (2, 0.37), (17, 0.25), (64, 0.5)]:
        ref = oracle.run(u0, r, nt)
        got = run_gpu(u0, np_, r, nt, form, T)
        assert same_bits(got, ref), (n, np_, nt, r, int(np.sum(got != ref)))


@pytest.mark.parametrize("form,T", FORMS_F64 + [("cluster", 0), ("tblock", 0)])
@pytest.mark.parametrize("r", [0.5, 0.25, -0.25])
def test_f64_power_of_two_r_with_out_of_domain_values(form, T, r):
    """r = +-2^k: tiles, groups or windows whose values pass the integer-pipe
    screen move the product's exponent on the integer pipes; the ones holding
    +0 next to -0, subnormals or tiny values take the plain FP64 update."""
    n = 4 * 4096 + 64                     # within the cluster form's limit
    u0 = workloads.uniform(n, 4242, -1, 1)
    u0[64:200] = 0.0
    u0[1000] = -0.0
    u0[5000:5008] = 4e-310
    u0[9000:9050] = 1e-290
    u0[12000:12003] = 1e300
    for nt in (1, 19):
        ref = oracle.run(u0, r, nt)
        assert same_bits(run_gpu(u0, 4, r, nt, form, T), ref), (form, T, nt)


@pytest.mark.parametrize("form,T", FORMS_F64)
def test_paper_config_small_ring(form, T):
    """np=4 x nx=1000, nt=100, k=0.5, dt=dx=1, u[g]=g (Section 2's initial condition)."""
    u0 = workloads.ramp(4000)
    r = oracle.coef(0.5, 1.0, 1.0)
    ref = oracle.run(u0, r, 100)
    with H.Heat(1000, 4, 0.5, 1.0, 1.0, form=form, T=T) as h:
        h.set(u0).run(100)
        got = h.get()
        assert h.sum() == 7998000.0
    assert same_bits(got, ref)


@pytest.mark.parametrize("form,T", FORMS_F64)
@pytest.mark.parametrize("n", [5, 64, 4000, 100003])
def test_f64_fma_form(form, T, n):
    u0 = workloads.uniform(n, 77, -3, 3)
    r, nt = 0.4, 50
    got = run_gpu(u0, 1, r, nt, form, T, arith=H.HEAT_ARITH_FMA)
    assert same_bits(got, oracle.run(u0, r, nt, fma=True))
    exact = oracle.run(u0, r, nt)
    assert np.max(np.abs(got - exact)) <= 1e-12 * np.max(np.abs(u0))


@pytest.mark.parametrize("form,T", FORMS_F32C)
@pytest.mark.parametrize("n", [1, 3, 128, 129, 4000, 100003])
def test_f32c_bitwise(form, T, n):
    u0 = workloads.uniform(n, 5 + n, -1, 1)
    u32 = u0.astype(np.float32)
    for nt, r in [(1, 0.5), (13, 0.3), (40, 0.25)]:
        with H.Heat(n, 1, r, 1.0, 1.0, dtype="f32c", form=form, T=T) as h:
            got = h.set(u0).run(nt).get()
            last_T = H.heat_last_run(h.ctx)["T"]
        Tb = T if form in ("tblock", "persist_tb") else 1
        if form == "persist":   # depth T (library default 32), or 1 on rings shorter than T
            assert last_T in (1, T or 32), last_T
            Tb = last_T
        ref = oracle.run_f32c(u32, np.float32(r), nt, max(Tb, 1)).astype(np.float64)
        assert np.array_equal(got, ref), (n, nt, r)


def test_restart_invariance():
    u0 = workloads.uniform(10007, 3, -1, 1)
    a = run_gpu(u0, 1, 0.3, 30, chunks=[7, 0, 13, 10])
    b = run_gpu(u0, 1, 0.3, 30)
    assert same_bits(a, b)


def test_sum_is_conserved_and_close_to_exact():
    n = 1 << 20
    u0 = workloads.uniform(n, 9, -1, 1)
    with H.Heat(n // 4, 4, 0.25, 1.0, 1.0) as h:
        h.set(u0)
        s0 = h.sum()
        assert abs(s0 - math.fsum(u0)) <= n * 1.2e-16 * np.sum(np.abs(u0))
        h.run(100)
        s1 = h.sum()
        u = h.get()
    assert abs(s1 - math.fsum(u)) <= n * 1.2e-16 * np.sum(np.abs(u))
    assert abs(s1 - s0) <= 4 * 100 * n * 2.2e-16


def test_sum_is_deterministic():
    n = 3 * 10**6 + 7
    u0 = workloads.uniform(n, 10, -1, 1)
    with H.Heat(n, 1, 0.25, 1.0, 1.0) as h:
        h.set(u0)
        vals = {h.sum() for _ in range(5)}
    assert len(vals) == 1


def test_device_transfers_match_host():
    import torch
    n = 12345
    u0 = workloads.uniform(n, 4, -1, 1)
    t = torch.from_numpy(u0).cuda()
    out = torch.empty_like(t)
    for dtype in ("f64", "f32c"):
        with H.Heat(n, 1, 0.25, 1.0, 1.0, dtype=dtype) as h:
            H.heat_set_device(h.ctx, t)
            h.run(5)
            H.heat_get_device(h.ctx, out)
            torch.cuda.synchronize()
            host = h.get()
        assert np.array_equal(out.cpu().numpy(), host)


def test_torch_stream_ordering():
    import torch
    n = 1 << 16
    u0 = workloads.uniform(n, 6, -1, 1)
    s = torch.cuda.Stream()
    with H.Heat(n, 1, 0.3, 1.0, 1.0, stream=s) as h:
        h.set(u0).run(20)
        got = h.get()
    assert same_bits(got, oracle.run(u0, 0.3, 20))


def test_argument_errors():
    with H.Heat(100, 2, 0.25, 1.0, 1.0) as h:
        with pytest.raises(H.HeatError) as e:
            H.heat_set(h.ctx, np.zeros(199))
        assert e.value.code == H.HEAT_EINVAL
        with pytest.raises(H.HeatError) as e:
            H.heat_run(h.ctx, -1)
        assert e.value.code == H.HEAT_EINVAL
        with pytest.raises(H.HeatError):
            H.heat_set_form(h.ctx, 9, 0)
        with pytest.raises(H.HeatError):
            H.heat_set_form(h.ctx, 2, 65)
        with pytest.raises(H.HeatError):
            H.heat_set_arith(h.ctx, 5)
        H.heat_run(h.ctx, 0)
        assert h.steps == 0


@pytest.mark.parametrize("T", [2, 5, 16])
def test_tblock_restart_matches_one_run_f64(T):
    """Binary64: any split of the steps into runs and blocks gives the same bits."""
    u0 = workloads.uniform(70001, 12, -1, 1)
    a = run_gpu(u0, 1, 0.45, 50, "tblock", T, chunks=[11, 39])
    b = run_gpu(u0, 1, 0.45, 50, "plain", 0)
    assert same_bits(a, b)


def test_tblock_default_depth_runs():
    u0 = workloads.uniform(5000, 2, -1, 1)
    with H.Heat(5000, 1, 0.3, 1.0, 1.0, form="tblock") as h:
        h.set(u0).run(9)
        got = h.get()
        info = H.heat_last_run(h.ctx)
    assert info["form"] == "tblock" and info["T"] >= 1
    assert same_bits(got, oracle.run(u0, 0.3, 9))


def test_tblock_rejects_depth_beyond_window():
    with H.Heat(1000, 1, 0.3, 1.0, 1.0, form="tblock", T=64) as h:
        h.set(np.zeros(1000)).run(3)           # 2T < window: fine
        with pytest.raises(H.HeatError) as e:
            H.heat_set_form(h.ctx, 2, 65)         # beyond the library's maximum depth
        assert e.value.code == H.HEAT_EINVAL


@pytest.mark.parametrize("dtype,T", [("f64", 1), ("f64", 4), ("f64", 9), ("f64", 64), ("f32c", 1), ("f32c", 16),
                                     ("f32c", 33)])
@pytest.mark.parametrize("n", [1, 5, 511, 513, 1024, 4000, 70001])
def test_contiguous_layout_bitwise(dtype, T, n):
    u0 = workloads.uniform(n, 60 + n, -1, 1)
    nt = 2 * T + 3
    with H.Heat(n, 1, 0.3, 1.0, 1.0, dtype=dtype, form="tblock", T=T) as h:
        H.heat_set_layout(h.ctx, 1)
        h.set(u0).run(nt)
        got = h.get()
    if dtype == "f64":
        ref = oracle.run(u0, 0.3, nt)
        assert same_bits(got, ref)
    else:
        ref = oracle.run_f32c(u0.astype(np.float32), np.float32(0.3), nt, T).astype(np.float64)
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("form,T", [("plain", 0), ("tblock", 4), ("tblock", 0)])
def test_graph_replay_matches_direct_launches(form, T):
    """The second identical run replays the captured CUDA graph."""
    u0 = workloads.uniform(50000, 8, -1, 1)
    ref = oracle.run(u0, 0.3, 33)
    with H.Heat(50000, 1, 0.3, 1.0, 1.0, form=form, T=T) as h:
        outs = []
        for _ in range(3):
            h.set(u0).run(33)
            outs.append(h.get())
        H.heat_set_graphs(h.ctx, False)
        h.set(u0).run(33)
        outs.append(h.get())
    for o in outs:
        assert same_bits(o, ref)


@pytest.mark.parametrize("form", ["tblock", "cluster", "persist"])
def test_checkpoint_and_resume_in_a_new_context(form):
    """heat_get + the step counter is a checkpoint; heat_set in a fresh context
    resumes it (binary64 runs are split-invariant, so the result is bitwise the
    uninterrupted run)."""
    n = 6000
    u0 = workloads.uniform(n, 77, -1, 1)
    with H.Heat(n // 4, 4, 0.4, 1.0, 1.0, form=form) as h:
        h.set(u0).run(13)
        saved, steps = h.get(), h.steps
    assert steps == 13
    with H.Heat(n // 4, 4, 0.4, 1.0, 1.0, form=form) as h2:
        h2.set(saved).run(30 - steps)
        resumed = h2.get()
    assert same_bits(resumed, oracle.run(u0, 0.4, 30))
