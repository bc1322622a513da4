"""mps_inner_noalloc: the inner product for callers that cannot allocate GPU
memory (its scratch is a fixed 16 MiB device array inside the library).

It must agree with mps_inner, the allocating entry point, within the inner-
product tolerances of the parity tests (float64: 1e-13, float32: 1e-6, both
relative to |phi||psi|), on two calls in a row (the shared scratch keeps the
previous call's contents), and reject inputs larger than its scratch.  The
file name makes pytest collect it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mps as OM  # noqa: E402
from paper_2409_12708_gb300.workloads import random_mps, sector_mps  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_12708_gb300 import binding
    return binding


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 1e-6)])
def test_noalloc_matches_allocating_inner_twice(B, dtype, tol):
    L, D = 16, 128
    a = sector_mps(L, 8, 8, D, seed=5, decay=12.0)
    b = sector_mps(L, 8, 8, D, seed=6, decay=12.0)
    c = random_mps(L, 32, seed=7)
    pa, pb, pc = ([dev(x, dtype) for x in m] for m in (a, b, c))
    scale_ab = OM.norm(a) * OM.norm(b)
    scale_ac = OM.norm(a) * OM.norm(c)
    for _ in range(2):  # two calls in a row share the scratch array
        ref = B.mps_inner(pa, pb)
        got = B.mps_inner_noalloc(pa, pb)
        assert abs(got - ref) <= tol * scale_ab
        ref2 = B.mps_inner(pa, pc)
        got2 = B.mps_inner_noalloc(pa, pc)
        assert abs(got2 - ref2) <= tol * scale_ac
    # and both agree with the oracle's float64 contraction
    assert abs(B.mps_inner_noalloc(pa, pb) - OM.inner(a, b)) <= max(tol, 1e-12) * 10 * scale_ab


def test_noalloc_rejects_inputs_beyond_its_scratch(B):
    # bond 700 on both sides: 5 * 700 * 700 float64 > 16 MiB
    big = [torch.ones(1, 4, 700, dtype=torch.float64, device="cuda"),
           torch.ones(700, 4, 1, dtype=torch.float64, device="cuda")]
    with pytest.raises(B.ThcError) as e:
        B.mps_inner_noalloc(big, big)
    assert e.value.status == B.EINVAL
    assert "scratch" in str(e.value)
    # a supported call right after the rejection still works
    small = [dev(x, torch.float64) for x in random_mps(6, 8, seed=1)]
    assert abs(B.mps_inner_noalloc(small, small) - B.mps_inner(small, small)) < 1e-10 * B.mps_inner(small, small)


def test_noalloc_refuses_a_capturing_stream(B):
    # it reads its result back and synchronises, which a stream under capture
    # cannot do: the call is refused before anything is enqueued, and the
    # capture around it stays valid
    small = [dev(x, torch.float64) for x in random_mps(6, 8, seed=1)]
    ref = B.mps_inner(small, small)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    x = torch.zeros(4, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            x.add_(1.0)
            with pytest.raises(B.ThcError) as e:
                B.mps_inner_noalloc(small, small)
    assert e.value.status == B.EUNSUPPORTED
    g.replay()
    torch.cuda.synchronize()
    assert float(x.sum()) == 4.0
    assert abs(B.mps_inner_noalloc(small, small) - ref) < 1e-10 * ref


def test_noalloc_accepts_the_inputs_mps_inner_accepts(B):
    one_site = [torch.ones(1, 4, 1, dtype=torch.float64, device="cuda")]
    for f in (B.mps_inner, B.mps_inner_noalloc):
        with pytest.raises(B.ThcError) as e:
            f(one_site, one_site)  # L = 1 is rejected by both
        assert e.value.status == B.EINVAL
