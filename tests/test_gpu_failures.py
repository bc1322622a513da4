"""Failure detection through the C ABI, injected on the host (no GPU fault):
an allocator that returns NULL part-way through a call, and non-finite values
in the inputs.  Both must come back as status codes with the context intact,
so the next call on the same device still works."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2409_12708_gb300.workloads import sector_mps, thc_hamiltonian  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_12708_gb300 import binding
    return binding


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _problem():
    L, N, D = 5, 3, 8
    t, chi, zeta = thc_hamiltonian(L, N, seed=21)
    psi = sector_mps(L, 2, 3, D, seed=22)
    return t, chi, zeta, psi, D


@pytest.mark.parametrize("fail_after", [0, 3, 12, 40])
def test_allocator_returning_null_gives_enomem_and_writes_nothing(B, fail_after):
    t, chi, zeta, psi, D = _problem()
    live = {}
    calls = [0]

    def alloc(size, stream):
        calls[0] += 1
        if calls[0] > fail_after:
            return None
        p = torch.cuda.caching_allocator_alloc(size, stream=int(stream or 0))
        live[p] = size
        return p

    def free(ptr, stream):
        live.pop(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    al = B.make_allocator(alloc, free)
    args = (dev(t), dev(chi), dev(zeta), [dev(a) for a in psi])
    with pytest.raises(B.ThcError) as e:
        B.thc_apply_H(*args, D_max=D, term_begin=0, term_end=20, allocator=al)
    assert e.value.status == B.ENOMEM
    assert not e.value.out_owner  # no output block was handed out
    torch.cuda.synchronize()
    assert live == {}  # every block obtained before the failure was released
    # the context is intact: a normal call right after works
    out = B.thc_apply_H(*args, D_max=D, term_begin=0, term_end=20)
    assert all(torch.isfinite(x).all() for x in out)


@pytest.mark.parametrize("where", ["chi", "psi"])
@pytest.mark.parametrize("path", ["fp64", "fp32"])
def test_nonfinite_input_gives_enonfinite(B, where, path):
    t, chi, zeta, psi, D = _problem()
    chi = chi.copy()
    psi = [a.copy() for a in psi]
    if where == "chi":
        chi[2, 1] = np.nan
    else:
        psi[2][0, 1, 0] = np.inf
    dt = torch.float64 if path == "fp64" else torch.float32
    with pytest.raises(B.ThcError) as e:
        B.thc_apply_H(dev(t), dev(chi), dev(zeta), [dev(a, dt) for a in psi], D_max=D, path=path)
    assert e.value.status == B.ENONFINITE
    t, chi, zeta, psi, D = _problem()
    out = B.thc_apply_H(dev(t), dev(chi), dev(zeta), [dev(a, dt) for a in psi], D_max=D, path=path)
    assert all(torch.isfinite(x).all() for x in out)
