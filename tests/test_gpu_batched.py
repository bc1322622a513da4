"""Independent instances of uneven L in one call (thc_apply_H_batched): each
output equals the single-instance call (same terms, same reduction tree, same
per-term kernels: float64 to 1e-12) and the oracle; bad input is rejected
before any work."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mps as OM  # noqa: E402
from oracle import thc as OT  # noqa: E402
from paper_2409_12708_gb300.workloads import sector_mps, thc_hamiltonian  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_12708_gb300 import binding
    return binding


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _instances(n_up_dn=((2, 2), (2, 3), (3, 3)), Ls=(4, 5, 6), D=8):
    out = []
    for k, (L, (u, d)) in enumerate(zip(Ls, n_up_dn)):
        t, chi, zeta = thc_hamiltonian(L, L, seed=50 + k)
        psi = sector_mps(L, u, d, D, seed=60 + k)
        out.append((t, chi, zeta, psi))
    return out


@pytest.mark.parametrize("path,tol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_batched_equals_single_instances(B, path, tol):
    D = 8
    inst = _instances(D=D)
    dt = torch.float64 if path == "fp64" else torch.float32
    hams = [(dev(t), dev(c), dev(z)) for t, c, z, _ in inst]
    psis = [[dev(a, dt) for a in p] for *_, p in inst]
    outs = B.thc_apply_H_batched(hams, psis, D_max=D, path=path)
    for h, p, o in zip(hams, psis, outs):
        ref = B.thc_apply_H(*h, p, D_max=D, path=path)
        a = OM.to_dense([x.double().cpu().numpy() for x in o])
        b = OM.to_dense([x.double().cpu().numpy() for x in ref])
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)


def test_batched_matches_oracle(B):
    D = 8
    inst = _instances(D=D)
    outs = B.thc_apply_H_batched([(dev(t), dev(c), dev(z)) for t, c, z, _ in inst],
                                 [[dev(a) for a in p] for *_, p in inst], D_max=D)
    for (t, c, z, p), o in zip(inst, outs):
        ref = OT.apply_H(p, t, c, z, D_max=D)
        a, b = OM.to_dense([x.cpu().numpy() for x in o]), OM.to_dense(ref)
        assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)


def test_batched_rejects_mismatched_instance(B):
    inst = _instances()
    hams = [(dev(t), dev(c), dev(z)) for t, c, z, _ in inst]
    psis = [[dev(a) for a in p] for *_, p in inst]
    hams[1], hams[2] = hams[2], hams[1]  # H of L = 6 with psi of L = 5
    with pytest.raises(B.ThcError) as e:
        B.thc_apply_H_batched(hams, psis, D_max=8)
    assert e.value.status == B.EINVAL
