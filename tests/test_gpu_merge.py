"""The spin-merged term list through the C ABI (thc_opts.merge_spin): the
merged H|psi> against the dense Eq. 1 operator (untruncated) and against the
oracle's merged list (truncated, term ranges across the block boundaries,
batching), the float32 paths, and a Lanczos run.  Tolerances as for the
unmerged list (float64 1e-10 dense / 1e-9 truncated; float32 untruncated 2e-6)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fock as F  # noqa: E402
from oracle import krylov as OK  # noqa: E402
from oracle import mps as OM  # noqa: E402
from oracle import thc as OT  # noqa: E402
from paper_2409_12708_gb300.workloads import sector_mps, thc_hamiltonian, workload  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_12708_gb300 import binding
    return binding


DT = {"fp64": torch.float64, "fp32": torch.float32, "tf32": torch.float32}


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def to_np(sites):
    return [s.detach().cpu().double().numpy() for s in sites]


def dense_rel(a, b):
    va, vb = OM.to_dense(a), OM.to_dense(b)
    return np.linalg.norm(va - vb) / max(np.linalg.norm(vb), 1e-300)


@pytest.mark.parametrize("path,tolr", [("fp64", 1e-10), ("fp32", 2e-6), ("tf32", 2e-6)])
def test_merged_untruncated_equals_dense(B, path, tolr):
    L, N = 4, 3
    t, chi, zeta = thc_hamiltonian(L, N, seed=31)
    psi = sector_mps(L, 2, 2, 16, seed=32)
    out = B.thc_apply_H(dev(t), dev(chi), dev(zeta), [dev(a, DT[path]) for a in psi], D_max=256, path=path,
                        merge_spin=True)
    ref = F.hamiltonian_eq1(t, F.thc_v(chi, zeta)) @ OM.to_dense(psi)
    got = OM.to_dense(to_np(out))
    assert np.linalg.norm(got - ref) <= tolr * np.linalg.norm(ref)


@pytest.mark.parametrize("batch", [1, 7, 0])
def test_merged_term_ranges_match_oracle(B, batch):
    # N^2 = 9: ranges inside the up blocks, across the up/down boundary, and into
    # the kinetic terms (3N^2 = 27 Coulomb terms, then 2L = 10 kinetic)
    L, N, D = 5, 3, 8
    t, chi, zeta = thc_hamiltonian(L, N, seed=33)
    psi = sector_mps(L, 2, 3, D, seed=34)
    for t0, t1 in [(0, 4), (5, 20), (25, 37), (0, 37)]:
        out = B.thc_apply_H(dev(t), dev(chi), dev(zeta), [dev(a) for a in psi], D_max=D, term_begin=t0,
                            term_end=t1, batch=batch, merge_spin=True)
        ref = OT.apply_H(psi, t, chi, zeta, D_max=D, term_begin=t0, term_end=t1, merge_spin=True)
        assert dense_rel(to_np(out), ref) < 1e-9


def test_merged_truncated_workload_matches_oracle(B):
    t, chi, zeta, psi, D = workload("L6_N12_D16")
    out = B.thc_apply_H(dev(t), dev(chi), dev(zeta), [dev(a) for a in psi], D_max=D, merge_spin=True)
    ref = OT.apply_H(psi, t, chi, zeta, D_max=D, merge_spin=True)
    assert dense_rel(to_np(out), ref) < 1e-9


def test_merged_lanczos_untruncated_equals_unmerged(B):
    L, N, K = 4, 3, 6
    t, chi, zeta = thc_hamiltonian(L, N, seed=35)
    psi = sector_mps(L, 2, 2, 16, seed=36)
    args = (dev(t), dev(chi), dev(zeta))
    e0, _, _ = B.krylov_lanczos_ground(*args, [dev(a) for a in psi], K, D_max=256)
    e1, _, _ = B.krylov_lanczos_ground(*args, [dev(a) for a in psi], K, D_max=256, merge_spin=True)
    Hop = lambda x: OT.apply_H(x, t, chi, zeta, D_max=256, merge_spin=True)
    e_ref, _, _ = OK.lanczos_ground(Hop, psi, K, 256)
    assert abs(e0 - e1) < 1e-9 and abs(e1 - e_ref[0]) < 1e-8
