"""Restarted Lanczos and excited states through the C ABI (Sec. 2.2), against
the oracle's lanczos_restarted (same restarts, same Gram-Schmidt sums) and the
exact levels of the sector: float64 path, energies within 1e-8 of the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fock as F  # noqa: E402
from oracle import krylov as OK  # noqa: E402
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


def mps_from_dense(vec, L):
    """Exact MPS of a dense 4^L vector by successive SVDs (test input only)."""
    sites, rest, left = [], vec.reshape(1, -1), 1
    for _ in range(L - 1):
        u, s, vh = np.linalg.svd(rest.reshape(left * 4, -1), full_matrices=False)
        k = int(np.sum(s > 1e-14 * s[0]))
        sites.append(u[:, :k].reshape(left, 4, k))
        rest, left = s[:k, None] * vh[:k], k
    sites.append(rest.reshape(left, 4, 1))
    return sites


def test_restarted_lanczos_untruncated_matches_oracle_and_ED(B):
    L = 4
    t, chi, zeta = thc_hamiltonian(L, 3, seed=40)
    psi = sector_mps(L, 2, 2, 256, seed=41)
    e, x = B.krylov_lanczos_restarted(dev(t), dev(chi), dev(zeta), [dev(a) for a in psi], 4, 8, D_max=256,
                                      want_state=True)
    ref, xr = OK.lanczos_restarted(lambda v: OT.apply_H(v, t, chi, zeta, D_max=256), psi, 4, 8, D_max=256)
    assert np.allclose(e, ref, atol=1e-8)
    H = F.hamiltonian_eq1(t, F.thc_v(chi, zeta))
    assert abs(e[-1] - F.ground_energy(H, L, 2, 2)) < 1e-6
    g = OM.to_dense([a.cpu().numpy() for a in x])
    assert abs(np.linalg.norm(g) - 1.0) < 1e-12
    assert abs(abs(np.vdot(g, OM.to_dense(xr))) - 1.0) < 1e-8


def test_excited_state_matches_oracle_and_first_excited_level(B):
    L = 4
    t, chi, zeta = thc_hamiltonian(L, 3, seed=41)
    H = F.hamiltonian_eq1(t, F.thc_v(chi, zeta))
    s = F.sector(L, 2, 2)
    E, Y = np.linalg.eigh(H[s][:, s].toarray())
    gvec = np.zeros(4 ** L)
    gvec[s] = Y[:, 0]
    ground = mps_from_dense(gvec, L)
    # the lower state's bonds padded up to the static profile of D_max = 256
    from paper_2409_12708_gb300.workloads import full_bond_profile
    ground_p = OM.pad_to_profile(ground, full_bond_profile(L, 256))
    psi = sector_mps(L, 2, 2, 256, seed=43)
    e, x = B.krylov_lanczos_restarted(dev(t), dev(chi), dev(zeta), [dev(a) for a in psi], 12, 2, D_max=256,
                                      lower=[[dev(a) for a in ground_p]], want_state=True)
    ref, _ = OK.lanczos_restarted(lambda v: OT.apply_H(v, t, chi, zeta, D_max=256), psi, 12, 2, D_max=256,
                                  lower=[ground])
    assert np.allclose(e, ref, atol=1e-8)
    assert abs(e[-1] - E[1]) < 1e-6
    assert abs(np.vdot(gvec, OM.to_dense([a.cpu().numpy() for a in x]))) < 1e-9


def test_restarted_lanczos_tolerance_truncated_matches_oracle(B):
    # discarded-weight truncation (tol = 1e-4) at L = 6, N = 6, D_max = 64: the
    # restarts also compress the Ritz vector with the same rule
    L, N, D, K, tol = 6, 6, 64, 5, 1e-4
    t, chi, zeta = thc_hamiltonian(L, N, seed=0)
    psi = sector_mps(L, 3, 3, 16, seed=1000)
    e, _ = B.krylov_lanczos_restarted(dev(t), dev(chi), dev(zeta), [dev(a) for a in psi], K, 3, D_max=D, tol=tol)
    ref, _ = OK.lanczos_restarted(lambda v: OT.apply_H(v, t, chi, zeta, D_max=D, tol=tol), psi, K, 3, D, tol)
    assert np.allclose(e, ref, atol=1e-8)
    assert np.all(np.diff(e) < 1e-8)


def test_restarted_rejects_bad_lower_states(B):
    L = 4
    t, chi, zeta = thc_hamiltonian(L, 3, seed=40)
    psi = [dev(a) for a in sector_mps(L, 2, 2, 16, seed=41)]
    other = [dev(a, torch.float32) for a in sector_mps(L, 2, 2, 16, seed=42)]
    with pytest.raises(B.ThcError) as e:
        B.krylov_lanczos_restarted(dev(t), dev(chi), dev(zeta), psi, 4, 2, D_max=16, lower=[other])
    assert e.value.status == B.EINVAL
    with pytest.raises(B.ThcError) as e:
        B.krylov_lanczos_restarted(dev(t), dev(chi), dev(zeta), psi, 4, 0, D_max=16)
    assert e.value.status == B.EINVAL
