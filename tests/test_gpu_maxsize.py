"""The largest supported shapes (D_max = 512): a layer on an L = 10 state whose
middle bond is 512 expands it to 1024, so the QR sweep factors a 2048 x 1024
matrix (narrow panels to fit shared memory) and the SVD sweep runs the
one-sided Jacobi on a 1024 x 1024 factor (32 columns per lane), with the rows
beyond shared memory in global memory.  Against the oracle's layer at the same
D_max: float64 1e-9; float32 1e-4 (truncation of a 1024-dimensional bond to
512 with Schmidt values decaying as exp(-k/8): the float32 rounding of the
inputs and of the kept vectors, amplified by the gaps at the cut).  A D_max
above 512 is refused before any work."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mps as OM  # noqa: E402
from oracle import thc as OT  # noqa: E402
from paper_2409_12708_gb300.workloads import sector_mps  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_12708_gb300 import binding
    return binding


DT = {"fp64": torch.float64, "fp32": torch.float32}


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


@pytest.fixture(scope="module")
def case():
    L, D = 10, 512
    psi = sector_mps(L, 5, 5, D, seed=70, decay=8.0)
    coef = np.random.default_rng(71).standard_normal(L)
    ref = OT.apply_layer(psi, coef, 0, False, D, 0.0)
    return psi, coef, ref, D


@pytest.mark.parametrize("path,tolr", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_layer_at_max_bond_matches_oracle(B, case, path, tolr):
    psi, coef, ref, D = case
    assert max(a.shape[2] for a in psi) == D
    B.profile_read()  # clears the counters
    out = B.thc_layer_apply([dev(a, DT[path]) for a in psi], dev(coef), 0, 0, D_max=D, path=path)
    # every Jacobi converged within its sweep budget (an exhausted budget is
    # counted, not raised: here it would mean unorthogonal kept rows)
    assert "jacobi_budget_exhausted" not in B.profile_read()
    assert [tuple(x.shape) for x in out] == [a.shape for a in ref]
    got = OM.to_dense([x.detach().cpu().double().numpy() for x in out])
    want = OM.to_dense(ref)
    assert np.linalg.norm(got - want) <= tolr * np.linalg.norm(want)


def test_bond_above_max_is_refused(B, case):
    psi, coef, _, _ = case
    with pytest.raises(B.ThcError) as e:
        B.thc_layer_apply([dev(a) for a in psi], dev(coef), 0, 0, D_max=513)
    assert e.value.status == B.EUNSUPPORTED
