"""Host-side checks of the density-control wrapper (CPU, no CUDA call): the
argument validation that runs before any library call."""
import types

import pytest

torch = pytest.importorskip("torch")

from paper_2503_06161_gb300 import density  # noqa: E402


def _params(P):
    return dict(means=torch.zeros(P, 3), log_scales=torch.zeros(P, 3), quats=torch.zeros(P, 4),
                opacity_logits=torch.zeros(P))


def test_densify_rejects_malformed_streams():
    P = 5
    st = density.DensityStats(P, "cpu")
    normals = torch.zeros(P, 2, 3)
    p = _params(P)
    del p["quats"]
    with pytest.raises(ValueError, match="quats"):
        density.densify(p, {}, st, normals, 2e-4, 0.01, 0.005)
    p = _params(P)
    p["feat"] = torch.zeros(P + 1, 8)                      # wrong row count
    with pytest.raises(ValueError, match="feat"):
        density.densify(p, {}, st, normals, 2e-4, 0.01, 0.005)
    p = _params(P)
    with pytest.raises(ValueError, match="m"):
        density.densify(p, {"m": torch.zeros(8, P).t()}, st, normals, 2e-4, 0.01, 0.005)   # not contiguous
    with pytest.raises(ValueError, match="normals"):
        density.densify(_params(P), {}, st, torch.zeros(P, 3), 2e-4, 0.01, 0.005)
    with pytest.raises(ValueError, match="normals"):
        density.densify(_params(P), {}, st, torch.zeros(P, 2, 3, dtype=torch.float64), 2e-4, 0.01, 0.005)


def test_statistics_follow_the_gaussian_count():
    st = density.DensityStats(4, "cpu")
    st.accum += 1.0
    st.count += 2
    st.reset()
    assert st.accum.sum().item() == 0.0 and st.count.sum().item() == 0
    st.reset(7)
    assert st.P == 7 and st.count.dtype == torch.int32
    with pytest.raises(ValueError, match="disagree"):
        st.record(types.SimpleNamespace(P=6))
