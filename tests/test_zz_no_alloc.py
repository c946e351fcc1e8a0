"""GPU test of ks_overlap_noalloc, the entry point for callers that cannot allocate device
memory (for example code whose device memory belongs to its own pool allocator).  Its
output must equal the Gram matrix the existing ks_orthonormalize entry point reports for the
same states, on two calls in a row (the second call reuses the library's fixed scratch).
Collected last so that a stop-at-first-failure run has already run every other test."""
import numpy as np
import pytest

from paper_2106_03872_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ks():
    from paper_2106_03872_gb300 import ks as mod
    mod.load()
    assert torch.cuda.is_available()
    return mod


TOL = {"fp64": 1e-12, "bf16x3": 2e-5}
DT = {"fp64": torch.complex128, "bf16x3": torch.complex64}


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("shape", [(10.0, 24, 9), (15.0, 48, 40)])
def test_overlap_noalloc_matches_orthonormalize(ks, prec, shape):
    L, N, ns = shape
    cell = inputs.small_cell(L, N, 3, ns, 31)
    g = ks.Grid(cell, prec=prec)
    c = inputs.random_coeffs(31, ns, g.nG)
    g.set_states(c)
    S_ref = g.orthonormalize(want_S=True)           # the existing entry point's Gram matrix
    g.close()
    a = torch.from_numpy(c).to("cuda", DT[prec])     # same rounding as ks_set_states
    for _ in range(2):
        out = torch.full((ns, ns), float("nan"), dtype=torch.complex128, device="cuda")
        ks.overlap_noalloc(a.data_ptr(), a.data_ptr(), ns, ns, a.shape[1], prec == "fp64", out.data_ptr())
        torch.cuda.synchronize()
        S = out.cpu().numpy()
        assert np.max(np.abs(S - S_ref)) <= TOL[prec] * np.max(np.abs(S_ref))


def test_overlap_noalloc_rejects_sizes_beyond_scratch(ks):
    a = torch.zeros((4, 8), dtype=torch.complex128, device="cuda")
    out = torch.zeros((4, 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(ks.KsError) as e:
        ks.overlap_noalloc(a.data_ptr(), a.data_ptr(), 513, 513, 8, True, out.data_ptr())
    assert e.value.status == ks.KS_ERR_ARG
    assert b"exceeds the scratch maximum" in ks.load().ks_last_error()
