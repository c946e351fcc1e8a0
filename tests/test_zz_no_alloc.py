"""GPU tests of ks_overlap_noalloc, the entry point for callers that cannot allocate device
memory (code whose device memory all belongs to its own pool allocator, or loops that cannot
take the synchronisation of an allocation).  Its output must equal the oracle's overlap
conj(A) B^T of the same blocks, and the Gram matrix the existing ks_orthonormalize entry point
reports for the same states, on two calls in a row (the second call reuses the library's
fixed scratch array), and the calls must leave the device's free memory unchanged.
Collected last so that a stop-at-first-failure run has already run every other test."""
import numpy as np
import pytest

from oracle import ks_oracle as ko
from paper_2106_03872_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ks():
    from paper_2106_03872_gb300 import ks as mod
    mod.load()
    assert torch.cuda.is_available()
    return mod


# FP64: 1e-12 relative.  complex64 inputs: rounding of the inputs (6e-8 relative) plus FP32
# accumulation over a K range of a few thousand terms (~sqrt(K) * 6e-8), bounded by 2e-5.
TOL = {"fp64": 1e-12, "bf16x3": 2e-5}
DT = {"fp64": torch.complex128, "bf16x3": torch.complex64}


def max_rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("shape", [(10.0, 24, 9), (15.0, 48, 40)])
def test_overlap_noalloc_matches_orthonormalize_and_oracle(ks, prec, shape):
    L, N, ns = shape
    cell = inputs.small_cell(L, N, 3, ns, 31)
    g = ks.Grid(cell, prec=prec)
    c = inputs.random_coeffs(31, ns, g.nG)
    g.set_states(c)
    S_ref = g.orthonormalize(want_S=True)           # the existing entry point's Gram matrix
    g.close()
    S_ora = ko.gram(c)
    a = torch.from_numpy(c).to("cuda", DT[prec])     # same rounding as ks_set_states
    for _ in range(2):
        out = torch.full((ns, ns), float("nan"), dtype=torch.complex128, device="cuda")
        ks.overlap_noalloc(a.data_ptr(), a.data_ptr(), ns, ns, a.shape[1], prec == "fp64", out.data_ptr())
        torch.cuda.synchronize()
        S = out.cpu().numpy()
        assert max_rel(S, S_ora) <= TOL[prec]
        assert max_rel(S, S_ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_overlap_noalloc_rectangular_on_a_stream_allocates_nothing(ks, prec):
    """m != n, distinct blocks, a non-default stream; against the oracle's conj(A) B^T.  After a
    first call (which may load the module and reserve the fixed array), further calls leave the
    device's free memory unchanged."""
    m, n, nG = 37, 101, 5003                           # ragged against every tile size
    A = inputs.random_coeffs(41, m, nG)
    B = inputs.random_coeffs(42, n, nG)
    expect = ko.gram(A, B)
    a = torch.from_numpy(A).to("cuda", DT[prec])
    b = torch.from_numpy(B).to("cuda", DT[prec])
    outs = [torch.full((m, n), float("nan"), dtype=torch.complex128, device="cuda") for _ in range(3)]
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    ks.overlap_noalloc(a.data_ptr(), b.data_ptr(), m, n, nG, prec == "fp64", outs[0].data_ptr(), st.cuda_stream)
    st.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for o in outs[1:]:
        ks.overlap_noalloc(a.data_ptr(), b.data_ptr(), m, n, nG, prec == "fp64", o.data_ptr(), st.cuda_stream)
    st.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for o in outs:
        assert max_rel(o.cpu().numpy(), expect) <= TOL[prec]


def test_overlap_noalloc_rejects_sizes_beyond_scratch(ks):
    a = torch.zeros((4, 8), dtype=torch.complex128, device="cuda")
    out = torch.zeros((4, 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(ks.KsError) as e:
        ks.overlap_noalloc(a.data_ptr(), a.data_ptr(), 513, 513, 8, True, out.data_ptr())
    assert e.value.status == ks.KS_ERR_ARG
    assert b"exceeds the scratch maximum" in ks.load().ks_last_error()
