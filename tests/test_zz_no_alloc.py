"""The allocation-free descriptor entry point against the context entry point.

aenet_descriptors_noalloc exists for callers that cannot call cudaMalloc when
they need descriptors (a program whose GPU memory comes only from its own fixed
pool, code running while another component owns the allocator, a plugin that
must not grow the device footprint after start-up). Its scratch is a fixed
static device array shared by every call, so this test makes two calls in a
row on different structures and checks that each matches aenet_descriptors()
within the descriptor tolerance of the parity tests, i.e. nothing of the first
call leaks into the second. It also checks the size limit. This file is named
to be collected last.
"""
import numpy as np
import pytest

from paper_2107_11311_gb300 import inputs
from tolerances import descriptor_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_descriptors_match_context_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2107_11311_gb300 import aenet
    cases = [("amorphous", inputs.amorphous(2000, seed=5)), ("water", inputs.water_192()),
             ("water", inputs.water(8, 6.6, seed=3))]
    for fam, st in cases:
        m = inputs.make_model(fam)
        ref = aenet.AenetGPU(m, "fp32").descriptors(st.pos, st.types, st.box)
        pos = torch.tensor(st.pos, device="cuda")
        types = torch.tensor(st.types, device="cuda")
        out = torch.full((st.n, m.D), float("nan"), dtype=torch.float32, device="cuda")
        aenet.descriptors_noalloc(m, pos, types, st.box, out)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        bad = np.abs(got - ref) > descriptor_tol(ref.astype(np.float64), m)
        assert not bad.any(), f"{fam} n={st.n}: {bad.sum()} coefficients differ"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2107_11311_gb300 import aenet
    n = aenet.NOALLOC_MAX_ATOMS + 1
    m = inputs.make_model("water")
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    types = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.zeros((n, m.D), dtype=torch.float32, device="cuda")
    with pytest.raises(aenet.AenetError) as ei:
        aenet.descriptors_noalloc(m, pos, types, np.full(3, 100.0), out)
    assert ei.value.code == -3
    assert "16384" in str(ei.value)
