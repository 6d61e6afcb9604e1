"""The allocation-free descriptor entry point against the FP64 oracle and the
context entry point.

aenet_descriptors_noalloc exists for callers that cannot call cudaMalloc when
they need descriptors (a program whose GPU memory comes only from its own fixed
pool, code running while another component owns the allocator, a plugin that
must not grow the device footprint after start-up). Its scratch is a fixed
static device array shared by every call, so these tests make calls in a row on
different structures and check that each matches the oracle's G (and
aenet_descriptors()) within the descriptor tolerance of the parity tests, i.e.
nothing of an earlier call leaks into a later one. One case overflows the
neighbour-list capacities the entry point derives from the mean density, so its
regrow-and-retry pass runs on scratch that still holds the first attempt; one
call runs on a non-default stream. The size limit is checked too. This file is
named to be collected last.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_11311_gb300 import inputs
from tolerances import descriptor_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _aenet():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2107_11311_gb300 import aenet
    return aenet


def _cluster():
    """The 192-atom water box (1.0 g/cm^3) placed, without its periodic
    images, in a 40 A box: the mean density is 3% of the cluster's, so the
    mean-density list capacities (64 entries within 6 A, 32 within 4 A) are
    below what the cluster's inner atoms need (up to 86 within 6 A): the first
    attempt overflows and the entry point retries with doubled capacities."""
    st = inputs.water_192()
    return inputs.Structure(pos=st.pos + 10.0, types=st.types, box=np.full(3, 40.0), n_species=st.n_species)


def _noalloc(aenet, m, st, stream=None):
    pos = torch.tensor(st.pos, device="cuda")
    types = torch.tensor(st.types, device="cuda")
    out = torch.full((st.n, m.D), float("nan"), dtype=torch.float32, device="cuda")
    if stream is not None:
        torch.cuda.current_stream().synchronize()  # inputs written before the other stream reads them
    aenet.descriptors_noalloc(m, pos, types, st.box, out, stream=stream)
    return out.cpu().numpy()


def _check(got, ref, m, what):
    assert np.isfinite(got).all(), what
    tol = descriptor_tol(ref.astype(np.float64), m)
    bad = np.abs(got - ref) > tol
    assert not bad.any(), f"{what}: {bad.sum()} coefficients differ (worst {(np.abs(got - ref) / tol).max():.2f}x)"


def test_noalloc_descriptors_match_oracle_and_context_in_a_row():
    aenet = _aenet()
    cases = [("amorphous", inputs.amorphous(2000, seed=5)), ("water", inputs.water_192()),
             ("water", inputs.water(8, 6.6, seed=3)), ("water", _cluster())]
    for k, (fam, st) in enumerate(cases):
        m = inputs.make_model(fam)
        got = _noalloc(aenet, m, st)
        oracle_G = O.compute(m, st.pos, st.types, st.box, want_G=True, want_forces=False)["G"]
        _check(got, oracle_G, m, f"call {k} ({fam}, n={st.n}) vs the oracle")
        ctx_G = aenet.AenetGPU(m, "fp32").descriptors(st.pos, st.types, st.box)
        _check(got, ctx_G.astype(np.float64), m, f"call {k} ({fam}, n={st.n}) vs aenet_descriptors")


def test_noalloc_on_a_side_stream_twice():
    aenet = _aenet()
    m = inputs.make_model("water")
    s = torch.cuda.Stream()
    for st in (_cluster(), inputs.water_192()):
        got = _noalloc(aenet, m, st, stream=s)
        ref = O.compute(m, st.pos, st.types, st.box, want_G=True, want_forces=False)["G"]
        _check(got, ref, m, f"side stream, n={st.n}, box {st.box[0]}")


def test_noalloc_rejects_bad_arguments():
    aenet = _aenet()
    m = inputs.make_model("water")
    st = inputs.water_192()
    pos = torch.tensor(st.pos, device="cuda")
    types = torch.tensor(st.types, device="cuda")
    with pytest.raises(ValueError):
        aenet.descriptors_noalloc(m, pos, types, st.box, torch.zeros((st.n, m.D - 1), device="cuda"))
    with pytest.raises(TypeError):
        aenet.descriptors_noalloc(m, pos, types, st.box,
                                  torch.zeros((st.n, m.D), dtype=torch.float16, device="cuda"))
    with pytest.raises(ValueError):
        aenet.descriptors_noalloc(m, pos, types[:-1], st.box, torch.zeros((st.n, m.D), device="cuda"))
    with pytest.raises(TypeError):
        aenet.descriptors_noalloc(m, pos.cpu(), types, st.box, torch.zeros((st.n, m.D), device="cuda"))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    aenet = _aenet()
    n = aenet.NOALLOC_MAX_ATOMS + 1
    m = inputs.make_model("water")
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    types = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.zeros((n, m.D), dtype=torch.float32, device="cuda")
    with pytest.raises(aenet.AenetError) as ei:
        aenet.descriptors_noalloc(m, pos, types, np.full(3, 100.0), out)
    assert ei.value.code == -3
    assert "16384" in str(ei.value)
