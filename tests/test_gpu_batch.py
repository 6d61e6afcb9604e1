"""Batched form: many independent periodic structures of uneven size
(log-uniform 32 ... 2,048 atoms, water and the 4-species solid, boxes down to
below the cutoff) evaluated in one call, against the oracle per structure and
against one-structure calls of the same context."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_11311_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_TOL, F_RMS_TOL = 5e-4, 1e-3


@pytest.fixture(scope="module")
def gpu_mod():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2107_11311_gb300 import aenet
    return aenet


@pytest.fixture(scope="module")
def batch():
    wat, amo = inputs.batch_structures(limit=6)
    # add a box shorter than the cutoff (self-images; staged in several chunks)
    return wat, amo + [inputs.amorphous(32, seed=4)]


@pytest.mark.parametrize("family,idx", [("water", 0), ("amorphous", 1)])
@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_batch_matches_oracle_per_structure(gpu_mod, batch, family, idx, precision):
    structs = batch[idx]
    m = inputs.make_model(family)
    off, pos, types, boxes = inputs.concat(structs)
    g = gpu_mod.AenetGPU(m, precision)
    out = g.compute_batch(off, pos, types, boxes)
    for s, st in enumerate(structs):
        ref = O.compute(m, st.pos, st.types, st.box)
        assert abs(out["energies"][s] - ref["energy"]) / st.n <= E_TOL
        df = out["forces"][off[s]:off[s + 1]] - ref["forces"]
        assert np.sqrt((df ** 2).mean()) <= F_RMS_TOL
        np.testing.assert_allclose(out["virials"][s], ref["virial"],
                                   atol=1e-4 * max(1.0, np.abs(ref["virial"]).max()))


def test_batch_equals_single_calls_and_device_pointers(gpu_mod, batch):
    structs = batch[1]
    m = inputs.make_model("amorphous")
    off, pos, types, boxes = inputs.concat(structs)
    g = gpu_mod.AenetGPU(m, "fp32")
    E = torch.zeros(len(structs), dtype=torch.float64, device="cuda")
    F = torch.zeros((int(off[-1]), 3), dtype=torch.float64, device="cuda")
    W = torch.zeros((len(structs), 3, 3), dtype=torch.float64, device="cuda")
    g.compute_batch(off, torch.tensor(pos, device="cuda"), torch.tensor(types, device="cuda"), boxes,
                    energies=E, forces=F, virials=W)
    torch.cuda.synchronize()
    for s, st in enumerate(structs):
        one = g.compute(st.pos, st.types, st.box)
        assert abs(E[s].item() - one["energy"]) / st.n < 1e-6
        np.testing.assert_allclose(F[off[s]:off[s + 1]].cpu().numpy(), one["forces"], atol=1e-4)


def test_batch_edge_cases(gpu_mod):
    m = inputs.make_model("water")
    g = gpu_mod.AenetGPU(m, "fp32")
    # an empty structure between two others, and a single isolated atom
    a = inputs.water(3, 8.0, seed=1)
    b = inputs.Structure(pos=np.array([[1.0, 1.0, 1.0]]), types=np.array([0], np.int32),
                         box=np.full(3, 20.0), n_species=2)
    e = inputs.Structure(pos=np.zeros((0, 3)), types=np.zeros(0, np.int32), box=np.full(3, 10.0), n_species=2)
    off, pos, types, boxes = inputs.concat([a, e, b])
    out = g.compute_batch(off, pos, types, boxes)
    assert out["energies"][1] == 0.0
    for s, st in ((0, a), (2, b)):
        ref = O.compute(m, st.pos, st.types, st.box)
        assert abs(out["energies"][s] - ref["energy"]) < 1e-4
    with pytest.raises(gpu_mod.AenetError):
        g.compute_batch(np.array([0, 5, 3]), pos, types, np.full((2, 3), 10.0))
