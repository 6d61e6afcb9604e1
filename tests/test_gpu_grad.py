"""Energy gradient with respect to the network parameters (Sec. II.C) and the
torch.autograd.Function wrapper, against the FP64 oracle's dE/dW (itself pinned
by finite differences and torch autograd in the oracle tests)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_11311_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu_mod():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2107_11311_gb300 import aenet
    return aenet


def _rel_err(got, ref):
    return float(np.abs(got - ref).max() / max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("family,hidden,precision", [
    ("water", None, "fp32"),          # fused kernel
    ("amorphous", None, "fp32"),      # fused kernel, 4 species
    ("water", (40, 36), "fp32"),      # split FP32 network kernel (widths > 32)
    ("water", (32, 32), "bf16x3"),    # tensor-core networks inside the fused kernel, split operands
    ("amorphous", None, "bf16x3"),    # the same, 4 species (staged in chunks)
    ("water", (32, 32), "bf16x3-split"),  # the three-kernel path's tensor-core network kernel
])
def test_grad_weights_matches_oracle(gpu_mod, family, hidden, precision):
    st = inputs.water_192() if family == "water" else inputs.amorphous(600, seed=6)
    m = inputs.make_model(family, hidden=hidden)
    g = gpu_mod.AenetGPU(m, precision.replace("-split", ""))
    if precision.endswith("-split"):
        g.fuse_network(False)
    g.keep_activations(True)
    g.compute(st.pos, st.types, st.box)
    dW = g.grad_weights()
    ref = O.compute(m, st.pos, st.types, st.box, want_dEdW=True, want_forces=False)["dEdW"]
    err = _rel_err(dW, ref)
    print(f"{family} {hidden} {precision}: max |dE/dW error| / max |dE/dW| = {err:.2e}")
    assert err < 2e-4


def test_grad_weights_plain_bf16_reported(gpu_mod):
    st = inputs.water_192()
    m = inputs.make_model("water", hidden=(32, 32))
    g = gpu_mod.AenetGPU(m, "bf16")
    g.keep_activations(True)
    g.compute(st.pos, st.types, st.box)
    ref = O.compute(m, st.pos, st.types, st.box, want_dEdW=True, want_forces=False)["dEdW"]
    err = _rel_err(g.grad_weights(), ref)
    print(f"plain bf16 dE/dW relative error {err:.2e}")
    assert err < 3e-2


def test_grad_weights_needs_activations(gpu_mod):
    st = inputs.water_192()
    g = gpu_mod.AenetGPU(inputs.make_model("water"), "fp32")
    g.compute(st.pos, st.types, st.box)
    with pytest.raises(gpu_mod.AenetError) as ei:
        g.grad_weights()
    assert ei.value.code == -8


def test_autograd_function(gpu_mod):
    """E.backward() gives -F for the positions and dE/dW for the parameters;
    a parameter update through the wrapper changes the energy as the oracle's."""
    st = inputs.water_192()
    m = inputs.make_model("water")
    g = gpu_mod.AenetGPU(m, "fp32")
    Fn = gpu_mod.energy_function()
    pos = torch.tensor(st.pos, device="cuda", requires_grad=True)
    params = torch.tensor(m.params, device="cuda", requires_grad=True)
    types = torch.tensor(st.types, device="cuda")
    E = Fn.apply(pos, params, g, types, st.box)
    E.backward()
    ref = O.compute(m, st.pos, st.types, st.box, want_dEdW=True)
    assert abs(E.item() - ref["energy"]) / st.n < 5e-4
    np.testing.assert_allclose(pos.grad.cpu().numpy(), -ref["forces"], atol=2e-3)
    assert _rel_err(params.grad.cpu().numpy(), ref["dEdW"]) < 2e-4
    # gradient step on the parameters: new energy matches the oracle with the new parameters
    with torch.no_grad():
        newp = params - 1e-3 * params.grad
    m2 = inputs.make_model("water")
    m2.params = newp.cpu().numpy()
    E2 = Fn.apply(pos.detach(), newp, g, types, st.box)
    assert abs(E2.item() - O.compute(m2, st.pos, st.types, st.box)["energy"]) / st.n < 5e-4


def test_full_size_water_331776_precision_form(gpu_mod):
    """The 110,592-molecule box with the widened 52-32-32-1 network: forces on 64
    seeded atoms against the oracle (whose forces are pinned by central
    differences with h = 1e-4 A), and dE/dW on 64 seeded parameters against the
    oracle's analytic gradient, in the FP32 form (the fused kernel's 32-wide
    form) and the split-BF16 and plain BF16 forms."""
    st = inputs.water_331776()
    m = inputs.make_model("water", hidden=(32, 32))
    rng = np.random.default_rng(43)
    atoms = rng.choice(st.n, 64, replace=False)
    Fo, _ = O.forces_subset(m, st.pos, st.types, st.box, atoms)
    ref_w = O.compute(m, st.pos, st.types, st.box, want_dEdW=True, want_forces=False)["dEdW"]
    wsel = [(int(rng.integers(m.n_species)), int(rng.integers(m.n_params))) for _ in range(64)]
    for prec, f_tol, w_tol in (("fp32", 1e-3, 2e-4), ("bf16x3", 1e-3, 1e-3), ("bf16", 3e-2, 5e-2)):
        g = gpu_mod.AenetGPU(m, prec)
        g.keep_activations(True)
        out = g.compute(st.pos, st.types, st.box)
        dW = g.grad_weights()
        df = out["forces"][atoms] - Fo
        rms = float(np.sqrt((df ** 2).mean()))
        wref = np.array([ref_w[t, k] for t, k in wsel])
        wgot = np.array([dW[t, k] for t, k in wsel])
        werr = float(np.abs(wgot - wref).max() / np.abs(ref_w).max())
        print(f"water_331776 {prec}: force RMS error on 64 atoms {rms:.2e} eV/A, dE/dW rel error {werr:.2e}")
        assert rms < f_tol and werr < w_tol
