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


def test_autograd_md_water_331776_bf16x3_1000_steps(gpu_mod):
    """The large water box as the differentiated run: 110,592 molecules with the
    52-32-32-1 network in the split-BF16 form, 1,000 velocity-Verlet steps at
    0.5 fs whose forces come from AenetEnergy's backward (E.backward() gives
    dE/dr = -F) with dE/dW computed in every step, all on the device through
    the autograd function (no host round trip per step). Checked against the
    FP64 oracle: forces on 64 seeded atoms at frames 0 and 1,000 (the GPU's own
    frame-1000 positions), dE/dW on 64 seeded parameters at frame 1,000, and the
    total-energy error of the run against the oracle's own 1,000-step error on
    the 12,288-atom box at the same density, temperature, network and step (an
    intensive quantity; the oracle cannot integrate 331,776 atoms for 1,000
    steps within a test)."""
    st = inputs.water_331776()
    m = inputs.make_model("water", hidden=(32, 32))
    v0 = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=42)
    dev = torch.device("cuda")
    g = gpu_mod.AenetGPU(m, "bf16x3")
    Fn = gpu_mod.energy_function()
    c_metal = 1.602176634e-19 / 1.66053906660e-27 * 1e-4   # A^2/ps^2 per eV/amu
    dt = 5e-4
    pos = torch.tensor(st.pos, device=dev)
    vel = torch.tensor(v0, device=dev)
    types = torch.tensor(st.types, device=dev)
    params = torch.tensor(m.params, device=dev, requires_grad=True)
    inv_m = torch.tensor(1.0 / m.masses[st.types], device=dev)[:, None]
    masses = torch.tensor(m.masses[st.types], device=dev)[:, None]

    def energy_forces(x):
        x = x.detach().requires_grad_(True)
        params.grad = None
        E = Fn.apply(x, params, g, types, st.box)
        E.backward()
        return E.detach(), -x.grad, params.grad

    rng = np.random.default_rng(43)
    atoms = rng.choice(st.n, 64, replace=False)
    E, F, dW = energy_forces(pos)
    Fo0, _ = O.forces_subset(m, st.pos, st.types, st.box, atoms)
    err0 = float(np.sqrt(((F[atoms].cpu().numpy() - Fo0) ** 2).mean()))
    et = [E.item() + 0.5 * float((masses * vel ** 2).sum()) / c_metal]
    for step in range(1000):
        vel = vel + (0.5 * dt * c_metal) * F * inv_m
        pos = pos + dt * vel
        E, F, dW = energy_forces(pos)
        vel = vel + (0.5 * dt * c_metal) * F * inv_m
        if (step + 1) % 100 == 0:
            g.check()  # device-side errors of the asynchronous evaluations
            et.append(E.item() + 0.5 * float((masses * vel ** 2).sum()) / c_metal)
    g.check()
    x1000 = pos.cpu().numpy()
    assert np.isfinite(x1000).all()
    Fo1, _ = O.forces_subset(m, x1000, st.types, st.box, atoms)
    err1 = float(np.sqrt(((F[atoms].cpu().numpy() - Fo1) ** 2).mean()))
    ref_w = O.compute(m, x1000, st.types, st.box, want_dEdW=True, want_forces=False)["dEdW"]
    wsel = [(int(rng.integers(m.n_species)), int(rng.integers(m.n_params))) for _ in range(64)]
    got_w = dW.cpu().numpy()
    werr = max(abs(got_w[t, k] - ref_w[t, k]) for t, k in wsel) / np.abs(ref_w).max()
    drift = np.abs(np.array(et) - et[0]).max() / st.n
    s2 = inputs.water_12288()
    v2 = inputs.maxwell_boltzmann(m.masses[s2.types], 300.0, seed=12)
    _, _, epo, eko = O.md_nve(m, s2.pos, v2, s2.types, s2.box, dt, 1000)
    ref_drift = np.abs((epo + eko) - (epo[0] + eko[0])).max() / s2.n
    print(f"water_331776 autograd bf16x3: force RMS error frame 0 {err0:.2e}, frame 1000 {err1:.2e} eV/A; "
          f"dE/dW rel. error {werr:.2e}; max |E_tot - E_tot(0)|/N {drift:.3e} (oracle, 12,288 atoms: "
          f"{ref_drift:.3e}) eV/atom")
    assert err0 <= 1e-3 and err1 <= 1e-3
    assert werr < 1e-3
    assert drift <= 2.0 * ref_drift + 5e-3
