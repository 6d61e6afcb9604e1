"""Verlet neighbour list with a skin for the MD path (the LAMMPS-style list the
paper credits for ænet-LAMMPS's speed, Sec. IV.B): the list of image-atoms
within rc_max + skin is rebuilt inside the captured step only when an atom has
moved more than skin/2. Checked against the oracle's own integration and
against the cell-list path on the same start."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_11311_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_TOL = 5e-4


@pytest.fixture(scope="module")
def gpu_mod():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2107_11311_gb300 import aenet
    return aenet


def _water192():
    st = inputs.water_192()
    m = inputs.make_model("water")
    v0 = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=2)
    return st, m, v0


def _run(gpu_mod, m, st, v0, n_steps, skin, dt=5e-4):
    g = gpu_mod.AenetGPU(m, "fp32")
    g.set_skin(skin)
    pos, vel = st.pos.copy(), v0.copy()
    ep, ek = np.zeros(n_steps + 1), np.zeros(n_steps + 1)
    g.md_nve(pos, vel, st.types, st.box, dt, n_steps, e_pot=ep, e_kin=ek)
    return g, pos, vel, ep, ek


def test_verlet_md_matches_oracle_trajectory(gpu_mod):
    st, m, v0 = _water192()
    xo, vo, epo, eko = O.md_nve(m, st.pos, v0, st.types, st.box, 5e-4, 10)
    g, pos, vel, ep, ek = _run(gpu_mod, m, st, v0, 10, 1.0)
    assert g.md_list_builds() >= 1
    assert np.abs(ep - epo).max() / st.n <= E_TOL
    np.testing.assert_allclose(ek, eko, rtol=1e-5)
    np.testing.assert_allclose(pos, xo, atol=1e-5)
    np.testing.assert_allclose(vel, vo, atol=1e-2)


@pytest.mark.parametrize("hidden", [(25, 25), (32, 32)])
def test_verlet_md_wide_network_matches_oracle(gpu_mod, hidden):
    """The list kernel's 32-wide form (water basis, hidden widths 17-32; the
    paper's 52-25-25-1 water model among them): 10 steps against the oracle's
    own integration with the same network."""
    st = inputs.water_192()
    m = inputs.make_model("water", hidden=hidden)
    v0 = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=2)
    xo, vo, epo, eko = O.md_nve(m, st.pos, v0, st.types, st.box, 5e-4, 10)
    g, pos, vel, ep, ek = _run(gpu_mod, m, st, v0, 10, 1.0)
    assert g.md_list_builds() >= 1
    assert np.abs(ep - epo).max() / st.n <= E_TOL
    np.testing.assert_allclose(ek, eko, rtol=1e-5)
    np.testing.assert_allclose(pos, xo, atol=1e-5)
    np.testing.assert_allclose(vel, vo, atol=1e-2)


def test_verlet_md_solid_matches_oracle(gpu_mod):
    """The list kernel on the 4-species solid's basis (angular order 6, whose
    angular sum runs through spherical harmonics), 10 steps of 600 atoms with
    a 1 A skin, against the oracle's own integration."""
    st = inputs.amorphous(600, seed=6)
    m = inputs.make_model("amorphous")
    v0 = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=4)
    xo, vo, epo, eko = O.md_nve(m, st.pos, v0, st.types, st.box, 5e-4, 10)
    g, pos, vel, ep, ek = _run(gpu_mod, m, st, v0, 10, 1.0)
    assert g.md_list_builds() >= 1
    assert np.abs(ep - epo).max() / st.n <= E_TOL
    np.testing.assert_allclose(ek, eko, rtol=1e-5)
    np.testing.assert_allclose(pos, xo, atol=1e-5)


def _stepwise(gpu_mod, m, st, v0, n_steps, skin):
    """One step per call (continuing): the energy the list path records after
    each step, and a fresh cell-list evaluation (another context) of the same
    positions."""
    g = gpu_mod.AenetGPU(m, "fp32")
    g.set_skin(skin)
    fresh = gpu_mod.AenetGPU(m, "fp32")
    p = torch.tensor(st.pos, device="cuda")
    v = torch.tensor(v0, device="cuda")
    t = torch.tensor(st.types, device="cuda")
    ep = torch.zeros(2, dtype=torch.float64, device="cuda")
    ek = torch.zeros(2, dtype=torch.float64, device="cuda")
    rec, ref = [], []
    for s in range(n_steps):
        g.md_nve(p, v, t, st.box, 5e-4, 1, e_pot=ep, e_kin=ek, flags=gpu_mod.AENET_MD_CONTINUE if s else 0)
        torch.cuda.synchronize()
        rec.append(ep[1].item())
        ref.append(fresh.compute(p.cpu().numpy(), st.types, st.box)["energy"])
    return g, np.array(rec), np.array(ref)


def test_verlet_energy_equals_fresh_evaluation_every_step(gpu_mod):
    """Between and across list builds, every step's energy from the list equals
    a fresh cell-list evaluation at the same positions (to FP32 summation order).
    The trajectory itself is chaotic (two identical cell-path runs part by
    ~1e-3 A within 60 steps through the FP32 atomic order), so the check is made
    per step on the same positions."""
    st, m, v0 = _water192()
    n = 60
    g, rec, ref = _stepwise(gpu_mod, m, st, v0, n, 1.0)
    builds = g.md_list_builds()
    print(f"skin 1.0 A: {builds} list builds in {n} steps; max |dE| {np.abs(rec - ref).max():.2e} eV")
    assert 2 <= builds < n // 2
    assert np.abs(rec - ref).max() / st.n < 2e-6
    # a skin far below the per-step displacement rebuilds every step
    g2, rec2, ref2 = _stepwise(gpu_mod, m, st, v0, 20, 1e-4)
    assert g2.md_list_builds() >= 19
    assert np.abs(rec2 - ref2).max() / st.n < 2e-6


def test_verlet_record_equals_fresh_evaluation(gpu_mod):
    """The energy the list path records after 100 steps of the 12,288-atom box
    equals a fresh cell-list evaluation of the final positions."""
    st = inputs.water_12288()
    m = inputs.make_model("water")
    v0 = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=12)
    g = gpu_mod.AenetGPU(m, "fp32")
    g.set_skin(1.0)
    pos = torch.tensor(st.pos, device="cuda")
    vel = torch.tensor(v0, device="cuda")
    types = torch.tensor(st.types, device="cuda")
    ep = torch.zeros(101, dtype=torch.float64, device="cuda")
    ek = torch.zeros(101, dtype=torch.float64, device="cuda")
    g.md_nve(pos, vel, types, st.box, 5e-4, 100, e_pot=ep, e_kin=ek)
    builds = g.md_list_builds()
    fresh = gpu_mod.AenetGPU(m, "fp32").compute(pos.cpu().numpy(), st.types, st.box)
    print(f"water_12288, skin 1.0 A: {builds} builds in 100 steps; E(list) {ep[-1].item():.6f}, "
          f"E(fresh) {fresh['energy']:.6f}")
    assert 1 <= builds < 50
    assert abs(ep[-1].item() - fresh["energy"]) / st.n < 1e-6


def test_verlet_continue_keeps_list_and_other_calls_invalidate_it(gpu_mod):
    st, m, v0 = _water192()
    ref = _run(gpu_mod, m, st, v0, 12, 0.0)[1]
    g = gpu_mod.AenetGPU(m, "fp32")
    g.set_skin(1.0)
    p = torch.tensor(st.pos, device="cuda")
    v = torch.tensor(v0, device="cuda")
    t = torch.tensor(st.types, device="cuda")
    g.md_nve(p, v, t, st.box, 5e-4, 4)
    b0 = g.md_list_builds()
    flags = gpu_mod.AENET_MD_ASYNC | gpu_mod.AENET_MD_CONTINUE
    for _ in range(4):
        g.md_nve(p, v, t, st.box, 5e-4, 1, flags=flags)
    g.check()
    assert g.md_list_builds() - b0 <= 1  # continuing reuses the list
    # an evaluation of another system rewrites the cell maps: the next MD call
    # must start again (frame 0 and a new list) and still follow the trajectory
    other = inputs.amorphous(64, seed=3)
    g.compute(other.pos, np.minimum(other.types, 1).astype(np.int32), other.box)
    b1 = g.md_list_builds()
    g.md_nve(p, v, t, st.box, 5e-4, 4, flags=gpu_mod.AENET_MD_CONTINUE)
    assert g.md_list_builds() > b1
    np.testing.assert_allclose(p.cpu().numpy(), ref, atol=1e-5)


def test_set_skin_rejects_bad_values(gpu_mod):
    st, m, v0 = _water192()
    g = gpu_mod.AenetGPU(m, "fp32")
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(gpu_mod.AenetError):
            g.set_skin(bad)
