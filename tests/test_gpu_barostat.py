"""Berendsen barostat of the MD path (aenet_set_barostat) against the oracle's
own barostat loop: cell, positions and per-frame energies, in an orthorhombic
and in a tilted cell, through the cell list and the Verlet list, with and
without the thermostat; plus the boundary's checks."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_11311_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_TOL = 5e-4  # eV/atom


@pytest.fixture(scope="module")
def gpu_mod():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2107_11311_gb300 import aenet
    return aenet


def _start(tilt_frac=(0.0, 0.0, 0.0)):
    st = inputs.water_192()
    m = inputs.make_model("water")
    L = np.asarray(st.box, dtype=float)
    tilt = (tilt_frac[0] * L[0], tilt_frac[1] * L[0], tilt_frac[2] * L[1])
    H = np.array([[L[0], tilt[0], tilt[1]], [0.0, L[1], tilt[2]], [0.0, 0.0, L[2]]])
    pos = (st.pos / L) @ H.T
    v0 = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=2)
    return st, m, pos, v0, tilt


# the random-weight water box sits near -3.3e5 bar: a 2.2e6 bar modulus keeps
# each coupling to a fraction of a percent of the volume
CASES = {
    "orthorhombic": ((0.0, 0.0, 0.0), 0.0, None, (0.0, 0.05, 2.2e6, 4), 12),
    "orthorhombic_partial_last_run": ((0.0, 0.0, 0.0), 0.0, None, (1e4, 0.05, 2.2e6, 5), 12),
    "tilted_verlet": ((0.3, -0.2, 0.25), 1.0, None, (0.0, 0.05, 2.2e6, 5), 10),
    "tilted_npt": ((0.2, 0.1, -0.15), 0.0, (300.0, 0.05), (-1e4, 0.05, 2.2e6, 3), 9),
}


@pytest.mark.parametrize("case", list(CASES))
def test_barostat_matches_oracle(gpu_mod, case):
    tilt_frac, skin, thermo, baro, n_steps = CASES[case]
    st, m, pos0, v0, tilt = _start(tilt_frac)
    dt = 5e-4
    xo, vo, epo, eko, boxo, tilto = O.md_npt(m, pos0, v0, st.types, st.box, tilt, dt, n_steps, baro,
                                              thermostat=thermo)
    g = gpu_mod.AenetGPU(m, "fp32")
    g.set_box_tilt(*tilt)
    g.set_skin(skin)
    if thermo:
        g.set_thermostat(*thermo)
    g.set_barostat(*baro)
    pos, vel = pos0.copy(), v0.copy()
    ep, ek = np.zeros(n_steps + 1), np.zeros(n_steps + 1)
    g.md_nve(pos, vel, st.types, st.box, dt, n_steps, e_pot=ep, e_kin=ek)
    box, tl = g.md_box()
    print(f"{case}: cell {st.box[0]:.4f} -> {box[0]:.4f} A (oracle {boxo[0]:.4f})")
    assert abs(box[0] / st.box[0] - 1.0) > 1e-4  # the cell did move
    np.testing.assert_allclose(box, boxo, rtol=1e-7)
    np.testing.assert_allclose(tl, tilto, rtol=1e-7, atol=1e-12)
    assert np.abs(ep - epo).max() / st.n <= E_TOL
    np.testing.assert_allclose(ek, eko, rtol=1e-5)
    np.testing.assert_allclose(pos, xo, atol=1e-5)
    np.testing.assert_allclose(vel, vo, atol=1e-2)


def test_barostat_with_infinite_modulus_is_the_fixed_cell_run(gpu_mod):
    st, m, pos0, v0, tilt = _start((0.2, 0.0, 0.1))
    runs = []
    for baro in (None, (0.0, 0.05, 1e300, 3)):
        g = gpu_mod.AenetGPU(m, "fp32")
        g.set_box_tilt(*tilt)
        if baro:
            g.set_barostat(*baro)
        pos, vel = pos0.copy(), v0.copy()
        ep = np.zeros(10)
        g.md_nve(pos, vel, st.types, st.box, 5e-4, 9, e_pot=ep)
        runs.append((pos, ep, g.md_box()))
    (p0, e0, (b0, t0)), (p1, e1, (b1, t1)) = runs
    np.testing.assert_array_equal(b1, b0)
    np.testing.assert_array_equal(t1, t0)
    np.testing.assert_allclose(p1, p0, atol=1e-6)  # FP32 atomics: run-dependent last bits
    assert np.abs(e1 - e0).max() / st.n < 1e-6


def test_barostat_boundary(gpu_mod):
    st, m, pos0, v0, tilt = _start()
    g = gpu_mod.AenetGPU(m, "fp32")
    with pytest.raises(gpu_mod.AenetError) as ei:  # no MD call yet
        g.md_box()
    assert ei.value.code == -8
    for bad in ((np.nan, 0.1, 1e4, 1), (0.0, 0.1, 0.0, 1), (0.0, 0.1, 1e4, 0)):
        with pytest.raises(gpu_mod.AenetError):
            g.set_barostat(*bad)
    g.set_barostat(0.0, 0.05, 2.2e6, 2)
    p = torch.tensor(pos0, device="cuda")
    v = torch.tensor(v0, device="cuda")
    t = torch.tensor(st.types, device="cuda")
    with pytest.raises(gpu_mod.AenetError):  # the barostat synchronises: no async steps
        g.md_nve(p, v, t, st.box, 5e-4, 4, flags=gpu_mod.AENET_MD_ASYNC)
    # a coupling far too strong for the pressure is reported, not applied
    g.set_barostat(1e9, 1e-3, 1.0, 1)
    with pytest.raises(gpu_mod.AenetError) as ei:
        g.md_nve(pos0.copy(), v0.copy(), st.types, st.box, 5e-4, 2)
    assert ei.value.code == -1
    g.set_barostat(0.0, 0.0, 0.0, 0)  # off again: a plain run works
    g.md_nve(pos0.copy(), v0.copy(), st.types, st.box, 5e-4, 2)
    box, _ = g.md_box()
    np.testing.assert_array_equal(box, st.box)
