"""Restricted triclinic cells on the GPU (a = (L_x, 0, 0), b = (xy, L_y, 0),
c = (xz, yz, L_z), set by aenet_set_box_tilt): every output against the
oracle's brute-force lattice images, descriptors within their rounding bound,
MD through the cell list and through the Verlet list against the oracle's
integration, and the boundary's handling of the tilt."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_11311_gb300 import inputs
from tolerances import descriptor_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_TOL = 5e-4      # eV/atom
F_RMS_TOL = 1e-3  # eV/A


@pytest.fixture(scope="module")
def gpu_mod():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2107_11311_gb300 import aenet
    return aenet


def _cell_matrix(box, tilt):
    lx, ly, lz = box
    xy, xz, yz = tilt
    return np.array([[lx, xy, xz], [0.0, ly, yz], [0.0, 0.0, lz]])


def _tilted(st, frac_tilt, shift=0.0):
    """The structure's fractional coordinates in a cell with tilts given as
    fractions of the edges (xy/L_x, xz/L_x, yz/L_y); shift adds a whole-cell
    displacement so that unwrapped input positions are exercised too."""
    L = np.asarray(st.box, dtype=float)
    tilt = (frac_tilt[0] * L[0], frac_tilt[1] * L[0], frac_tilt[2] * L[1])
    H = _cell_matrix(L, tilt)
    pos = (st.pos / L) @ H.T
    if shift:
        rng = np.random.default_rng(11)
        pos = pos + rng.integers(-2, 3, size=(st.n, 3)) @ H.T * shift
    return pos, tilt


def _check(ref, got, n, what):
    de = abs(got["energy"] - ref["energy"]) / max(n, 1)
    assert de <= E_TOL, f"{what}: |dE|/N = {de}"
    df = got["forces"] - ref["forces"]
    rms = float(np.sqrt((df ** 2).mean()))
    assert rms <= F_RMS_TOL, f"{what}: force RMS error {rms}"
    assert np.abs(df).max() <= 10 * F_RMS_TOL, f"{what}: max force error {np.abs(df).max()}"
    np.testing.assert_allclose(got["e_atom"], ref["e_atom"], atol=2e-4 * (1 + np.abs(ref["e_atom"]).max()))
    scale = max(1.0, np.abs(ref["virial"]).max())
    np.testing.assert_allclose(got["virial"], ref["virial"], atol=1e-4 * scale)


CASES = {
    # (family, structure, tilts as fractions of the edges, whole-cell shifts)
    "water_192_mild": ("water", inputs.water_192, (0.3, -0.2, 0.25), 0.0),
    "water_192_steep": ("water", inputs.water_192, (0.49, 0.45, -0.48), 1.0),
    "water_1536": ("water", lambda: inputs.water(512, None, 10), (0.2, 0.1, -0.3), 1.0),
    "amorphous_small_box": ("amorphous", lambda: inputs.amorphous(48, seed=4), (0.4, -0.35, 0.3), 1.0),
    "amorphous_2000": ("amorphous", lambda: inputs.amorphous(2000, seed=5), (-0.27, 0.13, 0.41), 0.0),
}


@pytest.mark.parametrize("case", list(CASES))
def test_tilted_cell_parity(gpu_mod, case):
    fam, make, ft, shift = CASES[case]
    st = make()
    m = inputs.make_model(fam)
    pos, tilt = _tilted(st, ft, shift)
    g = gpu_mod.AenetGPU(m, "fp32")
    g.set_box_tilt(*tilt)
    got = g.compute(pos, st.types, st.box)
    ref = O.compute_tri(m, pos, st.types, st.box, tilt)
    _check(ref, got, st.n, case)
    G = g.descriptors(pos, st.types, st.box)
    Gref = O.compute_tri(m, pos, st.types, st.box, tilt, want_G=True)["G"]
    tol = descriptor_tol(Gref, m)
    ratio = float((np.abs(G - Gref) / tol).max())
    print(f"{case}: worst descriptor error {ratio:.2f}x the rounding bound")
    assert ratio <= 1.0, f"{case}: descriptor coefficients off ({ratio:.2f}x the bound)"


def test_integer_tilt_is_the_orthorhombic_box(gpu_mod):
    """Tilts that are whole multiples of the edges describe the orthorhombic
    lattice again: the GPU result in that description equals the orthorhombic
    one (up to FP32 rounding: the cell grids differ)."""
    st = inputs.amorphous(2000, seed=5)
    m = inputs.make_model("amorphous")
    g = gpu_mod.AenetGPU(m, "fp32")
    ortho = g.compute(st.pos, st.types, st.box)
    L = st.box
    g.set_box_tilt(L[0], -L[0], 2 * L[1])
    tri = g.compute(st.pos, st.types, st.box)
    assert abs(tri["energy"] - ortho["energy"]) / st.n < 1e-6
    np.testing.assert_allclose(tri["forces"], ortho["forces"], atol=1e-4)
    np.testing.assert_allclose(tri["virial"], ortho["virial"], atol=1e-4 * max(1.0, np.abs(ortho["virial"]).max()))
    g.set_box_tilt(0.0, 0.0, 0.0)  # back to orthorhombic
    again = g.compute(st.pos, st.types, st.box)
    assert abs(again["energy"] - ortho["energy"]) / st.n < 1e-7


@pytest.mark.parametrize("skin", [0.0, 1.0])
def test_tilted_cell_md_matches_oracle(gpu_mod, skin):
    """NVE in a tilted cell (atoms cross the tilted faces), through the cell
    list every step and through the Verlet list, against the oracle."""
    st = inputs.water_192()
    m = inputs.make_model("water")
    pos0, tilt = _tilted(st, (0.35, -0.25, 0.3))
    v0 = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=2)
    n_steps = 10
    xo, vo, epo, eko = O.md_tri(m, pos0, v0, st.types, st.box, tilt, 5e-4, n_steps)
    g = gpu_mod.AenetGPU(m, "fp32")
    g.set_box_tilt(*tilt)
    g.set_skin(skin)
    pos, vel = pos0.copy(), v0.copy()
    ep, ek = np.zeros(n_steps + 1), np.zeros(n_steps + 1)
    g.md_nve(pos, vel, st.types, st.box, 5e-4, n_steps, e_pot=ep, e_kin=ek)
    if skin > 0:
        assert g.md_list_builds() >= 1
    assert np.abs(ep - epo).max() / st.n <= E_TOL
    np.testing.assert_allclose(ek, eko, rtol=1e-5)
    np.testing.assert_allclose(pos, xo, atol=1e-5)
    np.testing.assert_allclose(vel, vo, atol=1e-2)


def test_tilt_change_restarts_md(gpu_mod):
    """Changing the tilt between MD calls starts the next call from frame 0 in
    the new cell, even with AENET_MD_CONTINUE."""
    st = inputs.water_192()
    m = inputs.make_model("water")
    pos0, tilt = _tilted(st, (0.2, 0.0, 0.0))
    v0 = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=2)
    g = gpu_mod.AenetGPU(m, "fp32")
    pos, vel = pos0.copy(), v0.copy()
    g.md_nve(pos, vel, st.types, st.box, 5e-4, 3)  # orthorhombic cell
    g.set_box_tilt(*tilt)
    start = pos.copy()
    ep = np.zeros(4)
    g.md_nve(pos, vel, st.types, st.box, 5e-4, 3, e_pot=ep, flags=gpu_mod.AENET_MD_CONTINUE)
    assert abs(ep[0] - O.compute_tri(m, start, st.types, st.box, tilt)["energy"]) / st.n <= E_TOL
    assert abs(ep[-1] - O.compute_tri(m, pos, st.types, st.box, tilt)["energy"]) / st.n <= E_TOL


def test_set_box_tilt_rejects_non_finite(gpu_mod):
    m = inputs.make_model("water")
    g = gpu_mod.AenetGPU(m, "fp32")
    for bad in ((np.nan, 0.0, 0.0), (0.0, np.inf, 0.0), (0.0, 0.0, -np.inf)):
        with pytest.raises(gpu_mod.AenetError) as ei:
            g.set_box_tilt(*bad)
        assert ei.value.code == -1


def test_tilted_cell_edge_cases(gpu_mod):
    """No atoms in a tilted cell; a cell so small and oblique that its image
    window passes the 4,096-cell limit is refused before any launch."""
    m = inputs.make_model("water")
    g = gpu_mod.AenetGPU(m, "fp32")
    g.set_box_tilt(2.0, -1.0, 1.5)
    out = g.compute(np.zeros((0, 3)), np.zeros(0, dtype=np.int32), (10.0, 10.0, 10.0))
    assert out["energy"] == 0.0
    g.set_box_tilt(0.99, 0.99, 0.99)  # face distances ~0.7 A for a 6 A cutoff: 19 x 19 x 13 image cells
    with pytest.raises(gpu_mod.AenetError) as ei:
        g.compute(np.array([[0.1, 0.2, 0.3], [0.5, 0.5, 0.5]]), np.array([0, 1], dtype=np.int32), (1.0, 1.0, 1.0))
    assert ei.value.code == -1
