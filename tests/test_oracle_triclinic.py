"""Pins of the oracle's restricted triclinic cell (a = (L_x, 0, 0),
b = (xy, L_y, 0), c = (xz, yz, L_z), the box form of the MD codes the paper
plugs into): checks that hold for any correct periodic evaluation, none of
which reuses the tilted code path on both sides.

* integer tilts (multiples of the edges) describe the same lattice as the
  orthorhombic box: equal to the orthorhombic cell-list oracle;
* a supercell doubled along a, b or c of a tilted cell has twice the energy and
  virial and the same per-atom energies and forces on every copy;
* forces are minus the finite-difference gradient of the energy;
* the virial is minus the derivative of the energy under a homogeneous strain
  of positions and cell (upper-triangular strains keep the restricted form).

And of the Berendsen barostat of the oracle's MD loop (the cell scaled by
mu = (1 - (K dt / tau) (P0 - P) / B)^(1/3) after every K-th step): an infinite
bulk modulus is the fixed-cell run bit for bit; an ideal gas (no forces) is
driven to the ideal-gas volume 2 E_kin / (3 P0) with edges and tilts scaled
alike; a target above / below the pressure compresses / expands the cell.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_11311_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore")


def _cell_matrix(box, tilt):
    """Columns a, b, c."""
    lx, ly, lz = box
    xy, xz, yz = tilt
    return np.array([[lx, xy, xz], [0.0, ly, yz], [0.0, 0.0, lz]])


def _tilted(st, tilt):
    """The structure's fractional coordinates placed in the tilted cell."""
    H = _cell_matrix(st.box, tilt)
    frac = st.pos / np.asarray(st.box)
    return frac @ H.T


def _water():
    return inputs.water_192(), inputs.make_model("water")


def _amorphous():
    st = inputs.amorphous(96, seed=5)
    return st, inputs.make_model("amorphous")


@pytest.mark.parametrize("family", ["water", "amorphous"])
@pytest.mark.parametrize("k", [(1, 0, 0), (0, 1, -1), (2, -1, 1)])
def test_integer_tilts_are_the_orthorhombic_lattice(family, k):
    st, m = _water() if family == "water" else _amorphous()
    L = np.asarray(st.box)
    tilt = (k[0] * L[0], k[1] * L[0], k[2] * L[1])  # b + k0 a, c + k1 a + k2 b
    ref = O.compute(m, st.pos, st.types, st.box, mode=O.CELLS)
    got = O.compute_tri(m, st.pos, st.types, st.box, tilt)
    assert abs(got["energy"] - ref["energy"]) < 1e-9 * st.n
    np.testing.assert_allclose(got["forces"], ref["forces"], atol=1e-9)
    np.testing.assert_allclose(got["e_atom"], ref["e_atom"], atol=1e-10)
    np.testing.assert_allclose(got["virial"], ref["virial"], atol=1e-8)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_supercell_of_a_tilted_cell(axis):
    st, m = _amorphous()
    tilt = (0.31 * st.box[0], -0.22 * st.box[0], 0.17 * st.box[1])
    pos = _tilted(st, tilt)
    one = O.compute_tri(m, pos, st.types, st.box, tilt)
    H = _cell_matrix(st.box, tilt)
    H2 = H.copy()
    H2[:, axis] *= 2.0  # the lattice vector along `axis` doubled
    pos2 = np.vstack([pos, pos + H[:, axis]])
    types2 = np.concatenate([st.types, st.types])
    box2 = (H2[0, 0], H2[1, 1], H2[2, 2])
    tilt2 = (H2[0, 1], H2[0, 2], H2[1, 2])
    two = O.compute_tri(m, pos2, types2, box2, tilt2)
    assert abs(two["energy"] - 2.0 * one["energy"]) < 1e-9 * st.n
    np.testing.assert_allclose(two["virial"], 2.0 * one["virial"], atol=1e-8)
    for half in (slice(0, st.n), slice(st.n, 2 * st.n)):
        np.testing.assert_allclose(two["forces"][half], one["forces"], atol=1e-9)
        np.testing.assert_allclose(two["e_atom"][half], one["e_atom"], atol=1e-10)


def test_tilted_cell_is_not_the_orthorhombic_one():
    """A non-integer tilt changes the lattice, hence the energy (the test above
    would pass for an oracle that ignored the tilt only if this one failed)."""
    st, m = _amorphous()
    tilt = (0.31 * st.box[0], 0.0, 0.0)
    a = O.compute_tri(m, st.pos, st.types, st.box, tilt)
    b = O.compute(m, st.pos, st.types, st.box)
    assert abs(a["energy"] - b["energy"]) > 1e-3


def test_forces_are_the_energy_gradient_in_a_tilted_cell():
    st, m = _water()
    tilt = (0.4 * st.box[0], 0.25 * st.box[0], -0.3 * st.box[1])
    pos = _tilted(st, tilt)
    F = O.compute_tri(m, pos, st.types, st.box, tilt)["forces"]
    h = 1e-5
    rng = np.random.default_rng(3)
    for i in rng.choice(st.n, 6, replace=False):
        for a in range(3):
            p = pos.copy()
            p[i, a] += h
            ep = O.compute_tri(m, p, st.types, st.box, tilt)["energy"]
            p[i, a] -= 2 * h
            em = O.compute_tri(m, p, st.types, st.box, tilt)["energy"]
            fd = -(ep - em) / (2 * h)
            assert abs(fd - F[i, a]) < 1e-6 * max(1.0, abs(F[i, a])), (i, a, fd, F[i, a])


@pytest.mark.parametrize("ab", [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)])
def test_virial_is_the_strain_derivative_in_a_tilted_cell(ab):
    st, m = _amorphous()
    tilt = (0.31 * st.box[0], -0.22 * st.box[0], 0.17 * st.box[1])
    pos = _tilted(st, tilt)
    H = _cell_matrix(st.box, tilt)
    W = O.compute_tri(m, pos, st.types, st.box, tilt)["virial"]
    np.testing.assert_allclose(W, W.T, atol=1e-8 * max(1.0, np.abs(W).max()))
    a, b = ab
    h = 1e-6

    def energy(eps):
        S = np.eye(3)
        S[a, b] += eps
        H2 = S @ H  # stays upper triangular for a <= b
        return O.compute_tri(m, pos @ S.T, st.types, (H2[0, 0], H2[1, 1], H2[2, 2]),
                             (H2[0, 1], H2[0, 2], H2[1, 2]))["energy"]

    dE = (energy(h) - energy(-h)) / (2 * h)
    # x -> (I + eps E_ab) x moves every displacement d by eps d_b along a:
    # dE/deps = sum d_b dE/dd_a = -W_ba with W_ab = -sum d_a dE/dd_b
    assert abs(-dE - W[b, a]) < 1e-5 * max(1.0, np.abs(W).max()), (ab, -dE, W[b, a])


def test_tilt_must_be_finite():
    st, m = _water()
    with pytest.raises(O.OracleError):
        O.compute_tri(m, st.pos, st.types, st.box, (np.nan, 0.0, 0.0))


# ---------------------------------------------------------------- barostat

# 1 eV/A^3 in bar, from the SI elementary charge (1 eV = 1.602176634e-19 J, exact):
# e / (1e-30 m^3) Pa, and 1 bar = 1e5 Pa
EV_A3_BAR = 1.602176634e-19 / 1e-30 / 1e5


def test_barostat_with_infinite_modulus_is_nve():
    """mu = 1 exactly: the same trajectory as without the barostat, bit for bit
    (one thread: the same summation order), and the cell unchanged."""
    st, m = _water()
    tilt = (0.2 * st.box[0], 0.0, -0.1 * st.box[1])
    pos = _tilted(st, tilt)
    v = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=5)
    a = O.md_tri(m, pos, v, st.types, st.box, tilt, 5e-4, 6, n_threads=1)
    b = O.md_npt(m, pos, v, st.types, st.box, tilt, 5e-4, 6, (1.0, 0.1, 1e300, 2), n_threads=1)
    for x, y in zip(a, b[:4]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(b[4], st.box)
    np.testing.assert_array_equal(b[5], tilt)


def _free_gas(n=64, seed=1):
    """Atoms of a zero-weight network (no forces, zero virial): an ideal gas."""
    m = inputs.make_model("amorphous")
    m.params = np.zeros_like(m.params)
    m.masses = np.ones(m.n_species)
    rng = np.random.default_rng(seed)
    box = np.full(3, 20.0)
    pos = rng.uniform(0.0, 20.0, (n, 3))
    types = rng.integers(0, m.n_species, n).astype(np.int32)
    vel = rng.normal(0.0, 5.0, (n, 3))
    return m, pos, vel, types, box


def test_barostat_drives_an_ideal_gas_to_the_target_pressure():
    """Without forces the pressure is 2 E_kin / (3 V) and E_kin is constant, so
    repeated couplings take the volume to the ideal-gas value 2 E_kin / (3 P0)."""
    m, pos, vel, types, box = _free_gas()
    P0 = 50.0  # bar
    tilt = (3.0, -2.0, 1.5)
    _, _, ep, ek, box1, tilt1 = O.md_npt(m, pos, vel, types, box, tilt, 1e-3, 400, (P0, 0.01, 1.0e2, 1))
    assert np.all(ep == 0.0)
    assert np.ptp(ek) < 1e-12 * ek[0]
    V_star = 2.0 * ek[0] / (3.0 * P0 / EV_A3_BAR)
    V1 = np.prod(box1)
    assert abs(V1 / V_star - 1.0) < 1e-6, (V1, V_star)
    # isotropic: edges and tilts scaled by the same factor
    mu = box1[0] / box[0]
    np.testing.assert_allclose(box1, mu * box, rtol=1e-12)
    np.testing.assert_allclose(tilt1, mu * np.asarray(tilt), rtol=1e-12)


def test_barostat_direction():
    """A target above the current pressure (about -3.3e5 bar for this random-
    weight water box) compresses the cell; below it, expands it."""
    st, m = _water()
    v = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=5)
    tilt = (0.0, 0.0, 0.0)
    up = O.md_npt(m, st.pos, v, st.types, st.box, tilt, 5e-4, 4, (1e5, 0.05, 2.2e4, 2))
    down = O.md_npt(m, st.pos, v, st.types, st.box, tilt, 5e-4, 4, (-1e6, 0.05, 2.2e4, 2))
    assert np.all(up[4] < st.box) and np.all(down[4] > st.box)


def test_barostat_rejects_bad_parameters():
    st, m = _water()
    v = np.zeros_like(st.pos)
    for bad in ((1.0, 0.0, 1e4, 1), (1.0, 0.1, 0.0, 1), (1.0, 0.1, 1e4, 0)):
        with pytest.raises(O.OracleError):
            O.md_npt(m, st.pos, v, st.types, st.box, (0.0, 0.0, 0.0), 5e-4, 2, bad)


# ------------------------------------------------- image-window rule of the grid

def test_image_window_rule_covers_the_cutoff():
    """The cell grid of a tilted cell (nc_k cells along lattice vector k, at
    least one cutoff between opposite cell faces) scans m_k = ceil(rc nc_k / w_k)
    neighbour cells each way, w_k the distance between the faces of the whole
    cell across k (volume over the area of the face spanned by the other two
    vectors). Check on random oblique cells: two points within rc never lie in
    cells whose indices differ by more than m_k along any k."""
    rng = np.random.default_rng(17)
    rc = 6.0
    reached = 0
    for _ in range(200):
        L = rng.uniform(4.0, 30.0, 3)
        tilt = rng.uniform(-0.5, 0.5, 3) * np.array([L[0], L[0], L[1]])
        H = _cell_matrix(L, tilt)
        V = np.prod(L)
        w = np.array([V / np.linalg.norm(np.cross(H[:, 1], H[:, 2])),
                      V / np.linalg.norm(np.cross(H[:, 2], H[:, 0])),
                      V / np.linalg.norm(np.cross(H[:, 0], H[:, 1]))])
        nc = np.maximum(1, np.floor(w / rc)).astype(int)
        m = np.ceil(rc * nc / w).astype(int)
        Hinv = np.linalg.inv(H)
        p = rng.uniform(0.0, 1.0, (400, 3)) @ H.T
        d = rng.normal(size=(400, 3))
        d *= (rc * rng.uniform(0.0, 1.0, (400, 1)) ** (1 / 3)) / np.linalg.norm(d, axis=1, keepdims=True)
        q = p + d
        cp = np.floor((p @ Hinv.T) * nc).astype(int)
        cq = np.floor((q @ Hinv.T) * nc).astype(int)  # unwrapped cell index of the image
        assert (np.abs(cq - cp) <= m).all()
        reached += int((np.abs(cq - cp) == m).any())
    # the window is used to its edge (a window one cell narrower would miss pairs)
    assert reached > 100
