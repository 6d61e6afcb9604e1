"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
closed forms of the Chebyshev basis and the cosine cutoff, worked geometries
(a dimer and one water molecule) with hand-derived descriptor values, library
routines (numpy Chebyshev series, numpy/torch linear algebra and autograd),
finite differences, invariances, supercell additivity and NVE behaviour.

Each test names the passage of the paper it pins (Sec. II.A Eq. ANN-layer,
Sec. II.B Eqs. radial / angular / cos-cutoff and the Chebyshev recurrence).
"""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

from paper_2107_11311_gb300 import inputs
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cheb(alpha, x):
    c = np.zeros(alpha + 1)
    c[alpha] = 1.0
    return npcheb.chebval(x, c)


def _fc(r, rc):
    return 0.5 * (math.cos(math.pi * r / rc) + 1.0) if r <= rc else 0.0


# ------------------------------------------------------------------ basis

def test_chebyshev_closed_form():
    """Chebyshev recurrence (Sec. II.B): T_n(cos p) = cos(n p), and
    dT_n/dx = n sin(n p)/sin p at x = cos p."""
    rng = np.random.default_rng(0)
    for phi in rng.uniform(0.05, math.pi - 0.05, size=1000):
        T, dT = O.chebyshev(20, math.cos(phi))
        n = np.arange(21)
        np.testing.assert_allclose(T, np.cos(n * phi), rtol=0, atol=1e-13)
        np.testing.assert_allclose(dT, n * np.sin(n * phi) / math.sin(phi), rtol=1e-12, atol=1e-11)


def test_chebyshev_endpoints():
    """T_n(1) = 1, T_n(-1) = (-1)^n, T_n'(1) = n^2 (textbook values)."""
    T, dT = O.chebyshev(16, 1.0)
    np.testing.assert_allclose(T, 1.0)
    np.testing.assert_allclose(dT, np.arange(17) ** 2, rtol=1e-14)
    T, dT = O.chebyshev(16, -1.0)
    np.testing.assert_allclose(T, (-1.0) ** np.arange(17))


def test_cosine_cutoff_values_and_derivative():
    """Eq. cos-cutoff: f_c(0) = 1, f_c(Rc/2) = 1/2, f_c(Rc) = 0, zero beyond."""
    rc = 6.0
    assert O.cutoff(0.0, rc)[0] == pytest.approx(1.0, abs=1e-15)
    assert O.cutoff(rc / 2, rc)[0] == pytest.approx(0.5, abs=1e-15)
    assert O.cutoff(rc, rc)[0] == pytest.approx(0.0, abs=1e-15)
    assert O.cutoff(rc + 1e-9, rc) == (0.0, 0.0)
    assert O.cutoff(rc, rc)[1] == pytest.approx(0.0, abs=1e-15)
    h = 1e-6
    for r in (0.3, 1.7, 3.9, 5.5):
        fd = (O.cutoff(r + h, rc)[0] - O.cutoff(r - h, rc)[0]) / (2 * h)
        assert O.cutoff(r, rc)[1] == pytest.approx(fd, abs=1e-9)


# ------------------------------------------------------------- descriptor

def test_radial_dimer_worked_example():
    """Eq. radial for two atoms in a huge box: G_alpha = T_alpha(2r/Rc-1) f_c(r);
    the weighted copy carries s of the neighbour's species; no angular term."""
    m = inputs.make_model("water", identity_scaling=True)
    r = 2.5
    u = np.array([0.3, -0.5, 0.81])
    u /= np.linalg.norm(u)
    pos = np.array([[50.0, 50.0, 50.0], [50.0, 50.0, 50.0] + r * u])
    types = np.array([0, 1], dtype=np.int32)
    res = O.compute(m, pos, types, np.full(3, 100.0), mode=O.BRUTE, want_G=True)
    G = res["G"]
    Kr, Ka = 17, 9
    x = 2 * r / 6.0 - 1
    expect = np.array([_cheb(a, x) * _fc(r, 6.0) for a in range(Kr)])
    s = inputs.WATER_TYPE_WEIGHTS
    np.testing.assert_allclose(G[0, :Kr], expect, atol=1e-14)
    np.testing.assert_allclose(G[0, Kr + Ka:2 * Kr + Ka], s[1] * expect, atol=1e-14)
    np.testing.assert_allclose(G[1, Kr + Ka:2 * Kr + Ka], s[0] * expect, atol=1e-14)
    np.testing.assert_allclose(G[:, Kr:Kr + Ka], 0.0)
    np.testing.assert_allclose(G[:, 2 * Kr + Ka:], 0.0)


def test_angular_single_water_worked_example():
    """Eq. angular over ordered pairs for one H2O (O-H 0.96 A, H-O-H 104.5 deg):
    at O, G_alpha = 2 T_alpha(cos 104.5) f_c(0.96)^2; at H the angle between O and
    the other H is (180 - 104.5)/2 deg and the pair weight is s_O s_H."""
    m = inputs.make_model("water", identity_scaling=True)
    st = inputs.water(1, 100.0, seed=7)
    res = O.compute(m, st.pos, st.types, st.box, mode=O.BRUTE, want_G=True)
    G = res["G"]
    Kr, Ka = 17, 9
    sO, sH = inputs.WATER_TYPE_WEIGHTS
    roh = 0.96
    rhh = 2 * roh * math.sin(math.radians(104.5 / 2))
    # oxygen
    radO = np.array([2 * _cheb(a, 2 * roh / 6 - 1) * _fc(roh, 6) for a in range(Kr)])
    angO = np.array([2 * _cheb(a, math.cos(math.radians(104.5))) * _fc(roh, 4) ** 2 for a in range(Ka)])
    np.testing.assert_allclose(G[0, :Kr], radO, atol=1e-12)
    np.testing.assert_allclose(G[0, Kr:Kr + Ka], angO, atol=1e-12)
    np.testing.assert_allclose(G[0, Kr + Ka:2 * Kr + Ka], sH * radO, atol=1e-12)
    np.testing.assert_allclose(G[0, 2 * Kr + Ka:], sH * sH * angO, atol=1e-12)
    # hydrogens
    th = math.radians((180 - 104.5) / 2)
    for h in (1, 2):
        rad = np.array([_cheb(a, 2 * roh / 6 - 1) * _fc(roh, 6) for a in range(Kr)])
        rad2 = np.array([_cheb(a, 2 * rhh / 6 - 1) * _fc(rhh, 6) for a in range(Kr)])
        ang = np.array([2 * _cheb(a, math.cos(th)) * _fc(roh, 4) * _fc(rhh, 4) for a in range(Ka)])
        np.testing.assert_allclose(G[h, :Kr], rad + rad2, atol=1e-12)
        np.testing.assert_allclose(G[h, Kr:Kr + Ka], ang, atol=1e-12)
        np.testing.assert_allclose(G[h, Kr + Ka:2 * Kr + Ka], sO * rad + sH * rad2, atol=1e-12)
        np.testing.assert_allclose(G[h, 2 * Kr + Ka:], sO * sH * ang, atol=1e-12)


def test_descriptor_dimension_matches_paper():
    """The water descriptor has 52 components (Sec. IV.B: 2 x (17 + 9))."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    assert inputs.make_model("water").D == gold["water_descriptor_dim"]["value"]


# -------------------------------------------------------------- neighbours

@pytest.mark.parametrize("case", ["water192", "small_water", "small_amorphous", "noncubic"])
def test_cell_list_matches_brute_force(case):
    """Cell-list neighbour sets equal the brute-force definition (all images,
    only the zero-shift self excluded), also for boxes smaller than the cutoff."""
    if case == "water192":
        st, rc = inputs.water_192(), 6.0
        pos, box = st.pos, st.box
    elif case == "small_water":
        st, rc = inputs.water(8, 6.6, seed=3), 6.0
        pos, box = st.pos, st.box
    elif case == "small_amorphous":
        st, rc = inputs.amorphous(32, seed=4), 8.0
        pos, box = st.pos, st.box
    else:
        rng = np.random.default_rng(5)
        box = np.array([9.0, 13.0, 21.0])
        pos = rng.uniform(-5, 30, size=(60, 3))
        rc = 6.0
    a = O.neighbour_lists(pos, box, rc, mode=O.BRUTE)
    b = O.neighbour_lists(pos, box, rc, mode=O.CELLS)
    assert a == b
    if case == "small_amorphous":  # self-images are neighbours when L < rc
        assert any(e[0] == 0 for e in a[0])


# ------------------------------------------------------------------ network

def _numpy_network(model, t, g):
    P = model.params[t]
    x = g
    off = 0
    L = len(model.widths) - 1
    for l in range(1, L + 1):
        no, ni = model.widths[l], model.widths[l - 1]
        W = P[off:off + no * ni].reshape(no, ni)
        off += no * ni
        b = P[off:off + no]
        off += no
        z = W @ x + b
        x = np.tanh(z) if l < L else z
    return float(x[0])


def test_network_matches_numpy_matmul():
    """Eq. ANN-layer with tanh hidden layers and a linear output, evaluated with
    numpy matrix products on the oracle's own G, reproduces E_i."""
    m = inputs.make_model("water")
    st = inputs.water_192()
    r = O.compute(m, st.pos, st.types, st.box, want_G=True)
    for i in range(0, st.n, 17):
        t = st.types[i]
        g = (r["G"][i] - m.in_shift[t]) * m.in_scale[t]
        assert r["e_atom"][i] == pytest.approx(_numpy_network(m, t, g), abs=1e-12)
    assert r["energy"] == pytest.approx(r["e_atom"].sum(), abs=1e-10)


def test_dEdG_and_dEdW_against_torch_autograd():
    """Back-propagation (Sec. II.C) of the oracle against torch FP64 autograd of
    the same network on the oracle's G."""
    torch = pytest.importorskip("torch")
    m = inputs.make_model("amorphous", hidden=(7, 5))
    st = inputs.amorphous(60, seed=9)
    r = O.compute(m, st.pos, st.types, st.box, want_G=True, want_dEdG=True, want_dEdW=True)
    G = torch.tensor(r["G"], requires_grad=True)
    params = [torch.tensor(m.params[t], requires_grad=True) for t in range(m.n_species)]
    E = 0.0
    for i in range(st.n):
        t = int(st.types[i])
        x = (G[i] - torch.tensor(m.in_shift[t])) * torch.tensor(m.in_scale[t])
        off, L = 0, len(m.widths) - 1
        for l in range(1, L + 1):
            no, ni = m.widths[l], m.widths[l - 1]
            W = params[t][off:off + no * ni].reshape(no, ni)
            off += no * ni
            b = params[t][off:off + no]
            off += no
            x = W @ x + b
            if l < L:
                x = torch.tanh(x)
        E = E + x[0]
    E.backward()
    assert float(E.detach()) == pytest.approx(r["energy"], abs=1e-10)
    np.testing.assert_allclose(G.grad.numpy(), r["dEdG"], atol=1e-11)
    for t in range(m.n_species):
        np.testing.assert_allclose(params[t].grad.numpy(), r["dEdW"][t], atol=1e-10)


def test_dEdW_central_differences():
    """dE/dW by central finite differences in weight space (64 seeded weights)."""
    m = inputs.make_model("water")
    st = inputs.water(8, 6.6, seed=3)
    r = O.compute(m, st.pos, st.types, st.box, want_dEdW=True)
    rng = np.random.default_rng(11)
    h = 1e-6
    for _ in range(64):
        t = int(rng.integers(m.n_species))
        k = int(rng.integers(m.n_params))
        p0 = m.params[t, k]
        m.params[t, k] = p0 + h
        ep = O.compute(m, st.pos, st.types, st.box, want_forces=False)["energy"]
        m.params[t, k] = p0 - h
        em = O.compute(m, st.pos, st.types, st.box, want_forces=False)["energy"]
        m.params[t, k] = p0
        assert r["dEdW"][t, k] == pytest.approx((ep - em) / (2 * h), abs=2e-7)


# ---------------------------------------------------------- forces, virial

@pytest.mark.parametrize("family", ["water", "amorphous"])
def test_forces_central_differences(family):
    """F = -dE/dr against central differences with h = 1e-4 A, including a box
    smaller than the cutoff (images and self-images contribute)."""
    if family == "water":
        st = inputs.water_192()
        atoms = [0, 1, 2, 50, 101, 191]
    else:
        st = inputs.amorphous(32, seed=4)
        atoms = [0, 7, 23, 31]
    m = inputs.make_model(family)
    r = O.compute(m, st.pos, st.types, st.box)
    h = 1e-4
    for i in atoms:
        for a in range(3):
            p = st.pos.copy()
            p[i, a] += h
            ep = O.compute(m, p, st.types, st.box, want_forces=False)["energy"]
            p[i, a] -= 2 * h
            em = O.compute(m, p, st.types, st.box, want_forces=False)["energy"]
            fd = -(ep - em) / (2 * h)
            assert r["forces"][i, a] == pytest.approx(fd, abs=2e-5 + 1e-5 * abs(fd))


def test_zero_net_force_and_symmetric_virial():
    for family, st in (("water", inputs.water_192()), ("amorphous", inputs.amorphous(300, seed=2))):
        r = O.compute(inputs.make_model(family), st.pos, st.types, st.box)
        np.testing.assert_allclose(r["forces"].sum(0), 0.0, atol=1e-10)
        np.testing.assert_allclose(r["virial"], r["virial"].T, atol=1e-9)


def test_virial_against_strain_derivative():
    """Periodic box: W_aa = -dE/d(eps_aa) under a uniaxial affine strain of box and
    positions. Cluster in a large box: W_ba = -dE/d(eps_ab) for r -> (I + eps) r."""
    m = inputs.make_model("water")
    st = inputs.water_192()
    W = O.compute(m, st.pos, st.types, st.box)["virial"]
    h = 1e-6
    for a in range(3):
        s = np.ones(3)
        s[a] = 1 + h
        ep = O.compute(m, st.pos * s, st.types, st.box * s, want_forces=False)["energy"]
        s[a] = 1 - h
        em = O.compute(m, st.pos * s, st.types, st.box * s, want_forces=False)["energy"]
        assert W[a, a] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6, abs=1e-5)
    cl = inputs.water(12, 7.0, seed=8)
    pos = cl.pos - cl.pos.mean(0) + 40.0
    box = np.full(3, 80.0)
    W = O.compute(m, pos, cl.types, box)["virial"]
    c = pos.mean(0)
    for a in range(3):
        for b in range(3):
            e = np.zeros((3, 3))
            e[a, b] = h
            ep = O.compute(m, c + (pos - c) @ (np.eye(3) + e).T, cl.types, box, want_forces=False)["energy"]
            em = O.compute(m, c + (pos - c) @ (np.eye(3) - e).T, cl.types, box, want_forces=False)["energy"]
            assert W[b, a] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6, abs=1e-5)


# -------------------------------------------------------------- invariances

def test_translation_invariance():
    m = inputs.make_model("water")
    st = inputs.water_192()
    r0 = O.compute(m, st.pos, st.types, st.box)
    r1 = O.compute(m, st.pos + np.array([3.3, -17.1, 100.25]), st.types, st.box)
    assert r1["energy"] == pytest.approx(r0["energy"], rel=1e-12)
    np.testing.assert_allclose(r1["forces"], r0["forces"], atol=1e-9)


def test_rotation_invariance_cluster_and_cube_symmetries():
    m = inputs.make_model("water")
    cl = inputs.water(12, 7.0, seed=8)
    pos = cl.pos - cl.pos.mean(0)
    box = np.full(3, 80.0)
    r0 = O.compute(m, pos + 40.0, cl.types, box)
    q = np.random.default_rng(3).standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                  [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                  [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
    r1 = O.compute(m, pos @ R.T + 40.0, cl.types, box)
    assert r1["energy"] == pytest.approx(r0["energy"], rel=1e-12)
    np.testing.assert_allclose(r1["forces"], r0["forces"] @ R.T, atol=1e-9)
    # periodic cube: axis permutation and reflection are symmetries of the box
    st = inputs.water_192()
    r0 = O.compute(m, st.pos, st.types, st.box)
    r1 = O.compute(m, st.pos[:, [1, 2, 0]], st.types, st.box)
    assert r1["energy"] == pytest.approx(r0["energy"], rel=1e-12)
    np.testing.assert_allclose(r1["forces"], r0["forces"][:, [1, 2, 0]], atol=1e-9)
    r2 = O.compute(m, st.box - st.pos, st.types, st.box)
    assert r2["energy"] == pytest.approx(r0["energy"], rel=1e-12)
    np.testing.assert_allclose(r2["forces"], -r0["forces"], atol=1e-9)


def test_permutation_invariance():
    m = inputs.make_model("amorphous")
    st = inputs.amorphous(300, seed=2)
    r0 = O.compute(m, st.pos, st.types, st.box)
    p = np.random.default_rng(1).permutation(st.n)
    r1 = O.compute(m, st.pos[p], st.types[p], st.box)
    assert r1["energy"] == pytest.approx(r0["energy"], rel=1e-12)
    np.testing.assert_allclose(r1["forces"], r0["forces"][p], atol=1e-9)


@pytest.mark.parametrize("family", ["water", "amorphous"])
def test_supercell_additivity(family):
    """A 2x2x2 replica of a periodic cell has 8x the energy and the same per-atom
    descriptor, also when the cutoff exceeds half the box (image rule)."""
    st = inputs.water(8, 6.6, seed=3) if family == "water" else inputs.amorphous(32, seed=4)
    m = inputs.make_model(family)
    r0 = O.compute(m, st.pos, st.types, st.box, want_G=True)
    shifts = np.array([[i, j, k] for i in range(2) for j in range(2) for k in range(2)]) * st.box
    big = np.concatenate([st.pos + s for s in shifts])
    types = np.tile(st.types, 8)
    r1 = O.compute(m, big, types, 2 * st.box, want_G=True)
    assert r1["energy"] == pytest.approx(8 * r0["energy"], rel=1e-12)
    np.testing.assert_allclose(r1["G"], np.tile(r0["G"], (8, 1)), rtol=1e-12, atol=1e-11)
    np.testing.assert_allclose(r1["forces"], np.tile(r0["forces"], (8, 1)), atol=1e-9)
    np.testing.assert_allclose(r1["virial"], 8 * r0["virial"], rtol=1e-11, atol=1e-8)


def test_subset_forces_match_full():
    m = inputs.make_model("water")
    st = inputs.water_192()
    r = O.compute(m, st.pos, st.types, st.box)
    tg = [0, 5, 77, 190]
    F, Ea = O.forces_subset(m, st.pos, st.types, st.box, tg)
    np.testing.assert_allclose(F, r["forces"][tg], atol=1e-12)
    np.testing.assert_allclose(Ea, r["e_atom"][tg], atol=1e-13)


# --------------------------------------------------------------------- NVE

def _water_md_setup():
    m = inputs.make_model("water")
    st = inputs.water_192()
    v = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=2)
    return m, st, v


def test_nve_energy_error_scales_as_dt_squared():
    m, st, v = _water_md_setup()
    T = 0.01  # ps
    errs = []
    for dt in (5e-4, 2.5e-4):
        n = int(round(T / dt))
        _, _, ep, ek = O.md_nve(m, st.pos, v, st.types, st.box, dt, n)
        et = ep + ek
        errs.append(np.abs(et - et[0]).max())
    ratio = errs[0] / errs[1]
    assert 2.5 < ratio < 6.0, (errs, ratio)


def test_nve_time_reversibility():
    m, st, v = _water_md_setup()
    x1, v1, _, _ = O.md_nve(m, st.pos, v, st.types, st.box, 5e-4, 10)
    x2, v2, _, _ = O.md_nve(m, x1, -v1, st.types, st.box, 5e-4, 10)
    np.testing.assert_allclose(x2, st.pos, atol=1e-9)
    np.testing.assert_allclose(-v2, v, atol=1e-7)


def test_masses_are_the_papers():
    gold = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    assert inputs.MASS_H == gold["mass_H_amu"]["value"]
    assert inputs.MASS_O == gold["mass_O_amu"]["value"]


def test_berendsen_thermostat_closed_forms():
    """The thermostat (velocities scaled by sqrt(1 + dt/tau (T0/T - 1)) at the
    start of every step): a coupling time far beyond the run reproduces NVE
    exactly; with tau = dt and no forces (two atoms farther apart than every
    cutoff) one step sets the kinetic energy to (3N - 3) k_B T0 / 2 exactly."""
    m = inputs.make_model("water")
    st = inputs.water(8, 6.6, seed=3)
    v = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=5)
    a = O.md_nve(m, st.pos, v, st.types, st.box, 5e-4, 5)
    b = O.md_nve(m, st.pos, v, st.types, st.box, 5e-4, 5, thermostat=(1000.0, 1e30))
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    pos = np.array([[10.0, 10.0, 10.0], [60.0, 60.0, 60.0]])
    types = np.array([0, 1], dtype=np.int32)
    vel = np.array([[1.0, -2.0, 0.5], [-0.3, 0.7, 1.1]])
    box = np.full(3, 100.0)
    T0, dt = 450.0, 5e-4
    _, v1, ep, ek = O.md_nve(m, pos, vel, types, box, dt, 2, thermostat=(T0, dt))
    kB = 8.617333262e-5
    assert ek[1] == pytest.approx(1.5 * kB * T0, rel=1e-12)
    assert ek[2] == pytest.approx(1.5 * kB * T0, rel=1e-12)
    assert ep[0] == ep[1] == ep[2]
    # the scaling is uniform: the velocity directions are kept
    np.testing.assert_allclose(v1 / np.linalg.norm(v1), vel / np.linalg.norm(vel), rtol=1e-12)
