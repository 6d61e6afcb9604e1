"""The oracle's unit factors, derived here from SI constants instead of restated.

The paper's potential runs inside LAMMPS with ``units metal`` (Sec. III):
energies in eV, lengths in A, time in ps, masses in amu. Two factors follow:

* the kick v += (dt/2) F/m needs c = (1 eV / 1 amu) in A^2/ps^2. With the SI
  elementary charge e = 1.602176634e-19 J/eV (exact) and the atomic mass
  constant u = 1.66053906660e-27 kg (CODATA 2018), 1 eV/amu = e/u m^2/s^2, and
  1 m^2/s^2 = (1e10 A)^2 / (1e12 ps)^2 = 1e-4 A^2/ps^2;
* the barostat's pressure in bar: 1 eV/A^3 = e / 1e-30 Pa = e * 1e25 bar.

Releases of CODATA move u by a few parts in 1e10 (the oracle's c agrees with
the 2018 value to 4e-10), so c is compared to 1e-8 relative: any wrong digit
or unit still fails by orders of magnitude.

Each factor is checked through what the oracle computes with it (positions and
velocities after one step, kinetic energies, the cell scale of one barostat
coupling), so a wrong constant anywhere in the integrator fails here.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_11311_gb300 import inputs

E_CHARGE = 1.602176634e-19   # J per eV (SI, exact)
AMU_KG = 1.66053906660e-27   # kg (CODATA 2018, relative uncertainty 3e-10)
C_METAL = E_CHARGE / AMU_KG * 1e-4          # A^2/ps^2 per eV/amu
EV_A3_BAR = E_CHARGE / 1e-30 / 1e5          # bar per eV/A^3


def _water():
    m = inputs.make_model("water")
    st = inputs.water_192()
    v = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=2)
    return m, st, v


def test_kinetic_energy_uses_the_metal_unit_factor():
    m, st, v = _water()
    _, _, _, ek = O.md_nve(m, st.pos, v, st.types, st.box, 5e-4, 0)
    mass = m.masses[st.types]
    assert ek[0] == pytest.approx(0.5 * np.sum(mass[:, None] * v ** 2) / C_METAL, rel=1e-8)


def test_one_velocity_verlet_step_in_metal_units():
    """x1 = x0 + dt v0 + (dt^2 / 2) c F0 / m and v1 = v0 + (dt / 2) c (F0 + F1) / m,
    with F0, F1 the oracle's forces at x0 and x1 (pinned by finite differences
    elsewhere) and c derived from e and u."""
    m, st, v = _water()
    dt = 5e-4
    x1, v1, _, _ = O.md_nve(m, st.pos, v, st.types, st.box, dt, 1)
    F0 = O.compute(m, st.pos, st.types, st.box)["forces"]
    F1 = O.compute(m, x1, st.types, st.box)["forces"]
    inv_m = 1.0 / m.masses[st.types][:, None]
    drift = x1 - st.pos - dt * v
    np.testing.assert_allclose(drift, 0.5 * dt * dt * C_METAL * F0 * inv_m, rtol=1e-8, atol=1e-13)
    np.testing.assert_allclose(v1 - v, 0.5 * dt * C_METAL * (F0 + F1) * inv_m, rtol=1e-8, atol=1e-12)
    # the displacement term is not negligible: a wrong c would show
    assert np.abs(drift).max() > 1e-4


def test_barostat_pressure_in_bar():
    """One coupling of an ideal gas (zero weights: no forces, zero virial):
    P = 2 E_kin / (3 V) in eV/A^3, converted with the derived bar factor, sets
    the cell scale mu^3 = 1 - (dt / tau) (P0 - P) / B exactly."""
    m = inputs.make_model("amorphous")
    m.params = np.zeros_like(m.params)
    m.masses = np.ones(m.n_species)
    rng = np.random.default_rng(7)
    box = np.full(3, 20.0)
    pos = rng.uniform(0.0, 20.0, (48, 3))
    types = rng.integers(0, m.n_species, 48).astype(np.int32)
    vel = rng.normal(0.0, 5.0, (48, 3))
    dt, tau, B, P0 = 1e-3, 0.05, 500.0, 80.0
    _, _, _, ek, box1, _ = O.md_npt(m, pos, vel, types, box, (0.0, 0.0, 0.0), dt, 1, (P0, tau, B, 1))
    P = 2.0 * ek[0] / (3.0 * np.prod(box)) * EV_A3_BAR
    mu3 = 1.0 - (dt / tau) * (P0 - P) / B
    assert (box1[0] / box[0]) ** 3 == pytest.approx(mu3, rel=1e-12)
    assert abs(mu3 - 1.0) > 1e-3  # the coupling moved the cell measurably


def test_metal_factor_value():
    """The derived factors themselves, to the digits LAMMPS quotes for metal units."""
    assert C_METAL == pytest.approx(9648.53321, rel=1e-8)
    assert EV_A3_BAR == pytest.approx(1.602176634e6, rel=1e-15)
