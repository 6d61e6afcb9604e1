"""Precision forms of the network (Sec. II.A, Eq. ANN-layer): BF16 tensor-core layers with FP32
accumulation, and split BF16 (hi*hi + hi*lo + lo*hi), against the FP64 oracle.

Split BF16 carries ~16 significand bits per operand, so it must meet the FP32
form's bounds (<= 0.5 meV/atom, <= 1 meV/A RMS). Plain BF16 rounds every
network operand to 8 significand bits (relative 2^-9); its errors are reported
and checked only against a bound derived from that rounding: a few tenths of a
percent of the force and energy scales.
"""
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


CASES = {
    "water_192": ("water", inputs.water_192),
    "amorphous_2000": ("amorphous", lambda: inputs.amorphous(2000, seed=5)),
    "amorphous_small_box": ("amorphous", lambda: inputs.amorphous(32, seed=4)),
}


def _errors(got, ref, n):
    de = abs(got["energy"] - ref["energy"]) / n
    df = got["forces"] - ref["forces"]
    return de, float(np.sqrt((df ** 2).mean())), float(np.abs(df).max())


def _ctx(gpu_mod, m, prec, fused):
    g = gpu_mod.AenetGPU(m, prec)
    g.fuse_network(fused)
    return g


# fused: the tensor-core networks inside the fused potential kernel (one
# geometry pass); split: descriptor kernel, network kernel, force kernel
PATHS = [("fused", True), ("split", False)]


@pytest.mark.parametrize("path,fused", PATHS)
@pytest.mark.parametrize("case", list(CASES))
def test_split_bf16_meets_fp32_bounds(gpu_mod, case, path, fused):
    fam, make = CASES[case]
    st = make()
    m = inputs.make_model(fam)
    ref = O.compute(m, st.pos, st.types, st.box)
    got = _ctx(gpu_mod, m, "bf16x3", fused).compute(st.pos, st.types, st.box)
    de, rms, mx = _errors(got, ref, st.n)
    print(f"{case} bf16x3 {path}: |dE|/N {de:.2e} eV, force RMS {rms:.2e} eV/A, max {mx:.2e}")
    assert de <= 5e-4 and rms <= 1e-3 and mx <= 1e-2
    np.testing.assert_allclose(got["virial"], ref["virial"], atol=1e-4 * max(1.0, np.abs(ref["virial"]).max()))
    np.testing.assert_allclose(got["e_atom"], ref["e_atom"], atol=2e-4 * (1 + np.abs(ref["e_atom"]).max()))


@pytest.mark.parametrize("hidden", [(25, 25), (32, 32), (15, 15), (17, 30)])
@pytest.mark.parametrize("path,fused", PATHS)
def test_split_bf16_water_networks(gpu_mod, hidden, path, fused):
    """The water basis with hidden widths 15-32 (both tile widths of the
    tensor-core form, the paper's 52-25-25-1 model and the large box's
    52-32-32-1 network), on the 192-atom box and on the 8-molecule box shorter
    than the cutoff: every output against the oracle."""
    m = inputs.make_model("water", hidden=hidden)
    for st in (inputs.water_192(), inputs.water(8, 6.6, seed=3)):
        ref = O.compute(m, st.pos, st.types, st.box)
        got = _ctx(gpu_mod, m, "bf16x3", fused).compute(st.pos, st.types, st.box)
        de, rms, mx = _errors(got, ref, st.n)
        print(f"water {st.n} {hidden} bf16x3 {path}: |dE|/N {de:.2e}, force RMS {rms:.2e}, max {mx:.2e}")
        assert de <= 5e-4 and rms <= 1e-3 and mx <= 1e-2
        np.testing.assert_allclose(got["virial"], ref["virial"], atol=1e-4 * max(1.0, np.abs(ref["virial"]).max()))


@pytest.mark.parametrize("path,fused", PATHS)
@pytest.mark.parametrize("case", list(CASES))
def test_plain_bf16_error_is_at_the_rounding_level(gpu_mod, case, path, fused):
    fam, make = CASES[case]
    st = make()
    m = inputs.make_model(fam)
    ref = O.compute(m, st.pos, st.types, st.box)
    got = _ctx(gpu_mod, m, "bf16", fused).compute(st.pos, st.types, st.box)
    de, rms, mx = _errors(got, ref, st.n)
    f_scale = float(np.sqrt((ref["forces"] ** 2).mean()))
    print(f"{case} bf16: |dE|/N {de:.2e} eV, force RMS {rms:.2e} eV/A (force RMS {f_scale:.2f}), max {mx:.2e}")
    # 2^-9 relative rounding of inputs and weights through ~3 layers: allow 2 % of the force scale
    assert rms <= 0.02 * f_scale
    assert de <= 0.02 * max(np.abs(ref["e_atom"]).mean(), 0.1)


def test_full_size_amorphous_27000_precision_forms(gpu_mod):
    """The 27,000-atom 4-species solid: FP32 vs BF16 vs split BF16 against FP64."""
    st = inputs.amorphous_27000()
    m = inputs.make_model("amorphous")
    ref = O.compute(m, st.pos, st.types, st.box)
    out = {}
    for prec in ("fp32", "bf16", "bf16x3"):
        got = gpu_mod.AenetGPU(m, prec).compute(st.pos, st.types, st.box)
        out[prec] = _errors(got, ref, st.n)
        print(f"amorphous_27000 {prec}: |dE|/N {out[prec][0]:.2e} eV, force RMS {out[prec][1]:.2e} eV/A, "
              f"max {out[prec][2]:.2e}")
    for prec in ("fp32", "bf16x3"):
        assert out[prec][0] <= 5e-4 and out[prec][1] <= 1e-3


@pytest.mark.parametrize("path,fused", PATHS)
def test_bf16x3_md_matches_oracle_trajectory(gpu_mod, path, fused):
    """10 velocity-Verlet steps at 0.5 fs with split-BF16 networks: per-frame
    energies and final positions against the oracle's own integration."""
    st = inputs.water_192()
    m = inputs.make_model("water", hidden=(32, 32))
    v0 = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=2)
    xo, vo, epo, eko = O.md_nve(m, st.pos, v0, st.types, st.box, 5e-4, 10)
    g = _ctx(gpu_mod, m, "bf16x3", fused)
    pos, vel = st.pos.copy(), v0.copy()
    ep, ek = np.zeros(11), np.zeros(11)
    g.md_nve(pos, vel, st.types, st.box, 5e-4, 10, e_pot=ep, e_kin=ek)
    assert np.abs(ep - epo).max() / st.n <= 5e-4
    np.testing.assert_allclose(ek, eko, rtol=1e-4)
    np.testing.assert_allclose(pos, xo, atol=1e-5)


def test_full_size_water_331776_fused_bf16x3_forces(gpu_mod):
    """The 110,592-molecule box with the 52-32-32-1 network in the fused
    split-BF16 form (the benchmark's launch): forces on 64 seeded atoms and
    their atomic energies against the oracle."""
    st = inputs.water_331776()
    m = inputs.make_model("water", hidden=(32, 32))
    atoms = np.random.default_rng(43).choice(st.n, 64, replace=False)
    Fo, Eo = O.forces_subset(m, st.pos, st.types, st.box, atoms)
    out = _ctx(gpu_mod, m, "bf16x3", True).compute(st.pos, st.types, st.box)
    df = out["forces"][atoms] - Fo
    rms = float(np.sqrt((df ** 2).mean()))
    print(f"water_331776 fused bf16x3: force RMS error on 64 atoms {rms:.2e} eV/A")
    assert rms <= 1e-3 and np.abs(df).max() <= 1e-2
    np.testing.assert_allclose(out["e_atom"][atoms], Eo, atol=2e-4 * (1 + np.abs(Eo).max()))


def test_bf16x3_md_matches_fp32(gpu_mod):
    st = inputs.water_192()
    m = inputs.make_model("water")
    v0 = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=2)
    res = {}
    for prec in ("fp32", "bf16x3"):
        g = gpu_mod.AenetGPU(m, prec)
        pos, vel = st.pos.copy(), v0.copy()
        ep, ek = np.zeros(11), np.zeros(11)
        g.md_nve(pos, vel, st.types, st.box, 5e-4, 10, e_pot=ep, e_kin=ek)
        res[prec] = (pos, ep)
    np.testing.assert_allclose(res["bf16x3"][0], res["fp32"][0], atol=1e-5)
    assert np.abs(res["bf16x3"][1] - res["fp32"][1]).max() / st.n < 5e-4
