"""The pipelined form of the fused FP32 potential kernel (AENET_OPT_PIPELINE)
and the block-synchronous form, each against the FP64 oracle (Sec. II.A-B:
descriptor, network, chain rule to forces and virial).

The cases cover what the pipelined form does differently: items that are whole
cells and halves of cells (the last wave's worth of cells is split), fewer
cells than CTAs, boxes shorter than the cutoff (large image-offset tables), and
neighbourhoods larger than the staging buffer (a dense cluster in a large empty
box), which are scanned straight from global memory. The MD case checks that
the captured step runs the pipelined kernel (path flag) and follows the
oracle's trajectory.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_11311_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_TOL = 5e-4      # eV/atom
F_RMS_TOL = 1e-3  # eV/A


@pytest.fixture(scope="module")
def aenet():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2107_11311_gb300 import aenet as a
    return a


def _cluster():
    """The 192-atom water box without its periodic images in a 40 A box: the
    staging buffer is sized from the mean density (3% of the cluster's), so the
    cluster's cells have neighbourhoods larger than the buffer."""
    st = inputs.water_192()
    return inputs.Structure(pos=st.pos + 10.0, types=st.types, box=np.full(3, 40.0), n_species=st.n_species)


CASES = {
    "water_192": ("water", (15, 15), inputs.water_192),
    "water_192_wide": ("water", (32, 32), inputs.water_192),
    "water_small_box": ("water", (15, 15), lambda: inputs.water(8, 6.6, seed=3)),
    "water_cluster": ("water", (25, 25), _cluster),
    "amorphous_small_box": ("amorphous", None, lambda: inputs.amorphous(32, seed=4)),
    "amorphous_2000": ("amorphous", None, lambda: inputs.amorphous(2000, seed=5)),
    "water_12288": ("water", (15, 15), inputs.water_12288),
    "water_20736": ("water", (32, 32), lambda: inputs.water(6912, None, 10)),
}


def _model(fam, hidden):
    return inputs.make_model(fam) if hidden is None else inputs.make_model(fam, hidden=hidden)


def _check(ref, got, n, what):
    de = abs(got["energy"] - ref["energy"]) / n
    df = got["forces"] - ref["forces"]
    rms = float(np.sqrt((df ** 2).mean()))
    print(f"{what}: |dE|/N {de:.2e} eV, force RMS {rms:.2e} eV/A, max {np.abs(df).max():.2e}")
    assert de <= E_TOL and rms <= F_RMS_TOL and np.abs(df).max() <= 10 * F_RMS_TOL, what
    np.testing.assert_allclose(got["e_atom"], ref["e_atom"], atol=2e-4 * (1 + np.abs(ref["e_atom"]).max()))
    np.testing.assert_allclose(got["virial"], ref["virial"], atol=1e-4 * max(1.0, np.abs(ref["virial"]).max()))


@pytest.mark.parametrize("pipeline", [True, False])
@pytest.mark.parametrize("case", list(CASES))
def test_forms_match_oracle(aenet, case, pipeline):
    fam, hidden, make = CASES[case]
    st = make()
    m = _model(fam, hidden)
    ref = O.compute(m, st.pos, st.types, st.box)
    g = aenet.AenetGPU(m, "fp32")
    g.pipeline(pipeline)
    got = g.compute(st.pos, st.types, st.box)
    _check(ref, got, st.n, f"{case} pipeline={pipeline}")
    g.check()
    # a second evaluation on the same context (the work counters were left at zero)
    _check(ref, g.compute(st.pos, st.types, st.box), st.n, f"{case} pipeline={pipeline}, again")


@pytest.mark.parametrize("pipeline", [True, False])
def test_md_runs_the_selected_form(aenet, pipeline):
    """10 velocity-Verlet steps at 0.5 fs (captured graph): the path flag names
    the form that ran, and energies and positions follow the oracle."""
    st = inputs.water_192()
    m = inputs.make_model("water", hidden=(25, 25))
    v0 = inputs.maxwell_boltzmann(m.masses[st.types], 300.0, seed=2)
    xo, vo, epo, eko = O.md_nve(m, st.pos, v0, st.types, st.box, 5e-4, 10)
    g = aenet.AenetGPU(m, "fp32")
    g.pipeline(pipeline)
    pos, vel = st.pos.copy(), v0.copy()
    ep, ek = np.zeros(11), np.zeros(11)
    g.md_nve(pos, vel, st.types, st.box, 5e-4, 10, e_pot=ep, e_kin=ek)
    assert np.abs(ep - epo).max() / st.n <= E_TOL
    np.testing.assert_allclose(ek, eko, rtol=1e-4)
    np.testing.assert_allclose(pos, xo, atol=1e-5)
    p, v = st.pos.copy(), v0.copy()
    g.md_nve(p, v, st.types, st.box, 5e-4, 1, flags=aenet.AENET_MD_TIMING)
    flags = g.md_path_flags()
    assert flags & aenet.AENET_PATH_FUSED
    assert bool(flags & aenet.AENET_PATH_PIPELINED) == pipeline


def test_activation_records_and_weight_gradient(aenet):
    """dE/dW from the activation records the pipelined form writes, against the
    oracle's back-propagation (Sec. II.C)."""
    st = inputs.water_192()
    m = inputs.make_model("water", hidden=(25, 25))
    g = aenet.AenetGPU(m, "fp32")
    g.keep_activations(True)
    g.compute(st.pos, st.types, st.box)
    got = g.grad_weights()
    ref = O.compute(m, st.pos, st.types, st.box, want_dEdW=True, want_forces=False)["dEdW"]
    err = float(np.abs(got - ref).max() / max(1.0, np.abs(ref).max()))
    print(f"pipelined dE/dW: max error / max |dE/dW| = {err:.2e}")
    assert err < 2e-4
