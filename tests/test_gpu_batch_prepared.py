"""Prepared batch: one batch layout tuned once (persistent vs
one-CTA-per-cell launch, staging tile), captured as one CUDA graph and
replayed on new coordinates. Checked against the oracle per structure and
against the eager batched call."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_11311_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_TOL, F_RMS_TOL = 5e-4, 1e-3


@pytest.fixture(scope="module")
def gpu_mod():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2107_11311_gb300 import aenet
    return aenet


def _device_batch(structs):
    off, pos, types, boxes = inputs.concat(structs)
    S, N = len(structs), int(off[-1])
    d = dict(pos=torch.tensor(pos, device="cuda"), types=torch.tensor(types, device="cuda"),
             energies=torch.zeros(S, dtype=torch.float64, device="cuda"),
             forces=torch.zeros((N, 3), dtype=torch.float64, device="cuda"),
             virials=torch.zeros((S, 3, 3), dtype=torch.float64, device="cuda"))
    return off, boxes, d


def _check_against_oracle(m, structs, off, pos, d):
    for s, st in enumerate(structs):
        p = pos[off[s]:off[s + 1]]
        ref = O.compute(m, p, st.types, st.box)
        assert abs(d["energies"][s].item() - ref["energy"]) / max(st.n, 1) <= E_TOL
        df = d["forces"][off[s]:off[s + 1]].cpu().numpy() - ref["forces"]
        if st.n:
            assert np.sqrt((df ** 2).mean()) <= F_RMS_TOL
        np.testing.assert_allclose(d["virials"][s].cpu().numpy(), ref["virial"],
                                   atol=1e-4 * max(1.0, np.abs(ref["virial"]).max()))


@pytest.mark.parametrize("family", ["water", "amorphous"])
def test_prepared_batch_tunes_replays_and_matches_oracle(gpu_mod, family):
    wat, amo = inputs.batch_structures(limit=5)
    structs = wat if family == "water" else amo + [inputs.amorphous(32, seed=4)]
    m = inputs.make_model(family)
    off, boxes, d = _device_batch(structs)
    g = gpu_mod.AenetGPU(m, "fp32")
    tun = g.batch_prepare(off, boxes, d["pos"], d["types"], d["energies"], d["forces"], d["virials"])
    print(f"{family}: tuned launch {tun}")
    assert tun["tile"] in (256, 512, 1024, 2048) and tun["ctas"] >= 1 and tun["kernels"] >= 5 and tun["ms"] > 0
    for k in d:
        if k not in ("pos", "types"):
            d[k].zero_()
    g.batch_run()
    torch.cuda.synchronize()
    g.check()
    pos0 = d["pos"].cpu().numpy()
    _check_against_oracle(m, structs, off, pos0, d)
    # new coordinates in the same buffer: the replay reads them
    rng = np.random.default_rng(7)
    pos1 = pos0 + rng.uniform(-0.05, 0.05, pos0.shape)
    d["pos"].copy_(torch.tensor(pos1))
    g.batch_run()
    torch.cuda.synchronize()
    g.check()
    _check_against_oracle(m, structs, off, pos1, d)


def test_prepared_batch_equals_eager_batch_and_survives_reallocation(gpu_mod):
    wat, _ = inputs.batch_structures(limit=8)
    m = inputs.make_model("water")
    off, boxes, d = _device_batch(wat)
    g = gpu_mod.AenetGPU(m, "fp32")
    tun = g.batch_prepare(off, boxes, d["pos"], d["types"], d["energies"], d["forces"], d["virials"],
                          autotune=False)
    assert tun["persistent"]
    g.batch_run()
    torch.cuda.synchronize()
    eager = g.compute_batch(off, d["pos"].cpu().numpy(), d["types"].cpu().numpy(), boxes)
    # equal up to the run-dependent order of FP32 sums (atom order inside a cell)
    np.testing.assert_allclose(d["energies"].cpu().numpy(), eager["energies"], rtol=2e-7, atol=1e-6)
    np.testing.assert_allclose(d["forces"].cpu().numpy(), eager["forces"], atol=1e-4)
    # a larger system on the same context regrows the work buffers; the next
    # replay must capture again instead of using the old addresses
    big = inputs.water_12288()
    g.compute(big.pos, big.types, big.box)
    E_before = d["energies"].clone()
    d["energies"].zero_()
    g.batch_run()
    torch.cuda.synchronize()
    g.check()
    # same layout, same coordinates: equal up to the run-dependent order of FP32 sums
    torch.testing.assert_close(d["energies"], E_before, rtol=2e-7, atol=1e-6)


def test_prepared_batch_errors(gpu_mod):
    m = inputs.make_model("water")
    g = gpu_mod.AenetGPU(m, "fp32")
    with pytest.raises(gpu_mod.AenetError) as ei:
        g.batch_run()
    assert ei.value.code == -8  # AENET_E_STATE: nothing prepared
    a = inputs.water(3, 8.0, seed=1)
    off, pos, types, boxes = inputs.concat([a])
    with pytest.raises(gpu_mod.AenetError) as ei:  # host buffers are refused
        g.batch_prepare(off, boxes, pos, types)
    assert ei.value.code == -1


def test_full_batch_512_in_the_benchmark_launch(gpu_mod):
    """The benchmark's batch_512 workload at full size, prepared and replayed as
    the benchmark times it (tuned launch, one graph per model family): a seeded
    sample of structures per family (with the largest and the smallest) against
    the oracle, and on every structure finite energies and a net force that
    vanishes up to FP32 rounding."""
    wat, amo = inputs.batch_structures()
    rng = np.random.default_rng(7)
    for family, structs in (("water", wat), ("amorphous", amo)):
        m = inputs.make_model(family)
        off, boxes, d = _device_batch(structs)
        g = gpu_mod.AenetGPU(m, "fp32")
        g.batch_prepare(off, boxes, d["pos"], d["types"], d["energies"], d["forces"], d["virials"])
        g.batch_run()
        torch.cuda.synchronize()
        g.check()
        E = d["energies"].cpu().numpy()
        F = d["forces"].cpu().numpy()
        assert np.isfinite(E).all() and np.isfinite(F).all()
        for s, st in enumerate(structs):
            net = F[off[s]:off[s + 1]].sum(axis=0)
            assert np.abs(net).max() <= 5e-3 * np.sqrt(st.n), (family, s, net)
        sizes = np.array([st.n for st in structs])
        pick = {int(np.argmax(sizes)), int(np.argmin(sizes))} | set(int(i) for i in rng.choice(len(structs), 6,
                                                                                                 replace=False))
        pos = d["pos"].cpu().numpy()
        _check_against_oracle(m, [structs[i] for i in sorted(pick)],
                              np.concatenate([[0], np.cumsum([structs[i].n for i in sorted(pick)])]),
                              np.concatenate([pos[off[i]:off[i + 1]] for i in sorted(pick)]),
                              {k: _take(v, off, sorted(pick), k) for k, v in d.items()})


def _take(t, off, picks, key):
    """The rows of the picked structures (per-structure or per-atom tensors)."""
    if key in ("energies", "virials"):
        return t[picks]
    return torch.cat([t[off[i]:off[i + 1]] for i in picks])
