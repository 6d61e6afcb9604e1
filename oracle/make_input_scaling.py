"""Write the frozen input standardisation of the two basis families.

The paper's networks take a standardised descriptor (trained aenet models store
a per-feature shift and scale with their weights). Without trained models, this
script fixes g = (G - shift) * scale with shift = mean and scale = 1/std of
every descriptor component over one seeded frame, computed by the FP64 oracle
only:

* water:     the 4,096-molecule water box at 1.0 g/cm^3 (seed 10), water basis;
* amorphous: the 27,000-atom 4-species amorphous solid (seed 20), its basis.

Output: ``paper_2107_11311_gb300/input_scaling.json`` (model parameters read by
``inputs.make_model``). Run from the repository root:
``python -m oracle.make_input_scaling``.
"""
import json
import os

import numpy as np

from paper_2107_11311_gb300 import inputs
from oracle import oracle

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2107_11311_gb300", "input_scaling.json")


def stats(family, structure):
    m = inputs.make_model(family, identity_scaling=True)
    r = oracle.compute(m, structure.pos, structure.types, structure.box, mode=oracle.CELLS,
                       want_G=True, want_forces=False)
    G = r["G"]
    mean = G.mean(0)
    std = G.std(0)
    scale = np.where(std > 1e-12, 1.0 / np.maximum(std, 1e-300), 1.0)
    return {"shift": [float(x) for x in mean], "scale": [float(x) for x in scale],
            "frame": f"{structure.n} atoms, box {structure.box[0]:.6f} A"}


def main():
    data = {"water": stats("water", inputs.water_12288()),
            "amorphous": stats("amorphous", inputs.amorphous_27000())}
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
