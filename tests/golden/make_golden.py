"""Write the stored expected values in this folder from the CPU oracle.

Test infrastructure.  Calls only oracle/ (and the seeded input generators of
synthetic_inputs); nothing here comes from the CUDA library.  Re-run after a
change of the oracle's arithmetic that a passage of the paper justifies:

    python tests/golden/make_golden.py [case ...]

Each JSON file holds one workload's oracle results: per level the selected
counts m_i = min(nev_max, #{lambda < eta}) (Eq. coarse_space_def) and the
selected eigenvalues with the next one (Eq. theGEVP, exact dense GEVP), the
coarse dimensions, and the CG iteration counts to relative residuals 1e-8 and
1e-12 with x^0 = 0 (Section 5's stopping rule) and the 2-norm of the 1e-12
solution.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic_inputs as si  # noqa: E402
from oracle import fem, method  # noqa: E402

CASES = {
    "channels64": dict(n=(64, 64), parts=(4, 4), overlap=2, levels=2, group=(4, 4), nev=8, eta=0.3,
                       kappa=lambda: si.channels64().coefficient(),
                       recipe="synthetic_inputs.channels64(): kappa = 1, 8 one-element channels of 1e6"),
    "ragged3": dict(n=(52, 44), parts=(6, 5), overlap=2, levels=3, group=(2, 2), nev=6, eta=0.3,
                    kappa=lambda: si.grf_channels_inclusions_2d(52, seed=3, n_channels=3, n_inclusions=4,
                                                                inclusion_side=(3, 6))[: 52 * 44],
                    recipe="grf_channels_inclusions_2d(52, seed=3, n_channels=3, n_inclusions=4, "
                           "inclusion_side=(3, 6)), first 52 x 44 elements"),
    "three_level_3d": dict(n=(8, 8, 8), parts=(4, 4, 4), overlap=1, levels=3, group=(2, 2, 2), nev=4, eta=0.3,
                           kappa=lambda: si.layered_3d(8, seed=2),
                           recipe="layered_3d(8, seed=2): one-element z layers of kappa 1 and 1e4 times "
                                  "exp(0.5 g); null-pivot threshold 1e-6 on the middle level"),
}


def compute(name):
    c = CASES[name]
    mesh = fem.Mesh(c["n"], 0b1)
    H = method.Hierarchy(mesh, c["kappa"](), c["parts"], c["overlap"], c["levels"], c["group"], c["nev"], c["eta"])
    out = {"case": {k: (list(v) if isinstance(v, tuple) else v) for k, v in c.items() if k != "kappa"},
           "levels": {}}
    for l in range(H.L, 0, -1):
        lev = []
        for s in H.levels[l].subs:
            k = min(s["m"] + 1, len(s["lam"]))
            lev.append({"m": int(s["m"]), "lam": [float("%.13g" % v) for v in s["lam"][:k]]})
        out["levels"][str(l)] = lev
    out["coarse_dims"] = {str(k): int(v) for k, v in H.coarse_dims().items()}
    b = fem.load_vector(mesh)
    _, it8, *_ = method.pcg(H.A, b, H.apply_preconditioner, 1e-8)
    x12, it12, *_ = method.pcg(H.A, b, H.apply_preconditioner, 1e-12)
    out["pcg"] = {"iterations_1e-8": int(it8), "iterations_1e-12": int(it12),
                  "x_norm_1e-12": float("%.13g" % np.linalg.norm(x12))}
    return out


def main(names=None):
    for name in names or CASES:
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(compute(name), f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])
