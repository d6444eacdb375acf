"""Writes the stored expected values under tests/golden/.

Calls only the FP64 oracle (oracle/) and the seeded input generator; never
the CUDA path.  Re-run after a change to the oracle's arithmetic that the
paper justifies, and name that passage in the commit message.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1706_06750_gb300 import synth  # noqa: E402


def main():
    img = synth.workload_image("256x256")
    opt = oracle.Options.make(octaves=2, sublevels=4)
    lv, D, kp, k = oracle.kaze_detect(img, opt)
    out = {
        "workload": "256x256, 2 octaves x 4 sublevels, seed 1000",
        "source": "oracle (FP64), written by tests/golden/make_golden.py",
        "k": k,
        "level_mean": [float(x) for x in lv.reshape(lv.shape[0], -1).mean(axis=1)],
        "level_checksum": [float(np.sum(lv[i] * lv[i])) for i in range(lv.shape[0])],
        "doh_max": [float(D[i].max()) for i in range(D.shape[0])],
        "keypoints": [[int(r["level"]), int(r["iy"]), int(r["ix"]),
                       float(r["x"]), float(r["y"]), float(r["response"])] for r in kp],
    }
    with open(os.path.join(HERE, "oracle_256x256.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")

    # the same workload with the FED evolution (Eq. 5), and the orientation
    # and M-SURF descriptor (Sec. II-C) of the AOS keypoints
    from oracle import describe as od
    fopt = oracle.Options.make(octaves=2, sublevels=4, scheme=oracle.SCHEME_FED)
    flv, fD, fkp, fk = oracle.kaze_detect(img, fopt)
    sig, _ = oracle.scale_table(2, 4, 1.6)
    first = sorted(kp, key=lambda r: (int(r["level"]), int(r["iy"]), int(r["ix"])))[:12]
    desc = []
    for r in first:
        a, d = od.describe_level(lv[int(r["level"])], float(sig[int(r["level"])]), [(float(r["x"]), float(r["y"]))])
        desc.append([int(r["level"]), float(r["x"]), float(r["y"]), float(a[0])] + [float(v) for v in d[0]])
    out2 = {
        "workload": "256x256, 2 octaves x 4 sublevels, seed 1000",
        "source": "oracle (FP64), written by tests/golden/make_golden.py",
        "fed": {
            "k": fk,
            "level_mean": [float(x) for x in flv.reshape(flv.shape[0], -1).mean(axis=1)],
            "level_checksum": [float(np.sum(flv[i] * flv[i])) for i in range(flv.shape[0])],
            "keypoints": [[int(r["level"]), int(r["iy"]), int(r["ix"])] for r in fkp],
        },
        "describe": desc,
    }
    with open(os.path.join(HERE, "oracle_fed_describe_256x256.json"), "w") as f:
        json.dump(out2, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
