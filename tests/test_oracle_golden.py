"""Regression pin: the oracle reproduces its stored output on the 256x256
workload image (tests/golden/oracle_256x256.json, written by
tests/golden/make_golden.py from the oracle alone).  The paper prints no
worked example, so this fixture freezes the oracle after its independent pins
passed; any later change to its arithmetic must regenerate it deliberately."""
import json
import os

import numpy as np
import pytest

from paper_1706_06750_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_stored_golden(oracle_mod):
    with open(os.path.join(HERE, "golden", "oracle_256x256.json")) as f:
        gold = json.load(f)
    img = synth.workload_image("256x256")
    opt = oracle_mod.Options.make(octaves=2, sublevels=4)
    lv, D, kp, k = oracle_mod.kaze_detect(img, opt)
    assert k == pytest.approx(gold["k"], rel=1e-12)
    mean = lv.reshape(lv.shape[0], -1).mean(axis=1)
    assert np.allclose(mean, gold["level_mean"], rtol=1e-12, atol=0)
    chk = [float(np.sum(lv[i] * lv[i])) for i in range(lv.shape[0])]
    assert np.allclose(chk, gold["level_checksum"], rtol=1e-12, atol=0)
    assert np.allclose([D[i].max() for i in range(D.shape[0])], gold["doh_max"], rtol=1e-10)
    got = [[int(r["level"]), int(r["iy"]), int(r["ix"])] for r in kp]
    assert got == [g[:3] for g in gold["keypoints"]]
    assert np.allclose([[r["x"], r["y"]] for r in kp], [g[3:5] for g in gold["keypoints"]],
                       atol=1e-9)


def test_oracle_fed_and_description_match_stored_golden(oracle_mod):
    """The same freeze for the FED evolution (Eq. 5) of the workload and the
    orientation and descriptor (Sec. II-C) of its first AOS keypoints
    (tests/golden/oracle_fed_describe_256x256.json, from the oracle alone)."""
    from oracle import describe as od
    with open(os.path.join(HERE, "golden", "oracle_fed_describe_256x256.json")) as f:
        gold = json.load(f)
    img = synth.workload_image("256x256")
    fopt = oracle_mod.Options.make(octaves=2, sublevels=4, scheme=oracle_mod.SCHEME_FED)
    flv, fD, fkp, fk = oracle_mod.kaze_detect(img, fopt)
    g = gold["fed"]
    assert fk == pytest.approx(g["k"], rel=1e-12)
    assert np.allclose(flv.reshape(flv.shape[0], -1).mean(axis=1), g["level_mean"], rtol=1e-12, atol=0)
    assert np.allclose([float(np.sum(flv[i] * flv[i])) for i in range(flv.shape[0])], g["level_checksum"],
                       rtol=1e-12, atol=0)
    assert [[int(r["level"]), int(r["iy"]), int(r["ix"])] for r in fkp] == g["keypoints"]
    lv, _, _, _ = oracle_mod.kaze_detect(img, oracle_mod.Options.make(octaves=2, sublevels=4))
    sig, _ = oracle_mod.scale_table(2, 4, 1.6)
    for row in gold["describe"]:
        level, x, y, angle, ref = row[0], row[1], row[2], row[3], np.array(row[4:])
        a, d = od.describe_level(lv[level], float(sig[level]), [(x, y)])
        assert abs(a[0] - angle) <= 1e-12 and np.max(np.abs(d[0] - ref)) <= 1e-12
