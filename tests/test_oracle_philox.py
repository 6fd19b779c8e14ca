"""Oracle pins: Philox4x32-10 known-answer vectors and normal statistics."""
import json
import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")


def test_known_answer_vectors():
    for case in json.load(open(GOLDEN))["cases"]:
        ctr = [np.array([int(x, 16)], dtype=np.uint32) for x in case["ctr"]]
        key = [int(x, 16) for x in case["key"]]
        out = philox.philox4x32_10(*ctr, *key)
        assert [f"{int(o[0]):08x}" for o in out] == case["out"]


def test_normals_statistics_and_independence():
    z = philox.complex_noise(seed=123, sample=5, stream=0, n=200000)
    re, im = z.real, z.imag
    for v in (re, im):
        assert abs(v.mean()) < 0.01 and abs(v.std() - 1.0) < 0.01
        # fourth moment of a standard normal is 3
        assert abs(np.mean(v ** 4) - 3.0) < 0.05
    assert abs(np.corrcoef(re, im)[0, 1]) < 0.01
    other = philox.complex_noise(seed=123, sample=6, stream=0, n=1000)
    assert abs(np.corrcoef(z[:1000].real, other.real)[0, 1]) < 0.1
    # deterministic and prefix-stable (element i does not depend on n)
    assert np.array_equal(philox.complex_noise(123, 5, 0, 7), z[:7])
