"""The oracle's Philox4x32-10 against a second independent implementation,
cuRAND's device block function (curand_Philox4x32_10, called from a tiny
CUDA checker built here), on the same (seed, counter, attempt, domain)
cases as the ATen check, including both domains of the packed keying."""
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path_factory.mktemp("curand") / "philox_curand_check")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O1",
                        os.path.join(HERE, "philox_curand_check.cu"), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-500:]
    return exe


def test_philox_matches_curand(orc, curand_checker):
    rng = np.random.default_rng(2011)
    cases = []
    for g in (0, 1, 2**32 - 1, 2**32, 2**64 - 1, 2**63):
        for seed in (0, 0x0123456789ABCDEF, 2**64 - 1):
            for a in (0, 1, 2**31 + 5):
                for dom in (0, 1):
                    cases.append((seed, g, a, dom))
    for _ in range(3000):
        cases.append((int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2)),
                      int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2)),
                      int(rng.integers(0, 64)), int(rng.integers(0, 2))))
    inp = "\n".join(f"{s} {g} {a} {d}" for s, g, a, d in cases) + "\n"
    out = subprocess.run([curand_checker], input=inp, capture_output=True, text=True,
                         check=True, timeout=120).stdout
    ref = [tuple(int(v) for v in line.split()) for line in out.strip().splitlines()]
    assert len(ref) == len(cases)
    for (s, g, a, d), r in zip(cases, ref):
        mine = orc.philox([g & 0xFFFFFFFF, g >> 32, d, a], [s & 0xFFFFFFFF, s >> 32])
        assert mine == r, (s, g, a, d)
