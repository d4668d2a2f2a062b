"""Pins the oracle's Philox-4x32-10 (Salmon et al., SC'11) against NVIDIA's
independent implementation in the CUDA toolkit header curand_philox4x32_x.h,
compiled for the host with nvcc (no GPU needed)."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_host():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp(prefix="crbm_philox_")
    exe = os.path.join(d, "curand_philox_host")
    subprocess.check_call([nvcc, "-O1", "-o", exe, os.path.join(HERE, "curand_philox_host.cu")])
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def _cases():
    rng = np.random.default_rng(20251120)
    cases = [(0, 0, 0, 0, 0, 0), (0xFFFFFFFF,) * 6, (1, 2, 3, 4, 5, 6),
             (0, 0, 0, 5, 1, 0), (80, 99999, 4095, 4, 0xDEADBEEF, 0x12345678)]
    for _ in range(400):
        cases.append(tuple(int(x) for x in rng.integers(0, 2**32, size=6, dtype=np.uint64)))
    return cases


def test_oracle_philox_matches_cuda_header(orc, curand_host):
    cases = _cases()
    inp = "".join("%x %x %x %x %x %x\n" % c for c in cases)
    out = subprocess.run([curand_host], input=inp, capture_output=True, text=True, check=True)
    lines = out.stdout.strip().split("\n")
    assert len(lines) == len(cases)
    for c, line in zip(cases, lines):
        ref = [int(x, 16) for x in line.split()]
        assert orc.philox(c[:4], c[4:]) == ref, c


def test_philox_counter_and_key_sensitivity(orc):
    base = orc.philox([7, 8, 9, 10], [11, 12])
    for i in range(4):
        ctr = [7, 8, 9, 10]
        ctr[i] ^= 1
        assert orc.philox(ctr, [11, 12]) != base
    assert orc.philox([7, 8, 9, 10], [11, 13]) != base
