"""The K operator's block table (csrc/kblock.h), compiled with g++ and run on the CPU, against the
oracle's K entries: every entry K^{ab}(d) is sign(a, b) times the stored tensor tensor(a, b)
(zero blocks where p = q), and reflection(a, b, i) is the parity of K^{ab} under x_i -> -x_i."""

import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import green as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "paper_1902_02196_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "kblock.h"
int main() {
    for (int a = 0; a < 12; ++a)
        for (int b = 0; b < 12; ++b)
            std::printf("%d %d %d %d %d %d %d\n", a, b, kblock::tensor(a, b), kblock::sign(a, b),
                        kblock::reflection(a, b, 0), kblock::reflection(a, b, 1), kblock::reflection(a, b, 2));
    return 0;
}
"""

LL = [(1, 1), (1, 2), (1, 3), (1, 4), (2, 2), (2, 3), (2, 4), (3, 3), (3, 4), (4, 4)]


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("kblock")
    (d / "main.cpp").write_text(DRIVER)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", HEADER_DIR, str(d / "main.cpp"), "-o", str(d / "kb")], check=True)
    out = subprocess.run([str(d / "kb")], capture_output=True, text=True, check=True).stdout
    return np.array([[int(v) for v in ln.split()] for ln in out.strip().splitlines()])


def test_entries_from_the_thirty_tensors(table):
    delta = np.array([0.004, 0.005, 0.0045])
    rng = np.random.Generator(np.random.PCG64(11))
    D = rng.integers(0, 4, size=(12, 3))
    D[0] = 0
    K = G.k_entries(delta, 9.0, D)
    # the stored tensors, P_{10 j + ll} = -eps_pjq K^{(p,la),(q,lb)} with (p, j, q) = (j+1, j, j+2) mod 3
    P = np.zeros((30, len(D)), dtype=complex)
    for j in range(3):
        for lli, (la, lb) in enumerate(LL):
            P[10 * j + lli] = K[4 * ((j + 1) % 3) + la - 1, 4 * ((j + 2) % 3) + lb - 1]
    scale = np.max(np.abs(K))
    nonzero = 0
    for a, b, t, s, *_ in table:
        if t < 0:
            assert s == 0 and a // 4 == b // 4
            assert np.max(np.abs(K[a, b])) == 0.0
            continue
        nonzero += 1
        assert s in (-1, 1)
        assert np.max(np.abs(K[a, b] - s * P[t])) < 1e-13 * scale, (a, b, t, s)
    assert nonzero == 96


def test_reflection_parities(table):
    delta = np.array([0.004, 0.005, 0.0045])
    D = np.array([[1, 2, 0], [2, 1, 3], [0, 1, 1], [3, 0, 2]])
    Ds = [D]
    for i in range(3):
        Di = D.copy()
        Di[:, i] *= -1
        Ds.append(Di)
    K = G.k_entries(delta, 9.0, np.concatenate(Ds))
    n = len(D)
    scale = np.max(np.abs(K))
    for a, b, t, s, r0, r1, r2 in table:
        for i, r in enumerate((r0, r1, r2)):
            assert np.max(np.abs(K[a, b, (1 + i) * n:(2 + i) * n] - r * K[a, b, :n])) < 1e-13 * scale
