"""The K matvec's construction (csrc/kmatvec.cu) restated in NumPy and run on the CPU with the
compiled block table (csrc/kblock.h): the 30 tensors embedded into full circulants with the
table's reflection parities at negative offsets, the signed 12 x 12 block at every
frequency point, and the inverse transform taken as conj(FFT(conj(.))) / (Lx Ly Lz).  It must
reproduce the oracle's K operator, which embeds all 144 entries at every offset."""

import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import green as G
from oracle import operator as O
from synth import Grid, random_coefficients

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DRIVER = r"""
#include <cstdio>
#include "kblock.h"
int main() {
    for (int a = 0; a < 12; ++a)
        for (int b = 0; b < 12; ++b)
            std::printf("%d %d %d %d %d %d %d\n", a, b, kblock::tensor(a, b), kblock::sign(a, b),
                        kblock::reflection(a, b, 0), kblock::reflection(a, b, 1), kblock::reflection(a, b, 2));
}
"""
LL = [(1, 1), (1, 2), (1, 3), (1, 4), (2, 2), (2, 3), (2, 4), (3, 3), (3, 4), (4, 4)]


def next_pow2(v):
    n = 2
    while n < v:
        n *= 2
    return n


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("kmv")
    (d / "main.cpp").write_text(DRIVER)
    subprocess.run(["g++", "-std=c++17", "-I", os.path.join(ROOT, "paper_1902_02196_gb300", "csrc"),
                    str(d / "main.cpp"), "-o", str(d / "kb")], check=True)
    out = subprocess.run([str(d / "kb")], capture_output=True, text=True, check=True).stdout
    return {(r[0], r[1]): r[2:] for r in ([int(v) for v in ln.split()] for ln in out.strip().splitlines())}


def embed_axis(n, L):
    """Per circulant position j: (offset |d|, True when the offset is negative) or None (zero)."""
    out = []
    for j in range(L):
        out.append((j, False) if j < n else ((L - j, True) if j > L - n else None))
    return out


@pytest.mark.parametrize("shape,nrhs", [((4, 3, 5), 2), ((3, 5, 2), 1)])
def test_k_matvec_construction(table, shape, nrhs):
    g = Grid(*shape, 0.004, 0.005, 0.0045)
    k0 = O.k0_of(298e6)
    nx, ny, nz = shape
    L = (next_pow2(2 * nx - 1), next_pow2(2 * ny - 1), next_pow2(2 * nz - 1))
    dz, dy, dx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    D = np.stack([dx.ravel(), dy.ravel(), dz.ravel()], 1)
    K = G.k_entries((g.dx, g.dy, g.dz), k0, D)
    P = np.zeros((30, nz, ny, nx), dtype=complex)
    for j in range(3):
        for lli, (la, lb) in enumerate(LL):
            P[10 * j + lli] = K[4 * ((j + 1) % 3) + la - 1, 4 * ((j + 2) % 3) + lb - 1].reshape(nz, ny, nx)
    axes = [embed_axis(n, Ln) for n, Ln in zip(shape, L)]
    C = np.zeros((30, L[2], L[1], L[0]), dtype=complex)
    for t in range(30):
        jd, ll = divmod(t, 10)
        la, lb = LL[ll]
        refl = table[(4 * ((jd + 1) % 3) + la - 1, 4 * ((jd + 2) % 3) + lb - 1)][2:]
        for jz, ez in enumerate(axes[2]):
            for jy, ey in enumerate(axes[1]):
                for jx, ex in enumerate(axes[0]):
                    if ez is None or ey is None or ex is None:
                        continue
                    sgn = np.prod([refl[i] for i, e in enumerate((ex, ey, ez)) if e[1]])
                    C[t, jz, jy, jx] = sgn * P[t, ez[0], ey[0], ex[0]]
    KS = np.fft.fftn(C, axes=(-3, -2, -1))
    x = random_coefficients(g, nrhs, seed=31)
    W = np.zeros((nrhs, 12, L[2], L[1], L[0]), dtype=complex)
    W[..., :nz, :ny, :nx] = x
    W = np.fft.fftn(W, axes=(-3, -2, -1))
    Y = np.zeros_like(W)
    for (a, b), (t, s, *_) in table.items():
        if t >= 0:
            Y[:, a] += s * KS[t] * W[:, b]
    Y = np.conj(np.fft.fftn(np.conj(Y / np.prod(L)), axes=(-3, -2, -1)))
    y = Y[..., :nz, :ny, :nx]
    ref = O.KOperator(g, k0).apply(x)
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)
