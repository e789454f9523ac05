// Block structure of the K operator (K u = curl S u, Eq. 8) on the PWL functions (Eq. 19-22):
// the 12 x 12 Galerkin block K^{(p,l),(q,l')}(d) (Eq. 25) in terms of the 30 tensors
// P_t(d) = int int (d_j N^l) g N^l' for t = 10 j + ll(l, l'), l <= l', stored for d >= 0
// (vie_green_toeplitz_k).  Plain C++ (no CUDA types), for the device kernels and host tests.
//
//   K^{(p,l),(q,l')}(d) = -eps_pjq P_j^{l l'}(d), j the third axis; zero when p = q.
//   For l > l' the pair is stored as (l', l): reflecting all three axes maps d to -d and
//   multiplies P_j^{l l'} by -(-1)^{[l > 1] + [l' > 1]}, and swapping the two voxels gives
//   P_j^{l' l}(d) = -P_j^{l l'}(-d), so P_j^{l l'}(d) = (-1)^{[l > 1] + [l' > 1]} P_j^{l' l}(d).
//   Reflection of axis i (circulant embedding): K^{ab}(R_i d) = -s^i_a s^i_b K^{ab}(d), with the
//   parities s^i_(p,l) = (-1)^[p = i] (-1)^[l linear along i] of the N operator.
#pragma once

#ifdef __CUDACC__
#define KBLOCK_HD __host__ __device__
#else
#define KBLOCK_HD
#endif

namespace kblock {

KBLOCK_HD constexpr int levi_civita(int p, int j, int q) {
    return (p == j || j == q || p == q) ? 0 : (((j - p + 3) % 3 == 1) ? 1 : -1);
}

// index of the ordered scalar pair (l, l'), 1-based, l <= l': (1,1),(1,2),(1,3),(1,4),(2,2),...,(4,4)
KBLOCK_HD constexpr int ll_pair(int l, int lp) {
    return l > lp ? ll_pair(lp, l) : (l == 1 ? lp - 1 : (l == 2 ? 2 + lp : (l == 3 ? 4 + lp : 9)));
}

// stored tensor of entry (a, b), a = 4 p + l - 1, b = 4 q + l' - 1; -1 when the entry is zero (p = q)
KBLOCK_HD constexpr int tensor(int a, int b) {
    const int p = a / 4, q = b / 4;
    return p == q ? -1 : 10 * (3 - p - q) + ll_pair(a % 4 + 1, b % 4 + 1);
}

// sign s with K^{ab}(d) = s P_tensor(a,b)(d); 0 when the entry is zero
KBLOCK_HD constexpr int sign(int a, int b) {
    const int p = a / 4, q = b / 4, l = a % 4 + 1, lp = b % 4 + 1;
    if (p == q) return 0;
    const int e = -levi_civita(p, 3 - p - q, q);
    const int swap = (l > lp && ((l > 1) + (lp > 1)) % 2 == 1) ? -1 : 1;
    return e * swap;
}

// reflection parity of entry (a, b) under x_i -> -x_i (the curl's extra sign times N's parities)
KBLOCK_HD constexpr int reflection(int a, int b, int i) {
    const int pa = ((a / 4 == i) ? -1 : 1) * ((a % 4 == i + 1) ? -1 : 1);
    const int pb = ((b / 4 == i) ? -1 : 1) * ((b % 4 == i + 1) ? -1 : 1);
    return -pa * pb;
}

// every stored tensor is used, by 96 non-zero entries in all (12 x 12 minus the 3 diagonal 4 x 4 blocks)
constexpr bool table_complete() {
    int used[30] = {};
    int nonzero = 0;
    for (int a = 0; a < 12; ++a)
        for (int b = 0; b < 12; ++b) {
            const int t = tensor(a, b);
            if (t < 0) continue;
            if (t >= 30 || sign(a, b) == 0) return false;
            ++used[t];
            ++nonzero;
        }
    for (int t = 0; t < 30; ++t)
        if (used[t] == 0) return false;
    return nonzero == 96;
}

}  // namespace kblock
