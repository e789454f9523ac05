// FP64 z pass with the fused 12 x 12 block product (zpass_f64.cu).
#pragma once

#include "common.cuh"

struct ZDArgs {
    double2* w;                // spectrum [R*12][Nz][Ly][Lx], in place
    const double2* green_t;    // [Oy][Ox][Oz][60] (N), [Oy][Ox][Oz][30] (K)
    const int* colkx;          // [Lx] kx of each stored column (mirror pairs)
    int R, nz, Lx, Ly, Ox, Oy, Oz;
    int ay, by;                // row py holds ky = py / by + ay * (py % by)
    unsigned mx, my, mz;
    const int* nact;             // optional device count of the right-hand sides (as ZFArgs)
    unsigned long long* bctr;
};

// Launches the FP64 z pass (Lz in 8..512, Lx >= 4).
int zpass_f64_fused(const vie_handle* h, const ZDArgs& z, cudaStream_t s);
// The same z pass with the K block (VIE_OP_K) on the K octant [Oy][Ox][Oz][30].
int zpass_f64_fused_k(const vie_handle* h, const ZDArgs& z, cudaStream_t s);
