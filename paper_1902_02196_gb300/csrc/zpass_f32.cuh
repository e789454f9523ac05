// FP32 z pass with the fused 12 x 12 block product (zpass_f32.cu).
#pragma once

#include "common.cuh"

struct ZFArgs {
    float2* w;                    // spectrum [R*12][Nz][Ly][Lx], in place
    const float2* green_t;        // [Oy][Ox][Oz][60] (N), [Oy][Ox][Oz][30] (K)
    const int* colkx;             // [Lx] kx of each stored column
    int R, nz, Lx, Ly, Ox, Oy, Oz;
    int ay, by;                   // split of Ly: row py holds ky = py / by + ay * (py % by)
    unsigned mx, my, mz;
    // optional: right-hand sides transformed = min(*nact, R) (a count kept on the device), with
    // the launch's algorithmic bytes added to *bctr
    const int* nact;
    unsigned long long* bctr;
};

// Launches the z pass (Lz in 8..512, Lx >= 4) on a spectrum whose row py holds
// ky = py / by + ay (py % by) and whose stored columns follow colkx (mirror pairs).
int zpass_f32_fused(const vie_handle* h, const ZFArgs& z, cudaStream_t s);
// The same z pass with the K block (VIE_OP_K): green_t then holds the K octant [Oy][Ox][Oz][30].
int zpass_f32_fused_k(const vie_handle* h, const ZFArgs& z, cudaStream_t s);
// Autotuner measurement of the z passes' tile widths outside any stream capture (autotune.h).
int zpass_f32_tune(const vie_handle* h, const ZFArgs& z, cudaStream_t s);
int zpass_f32_tune_k(const vie_handle* h, const ZFArgs& z, cudaStream_t s);
