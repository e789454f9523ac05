// Line transforms of the matvec's line path with the two-pass register FFT (line2.cu).
#pragma once

#include "fft.cuh"

// FFT lengths the two-pass line kernels take (8..512, powers of two)
bool line2_ok(int L);

// Forward transform of the lines of `a` (natural order in, a.n_in <= L/2 elements, the rest
// zero): every frequency stored, at position q = colkx^-1 (colkx[q] = the frequency stored at q)
// or, with colkx NULL, in fft2's transposed order.  FP64 (double pairs) or FP32 (float pairs).
int line2_forward(const char* name, const vie_handle* h, int L, bool fp64, const LineArgs& a, const int* colkx,
                  cudaStream_t s);

// Inverse (unnormalised) transform of the lines of `a`, spectrum in the order line2_forward
// stores, outputs l < a.n_out (<= L/2) written in natural order.
int line2_inverse(const char* name, const vie_handle* h, int L, bool fp64, const LineArgs& a, const int* colkx,
                  cudaStream_t s);
