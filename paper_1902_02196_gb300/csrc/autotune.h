// Launch-configuration autotuner of the z-pass kernels (autotune.cu).
#pragma once

#include <functional>
#include <string>

#include "zpass_f32.cuh"

// Index of the configuration (0..n-1) to launch for `key` = (kernel kind, Lz, Lx, Ly, nz) and
// the launch's right-hand side count z.R rounded up to a power of two, at most 8 (rt).  The first
// time a key is seen outside stream capture, every configuration runs launch(c, stream, zt) on a
// scratch spectrum of rt right-hand sides (zeros, allocated for the measurement only) and the one
// with the shortest median device time over three launches is cached for the process.  Under stream capture an unseen key takes configuration 0 and is not
// cached.  label(c) names configuration c in the report.
int autotune_pick(const int key[5], int n, cudaStream_t s,
                  const std::function<int(int, cudaStream_t, const ZFArgs&)>& launch, const ZFArgs& z,
                  const std::function<std::string(int)>& label);
