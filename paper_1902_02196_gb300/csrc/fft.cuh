// Shared-memory Stockham FFT used by every pass of the matvec and by the Green-tensor setup.
//
// A CTA holds a set of lines in shared memory; line (g, tb) has its element l
// at s[g * GS + l * TBP + tb] (tb = index among TB adjacent lines, g = group).
// Each radix-R stage reads R elements per butterfly into registers, applies
// the twiddles and an R-point DFT, and writes them back in self-sorting
// (Stockham) order, so the result is in natural order with no bit reversal
// (Stockham autosort formulation as in Govindaraju et al., SC'08).  Radix 4 is
// used while it divides the remaining length, radix 2 for a last odd stage.
// Twiddles come from a table tw[m] = exp(-2 pi i m / L) computed on the host
// in double precision; the inverse transform uses its conjugate.
#pragma once

#include "common.cuh"

template <typename C>
__device__ __forceinline__ C twiddle(const C* tw, int m, int dir) {
    C w = tw[m];
    return dir < 0 ? w : cconj(w);
}

template <typename C>
__device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3, int dir) {
    C a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = cmul_i(csub(v1, v3), dir);
    v0 = cadd(a0, a2);
    v2 = csub(a0, a2);
    v1 = cadd(a1, a3);
    v3 = csub(a1, a3);
}

// One FFT over G*TB lines of length L held in shared memory, NT threads.
template <typename C, int L, int G, int TB, int TBP, int GS, int NT>
__device__ __forceinline__ void fft_smem(C* s, const C* tw, int dir) {
    const int tid = threadIdx.x;
    constexpr int NB4 = G * TB * (L / 4);
    constexpr int MAXB4 = (NB4 + NT - 1) / NT;
    int Ns = 1;
    if constexpr (L >= 4) {
#pragma unroll 1
    for (; Ns * 4 <= L; Ns *= 4) {
        C v[MAXB4 > 0 ? MAXB4 : 1][4];
        int base[MAXB4 > 0 ? MAXB4 : 1];
#pragma unroll
        for (int i = 0; i < MAXB4; ++i) {
            int bf = tid + i * NT;
            if (bf < NB4) {
                int tb = bf % TB;
                int rest = bf / TB;
                int j = rest % (L / 4);
                int g = rest / (L / 4);
                C* line = s + g * GS + tb;
                int k = j % Ns;
                int step = L / (Ns * 4);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    C x = line[(j + r * (L / 4)) * TBP];
                    v[i][r] = r == 0 ? x : cmul(x, twiddle(tw, k * r * step, dir));
                }
                dft4(v[i][0], v[i][1], v[i][2], v[i][3], dir);
                base[i] = g * GS + tb + ((j / Ns) * Ns * 4 + k) * TBP;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < MAXB4; ++i) {
            int bf = tid + i * NT;
            if (bf < NB4) {
#pragma unroll
                for (int r = 0; r < 4; ++r) s[base[i] + r * Ns * TBP] = v[i][r];
            }
        }
        __syncthreads();
    }
    }
    if (Ns < L) {  // one radix-2 stage, Ns = L / 2
        constexpr int NB2 = G * TB * (L / 2);
        constexpr int MAXB2 = (NB2 + NT - 1) / NT;
        C v[MAXB2][2];
        int base[MAXB2];
#pragma unroll
        for (int i = 0; i < MAXB2; ++i) {
            int bf = tid + i * NT;
            if (bf < NB2) {
                int tb = bf % TB;
                int rest = bf / TB;
                int j = rest % (L / 2);
                int g = rest / (L / 2);
                C* line = s + g * GS + tb;
                int k = j % Ns;
                C x0 = line[j * TBP];
                C x1 = line[(j + L / 2) * TBP];
                if (k) x1 = cmul(x1, twiddle(tw, k * (L / (Ns * 2)), dir));
                v[i][0] = cadd(x0, x1);
                v[i][1] = csub(x0, x1);
                base[i] = g * GS + tb + ((j / Ns) * Ns * 2 + k) * TBP;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < MAXB2; ++i) {
            int bf = tid + i * NT;
            if (bf < NB2) {
                s[base[i]] = v[i][0];
                s[base[i] + Ns * TBP] = v[i][1];
            }
        }
        __syncthreads();
    }
}

// Lines of length L processed TB at a time.  The array is viewed as
// [na][L-axis][nb] with element strides (ia, il, ib) on input and (oa, ol, ob)
// on output; inputs l >= n_in are zero (padding), outputs l >= n_out are not
// stored (cropping).  When il == 1 the TB lines are consecutive inner indices
// whose elements are contiguous, otherwise they are adjacent along the inner
// axis (ib == 1) so that loads of one l coalesce across lines.
// pin / pout (optional, NULL = identity): element l of a line is read from position pin[l]
// / written to position pout[l] (the stored column order of the matvec spectrum).
struct LineArgs {
    const void* in;
    void* out;
    long long ia, il, ib;
    long long oa, ol, ob;
    int na, nb;
    int n_in, n_out;
    int dir;
    const int* pin;
    const int* pout;
};

// Optional epilogue of the last inverse pass of the matvec: crop + material and Gram terms.
struct MatvecEpi {
    const void* x;     // input vector [R][12][Nz][Ny][Nx] (or [R][12][ns] on a support, see Support)
    const void* c1;    // per-voxel complex coefficient multiplying x   (op A: none; op PA: 1/eps)
    const void* c2;    // per-voxel complex coefficient multiplying Nx  (op A: chi; op PA: tau)
    int op;            // VIE_OP_*
    int nx, ny, nz;    // grid
    double g1, g234;   // Gram entries
    const int4* rows;  // support rows (x0, x1, offset) per (z, y) or NULL for the full grid
    long long ns;      // support size (voxels)
    const double2* shift;  // op PA only, optional: y -= shift[r] x per right-hand side r
    void* conv;            // optional: full-grid (N - G) x at every voxel, before the voxel-wise terms
    const int* rmap;       // optional (fused xy path): spectrum right-hand side k holds right-hand side rmap[k]
    // optional with rmap: the number of listed right-hand sides kept on the device (planes of the
    // others are skipped); the launch's algorithmic bytes bfix + bper * count go to *bctr
    const int* nact;
    unsigned long long* bctr;
    double bfix, bper;
    int nc;  // components per voxel and right-hand side: 12 (PWL) or 3 (PWC: the l = 1 functions only)
};

template <int L>
struct LineCfg {
    static constexpr int TB = (4096 / L) > 32 ? 32 : (4096 / L) < 1 ? 1 : (4096 / L);
    static constexpr int TBP = TB + 1;
    static constexpr int NT0 = TB * L / 4;
    static constexpr int NT = NT0 < 64 ? 64 : (NT0 > 512 ? 512 : NT0);
};

template <typename T, int L, bool EPI>
__global__ void __launch_bounds__(LineCfg<L>::NT) line_fft_kernel(LineArgs a, const typename CT<T>::C* twg,
                                                                  MatvecEpi epi) {
    using C = typename CT<T>::C;
    constexpr int TB = LineCfg<L>::TB, TBP = LineCfg<L>::TBP, NT = LineCfg<L>::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    C* tw = s + L * TBP;
    const int tid = threadIdx.x;
    for (int m = tid; m < L; m += NT) tw[m] = twg[m];

    const int ntile = (a.nb + TB - 1) / TB;
    const long long ai = blockIdx.x / ntile;
    const int b0 = (blockIdx.x % ntile) * TB;
    const C* in = reinterpret_cast<const C*>(a.in);
    C* out = reinterpret_cast<C*>(a.out);
    const C zero = mk(T(0), T(0));
    const bool contiguous = a.il == 1;

    for (int idx = tid; idx < L * TB; idx += NT) {
        int l, tb;
        if (contiguous) {
            tb = idx / L;
            l = idx % L;
        } else {
            l = idx / TB;
            tb = idx % TB;
        }
        int b = b0 + tb;
        C v = zero;
        if (l < a.n_in && b < a.nb) v = in[ai * a.ia + (a.pin ? a.pin[l] : l) * a.il + (long long)b * a.ib];
        s[l * TBP + tb] = v;
    }
    __syncthreads();
    fft_smem<C, L, 1, TB, TBP, 0, NT>(s, tw, a.dir);

    for (int idx = tid; idx < L * TB; idx += NT) {
        int l, tb;
        if (contiguous || EPI) {
            tb = idx / L;
            l = idx % L;
        } else {
            l = idx / TB;
            tb = idx % TB;
        }
        int b = b0 + tb;
        if (l >= a.n_out || b >= a.nb) continue;
        C v = s[l * TBP + tb];
        long long o = ai * a.oa + (a.pout ? a.pout[l] : l) * a.ol + (long long)b * a.ob;
        if (EPI && epi.conv) reinterpret_cast<C*>(epi.conv)[o] = v;  // full-grid output: o is the voxel index
        if (EPI) {
            // line b = ((r * nc + alpha) * nz + z) * ny + y, element l = x
            int alpha = (b / (epi.ny * epi.nz)) % epi.nc;
            long long vox = (long long)(b % (epi.ny * epi.nz)) * epi.nx + l;
            C xv = reinterpret_cast<const C*>(epi.x)[o];
            T gl = (T)(comp_is_constant(alpha, epi.nc) ? epi.g1 : epi.g234);
            if (epi.op == VIE_OP_A) {
                C c2 = reinterpret_cast<const C*>(epi.c2)[vox];
                v = csub(mk(gl * xv.x, gl * xv.y), cmul(c2, v));
            } else if (epi.op == VIE_OP_PA) {
                C c1 = reinterpret_cast<const C*>(epi.c1)[vox];
                C c2 = reinterpret_cast<const C*>(epi.c2)[vox];
                C t = cmul(c2, v);
                T ig = T(1) / gl;
                if (epi.shift) {
                    const double2 sh = epi.shift[b / (epi.nc * epi.ny * epi.nz)];
                    c1 = csub(c1, mk((T)sh.x, (T)sh.y));
                }
                v = csub(cmul(c1, xv), mk(ig * t.x, ig * t.y));
            }
        }
        out[o] = v;
    }
}

template <typename T, int L>
inline size_t line_fft_smem_bytes() {
    using C = typename CT<T>::C;
    return sizeof(C) * (size_t)(L * LineCfg<L>::TBP + L);
}
