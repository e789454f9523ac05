// Green-tensor setup on the GPU, FP64 (Section III-C, Eq. 25, Eq. 34, Eq. 42-43; Section IV-A).
//
// The Galerkin entries of N between PWL functions of voxels at offset d are
//   N^{pl,ql'}(d) = delta_d0 delta_pq delta_ll' G^l + k0^2 delta_pq S^{ll'}(d) - Q^{pl,ql'}(d),
// S the volume-volume integral of g against N^l N^l', Q the integral of g
// against the distributional divergences of the two vector functions (volume
// density plus face densities from their jumps), a consequence of
// (lap + k0^2) g = -delta (Eq. 10).  Every such integral of two product
// densities is an integral over t = s - s' of g(Delta (d + t)) times a product
// of 1-D correlation polynomials W_i(t_i), piecewise cubic with integer
// breakpoints, or a point mass for two parallel faces.  The library therefore
//   1. computes moments of g over every unit cell (3-D) and unit face (2-D) of
//      the offset lattice, mu[a][b][c] = int_cell g xi_x^a xi_y^b xi_z^c, with
//      tensor Gauss-Legendre rules whose order grows near the singular point
//      and, on the cells that touch u = 0, the Duffy transform (three pyramids
//      in 3-D, two triangles in 2-D, Jacobian tau^2 resp. tau cancelling 1/r);
//   2. assembles, per offset d in [0, N)^3, the 60 unique tensors of N - G
//      (6 vector pairs x 10 scalar pairs) as combinations of those moments;
//   3. embeds them in circulants of length L_i (offsets d_i < 0 from the
//      reflection parities), runs the 3-D FFT, keeps the octant k_i in
//      [0, L_i/2] (the rest follows from the same parities) and scales by 1/(Lx Ly Lz).
// The Gram term is left out of the FFT and applied exactly per voxel.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kblock.h"

// ---------------------------------------------------------------------------
// Gauss-Legendre rules on [0, 1], computed on the host by Newton iteration on
// the Legendre three-term recurrence.
// ---------------------------------------------------------------------------
static void gauss_legendre01(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(VIE_PI * (i + 0.75) / (n + 0.5));
        double dp = 0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double pn = n == 1 ? z : p1, pm = n == 1 ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // = 2/((1-z^2) P'^2) on [-1,1], halved for [0,1]
    }
}

// rule table in constant memory: orders and their offsets
constexpr int kNumRules = 7;
constexpr int kOrders[kNumRules] = {6, 7, 9, 12, 14, 12, 16};  // last two: Duffy tau and zeta rules
__constant__ double c_gx[128];
__constant__ double c_gw[128];
__constant__ int c_goff[kNumRules];

enum { R6 = 0, R7, R9, R12, R14, RDT, RDS };

__device__ __forceinline__ int rule_for_ratio(double ratio) {
    return ratio < 1.5 ? R14 : ratio < 3.0 ? R12 : ratio < 6.0 ? R9 : ratio < 12.0 ? R7 : R6;
}
__device__ __forceinline__ int rule_n(int r) {
    return r == R6 ? 6 : r == R7 ? 7 : r == R9 ? 9 : r == R12 ? 12 : r == R14 ? 14 : r == RDT ? 12 : 16;
}

struct GreenGeo {
    int nx, ny, nz;
    double d[3];
    double k0;
};

__device__ __forceinline__ double2 gfun(double r, double k0) {
    double s, c;
    sincos(k0 * r, &s, &c);
    double f = 1.0 / (4.0 * VIE_PI * r);
    return make_double2(c * f, -s * f);
}

// 3-D cell moments: thread per (cell, a); cells k in [-1, N-1]^3.
__global__ void moments3_kernel(GreenGeo g, double2* __restrict__ mu) {
    const long long ncell = (long long)(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= ncell * 4) return;
    const int a = (int)(gid & 3);
    const long long cell = gid >> 2;
    const int kx = (int)(cell % (g.nx + 1)) - 1;
    const int ky = (int)((cell / (g.nx + 1)) % (g.ny + 1)) - 1;
    const int kz = (int)(cell / ((long long)(g.nx + 1) * (g.ny + 1))) - 1;
    const int k[3] = {kx, ky, kz};
    double2 acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = make_double2(0, 0);
    const bool touching = (kx == 0 || kx == -1) && (ky == 0 || ky == -1) && (kz == 0 || kz == -1);
    if (!touching) {
        double dist2 = 0, dmax = fmax(g.d[0], fmax(g.d[1], g.d[2]));
        for (int i = 0; i < 3; ++i) {
            int e = k[i] >= 0 ? k[i] : -k[i] - 1;
            dist2 += (e * g.d[i]) * (e * g.d[i]);
        }
        const int rule = rule_for_ratio(sqrt(dist2) / dmax);
        const int n = rule_n(rule), off = c_goff[rule];
        for (int i = 0; i < n; ++i) {
            const double xi = c_gx[off + i], wx = c_gw[off + i];
            const double ux = g.d[0] * (kx + xi);
            double xa = 1.0;
            for (int p = 0; p < a; ++p) xa *= xi;
            for (int j = 0; j < n; ++j) {
                const double yj = c_gx[off + j], wy = c_gw[off + j];
                const double uy = g.d[1] * (ky + yj);
                double yb[4] = {1.0, yj, yj * yj, yj * yj * yj};
                double2 t[4] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
                for (int l = 0; l < n; ++l) {
                    const double zl = c_gx[off + l], wz = c_gw[off + l];
                    const double uz = g.d[2] * (kz + zl);
                    double2 gv = gfun(sqrt(ux * ux + uy * uy + uz * uz), g.k0);
                    double zc = wz;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        t[c].x = fma(zc, gv.x, t[c].x);
                        t[c].y = fma(zc, gv.y, t[c].y);
                        zc *= zl;
                    }
                }
                const double f = wx * wy * xa;
#pragma unroll
                for (int b = 0; b < 4; ++b)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        acc[b * 4 + c].x = fma(f * yb[b], t[c].x, acc[b * 4 + c].x);
                        acc[b * 4 + c].y = fma(f * yb[b], t[c].y, acc[b * 4 + c].y);
                    }
            }
        }
    } else {
        // Duffy: eta = distance from the singular vertex per axis; pyramid m has eta_m = tau.
        const int nt = rule_n(RDT), ns = rule_n(RDS), ot = c_goff[RDT], os = c_goff[RDS];
        for (int m = 0; m < 3; ++m) {
            const int o1 = m == 0 ? 1 : 0, o2 = m == 2 ? 1 : 2;
            for (int it = 0; it < nt; ++it) {
                const double tau = c_gx[ot + it], wt = c_gw[ot + it] * tau * tau;
                for (int i1 = 0; i1 < ns; ++i1) {
                    const double z1 = c_gx[os + i1], w1 = c_gw[os + i1];
                    for (int i2 = 0; i2 < ns; ++i2) {
                        const double z2 = c_gx[os + i2], w2 = c_gw[os + i2];
                        double eta[3];
                        eta[m] = tau;
                        eta[o1] = tau * z1;
                        eta[o2] = tau * z2;
                        double r2 = 0, xi[3];
                        for (int q = 0; q < 3; ++q) {
                            r2 += (g.d[q] * eta[q]) * (g.d[q] * eta[q]);
                            xi[q] = k[q] == 0 ? eta[q] : 1.0 - eta[q];
                        }
                        double2 gv = gfun(sqrt(r2), g.k0);
                        double f = wt * w1 * w2;
                        for (int p = 0; p < a; ++p) f *= xi[0];
                        double yb = 1.0;
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            double zc = 1.0;
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                acc[b * 4 + c].x = fma(f * yb * zc, gv.x, acc[b * 4 + c].x);
                                acc[b * 4 + c].y = fma(f * yb * zc, gv.y, acc[b * 4 + c].y);
                                zc *= xi[2];
                            }
                            yb *= xi[1];
                        }
                    }
                }
            }
        }
    }
    double2* out = mu + cell * 64 + a * 16;
#pragma unroll
    for (int i = 0; i < 16; ++i) out[i] = acc[i];
}

// 2-D face moments for faces normal to `axis`: levels lev in [-1, N_axis], in-plane
// cells kj in [-1, N_j - 1], kk in [-1, N_k - 1] (j < k the other axes); thread per (face, a).
__global__ void moments2_kernel(GreenGeo g, int axis, double2* __restrict__ mu) {
    const int j = axis == 0 ? 1 : 0, k = axis == 2 ? 1 : 2;
    const int n[3] = {g.nx, g.ny, g.nz};
    const long long nj = n[j] + 1, nk = n[k] + 1, nl = n[axis] + 2;
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= nl * nj * nk * 4) return;
    const int a = (int)(gid & 3);
    const long long face = gid >> 2;
    const int cj = (int)(face % nj) - 1;
    const int ck = (int)((face / nj) % nk) - 1;
    const int lev = (int)(face / (nj * nk)) - 1;
    double2 acc[4] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    const bool touching = lev == 0 && (cj == 0 || cj == -1) && (ck == 0 || ck == -1);
    const double ui = g.d[axis] * lev;
    if (!touching) {
        int ej = cj >= 0 ? cj : -cj - 1, ek = ck >= 0 ? ck : -ck - 1;
        double dist = sqrt(ui * ui + (ej * g.d[j]) * (ej * g.d[j]) + (ek * g.d[k]) * (ek * g.d[k]));
        const int rule = rule_for_ratio(dist / fmax(g.d[0], fmax(g.d[1], g.d[2])));
        const int nn = rule_n(rule), off = c_goff[rule];
        for (int p = 0; p < nn; ++p) {
            const double xp = c_gx[off + p], wp = c_gw[off + p];
            const double uj = g.d[j] * (cj + xp);
            double xa = wp;
            for (int q = 0; q < a; ++q) xa *= xp;
            for (int q = 0; q < nn; ++q) {
                const double yq = c_gx[off + q], wq = c_gw[off + q];
                const double uk = g.d[k] * (ck + yq);
                double2 gv = gfun(sqrt(ui * ui + uj * uj + uk * uk), g.k0);
                double f = xa * wq;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc[b].x = fma(f, gv.x, acc[b].x);
                    acc[b].y = fma(f, gv.y, acc[b].y);
                    f *= yq;
                }
            }
        }
    } else {
        const int nt = rule_n(RDT), ns = rule_n(RDS), ot = c_goff[RDT], os = c_goff[RDS];
        for (int m = 0; m < 2; ++m) {
            for (int it = 0; it < nt; ++it) {
                const double tau = c_gx[ot + it], wt = c_gw[ot + it] * tau;
                for (int i1 = 0; i1 < ns; ++i1) {
                    const double z1 = c_gx[os + i1], w1 = c_gw[os + i1];
                    double eta[2];
                    eta[m] = tau;
                    eta[1 - m] = tau * z1;
                    double xj = cj == 0 ? eta[0] : 1.0 - eta[0];
                    double xk = ck == 0 ? eta[1] : 1.0 - eta[1];
                    double r = sqrt((g.d[j] * eta[0]) * (g.d[j] * eta[0]) + (g.d[k] * eta[1]) * (g.d[k] * eta[1]));
                    double2 gv = gfun(r, g.k0);
                    double f = wt * w1;
                    for (int q = 0; q < a; ++q) f *= xj;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        acc[b].x = fma(f, gv.x, acc[b].x);
                        acc[b].y = fma(f, gv.y, acc[b].y);
                        f *= xk;
                    }
                }
            }
        }
    }
    double2* out = mu + face * 16 + a * 4;
#pragma unroll
    for (int b = 0; b < 4; ++b) out[b] = acc[b];
}

// ---------------------------------------------------------------------------
// 1-D factors: 0 = interval weight 1, 1 = interval weight s, 2 = point s = -1/2, 3 = point s = +1/2.
// Correlation W(t) = int a(s) b(s - t) ds in the local coordinate xi = t - lo of each unit cell.
// ---------------------------------------------------------------------------
struct Corr {
    int npieces;  // 1 or 2 cells, or 0 for a point mass at t0
    int lo[2];
    double c[2][4];
    int t0;
};

__device__ __forceinline__ void set4(double* c, double a0, double a1, double a2, double a3) {
    c[0] = a0, c[1] = a1, c[2] = a2, c[3] = a3;
}

__device__ Corr correlate(int fa, int fb) {
    Corr r;
    r.t0 = 0;
    if (fa < 2 && fb < 2) {
        r.npieces = 2;
        r.lo[0] = -1;
        r.lo[1] = 0;
        if (fa == 0 && fb == 0) {  // triangle 1 - |t|
            set4(r.c[0], 0, 1, 0, 0);
            set4(r.c[1], 1, -1, 0, 0);
        } else if (fa == 1 && fb == 0) {  // t (1 - |t|) / 2
            set4(r.c[0], 0, -0.5, 0.5, 0);
            set4(r.c[1], 0, 0.5, -0.5, 0);
        } else if (fa == 0 && fb == 1) {  // -t (1 - |t|) / 2
            set4(r.c[0], 0, 0.5, -0.5, 0);
            set4(r.c[1], 0, -0.5, 0.5, 0);
        } else {  // |t|^3/6 - |t|/4 + 1/12
            set4(r.c[0], 0, -0.25, 0.5, -1.0 / 6.0);
            set4(r.c[1], 1.0 / 12.0, -0.25, 0, 1.0 / 6.0);
        }
    } else if (fa >= 2 && fb < 2) {  // point sigma/2 (x) interval: b(sigma/2 - t)
        r.npieces = 1;
        r.lo[0] = fa == 3 ? 0 : -1;
        if (fb == 0)
            set4(r.c[0], 1, 0, 0, 0);
        else
            set4(r.c[0], 0.5, -1, 0, 0);
    } else if (fa < 2 && fb >= 2) {  // interval (x) point sigma'/2: a(t + sigma'/2)
        r.npieces = 1;
        r.lo[0] = fb == 3 ? -1 : 0;
        if (fa == 0)
            set4(r.c[0], 1, 0, 0, 0);
        else
            set4(r.c[0], -0.5, 1, 0, 0);
    } else {  // two points
        r.npieces = 0;
        int sa = fa == 3 ? 1 : -1, sb = fb == 3 ? 1 : -1;
        r.t0 = (sa - sb) / 2;
    }
    return r;
}

struct Density {
    int n;
    double coef[3];
    int f[3][3];  // per piece, per axis factor code
};

// Scalar PWL function N^l (l = 1..4) as a single product density.
__device__ Density basis_density(int l) {
    Density d;
    d.n = 1;
    d.coef[0] = 1.0;
    for (int i = 0; i < 3; ++i) d.f[0][i] = (l - 2 == i) ? 1 : 0;
    return d;
}

// d/ds_p [N^l P]: volume part (1 if N^l is linear along p) and the two face parts.
__device__ Density divergence_density(int p, int l) {
    Density d;
    d.n = 0;
    const int la = l - 2;
    if (la == p) {
        d.coef[d.n] = 1.0;
        d.f[d.n][0] = d.f[d.n][1] = d.f[d.n][2] = 0;
        ++d.n;
    }
    for (int sg = -1; sg <= 1; sg += 2) {
        d.coef[d.n] = -sg * (la == p ? 0.5 * sg : 1.0);
        for (int i = 0; i < 3; ++i) d.f[d.n][i] = (la == i) ? 1 : 0;
        d.f[d.n][p] = sg > 0 ? 3 : 2;
        ++d.n;
    }
    return d;
}

struct GreenArgs {
    GreenGeo g;
    const double2* mu3;
    const double2* mu2[3];
    double2* out;  // [60][nz][ny][nx]
};

__device__ __forceinline__ const double2* cell3(const GreenArgs& A, int kx, int ky, int kz) {
    const long long idx = ((long long)(kz + 1) * (A.g.ny + 1) + (ky + 1)) * (A.g.nx + 1) + (kx + 1);
    return A.mu3 + idx * 64;
}
__device__ __forceinline__ const double2* face2(const GreenArgs& A, int axis, int lev, int cj, int ck) {
    const int n[3] = {A.g.nx, A.g.ny, A.g.nz};
    const int j = axis == 0 ? 1 : 0, k = axis == 2 ? 1 : 2;
    const long long idx = ((long long)(lev + 1) * (n[k] + 1) + (ck + 1)) * (n[j] + 1) + (cj + 1);
    return A.mu2[axis] + idx * 16;
}

// I(d) = int prod_i W_i(t_i) g(Delta (d + t)) dt for one pair of product densities.
__device__ double2 pair_integral(const GreenArgs& A, const int* fa, const int* fb, const int* dd) {
    Corr c[3];
    int point_axis = -1;
    for (int i = 0; i < 3; ++i) {
        c[i] = correlate(fa[i], fb[i]);
        if (c[i].npieces == 0) point_axis = i;
    }
    double2 sum = make_double2(0, 0);
    if (point_axis < 0) {
        for (int px = 0; px < c[0].npieces; ++px)
            for (int py = 0; py < c[1].npieces; ++py)
                for (int pz = 0; pz < c[2].npieces; ++pz) {
                    const double2* m = cell3(A, dd[0] + c[0].lo[px], dd[1] + c[1].lo[py], dd[2] + c[2].lo[pz]);
                    const double* cx = c[0].c[px];
                    const double* cy = c[1].c[py];
                    const double* cz = c[2].c[pz];
                    for (int a = 0; a < 4; ++a) {
                        if (cx[a] == 0.0) continue;
                        double2 sa = make_double2(0, 0);
                        for (int b = 0; b < 4; ++b) {
                            if (cy[b] == 0.0) continue;
                            double2 sb = make_double2(0, 0);
                            for (int e = 0; e < 4; ++e) {
                                if (cz[e] == 0.0) continue;
                                double2 v = m[a * 16 + b * 4 + e];
                                sb.x = fma(cz[e], v.x, sb.x);
                                sb.y = fma(cz[e], v.y, sb.y);
                            }
                            sa.x = fma(cy[b], sb.x, sa.x);
                            sa.y = fma(cy[b], sb.y, sa.y);
                        }
                        sum.x = fma(cx[a], sa.x, sum.x);
                        sum.y = fma(cx[a], sa.y, sum.y);
                    }
                }
        return sum;
    }
    const int ax = point_axis, j = ax == 0 ? 1 : 0, k = ax == 2 ? 1 : 2;
    const int lev = dd[ax] + c[ax].t0;
    for (int pj = 0; pj < c[j].npieces; ++pj)
        for (int pk = 0; pk < c[k].npieces; ++pk) {
            const double2* m = face2(A, ax, lev, dd[j] + c[j].lo[pj], dd[k] + c[k].lo[pk]);
            const double* cj = c[j].c[pj];
            const double* ck = c[k].c[pk];
            for (int a = 0; a < 4; ++a) {
                if (cj[a] == 0.0) continue;
                double2 sa = make_double2(0, 0);
                for (int b = 0; b < 4; ++b) {
                    double2 v = m[a * 4 + b];
                    sa.x = fma(ck[b], v.x, sa.x);
                    sa.y = fma(ck[b], v.y, sa.y);
                }
                sum.x = fma(cj[a], sa.x, sum.x);
                sum.y = fma(cj[a], sa.y, sum.y);
            }
        }
    return sum;
}

__device__ __forceinline__ void tensor_indices(int t, int& p, int& q, int& la, int& lb) {
    const int pq = t / 10, ll = t % 10;
    const int P[6] = {0, 0, 0, 1, 1, 2}, Q[6] = {0, 1, 2, 1, 2, 2};
    const int LA[10] = {1, 1, 1, 1, 2, 2, 2, 3, 3, 4}, LB[10] = {1, 2, 3, 4, 2, 3, 4, 3, 4, 4};
    p = P[pq], q = Q[pq], la = LA[ll], lb = LB[ll];
}

// U_t(d) = k0^2 delta_pq S^{la lb}(d) - Q^{p la, q lb}(d) for d in [0, N)^3; thread per (d, t).
__global__ void assemble_kernel(GreenArgs A) {
    const long long nd = (long long)A.g.nx * A.g.ny * A.g.nz;
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= nd * 60) return;
    const int t = (int)(gid % 60);
    const long long di = gid / 60;
    const int dd[3] = {(int)(di % A.g.nx), (int)((di / A.g.nx) % A.g.ny), (int)(di / ((long long)A.g.nx * A.g.ny))};
    int p, q, la, lb;
    tensor_indices(t, p, q, la, lb);
    const double dV = A.g.d[0] * A.g.d[1] * A.g.d[2];
    double2 val = make_double2(0, 0);
    if (p == q) {
        Density da = basis_density(la), db = basis_density(lb);
        double2 s = pair_integral(A, da.f[0], db.f[0], dd);
        const double f = A.g.k0 * A.g.k0 * dV * dV;
        val.x += f * s.x;
        val.y += f * s.y;
    }
    Density ra = divergence_density(p, la), rb = divergence_density(q, lb);
    double2 qs = make_double2(0, 0);
    for (int i = 0; i < ra.n; ++i)
        for (int jj = 0; jj < rb.n; ++jj) {
            double2 v = pair_integral(A, ra.f[i], rb.f[jj], dd);
            const double cc = ra.coef[i] * rb.coef[jj];
            qs.x = fma(cc, v.x, qs.x);
            qs.y = fma(cc, v.y, qs.y);
        }
    const double fq = dV * dV / (A.g.d[p] * A.g.d[q]);
    val.x -= fq * qs.x;
    val.y -= fq * qs.y;
    A.out[(long long)t * nd + di] = val;
}

static_assert(kblock::table_complete(), "K block table: 30 tensors, 96 non-zero entries");

// K operator (K u = curl S u): P_t(d) = (dV^2 / Delta_j) int int (D_j N^la) g N^lb for
// t = 10 j + ll(la, lb), la <= lb, d in [0, N)^3; thread per (d, t).  D_j N^la is the
// distributional derivative (volume part and face masses), the testing-side integration by
// parts that turns the weakly singular d_j g into g.  K^{(p,la),(q,lb)}(d) = -eps_pjq P_t(d).
__global__ void assemble_k_kernel(GreenArgs A) {
    const long long nd = (long long)A.g.nx * A.g.ny * A.g.nz;
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= nd * 30) return;
    const int t = (int)(gid % 30);
    const long long di = gid / 30;
    const int dd[3] = {(int)(di % A.g.nx), (int)((di / A.g.nx) % A.g.ny), (int)(di / ((long long)A.g.nx * A.g.ny))};
    const int j = t / 10, ll = t % 10;
    const int LA[10] = {1, 1, 1, 1, 2, 2, 2, 3, 3, 4}, LB[10] = {1, 2, 3, 4, 2, 3, 4, 3, 4, 4};
    Density ra = divergence_density(j, LA[ll]), rb = basis_density(LB[ll]);
    double2 acc = make_double2(0, 0);
    for (int i = 0; i < ra.n; ++i) {
        const double2 v = pair_integral(A, ra.f[i], rb.f[0], dd);
        acc.x = fma(ra.coef[i], v.x, acc.x);
        acc.y = fma(ra.coef[i], v.y, acc.y);
    }
    const double dV = A.g.d[0] * A.g.d[1] * A.g.d[2];
    const double f = dV * dV / A.g.d[j];
    A.out[(long long)t * nd + di] = make_double2(f * acc.x, f * acc.y);
}

// Circulant embedding of tensors [t0, t0 + nt) into [nt][Lz][Ly][Lx].
__global__ void embed_kernel(const double2* __restrict__ T, int nx, int ny, int nz, int Lx, int Ly, int Lz, int t0,
                             int nt, double2* __restrict__ C) {
    const long long vol = (long long)Lx * Ly * Lz;
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= vol * nt) return;
    const int tl = (int)(gid / vol);
    const long long j = gid % vol;
    const int jx = (int)(j % Lx), jy = (int)((j / Lx) % Ly), jz = (int)(j / ((long long)Lx * Ly));
    const int J[3] = {jx, jy, jz}, N[3] = {nx, ny, nz}, Lv[3] = {Lx, Ly, Lz};
    int d[3];
    bool neg[3];
    bool zero = false;
    for (int i = 0; i < 3; ++i) {
        if (J[i] < N[i]) {
            d[i] = J[i];
            neg[i] = false;
        } else if (J[i] > Lv[i] - N[i]) {
            d[i] = Lv[i] - J[i];
            neg[i] = true;
        } else {
            zero = true;
            d[i] = 0;
            neg[i] = false;
        }
    }
    double2 v = make_double2(0, 0);
    if (!zero) {
        const int t = t0 + tl;
        const int pq = t / 10, ll = t % 10;
        const int P[6] = {0, 0, 0, 1, 1, 2}, Q[6] = {0, 1, 2, 1, 2, 2};
        const int LA[10] = {1, 1, 1, 1, 2, 2, 2, 3, 3, 4}, LB[10] = {1, 2, 3, 4, 2, 3, 4, 3, 4, 4};
        const int alpha = 4 * P[pq] + LA[ll] - 1, beta = 4 * Q[pq] + LB[ll] - 1;
        int sgn = 1;
        for (int i = 0; i < 3; ++i)
            if (neg[i]) sgn *= parity_of(alpha, i) * parity_of(beta, i);
        v = T[(long long)t * nx * ny * nz + ((long long)d[2] * ny + d[1]) * nx + d[0]];
        if (sgn < 0) v = make_double2(-v.x, -v.y);
    }
    C[gid] = v;
}

// Octant k_i in [0, L_i/2] of the transformed circulants, scaled, into FP64 and FP32 tables [60][Oz][Oy][Ox].
__global__ void octant_kernel(const double2* __restrict__ C, int Lx, int Ly, int Lz, int t0, int nt, double scale,
                              double2* __restrict__ g64, float2* __restrict__ g32, float2* __restrict__ g32t,
                              double2* __restrict__ g64t) {
    const int Ox = Lx / 2 + 1, Oy = Ly / 2 + 1, Oz = Lz / 2 + 1;
    const long long ovol = (long long)Ox * Oy * Oz;
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= ovol * nt) return;
    const int tl = (int)(gid / ovol);
    const long long o = gid % ovol;
    const int kx = (int)(o % Ox), ky = (int)((o / Ox) % Oy), kz = (int)(o / ((long long)Ox * Oy));
    double2 v = C[(long long)tl * Lx * Ly * Lz + ((long long)kz * Ly + ky) * Lx + kx];
    v.x *= scale;
    v.y *= scale;
    const long long dst = (long long)(t0 + tl) * ovol + o;
    g64[dst] = v;
    g32[dst] = make_float2((float)v.x, (float)v.y);
    const long long tdst = (((long long)ky * Ox + kx) * Oz + kz) * 60 + t0 + tl;
    g32t[tdst] = make_float2((float)v.x, (float)v.y);
    g64t[tdst] = v;
}

// Gauss-Legendre tables of the cell-moment kernels in constant memory (current device)
static int quad_tables() {
    double gx[128], gw[128];
    int off[kNumRules];
    int pos = 0;
    for (int r = 0; r < kNumRules; ++r) {
        off[r] = pos;
        gauss_legendre01(kOrders[r], gx + pos, gw + pos);
        pos += kOrders[r];
    }
    VIE_CUDA(cudaMemcpyToSymbol(c_gx, gx, sizeof(double) * pos));
    VIE_CUDA(cudaMemcpyToSymbol(c_gw, gw, sizeof(double) * pos));
    VIE_CUDA(cudaMemcpyToSymbol(c_goff, off, sizeof(off)));
    return VIE_OK;
}

int green_embed(vie_handle* h, double2* T, bool keep_table = true);

int green_setup(vie_handle* h) {
    VIE_TRY(quad_tables());
    cudaStream_t s = h->stream;
    GreenGeo g;
    g.nx = h->nx, g.ny = h->ny, g.nz = h->nz;
    g.d[0] = h->dx, g.d[1] = h->dy, g.d[2] = h->dz;
    g.k0 = h->k0;
    const long long n3 = (long long)(h->nx + 1) * (h->ny + 1) * (h->nz + 1);
    size_t n2[3];
    const int n[3] = {h->nx, h->ny, h->nz};
    for (int ax = 0; ax < 3; ++ax) {
        int j = ax == 0 ? 1 : 0, k = ax == 2 ? 1 : 2;
        n2[ax] = (size_t)(n[ax] + 2) * (n[j] + 1) * (n[k] + 1);
    }
    const long long nd = (long long)h->nx * h->ny * h->nz;
    double2 *mu3 = nullptr, *mu2[3] = {nullptr, nullptr, nullptr}, *T = nullptr;
    auto fail = [&](int code) {
        cudaFree(mu3);
        for (int ax = 0; ax < 3; ++ax) cudaFree(mu2[ax]);
        cudaFree(T);
        return code;
    };
    if (cudaMalloc(&mu3, sizeof(double2) * 64 * n3) != cudaSuccess) return fail((set_error("moments alloc"), VIE_ENOMEM));
    for (int ax = 0; ax < 3; ++ax)
        if (cudaMalloc(&mu2[ax], sizeof(double2) * 16 * n2[ax]) != cudaSuccess)
            return fail((set_error("face moments alloc"), VIE_ENOMEM));
    if (cudaMalloc(&T, sizeof(double2) * 60 * nd) != cudaSuccess) return fail((set_error("toeplitz alloc"), VIE_ENOMEM));
    {
        long long th = n3 * 4;
        VIE_KLAUNCH("moments3", s, moments3_kernel<<<(unsigned)((th + 127) / 128), 128, 0, s>>>(g, mu3));
        for (int ax = 0; ax < 3; ++ax) {
            long long th2 = (long long)n2[ax] * 4;
            VIE_KLAUNCH("moments2", s, moments2_kernel<<<(unsigned)((th2 + 127) / 128), 128, 0, s>>>(g, ax, mu2[ax]));
        }
        GreenArgs A;
        A.g = g;
        A.mu3 = mu3;
        for (int ax = 0; ax < 3; ++ax) A.mu2[ax] = mu2[ax];
        A.out = T;
        long long tha = nd * 60;
        VIE_KLAUNCH("assemble", s, assemble_kernel<<<(unsigned)((tha + 127) / 128), 128, 0, s>>>(A));
        if (cudaGetLastError() != cudaSuccess) return fail((set_error("green kernels launch"), VIE_EDEVICE));
    }
    cudaFree(mu3);
    for (int ax = 0; ax < 3; ++ax) cudaFree(mu2[ax]);
    return green_embed(h, T);  // takes T
}

// Circulant embedding, 3-D FFT and octant storage of the 60 Toeplitz tensors T [60][nz][ny][nx]
// (device, N - G at offsets d >= 0) in FP64 and FP32 (Section IV-A).  Takes ownership of T, also
// on failure: the handle keeps it for vie_green_toeplitz when keep_table is set, else frees it.
// The spectra are allocated on the first call and overwritten by later ones.
int green_embed(vie_handle* h, double2* T, bool keep_table) {
    cudaStream_t s = h->stream;
    const long long nd = (long long)h->nx * h->ny * h->nz;
    double2* C = nullptr;
    auto fail = [&](int code) {
        cudaFree(T);
        cudaFree(C);
        return code;
    };
    int rc = VIE_OK;
    const int Lx = h->L[0], Ly = h->L[1], Lz = h->L[2];
    const long long vol = (long long)Lx * Ly * Lz;
    const long long ovol = (long long)h->O[0] * h->O[1] * h->O[2];
    if (!h->green64) {
        if (cudaMalloc(&h->green64, sizeof(double2) * 60 * ovol) != cudaSuccess ||
            cudaMalloc(&h->green32, sizeof(float2) * 60 * ovol) != cudaSuccess ||
            cudaMalloc(&h->green32t, sizeof(float2) * 60 * ovol) != cudaSuccess ||
            cudaMalloc(&h->green64t, sizeof(double2) * 60 * ovol) != cudaSuccess ||
            cudaMalloc(&h->greenbf, sizeof(uint2) * 60 * ovol) != cudaSuccess)
            return fail((set_error("green alloc"), VIE_ENOMEM));
        h->bytes_held += (2 * sizeof(double2) + 2 * sizeof(float2) + sizeof(uint2)) * 60 * ovol;
    }
    int chunk = (int)std::max<long long>(1, std::min<long long>(60, (4LL << 30) / (vol * (long long)sizeof(double2))));
    if (cudaMalloc(&C, sizeof(double2) * vol * chunk) != cudaSuccess) return fail((set_error("embed alloc"), VIE_ENOMEM));
    for (int t0 = 0; t0 < 60; t0 += chunk) {
        int nt = std::min(chunk, 60 - t0);
        long long th = vol * nt;
        VIE_KLAUNCH("embed", s, embed_kernel<<<(unsigned)((th + 255) / 256), 256, 0, s>>>(T, h->nx, h->ny, h->nz, Lx, Ly, Lz, t0, nt, C));
        if (cudaGetLastError() != cudaSuccess) return fail((set_error("embed launch"), VIE_EDEVICE));
        rc = fft3d_inplace64(h, C, nt, s);
        if (rc < 0) return fail(rc);
        long long tho = ovol * nt;
        VIE_KLAUNCH("octant", s, octant_kernel<<<(unsigned)((tho + 255) / 256), 256, 0, s>>>(C, Lx, Ly, Lz, t0, nt, 1.0 / (double)vol,
                                                                     h->green64, h->green32, h->green32t,
                                                                     h->green64t));
        if (cudaGetLastError() != cudaSuccess) return fail((set_error("octant launch"), VIE_EDEVICE));
    }
    rc = green_split_bf16(h);
    if (rc < 0) return fail(rc);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail((set_error("green setup sync"), VIE_EDEVICE));
    cudaFree(C);
    if (!keep_table) {
        cudaFree(T);
        return VIE_OK;
    }
    // The Toeplitz table is kept for inspection (vie_green_toeplitz)
    h->toeplitz = T;
    h->bytes_held += sizeof(double2) * 60 * nd;
    return VIE_OK;
}

// T[t][d] = the representative entry (alpha, beta) of unique tensor t at offset d >= 0, taken
// from a caller's full table E[144][2nz-1][2ny-1][2nx-1] (entry alpha * 12 + beta, offset d at
// index d + N - 1 per axis), minus the Gram term G^l on the diagonal at d = 0 (the device keeps
// N - G).
__global__ void external_pick_kernel(const double2* __restrict__ E, int nx, int ny, int nz, double g1, double g234,
                                     double2* __restrict__ T) {
    const long long nd = (long long)nx * ny * nz;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= 60 * nd) return;
    const int t = (int)(gid / nd);
    const long long d = gid % nd;
    const int dx = (int)(d % nx), dy = (int)((d / nx) % ny), dz = (int)(d / ((long long)nx * ny));
    const int pq = t / 10, ll = t % 10;
    const int P[6] = {0, 0, 0, 1, 1, 2}, Q[6] = {0, 1, 2, 1, 2, 2};
    const int LA[10] = {1, 1, 1, 1, 2, 2, 2, 3, 3, 4}, LB[10] = {1, 2, 3, 4, 2, 3, 4, 3, 4, 4};
    const int alpha = 4 * P[pq] + LA[ll] - 1, beta = 4 * Q[pq] + LB[ll] - 1;
    const long long ex = 2LL * nx - 1, ey = 2LL * ny - 1, ez = 2LL * nz - 1;
    double2 v = E[(long long)(alpha * 12 + beta) * ex * ey * ez + ((dz + nz - 1) * ey + (dy + ny - 1)) * ex + dx + nx - 1];
    if (d == 0 && alpha == beta) v.x -= LA[ll] == 1 ? g1 : g234;
    T[gid] = v;
}

// Green tensors of a handle from a caller's Toeplitz table (vie_setup_green_external): `ext` is
// device memory [144][2nz-1][2ny-1][2nx-1] complex128.
int green_setup_external(vie_handle* h, const double2* ext) {
    VIE_TRY(quad_tables());  // for the K tensors, which the device still computes
    const long long nd = (long long)h->nx * h->ny * h->nz;
    double2* T = nullptr;
    if (cudaMalloc(&T, sizeof(double2) * 60 * nd) != cudaSuccess) {
        cudaGetLastError();
        set_error("toeplitz alloc");
        return VIE_ENOMEM;
    }
    const double dV = h->dx * h->dy * h->dz;
    cudaStream_t s = h->stream;
    VIE_KLAUNCH("green_external", s,
                external_pick_kernel<<<(unsigned)((60 * nd + 255) / 256), 256, 0, s>>>(ext, h->nx, h->ny, h->nz, dV,
                                                                                      dV / 12.0, T));
    if (cudaGetLastError() != cudaSuccess) {
        cudaFree(T);
        set_error("green_external launch");
        return VIE_EDEVICE;
    }
    return green_embed(h, T);
}

// The 30 Toeplitz tensors of the K operator into out [30][nz][ny][nx] (device), from the same
// cell moments as green_setup (computed again here; the handle keeps none of them).
int green_k_toeplitz(vie_handle* h, double2* out, cudaStream_t s) {
    GreenGeo g;
    g.nx = h->nx, g.ny = h->ny, g.nz = h->nz;
    g.d[0] = h->dx, g.d[1] = h->dy, g.d[2] = h->dz;
    g.k0 = h->k0;
    const long long n3 = (long long)(h->nx + 1) * (h->ny + 1) * (h->nz + 1);
    size_t n2[3];
    const int n[3] = {h->nx, h->ny, h->nz};
    for (int ax = 0; ax < 3; ++ax) {
        int j = ax == 0 ? 1 : 0, k = ax == 2 ? 1 : 2;
        n2[ax] = (size_t)(n[ax] + 2) * (n[j] + 1) * (n[k] + 1);
    }
    const long long nd = (long long)h->nx * h->ny * h->nz;
    double2 *mu3 = nullptr, *mu2[3] = {nullptr, nullptr, nullptr};
    auto done = [&](int code) {
        cudaFree(mu3);
        for (int ax = 0; ax < 3; ++ax) cudaFree(mu2[ax]);
        return code;
    };
    if (cudaMalloc(&mu3, sizeof(double2) * 64 * n3) != cudaSuccess) return done((set_error("moments alloc"), VIE_ENOMEM));
    for (int ax = 0; ax < 3; ++ax)
        if (cudaMalloc(&mu2[ax], sizeof(double2) * 16 * n2[ax]) != cudaSuccess)
            return done((set_error("face moments alloc"), VIE_ENOMEM));
    const long long th = n3 * 4;
    VIE_KLAUNCH("moments3", s, moments3_kernel<<<(unsigned)((th + 127) / 128), 128, 0, s>>>(g, mu3));
    for (int ax = 0; ax < 3; ++ax) {
        const long long th2 = (long long)n2[ax] * 4;
        VIE_KLAUNCH("moments2", s, moments2_kernel<<<(unsigned)((th2 + 127) / 128), 128, 0, s>>>(g, ax, mu2[ax]));
    }
    GreenArgs A;
    A.g = g;
    A.mu3 = mu3;
    for (int ax = 0; ax < 3; ++ax) A.mu2[ax] = mu2[ax];
    A.out = out;
    const long long tha = nd * 30;
    VIE_KLAUNCH("assemble_k", s, assemble_k_kernel<<<(unsigned)((tha + 127) / 128), 128, 0, s>>>(A));
    if (cudaGetLastError() != cudaSuccess) return done((set_error("K tensor kernels launch"), VIE_EDEVICE));
    if (cudaStreamSynchronize(s) != cudaSuccess) return done((set_error("K tensor sync"), VIE_EDEVICE));
    return done(VIE_OK);
}
