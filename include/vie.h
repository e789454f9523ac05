/*
 * vie.h -- C ABI of the GB300 library for the FFT-accelerated PWL current-based
 * volume integral equation of Georgakis, Giannakopoulos, Litsarev and
 * Polimeridis, "A Fast Volume Integral Equation Solver with Linear Basis
 * Functions for the Accurate Computation of EM Fields in MRI" (arXiv 1902.02196).
 *
 * Problem (Section II, Eq. 16):  (M_eps - M_chi N) j = c_e M_chi e_inc, dielectric body,
 * time factor exp(i omega t), c_e = i omega eps0, chi = eps - 1, eps = eps' - i sigma/(omega eps0).
 * Discretisation (Section III): Galerkin MoM with 4 scalar PWL functions
 * {1, (x-xn)/dx, (y-yn)/dy, (z-zn)/dz} x 3 vector components = 12 unknowns per
 * voxel (Eq. 19-22), system A x = b with A = M_eps G - M_chi N, b = c_e M_chi e_inc (Eq. 24).
 *
 * Data conventions used by every entry point:
 *  - grid of nx*ny*nz voxels, box centred at the origin; voxel (ix,iy,iz) has its
 *    centre at ((ix+1/2-nx/2) dx, (iy+1/2-ny/2) dy, (iz+1/2-nz/2) dz); N_V = nx*ny*nz;
 *  - per-voxel real maps: double[nz][ny][nx] (x fastest);
 *  - coefficient vectors: complex numbers stored as interleaved (re, im) pairs,
 *    layout [nrhs][12][nz][ny][nx]; component alpha = 4 p + (l - 1) with p = 0,1,2
 *    for the x,y,z vector component and l = 1..4 the scalar PWL function;
 *  - "C128" buffers hold double pairs, "C64" buffers hold float pairs;
 *  - every buffer is owned by the caller.  Pointers may be host or device memory
 *    (detected with cudaPointerGetAttributes); host buffers are staged through
 *    device memory owned by the handle and copied back before the call returns;
 *  - `stream` is a cudaStream_t passed as void* (NULL = the handle's own stream).
 *    Calls with device buffers are asynchronous with respect to the host unless
 *    stated otherwise; calls with host buffers synchronise the stream.
 *
 * Errors: every int-returning function returns VIE_OK (0), a negative error
 * code, or the positive VIE_NOT_CONVERGED.  No exception or abort crosses the
 * ABI.  vie_strerror() gives a static description; vie_last_error() the detail
 * of the most recent failure on the calling thread.
 */
#ifndef VIE_H
#define VIE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VIE_OK 0
#define VIE_EINVAL (-1)        /* invalid argument (sizes, NULL pointer, NaN input, unknown flag) */
#define VIE_ENOMEM (-2)        /* device or host allocation failed */
#define VIE_EDEVICE (-3)       /* a CUDA call or kernel launch failed */
#define VIE_ETIMEOUT (-4)      /* a bounded wait ran out */
#define VIE_NOT_CONVERGED 1    /* solver hit its iteration limit; best iterate returned */

/* Compute precision of a matvec; also the element type of its vectors. */
#define VIE_FP64 0 /* complex128 vectors, FP64 FFT and block product */
#define VIE_FP32 1 /* complex64 vectors, FP32 FFT and block product */
#define VIE_BF16X3 2 /* complex64 vectors, FP32 FFT; block product on the tensor cores from bf16
                        (hi, lo) splits of both operands, x_lo B_hi + x_hi B_lo + x_hi B_hi with FP32
                        accumulation (each real product within 3 * 2^-16 relative); FFT lengths
                        along z of 8..512 */

/* Operator applied by vie_matvec. */
#define VIE_OP_A 0      /* y = A x = M_eps G x - M_chi N x                     (Eq. 24) */
#define VIE_OP_PA 1     /* y = P^-1 A x, P = M_eps G: x/eps - tau G^-1 (N - G) x (Section IV-B, Eq. 17) */
#define VIE_OP_NSCAT 2  /* y = (N - G) x, the Galerkin "N - I" operator (tested scattered field * c_e) */
#define VIE_OP_K 3      /* y = K x, K u = curl S u (Eq. 8): the tested scattered magnetic field (Eq. 13); FP64 or FP32 */

/* Solver modes of vie_solve. */
#define VIE_SOLVE_FP64 0         /* plain FP64 GMRES */
#define VIE_SOLVE_FP32_REFINE 1  /* FP32 inner GMRES inside FP64 iterative refinement */
#define VIE_SOLVE_BF16X3_REFINE 2 /* as VIE_SOLVE_FP32_REFINE with the VIE_BF16X3 matvec in the inner GMRES */

/* vie_setup flags */
#define VIE_SETUP_PWC 1 /* piecewise-constant basis: 3 unknowns per voxel (Section V-A comparison) */

typedef struct vie_handle vie_handle;

typedef struct {
    int nx, ny, nz;    /* voxels per axis, >= 1 */
    double dx, dy, dz; /* voxel side lengths in metres, > 0 */
} vie_grid;

typedef struct {
    int converged;       /* 1 if resid <= tol */
    int iterations;      /* GMRES (Arnoldi) steps taken, all precisions */
    int fp64_matvecs;    /* FP64 operator applications (refinement residuals, plain FP64 steps) */
    int fp32_matvecs;    /* FP32 (or BF16x3) operator applications */
    int refinements;     /* outer refinement sweeps (mode VIE_SOLVE_FP32_REFINE) */
    double resid;        /* final ||P^-1 (b - A x)|| / ||P^-1 b||, recomputed in FP64 */
    double true_resid;   /* final ||b - A x|| / ||b|| in FP64 when requested (flags bit 1), else -1 */
    double err_est;      /* estimated relative error ||x - x*|| / ||x|| of the returned x (x* the exact
                            solution of A x = b): the last refinement sweep's (mixed) or restart cycle's
                            (FP64) correction dx, scaled by the residual reduction it left,
                            ||dx|| / ||x|| * ||r_end|| / ||r_start|| (preconditioned residuals) */
} vie_solve_info;

/*
 * vie_setup -- build a handle for one grid, frequency and dielectric map.
 * Computes on the GPU, in FP64: the Galerkin entries of N for every offset
 * (Section III-C, Eq. 25, Eq. 34, Eq. 42-43), their circulant embedding and 3-D
 * FFT (Section IV-A), stored once in FP64 and once in FP32; and the per-voxel
 * material coefficients eps, chi = eps - 1, tau = chi/eps (Eq. 7, Eq. 17, Eq. 29).
 *   grid          : voxel counts and sizes (see above)
 *   freq_hz       : frequency f > 0; omega = 2 pi f, k0 = omega / c0
 *   eps_real      : double[nz][ny][nx], eps' >= 1 (1 in air), host or device
 *   sigma         : double[nz][ny][nx], conductivity in S/m >= 0, host or device
 *   flags         : 0, or VIE_SETUP_PWC for the piecewise-constant system (below)
 *   out           : receives the handle; release with vie_destroy
 * VIE_SETUP_PWC: the comparison solver of Section V-A with one constant basis function per
 * vector component and voxel (3 unknowns per voxel), whose Galerkin system is exactly the
 * l = 1 sub-block of the PWL system (Eq. 19-22, 24, 33 with l = l' = 1).  Every vector of the
 * handle is then [nrhs][3][nz][ny][nx] (component p = x, y, z), the block product is the 3 x 3
 * block of the six (1,1) tensors, and the Gram entry of every component is DV.  vie_matvec
 * (VIE_FP64, VIE_FP32; not VIE_BF16X3 or VIE_OP_K), vie_solve, vie_rhs_planewave,
 * vie_rhs_dipoles and vie_fields accept it; the magnetic-field calls do not.
 * Synchronous.  Returns VIE_EINVAL on bad sizes/NaN, VIE_ENOMEM, VIE_EDEVICE.
 */
int vie_setup(const vie_grid* grid, double freq_hz, const double* eps_real, const double* sigma, int flags,
              vie_handle** out);

/*
 * vie_setup_green_external -- vie_setup with the Galerkin entries of N supplied by the
 * caller instead of computed on the GPU: a test hook that checks the matvec apart from the
 * Green-tensor setup.  Everything else (circulant embedding and FFT of Section IV-A, octant
 * storage in FP64 and FP32, material maps) is as in vie_setup.
 *   grid, freq_hz, eps_real, sigma : as for vie_setup
 *   toeplitz_fp64 : complex128 [144][2nz-1][2ny-1][2nx-1], host or device, read during the
 *                   call only: entry alpha * 12 + beta holds N^{alpha beta}(d) (Eq. 25, Eq. 42-43,
 *                   the Gram term G^l of Eq. 33 included at d = 0 on the diagonal) for the voxel
 *                   offset d = m - n, stored at index d + N - 1 per axis.  Only the 60 entries
 *                   (alpha, beta) = (4p + l - 1, 4q + l' - 1) with p <= q and l <= l' at offsets
 *                   d >= 0 are read; the others must follow from them by reciprocity and the
 *                   reflection parities (Section III-C), as the exact entries do.
 * The K tensors (VIE_OP_K, vie_green_toeplitz_k) are still computed on the GPU.
 * Synchronous.  Errors as for vie_setup; VIE_EINVAL for a NULL table.
 */
int vie_setup_green_external(const vie_grid* grid, double freq_hz, const double* eps_real, const double* sigma,
                             const void* toeplitz_fp64, vie_handle** out);

/* Release every device buffer of the handle.  NULL is ignored. */
void vie_destroy(vie_handle* h);

/*
 * vie_matvec -- apply the operator `op` (VIE_OP_*) to nrhs vectors at once by the
 * FFT-accelerated circulant product (Section IV-A): zero-pad to the embedding
 * grid, 3-D FFT, 12x12 block product with the Green tensor at every frequency
 * point, inverse FFT, crop, then the per-voxel material and Gram terms.
 *   nrhs      : number of vectors >= 1
 *   x, y      : [nrhs][12][nz][ny][nx] complex, element type by `precision`
 *               (VIE_FP64: double pairs, VIE_FP32 and VIE_BF16X3: float pairs); x and y must not overlap
 *   precision : VIE_FP64, VIE_FP32 or VIE_BF16X3 (VIE_OP_K: VIE_FP64 or VIE_FP32)
 *   op        : VIE_OP_A, VIE_OP_PA, VIE_OP_NSCAT or VIE_OP_K.  VIE_OP_K transforms the 30
 *               tensors of vie_green_toeplitz_k once per handle into octant spectra (30 Ox Oy Oz
 *               values in FP64 and FP32, each in two layouts: 48 bytes per value in all, kept
 *               until vie_destroy and counted by vie_info) and runs
 *               the same transforms as the N operator with the K block (96 signed entries) at
 *               every frequency point, the other octants from the K parities.
 */
int vie_matvec(vie_handle* h, int nrhs, const void* x, void* y, int precision, int op, void* stream);

/*
 * vie_matvec_noalloc -- the same operator as vie_matvec, for callers that cannot
 * allocate GPU memory at call time: code that hands all device memory to its
 * own pool at start-up, loops that must not stall on the device-wide
 * synchronisation an allocation can cause, or runtimes with a fixed memory
 * budget.  The paper has no counterpart; this is an interface choice only.
 *
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Its
 * scratch (the spectrum buffers) is one static device array of 64 MiB
 * compiled into the library, which every GPU that loads the library holds
 * until the process exits.  A call needs nrhs * 12 * nz * L_y * L_x complex
 * values of the precision (8 or 16 bytes each) plus 256 bytes, where L_i is
 * the FFT length of vie_info; grids whose xy circulant is not square or is
 * longer than 128 take the line-transform path, which needs nrhs * 12 * nz *
 * ny * L_x more.  A call that needs more than the array returns VIE_EINVAL
 * without doing anything: use fewer right-hand sides per call, or vie_matvec.
 *   h, nrhs, precision     : as for vie_matvec
 *   op                     : VIE_OP_A, VIE_OP_PA or VIE_OP_NSCAT (not VIE_OP_K,
 *                            whose spectra are held by the handle)
 *   x, y                   : device memory of the handle's device only (host
 *                            buffers would need staging memory); VIE_EINVAL
 *                            otherwise
 *   stream                 : cudaStream_t as void*, NULL = the handle's stream
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  The current device must be the handle's device.
 * All calls share the one array, and it keeps whatever the last call left in
 * it; no part of it needs to start at zero, since each call writes every
 * element it reads before reading it.  Calls whose work overlaps on the GPU
 * (on different streams, or from different host threads) race on the array:
 * order them on one stream or serialise them.
 */
int vie_matvec_noalloc(vie_handle* h, int nrhs, const void* x, void* y, int precision, int op, void* stream);

/*
 * vie_rhs_planewave -- tested incident field of e_inc = pol exp(-i k0 dir.r)
 * (Eq. 27, Eq. 30; Section V-A uses pol = x, dir = z) in closed form, and the
 * right-hand side b = c_e chi e_inc (Eq. 31).
 *   pol, dir : 3-vectors (dir normalised by the library; pol used as given, V/m)
 *   e_inc    : [12][nz][ny][nx] C128 output or NULL
 *   b        : [12][nz][ny][nx] C128 output or NULL
 */
int vie_rhs_planewave(vie_handle* h, const double pol[3], const double dir[3], void* e_inc, void* b, void* stream);

/*
 * vie_rhs_dipoles -- tested incident fields of nrhs Hertzian dipoles, one per
 * right-hand side: e_inc = (1/c_e)(k0^2 g p + grad(p . grad g)) (Eq. 13 with a
 * point current p = I l, g of Eq. 10), tested with a 6x6x6 Gauss-Legendre rule
 * per voxel, and b = c_e chi e_inc (Eq. 31).
 *   pos : double[nrhs][3] positions (m);  mom : double[nrhs][3] moments (A m); host memory
 *   e_inc, b : [nrhs][12][nz][ny][nx] C128 outputs, either may be NULL
 */
int vie_rhs_dipoles(vie_handle* h, int nrhs, const double* pos, const double* mom, void* e_inc, void* b,
                    void* stream);

/*
 * vie_solve -- solve A x = b for nrhs right-hand sides with left-preconditioned
 * restarted GMRES, P = M_eps G (Section IV-B, Section V: GMRES(restart), at most
 * maxit restart cycles), stopping when ||P^-1 (b - A x)|| / ||P^-1 b|| <= tol.
 *   b       : [nrhs][12][nz][ny][nx] C128
 *   x       : [nrhs][12][nz][ny][nx] C128; on entry the initial guess when
 *             (flags & 1), else ignored (zero guess); on exit the solution
 *   restart : Krylov dimension m in [1, 128];  maxit: cap on restart cycles, counted
 *             over all refinement sweeps in mixed mode
 *   mode    : VIE_SOLVE_BF16X3_REFINE is VIE_SOLVE_FP32_REFINE below with the VIE_BF16X3 matvec in
 *             the FP32 GMRES cycles (the refinement residuals unchanged);
 *             VIE_SOLVE_FP64 (plain FP64: every restart recomputes the residual with
 *             the FP64 matvec) or VIE_SOLVE_FP32_REFINE (FP32 GMRES with FP64 iterative
 *             refinement: each sweep takes the residual in FP64, then runs FP32 cycles
 *             on the correction until every right-hand side is below
 *             max(2e-5 ||r||, tol ||P^-1 b|| / 2), restarting from the residual carried
 *             by the Krylov basis; Hessenberg matrix, rotations and the solution in
 *             FP64, Krylov vectors in FP32.  The first sweep's residual is b - A x with
 *             the FP64 matvec; a later one is the previous residual minus A d, d the
 *             sweep's correction, with A d from the FP32 matvec when |d| <=
 *             min(1e-3, 1e5 tol) |x| for every right-hand side, else the FP64 matvec)
 *   flags   : bit 0 = use x as initial guess; bit 1 = also compute true_resid
 *             (one more FP64 matvec), else true_resid = -1; bit 2 = keep no point for
 *             vie_fields (below); bit 3 = launch every kernel directly instead of replaying
 *             each restart cycle as a CUDA graph (same results, bit for bit)
 * Each restart cycle runs on the device without host round trips: the Arnoldi steps work on a
 * device list of the right-hand sides still above their target, and the host reads the list
 * once per cycle.  On a stream other than the legacy or per-thread default stream, the cycle is
 * captured once per solve as a CUDA graph (m Arnoldi steps of about 15 kernels each) and replayed.
 * Where chi, b and the guess all vanish (air), the rows of P^-1 A are the identity and
 * the solution is zero; the solver's vectors cover only each grid row's span of the
 * other voxels (the whole grid when that span covers it), so air costs no iterations'
 * memory traffic.  x is zero outside that span on exit.
 *   info    : vie_solve_info[nrhs] host array or NULL
 * Unless flags bit 2 is set, the handle keeps the point x1 of the solve's last FP64
 * residual matvec and the FP64 convolution (N - G) x1 on the full grid (2 x 16 bytes per
 * unknown of device memory) for vie_fields; a new solve on the handle drops them.  In FP64
 * mode x1 is the returned x.
 * Synchronous.  Returns VIE_NOT_CONVERGED (x = best iterate) when a right-hand side misses tol.
 */
int vie_solve(vie_handle* h, int nrhs, const void* b, void* x, double tol, int restart, int maxit, int mode,
              int flags, vie_solve_info* info, void* stream);

/*
 * vie_fields -- post-processing (Section IV-C): tested total field
 * e~ = e_inc + (1/c_e)(N - G) x, PWL field coefficients e = G^-1 e~, and the
 * absorbed power (Eq. 44) P_abs = 1/2 Re{x^* (c_e M_chi)^-1 G x}, as a per-voxel
 * density p_abs (W/m^3, zero in air) and its total, all in FP64.
 *   x, e_inc : [nrhs][12][nz][ny][nx] C128
 *   e_coeff  : [nrhs][12][nz][ny][nx] C128 output or NULL
 *   p_abs    : double[nrhs][nz][ny][nx] output or NULL
 *   P_abs    : double[nrhs] host output or NULL
 * The field map needs (N - G) x.  When the handle holds the point x1 of a vie_solve (same
 * nrhs) and |x - x1| <= 1e-3 |x| for every right-hand side, that product is the solver's
 * FP64 (N - G) x1 plus the FP32 product of d = x - x1: the FP32 term adds a relative error
 * of at most about 1e-6 |d| / |x| <= 1e-9 (none when x = x1, as after an FP64 solve).
 * Otherwise one FP64 matvec.  p_abs and P_abs depend on x alone.
 * Synchronous.
 */
int vie_fields(vie_handle* h, int nrhs, const void* x, const void* e_inc, void* e_coeff, double* p_abs,
               double* P_abs, void* stream);

/*
 * vie_green_toeplitz -- copy the 60 unique Toeplitz tensors of N - G computed by
 * vie_setup (the Gram term at offset 0 excluded) for offsets d in [0,nx)x[0,ny)x[0,nz):
 * out[t][dz][dy][dx] C128 with t = 10 * pq + ll, pq indexing the unordered
 * vector pair (xx,xy,xz,yy,yz,zz) and ll the ordered scalar pair l <= l'
 * ((1,1),(1,2),(1,3),(1,4),(2,2),(2,3),(2,4),(3,3),(3,4),(4,4)) (Section III-C: 6 x 10 = 60).
 * Entries for negative offsets follow from the reflection parities.  After vie_green_tucker with
 * VIE_TUCKER_APPLY the table is the Tucker reconstruction.  Synchronous.
 */
int vie_green_toeplitz(vie_handle* h, void* out);

/*
 * vie_green_tucker -- low multilinear rank (Tucker) compression of the handle's 60 Toeplitz
 * tensors of N - G (Section III-C: the defining tensors compress by low multilinear rank
 * decompositions).  Each tensor T [nz][ny][nx] becomes a core C [rz][ry][rx] and orthonormal
 * factors U_x [nx][rx], U_y [ny][ry], U_z [nz][rz], T~ = C x_z U_z x_y U_y x_x U_x, with
 * ||T - T~||_F <= tol ||T||_F: every factor spans its mode's unfolding up to a discarded energy of
 * tol^2 ||T||^2 / 3 (range from the unfolding's Gram matrix by pivoted Cholesky, so the ranks are
 * at least, and usually close to, those of the truncated HOSVD).  FP64 on the device.
 *   tol   : relative tolerance in [1e-7, 1) (the Gram matrices square the singular values, so
 *           smaller tolerances are not resolved in FP64)
 *   flags : VIE_TUCKER_APPLY = rebuild the handle's Green spectra from T~ (every later matvec
 *           and solve uses the compressed Green function) and keep the Tucker form in place of
 *           the full table (vie_green_toeplitz then returns T~; vie_info's bytes drop by the
 *           difference).  Without it the handle is unchanged apart from holding the form.
 *   ranks : int[60][3] host output (rx, ry, rz) per tensor, or NULL
 *   rel_err : double[60] host output ||T - T~||_F / ||T||_F per tensor, or NULL
 *   compressed_bytes : bytes of the Tucker form (cores and factors), or NULL
 * The K tensors are not compressed.  Synchronous.  Errors: VIE_EINVAL (tol out of range, a handle
 * sharing a server template's tensors), VIE_ENOMEM.
 */
#define VIE_TUCKER_APPLY 1
int vie_green_tucker(vie_handle* h, double tol, int flags, int* ranks, double* rel_err, size_t* compressed_bytes);

/*
 * vie_green_toeplitz_k -- the 30 unique Toeplitz tensors of the K operator, K u = curl S u
 * (Eq. 8; Galerkin entries of Eq. 25), for offsets d in [0,nx)x[0,ny)x[0,nz):
 * out[t][dz][dy][dx] C128 with t = 10 j + ll, j the axis of the derivative (x, y, z) and ll
 * the ordered scalar pair l <= l' as for vie_green_toeplitz (Section III-C: the
 * anti-symmetric kernel has 3 unique dyadic components, 3 x 10 = 30 tensors):
 *   P_t(d) = int int (d_j N^l)(r) g(r - r') N^l'(r') dr dr'   (d_j N^l with its face jumps),
 *   K^{(p,l),(q,l')}(d) = -eps_pjq P_t(d)   (eps the Levi-Civita symbol).
 * Computed on the device at each call (the handle keeps the cell moments of vie_setup for
 * no longer than setup, so they are computed again).  out: host or device memory of
 * 30 nx ny nz complex values.  Entries for negative offsets follow from the reflection
 * parities of N times -1.  Synchronous.  Errors: VIE_EINVAL (NULL), VIE_ENOMEM, VIE_EDEVICE.
 */
int vie_green_toeplitz_k(vie_handle* h, void* out);

/*
 * vie_rhs_dipoles_h -- tested incident magnetic fields of nrhs Hertzian dipoles, one per
 * right-hand side: h_inc = curl (g p) = grad g x p (Eq. 8, g of Eq. 10, p = I l), tested
 * with the 6x6x6 Gauss-Legendre rule per voxel of vie_rhs_dipoles.
 *   pos, mom : double[nrhs][3] (m, A m), host memory
 *   h_inc    : [nrhs][12][nz][ny][nx] C128 output (host or device)
 * Synchronous.
 */
int vie_rhs_dipoles_h(vie_handle* h, int nrhs, const double* pos, const double* mom, void* h_inc, void* stream);

/*
 * vie_hfields -- magnetic post-processing (Section II total fields: h_tot = h_inc + K j): tested field
 * h~ = h_inc + K x (K in FP64 as vie_matvec VIE_OP_K), PWL coefficients h = G^-1 h~, the
 * transmit field b1+ = mu0 (h_x + i h_y) of the voxel-average (l = 1) coefficients
 * (Section V-D), and the magnetic energy W_m = 1/4 int mu0 |h|^2 over the scatterer
 * (chi != 0; Section V-D, exact for the PWL field since the four functions of a voxel are
 * orthogonal).
 *   x, h_inc : [nrhs][12][nz][ny][nx] C128 (x: current coefficients of vie_solve)
 *   h_coeff  : [nrhs][12][nz][ny][nx] C128 output or NULL
 *   b1_plus  : [nrhs][nz][ny][nx] C128 output (T per unit source) or NULL
 *   W_m      : double[nrhs] host output (J) or NULL
 * Synchronous.
 */
int vie_hfields(vie_handle* h, int nrhs, const void* x, const void* h_inc, void* h_coeff, void* b1_plus, double* W_m,
                void* stream);

/*
 * Full JM-VIE (Eq. 14-15): polarization current j and magnetization current m of a scatterer
 * with relative permeability mu_r = mu' - i mu'' (Eq. 1-2; chi_m = mu_r - 1, Eq. 7).  PWL
 * handles only, FP64 (the K products are those of VIE_OP_K; vie_jm_solve can run its inner
 * GMRES in FP32).
 *
 * Unknowns: both currents in the PWL functions of Section III, with the magnetization scaled,
 * m' = m / eta0 (eta0 = sqrt(mu0/eps0)), and the second row of Eq. 15 divided by eta0.  Since
 * c_e eta0 = c_m / eta0 = i k0 the Galerkin system reads
 *     [ M_eps G - M_chie N      i k0 M_chie K      ] [j ]   [ c_e M_chie e_inc  ]
 *     [ -i k0 M_chim K          M_mu G - M_chim N  ] [m'] = [ i k0 M_chim h_inc ]
 * (the same solution as Eq. 15, with m = eta0 m'), preconditioned by P = diag(M_eps G, M_mu G).
 * Vectors of this system: [nrhs][2][12][nz][ny][nx] C128, index 0 of the axis of length 2 = j,
 * index 1 = m'.  With mu_r = 1 the second current vanishes and j solves Eq. 16.
 * Host or device buffers as for vie_matvec; vie_jm_matvec and vie_jm_rhs follow the stream rule
 * above, vie_jm_solve and vie_jm_fields are synchronous.  Scratch: 2 x 24 nrhs nv complex values
 * for the two products plus the K path's padded spectra (VIE_OP_K).
 */

/*
 * vie_set_permeability -- relative permeability per voxel, mu_r = mu_real - i mu_imag
 * (mu_real > 0, mu_imag >= 0, finite; [nz][ny][nx] doubles, host or device).  Until it is
 * called the JM calls take mu_r = 1.  Errors: VIE_EINVAL (NULL, a PWC handle, an entry out of
 * range), VIE_ENOMEM.
 */
int vie_set_permeability(vie_handle* h, const double* mu_real, const double* mu_imag);

/*
 * vie_jm_matvec -- y = A x (op VIE_OP_A) or y = P^-1 A x (op VIE_OP_PA) of the JM system above
 * for nrhs vectors.  precision VIE_FP64 (x, y double pairs) or VIE_FP32 (float pairs: both
 * products and the combination in FP32, the operator of vie_jm_solve's inner GMRES in
 * VIE_SOLVE_FP32_REFINE).  x and y must not overlap.  Errors: VIE_EINVAL (NULL, PWC handle,
 * another precision or operator), VIE_ENOMEM.
 */
int vie_jm_matvec(vie_handle* h, int nrhs, const void* x, void* y, int precision, int op, void* stream);

/*
 * vie_jm_rhs -- right-hand sides b = (c_e chi_e e_inc, i k0 chi_m h_inc) (Eq. 14, second row
 * divided by eta0) from tested incident fields e_inc, h_inc [nrhs][12][nz][ny][nx] C128
 * (vie_rhs_dipoles / vie_rhs_planewave and vie_rhs_dipoles_h); b: [nrhs][2][12][nz][ny][nx].
 */
int vie_jm_rhs(vie_handle* h, int nrhs, const void* e_inc, const void* h_inc, void* b, void* stream);

/*
 * vie_jm_solve -- restarted GMRES(restart) on P^-1 A x = P^-1 b of the JM system with the
 * batched device Arnoldi steps of vie_solve (chunks of steps replayed as CUDA graphs, as there),
 * stopping when ||P^-1 (b - A x)|| / ||P^-1 b|| <= tol.  The solver's vectors cover the
 * voxels where chi_e, chi_m, b or the guess is non-zero (rows of the grid as for vie_solve).
 *   b, x  : [nrhs][2][12][nz][ny][nx] C128; x is the initial guess when (flags & 1)
 *   mode  : VIE_SOLVE_FP64, or VIE_SOLVE_FP32_REFINE (FP32 inner GMRES, both products of the
 *           operator in FP32, inside FP64 iterative refinement as vie_solve's mode of that name);
 *           VIE_SOLVE_BF16X3_REFINE is refused (the K block has no BF16x3 z pass)
 *   flags : bit 0 = use x as initial guess; bit 1 = also compute true_resid (||b - A x|| / ||b||);
 *           bit 3 = launch the steps directly instead of replaying CUDA graphs
 *   info  : vie_solve_info[nrhs] or NULL
 * Returns VIE_NOT_CONVERGED (x = best iterate) when a right-hand side misses tol; VIE_EINVAL for
 * an unknown mode or flag.
 */
int vie_jm_solve(vie_handle* h, int nrhs, const void* b, void* x, double tol, int restart, int maxit, int mode,
                 int flags, vie_solve_info* info, void* stream);

/*
 * vie_jm_fields -- total fields of the JM solution (Eq. 13, tested, then divided by G):
 *   e = (e_inc + (1/c_e)(N - G) j - eta0 K m') / G,   h = (h_inc + K j + (1/(i k0))(N - G) m') / G,
 * and the absorbed power, electric plus magnetic loss:
 *   P_abs = 1/2 Re{ j^* (c_e M_chie)^-1 G j } + 1/2 Re{ eta0 m'^* (i k0 M_chim)^-1 G m' }
 * (Eq. 44 and its magnetic analogue, 1/2 int omega mu0 mu'' |h|^2), per voxel in W/m^3 and summed.
 *   x            : [nrhs][2][12][nz][ny][nx] C128;  e_inc, h_inc : [nrhs][12][nz][ny][nx] C128
 *   e_coeff, h_coeff : [nrhs][12][nz][ny][nx] C128 outputs or NULL
 *   p_abs        : double[nrhs][nz][ny][nx] output or NULL;  P_abs : double[nrhs] host output or NULL
 */
int vie_jm_fields(vie_handle* h, int nrhs, const void* x, const void* e_inc, const void* h_inc, void* e_coeff,
                  void* h_coeff, double* p_abs, double* P_abs, void* stream);

/* Sizes used by the handle: FFT lengths per axis and bytes of device memory held. */
int vie_info(vie_handle* h, int* fft_len_xyz, size_t* device_bytes);

/*
 * Launch accounting.  The library counts every kernel it launches, per kernel
 * name; with timing enabled it also records a CUDA event pair on the launch
 * stream around each launch and accumulates the device time per name.
 * vie_stats_reset clears the counters and switches timing on (1) or off (0).
 * vie_stats_read synchronises on the recorded events and returns up to
 * max_entries rows: names (max_entries x 48 chars, NUL-terminated), launch
 * counts, milliseconds (0 without timing) and algorithmic bytes (the bytes
 * each launch must read and write at minimum: its inputs once, its outputs
 * once); *n_entries rows written and *total_launches over all names.  Any
 * output pointer may be NULL.  Host memory.  Counters are process-wide.
 * Launches inside a solver cycle that find no active right-hand side return at once: they are
 * not in the per-name counts but are in *total_launches (every launch issued).  Kernels
 * replayed from a CUDA graph are counted (and timed) per replay.
 * vie_stats_read synchronises the device first.
 */
int vie_stats_reset(int enable_timing);
int vie_stats_read(int max_entries, char* names, long long* launches, double* ms, double* bytes, int* n_entries,
                   long long* total_launches);

/*
 * Serving: a request loop with continuous batching (no counterpart in the paper, which
 * runs one solve at a time).  A request is one dielectric solve of the method: setup of
 * the grid, voxel size, frequency and material map (as vie_setup), nrhs dipole
 * right-hand sides (as vie_rhs_dipoles), GMRES (as vie_solve, flags 0) and the fields
 * and absorbed power (as vie_fields).  Up to max_concurrent requests run at once, each
 * on its own host thread and CUDA stream, so their kernels overlap on the device; when
 * one finishes, the next admissible request starts at once.  A request is admitted when
 * its device working set, plus its Green tensors if not yet cached, fits in the budget
 * (least recently used idle Green tensors are evicted first); requests are served in
 * submission order, except that a later request may start ahead of one that does not
 * fit yet (at most 4 times per waiting request).  Green tensors depend only on (grid,
 * voxel size, frequency): each key is built once and shared by every request with it.
 * Each result is the one the four calls above give on their own.
 */
typedef struct vie_server vie_server;

typedef struct {
    vie_grid grid;
    double freq_hz;
    const double* eps_real;  /* [nz][ny][nx] host, copied by vie_submit */
    const double* sigma;     /* [nz][ny][nx] host (S/m), copied by vie_submit */
    int nrhs;
    const double* dip_pos;   /* [nrhs][3] host positions (m), copied */
    const double* dip_mom;   /* [nrhs][3] host moments (A m), copied */
    double tol;              /* GMRES tolerance (as vie_solve) */
    int restart, maxit, mode;
    /* optional caller-owned host outputs (NULL to skip), written before the result is
       ready; they must stay valid until vie_poll has returned the result */
    void* x_out;             /* [nrhs][12][nz][ny][nx] C128 solution */
    double* p_abs_out;       /* [nrhs][nz][ny][nx] absorbed power density (W/m^3) */
    double* P_abs_out;       /* [nrhs] absorbed power (W) */
} vie_request;

typedef struct {
    int status;        /* VIE_OK, VIE_NOT_CONVERGED, or the negative error of the failed step */
    int nrhs;
    int iterations;    /* largest GMRES iteration count over the right-hand sides */
    int green_cached;  /* 1 when the request found its Green tensors in the cache */
    double queued_s;   /* seconds from vie_submit to the start of the solve */
    double run_s;      /* seconds of setup, solve and post-processing */
    double resid;      /* largest final relative residual */
    double start_s, end_s;          /* host span of the request, seconds since vie_server_create */
    double dev_start_s, dev_end_s;  /* device span: CUDA events on the request's stream before its
                                       first and after its last kernel, seconds after an event
                                       recorded at vie_server_create (-1 if unavailable) */
} vie_result;

/*
 * vie_server_create -- start a request loop on the current device.
 *   hbm_budget_bytes : device memory the loop may use for working sets and cached
 *                      Green tensors; 0 = 85% of the free memory now
 *   max_concurrent   : requests in flight at once, 1..64
 * VIE_EINVAL for a budget above the free memory or a bad count.
 */
int vie_server_create(size_t hbm_budget_bytes, int max_concurrent, vie_server** out);
/* Stops the loop: queued requests are dropped, running ones finish first; frees the cache. */
void vie_server_destroy(vie_server* s);
/* Queue a request (its host inputs are copied); *ticket identifies it.  VIE_ENOMEM when
   it could never fit in the budget, VIE_EINVAL for invalid fields. */
int vie_submit(vie_server* s, const vie_request* req, unsigned long long* ticket);
/* Wait at most timeout_us (>= 0) microseconds for the request: VIE_OK with *out filled
   (the ticket is then retired), VIE_ETIMEOUT when it is still queued or running,
   VIE_EINVAL for an unknown or retired ticket. */
int vie_poll(vie_server* s, unsigned long long ticket, int timeout_us, vie_result* out);
/* Snapshot: queued requests, requests running, device bytes reserved, cached Green keys. */
int vie_server_stats(vie_server* s, int* queued, int* running, size_t* bytes_in_use, int* cache_entries);

/*
 * Host-side fault injection for tests of the failure paths (no counterpart in the paper).
 * Nothing here touches the GPU: an injected failure is returned by the host code at the point
 * where the real one would be detected, and the handle stays usable.
 *   VIE_INJECT_OOM  : the next `count` growths of a handle's device workspace (matvec spectra,
 *                     solver vectors, staging, post-processing scratch) fail with VIE_ENOMEM
 *                     before allocating
 *   VIE_INJECT_NONE : clear every pending injection (count ignored)
 * Process-wide.  VIE_EINVAL for an unknown kind or count < 0.
 */
#define VIE_INJECT_NONE 0
#define VIE_INJECT_OOM 1
int vie_fault_inject(int kind, int count);

/*
 * vie_tuning -- the launch configurations the library's autotuner measured and chose (no
 * counterpart in the paper).  The z-pass kernels are compiled for several tile widths (column
 * lines per CTA); the first time a grid shape and right-hand side class (the count rounded up to
 * a power of two, at most 8) is seen outside stream capture, each width runs on a scratch
 * spectrum of that many right-hand sides (allocated for the measurement) and the fastest median
 * device time wins for the process.  Writes one line per measured shape, NUL-terminated,
 * into out[len] (truncated to fit; out may be NULL); returns the full text length.
 */
int vie_tuning(char* out, size_t len);

/* Static description of an error code. */
const char* vie_strerror(int code);

/* Detail of the most recent error on the calling thread ("" if none). */
const char* vie_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VIE_H */
