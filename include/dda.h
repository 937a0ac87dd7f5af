/*
 * dda.h -- C-ABI of the GB300 (sm_103a) discrete dipole approximation library.
 *
 * The library computes the DDA of Yurkin, Maltsev & Hoekstra
 * (arXiv:0704.0037): the dipole polarizations P of Eq. (1), obtained by
 * solving the Jacobi-symmetrised system of Eqs. (2)-(3),
 *
 *     x_i - sum_{j != i} beta_i G_ij beta_j x_j = beta_i E_inc,i ,   P_i = beta_i x_i,
 *
 * with the interaction-matrix product done by zero-padded FFT convolution
 * split into 1D transforms with pruning (Sec. 2, performance paragraph),
 * inside the complex-symmetric Krylov solvers of Sec. 2 (QMR, Bi-CG,
 * Bi-CGSTAB, CGNR), stopped on the relative residual norm (default 1e-5).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns an int status (enum dda_status); no exception, abort
 *   or longjmp crosses the ABI.  A negative status sets a per-handle message
 *   readable with dda_last_error().  Nothing is silently downgraded: there is
 *   no CPU fallback, and a missing or failing GPU gives DDA_ERR_CUDA.
 * - Units: lengths in dipole sizes d; kd = k d; |E0| = 1; the polarizations
 *   are dimensionless (alpha in units of d^3), Gaussian units.
 * - Lattice: a box of nx*ny*nz cells, host arrays with x fastest
 *   (index = (iz*ny + iy)*nx + ix); cell centres r = ((2i+1-n)/2) per axis, so
 *   the origin (and the phase origin of E_inc) is the box centre.
 * - Occupied ("real") dipoles are numbered 0..N_occ-1 in that x-fastest scan
 *   order.  A complex vector on the dipoles is laid out [nrhs][3][N_occ],
 *   interleaved (re, im): complex128 (16 B) or complex64 (8 B) per element.
 * - The handle owns all its device workspace (FFT of G, padded FFT buffers,
 *   Krylov vectors).  Buffers passed as *_dev are caller-owned device memory
 *   (e.g. torch tensors); *_host pointers are caller-owned host memory.
 * - All device work is enqueued on the stream given at dda_init_lattice
 *   (NULL = legacy default stream).  Calls that return host results
 *   (dda_solve, dda_scatter) synchronise that stream before returning.
 * - A handle is not thread-safe: use one handle per host thread.
 * - A handle belongs to the device that was current at dda_init_lattice.
 *   Every call taking a handle makes that device current while it runs and
 *   gives the calling thread its previous current device back before it
 *   returns (dda_farfield_noalloc excepted: it switches no device and
 *   requires the handle's device to be current).
 */
#ifndef DDA_H
#define DDA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dda_ctx* dda_t;                 /* opaque handle */

enum dda_status {
  DDA_OK = 0,
  DDA_NOT_CONVERGED = 1,   /* maxiter reached; results are those of the last iterate   */
  DDA_BREAKDOWN = 2,       /* Lanczos/Bi-CG breakdown (a zero pivot), no look-ahead       */
  DDA_ERR_ARG = -1,        /* invalid argument (NULL pointer, size, enum value)          */
  DDA_ERR_CUDA = -2,       /* a CUDA call failed (message holds cudaGetErrorString)      */
  DDA_ERR_OOM = -3,        /* device allocation failed                                   */
  DDA_ERR_STATE = -4,      /* call out of order (e.g. product before dda_build_Dmatrix)  */
  DDA_ERR_NONFINITE = -5,  /* a NaN/Inf appeared in a solver reduction                   */
  DDA_ERR_TIMEOUT = -6     /* reserved: a bounded device wait gave up                    */
};

/* Polarizability prescriptions of Sec. 2: Clausius-Mossotti, radiative
 * reaction, lattice dispersion relation, corrected LDR.  All are diagonal. */
enum dda_pol { DDA_CM = 0, DDA_RR = 1, DDA_LDR = 2, DDA_CLDR = 3 };

/* Iterative solvers of Sec. 2; QMR and Bi-CG use the complex symmetry of A. */
enum dda_solver { DDA_QMR_CS = 0, DDA_BICG_CS = 1, DDA_BICGSTAB = 2, DDA_CGNR = 3 };

/* Arithmetic of the product / solve.  DDA_FP64: complex128 everywhere (the
 * paper's choice, Sec. 2).  DDA_FP32_REFINED: complex64 vectors and FFTs with
 * an FP64-class D-matrix build, FP64 Krylov scalars and inner products, and
 * an outer iterative refinement on the true residual computed from complex128
 * vectors.  On grids whose three padded lengths have register-resident passes
 * in every precision (32, 40, 48, 64, 80, 96, 128, 256, 270) the
 * FP32_REFINED D-matrix build and its residual
 * products run in double-float arithmetic (pairs of floats, about 48
 * significant bits, on the FP32 pipe); elsewhere in FP64.
 * DDA_FP64_PAIR (dda_matvec only): that double-float product on complex128
 * vectors; needs a DDA_FP32_REFINED build on such a grid, no adjoint. */
enum dda_prec { DDA_FP64 = 0, DDA_FP32_REFINED = 1, DDA_FP64_PAIR = 2 };

/*
 * dda_init_lattice -- create a handle for one particle (Sec. 2 Eq. (1); the
 * lattice and the volume correction of Sec. 3.1).
 *   out        : receives the new handle (set to NULL on failure).
 *   nx,ny,nz   : box size in cells, each >= 1.
 *   occ_host   : nx*ny*nz bytes, x fastest; 0 = void, k in 1..n_mat = material k.
 *   n_mat      : number of materials, 1..255.
 *   m_host     : 2*n_mat doubles, refractive index of material k as (re, im).
 *   kd         : k*d if volume_corrected == 0; otherwise the size parameter
 *                x = k a_eq and the library sets kd = x (4 pi / (3 N_occ))^(1/3)
 *                so that N_occ d^3 equals the sphere volume (Sec. 3.1).
 *   cuda_stream: cudaStream_t on which all device work is enqueued.
 * Errors: DDA_ERR_ARG (bad sizes, no occupied cell, material index > n_mat),
 *   DDA_ERR_CUDA / DDA_ERR_OOM.  Copies what it needs from the host arrays.
 * The FFT passes use register-resident kernels for padded lengths with a
 * compiled split (32, 40, 48, 64, 80, 96, 128, 256, 270; for complex64 also
 * 512 and 1080) and shared-memory Stockham kernels otherwise;
 * dda_set_fft_engine selects the latter for every length.  An axis is padded
 * to the smallest compiled length >= 2n - 1 when that is within 1.35x of the
 * smallest 7-smooth one, else to the 7-smooth one.
 */
int dda_init_lattice(dda_t* out, int nx, int ny, int nz, const uint8_t* occ_host,
                     int n_mat, const double* m_host, double kd, int volume_corrected,
                     void* cuda_stream);

/*
 * dda_set_fft_engine -- which FFT kernels the handle's products use.
 *   engine : DDA_ENGINE_AUTO (the default) -- register-resident two-level
 *            passes for padded lengths with a compiled split, shared-memory
 *            Stockham passes otherwise; DDA_ENGINE_STOCKHAM -- the Stockham
 *            passes for every length (both give the same product to rounding;
 *            the FP32_REFINED build then uses FP64 instead of double-float).
 * Must precede the first dda_build_Dmatrix of the handle (DDA_ERR_STATE after
 * it); DDA_ERR_ARG for an unknown value.  No counterpart in the paper (Sec. 2
 * names the FFT libraries ADDA can use).
 */
enum dda_engine { DDA_ENGINE_AUTO = 0, DDA_ENGINE_STOCKHAM = 1 };
int dda_set_fft_engine(dda_t h, int engine);

/*
 * dda_set_pass_tiles / dda_get_pass_tiles -- tile variants of the
 * register-resident product passes: lines per block of the y forward pass,
 * the fused z pass and the y inverse pass (tiles[0..2]), for the products of
 * one arithmetic (prec: DDA_FP32_REFINED the complex64 products, DDA_FP64 the
 * complex128 ones, DDA_FP64_PAIR the double-float ones).
 *   0  : the default lines per block (16 columns complex64, 8 wider; fewer
 *        where the z pass's spectra would not fit in shared memory);
 *   1  : half as many lines per block (twice the blocks);
 *   -1 : chosen by dda_build_Dmatrix, which times both variants of each pass
 *        on the handle's own buffers (CUDA events, three launches) and takes
 *        the half tiles when they are at least 3 % faster (cached per device
 *        and grid shape).  The default.
 * Every variant computes each line with the same arithmetic: the products
 * agree bit for bit.  dda_set_pass_tiles with tiles == NULL sets -1 for all
 * three; an entry set to 0 or 1 is kept by later builds.  dda_get_pass_tiles
 * writes the current entries to tiles[0..2] (-1 before the first build).
 * Errors: DDA_ERR_ARG (null handle, unknown precision, a value outside
 * -1..1, null tiles for the get).  No counterpart in the paper (Sec. 2 names
 * the FFT libraries ADDA can use; FFTW plans its transforms by timing).
 */
int dda_set_pass_tiles(dda_t h, int prec, const int* tiles);
int dda_get_pass_tiles(dda_t h, int prec, int* tiles);

/*
 * dda_build_Dmatrix -- FFT of the Green's tensor on the padded grid (Sec. 2:
 * the product is an FFT convolution and the symmetry of the interaction
 * matrix reduces the memory of its Fourier transform).
 * Builds G (FP64) on an M_x*M_y*M_z grid with M >= 2n - 1 (7-smooth), takes
 * its 3D FFT in FP64 and keeps the 6 components on the octant
 * k_mu in [0, M_mu/2] (the rest follows from parity), pre-scaled by
 * 1/(M_x M_y M_z).  prec = DDA_FP32_REFINED also keeps a complex64 copy.
 * Errors: DDA_ERR_ARG, DDA_ERR_CUDA, DDA_ERR_OOM.
 */
int dda_build_Dmatrix(dda_t h, int prec);

/*
 * dda_set_beta -- polarizability and beta = sqrt(alpha) (Eq. (2), principal
 * branch) used by dda_matvec for each right-hand side.
 *   pol_prescription : enum dda_pol.
 *   nrhs             : number of right-hand sides, >= 1.
 *   prop_host        : 3*nrhs doubles, unit propagation vectors a (LDR's S term
 *                      and CLDR's a_mu^2 depend on them).
 *   polvec_host      : 6*nrhs doubles, polarisation e of each RHS as 3 complex
 *                      (re, im) -- LDR's S = sum_mu (a_mu e_mu)^2.
 * Errors: DDA_ERR_ARG.  The beta table is computed on the device in FP64.
 */
int dda_set_beta(dda_t h, int pol_prescription, int nrhs, const double* prop_host,
                 const double* polvec_host);

/*
 * dda_matvec -- y = A x with A of Eq. (2), for nrhs right-hand sides:
 *   y_i = x_i - beta_i sum_{j != i} G_ij beta_j x_j.
 *   prec  : DDA_FP64 -> x, y are complex128; DDA_FP32_REFINED -> complex64.
 *   x_dev : caller-owned device buffer [nrhs][3][N_occ] (read only).
 *   y_dev : caller-owned device buffer [nrhs][3][N_occ] (written); must not
 *           alias x_dev.
 *   nrhs  : must not exceed the nrhs of the last dda_set_beta; RHS r uses
 *           beta table r.
 * Errors: DDA_ERR_STATE (no D-matrix of that precision, no beta),
 *   DDA_ERR_ARG, DDA_ERR_CUDA.  Asynchronous on the handle's stream.
 */
int dda_matvec(dda_t h, int prec, const void* x_dev, void* y_dev, int nrhs);

/*
 * dda_matvec_adjoint -- y = A^H x = conj(A conj(x)) (A is complex symmetric,
 * Eq. (2)); the product CGNR needs.  Same arguments as dda_matvec.
 */
int dda_matvec_adjoint(dda_t h, int prec, const void* x_dev, void* y_dev, int nrhs);

typedef struct {
  int solver;           /* enum dda_solver                                       */
  int pol;              /* enum dda_pol: polarizability prescription             */
  int prec;             /* enum dda_prec                                         */
  double tol;           /* stop when ||b - A x||_2 / ||b||_2 < tol (Sec. 2: 1e-5) */
  int maxiter;          /* iterations per RHS (inner iterations summed for FP32)  */
  double inner_tol;     /* FP32_REFINED: relative tolerance of each inner solve   */
  int checkpoint_every; /* > 0: save the solve's state into checkpoint_host
                           every this many iterations (QMR-CS without a
                           residual history only; FP64: at the first host
                           synchronisation, every 8 steps, at or after each
                           multiple; FP32_REFINED: between refinement steps,
                           at the first one after each multiple of inner
                           iterations); 0: none                                */
  int inner_cap;        /* FP32_REFINED: complex64 steps an inner solve may take
                           before the later inner solves switch to complex128
                           vectors and FP64-class products; <= 0: 1000          */
  void* checkpoint_host;       /* host buffer of the solver state (or NULL)      */
  long long checkpoint_bytes;  /* its size, >= dda_checkpoint_bytes()            */
  int checkpoint_stop;  /* nonzero: return right after the first save; the
                           right-hand sides not yet converged report
                           DDA_NOT_CONVERGED and P holds the current iterate   */
  int resume;           /* nonzero: continue the solve saved in checkpoint_host
                           (same handle lattice, precision, right-hand sides
                           and incidences, else DDA_ERR_ARG) instead of starting
                           from x0 = 0; maxiter counts the iterations before the
                           save too, and the continued solve is the one an
                           uninterrupted solve would have done, bit for bit    */
} dda_solve_opts;

/*
 * dda_checkpoint_bytes -- size of the host buffer that dda_solve_opts'
 * checkpoints of a QMR-CS solve of nrhs right-hand sides in precision prec
 * need on this handle (ADDA's checkpoints, Sec. 2, let a long solve be
 * stopped and resumed; here the caller owns the buffer and may write it to
 * a file).  FP64: about 8 x nrhs x 3 N_occ x 16 bytes; FP32_REFINED: about
 * 3 x nrhs x 3 N_occ x 16 bytes.  DDA_ERR_ARG on bad arguments.
 */
int dda_checkpoint_bytes(dda_t h, int prec, int nrhs, long long* bytes);

typedef struct {
  int status;           /* enum dda_status of this RHS                           */
  int iters;            /* solver iterations (all inner iterations for FP32)      */
  int matvecs;          /* products with A or A^H (any precision)                 */
  int matvecs_fp64;     /* of which FP64-class (native FP64, or double-float)     */
  int outer;            /* FP32_REFINED: refinement steps; FP64: 0                */
  double rel_res_true;  /* ||b - A x|| / ||b|| recomputed at exit with an FP64-class
                           product: native FP64, or for FP32_REFINED on grids with
                           register-resident passes double-float (about 48
                           significant bits); dda_residual gives the native FP64 one */
  double rel_res_recur; /* the solver's own residual estimate at exit             */
  double seconds;       /* wall time of this RHS                                  */
} dda_solve_info;

/*
 * dda_solve -- solve Eq. (3) for nrhs incident plane waves and return
 * P = beta x (Eq. (3)).  Starts from x0 = 0.
 *   opts      : solver options (host).
 *   prop_host : 3*nrhs doubles, unit propagation vectors.
 *   pol_host  : 6*nrhs doubles, unit polarisations (complex, re/im pairs).
 *   P_dev     : caller-owned device buffer [nrhs][3][N_occ] complex128 (out).
 *   res_hist  : optional host [nrhs][hist_len] relative residual per iteration
 *               (index 0 = 1.0 before the first iteration); unused tail = -1.
 *   info      : host array of nrhs dda_solve_info.
 * Also leaves beta set for these RHS (as dda_set_beta).  Requires
 * dda_build_Dmatrix for DDA_FP64, and with DDA_FP32_REFINED for that mode.
 * With DDA_QMR_CS and no res_hist the right-hand sides are solved together as
 * dda_solve_batch does (same iterates; info[r].seconds is then the whole
 * call's time); otherwise one after the other, with the scalars read every
 * step.  Returns the worst per-RHS status (errors first, then BREAKDOWN,
 * NOT_CONVERGED).  Synchronises the stream.
 */
int dda_solve(dda_t h, const dda_solve_opts* opts, int nrhs, const double* prop_host,
              const double* pol_host, void* P_dev, double* res_hist, int hist_len,
              dda_solve_info* info);

/*
 * dda_solve_batch -- dda_solve for all nrhs right-hand sides at once (QMR-CS
 * only; no counterpart in the paper, which solves one right-hand side at a
 * time): every QMR step is one launch per product pass and per solver kernel
 * for all right-hand sides (the products of converged ones are skipped), and
 * the host reads the solver scalars every 8 steps instead of every step.  The
 * arithmetic per right-hand side is that of dda_solve with QMR-CS (the
 * iterates agree to rounding), and FP32_REFINED runs the same refinement per
 * right-hand side (inner complex64 solves of all unfinished right-hand sides
 * together, then one batched FP64-class residual product: double-float on
 * grids with register-resident passes, else FP64).  An inner complex64 solve
 * gets at most opts->inner_cap steps (1000 when inner_cap <= 0);
 * if it needs more, the following inner solves keep complex128 Krylov vectors
 * and use the FP64-class product, which converges hard problems at the FP64
 * rate where complex64 Lanczos vectors stall.  Arguments as dda_solve
 * (no history); opts->solver must be DDA_QMR_CS (else DDA_ERR_ARG).
 * info[r].seconds is the wall time of the whole call.  Allocates per call
 * about nrhs x (8 complex64 + 4 complex128) x 3 N_occ (FP32_REFINED) or
 * nrhs x 8 complex128 x 3 N_occ (FP64) of device memory, kept by the handle,
 * and grows the product buffers to up to 64 right-hand sides.
 * Synchronises the stream.
 */
int dda_solve_batch(dda_t h, const dda_solve_opts* opts, int nrhs, const double* prop_host,
                    const double* pol_host, void* P_dev, dda_solve_info* info);

/*
 * dda_solve_many -- many particles at once (no counterpart in the paper): a
 * pool of n_threads host threads takes the particles in order; each builds
 * the particle's D-matrix for opts->prec if it is missing and runs
 * dda_solve_batch on it, so the kernels of different particles overlap on
 * the device.  Each handle must be distinct (a handle is not thread-safe)
 * and should own a distinct non-default stream (dda_init_lattice) for the
 * particles to overlap.
 *   hs[i], nrhs[i], prop[i], pol[i], P[i], info[i] : as dda_solve_batch for
 *   particle i (arrays of n_part pointers).
 *   status_out : n_part ints, the status of each particle.
 * Returns the worst status (errors before NOT_CONVERGED before OK), or
 * DDA_ERR_ARG for null or repeated arguments (nothing runs then).
 */
int dda_solve_many(int n_part, dda_t const* hs, const dda_solve_opts* opts, const int* nrhs,
                   const double* const* prop_host, const double* const* pol_host,
                   void* const* P_dev, dda_solve_info* const* info, int n_threads,
                   int* status_out);

/*
 * dda_residual -- the relative residual ||b - A x||_2 / ||b||_2 of Sec. 2's
 * stopping criterion for given polarizations P, evaluated outside any solver
 * with the native FP64 (complex128) product: x = P / beta, b = beta E_inc
 * (Eq. (3)).  Used to check a solution whatever precision produced it.
 *   pol_prescription, nrhs, prop_host, pol_host : as dda_solve (also leaves
 *                      beta set for these right-hand sides, as dda_set_beta).
 *   P_dev        : device [nrhs][3][N_occ] complex128 (read only).
 *   res_out_host : nrhs doubles (0 where b = 0).
 * Requires dda_build_Dmatrix (either precision; a FP32_REFINED build derives
 * its FP64 octant on first use).  Uses 4 x 3 N_occ complex128 of the handle's
 * solver workspace.  Synchronises the stream.
 */
int dda_residual(dda_t h, int pol_prescription, int nrhs, const double* prop_host,
                 const double* pol_host, const void* P_dev, double* res_out_host);

/*
 * dda_scatter -- scattering quantities of Sec. 3.1 from P (FP64 sums).
 *   pol_prescription : the prescription P was computed with (Q_abs needs alpha).
 *   P_dev     : device [nrhs][3][N_occ] complex128.
 *   prop_host, pol_host : as in dda_solve (E_inc for Q_ext, alpha for Q_abs).
 *   n_dir, dirs_host : n_dir unit directions n (3 doubles each), may be 0.
 *   weights_host     : optional n_dir quadrature weights (sum 4 pi); when given,
 *                      Q_sca = (1/(pi x^2)) sum_k w_k |F(n_k)|^2.
 *   F_out_host : host [nrhs][n_dir][3] complex (re, im): the amplitude
 *                F(n) = -i kd^3 (I - n n) sum_j P_j exp(-i kd n.r_j).
 *   q_out_host : host [nrhs][3] = (Q_ext, Q_abs, Q_sca); Q_sca is NaN without
 *                weights.  x = kd (3 N_occ / (4 pi))^(1/3) normalises Q.
 * Synchronises the stream.
 */
int dda_scatter(dda_t h, int pol_prescription, const void* P_dev, int nrhs,
                const double* prop_host, const double* pol_host, int n_dir,
                const double* dirs_host, const double* weights_host, double* F_out_host,
                double* q_out_host);

/*
 * dda_mueller_plane -- S11(theta) in the xz scattering plane (Sec. 3.1: all
 * Mueller elements in one scattering plane; S11 is the one the paper plots)
 * from the amplitudes of x- and y-polarised incidence along +z evaluated at
 * n = (sin t, 0, cos t): S2 = theta.F_x, S4 = -y.F_x, S3 = -theta.F_y,
 * S1 = y.F_y (Bohren-Huffman amplitude matrix), S11 = (|S1|^2+...+|S4|^2)/2.
 *   F_xpol_host, F_ypol_host : [n_theta][3] complex (as dda_scatter returns).
 *   theta_deg_host : n_theta angles in degrees.   s11_out_host : n_theta doubles.
 * Host-only arithmetic; no device work.
 */
int dda_mueller_plane(int n_theta, const double* theta_deg_host, const double* F_xpol_host,
                      const double* F_ypol_host, double* s11_out_host);

/*
 * dda_mueller_plane_full -- all 16 Mueller elements in the xz scattering
 * plane (Sec. 3.1: "all Mueller matrix elements in one scattering plane"),
 * from the same amplitudes as dda_mueller_plane.  With the amplitude matrix
 * [[S2, S3], [S4, S1]] acting on (E_par, E_perp) and Stokes vectors
 * (I, Q, U, V) = (|E_par|^2+|E_perp|^2, |E_par|^2-|E_perp|^2,
 * 2 Re(E_par E_perp^*), -2 Im(E_par E_perp^*)) (Bohren-Huffman), the scattered
 * Stokes vector is M times the incident one.
 *   M_out_host : n_theta x 16 doubles, row-major M[i][j] (M11 first).
 * Host-only arithmetic; no device work.  DDA_ERR_ARG on a null pointer.
 */
int dda_mueller_plane_full(int n_theta, const double* theta_deg_host, const double* F_xpol_host,
                           const double* F_ypol_host, double* M_out_host);

/*
 * dda_asymmetry -- the asymmetry parameter <cos theta> (Sec. 3.1) from the
 * amplitudes F (as dda_scatter returns them) at n_dir quadrature directions:
 *   g_vec = sum_k w_k |F_k|^2 n_k / sum_k w_k |F_k|^2,  <cos theta> = g_vec . a.
 *   dirs_host : n_dir x 3 unit directions;  weights_host : n_dir weights;
 *   F_host : n_dir x 3 complex (re, im);  prop_host : the incidence direction a.
 *   g_out_host : 4 doubles = (<cos theta>, g_x, g_y, g_z).
 * Host-only arithmetic.  DDA_ERR_ARG on a null pointer, n_dir < 1 or a zero
 * total scattered power.
 */
int dda_asymmetry(int n_dir, const double* dirs_host, const double* weights_host,
                  const double* F_host, const double* prop_host, double* g_out_host);

/*
 * dda_symmetry -- symmetries of the lattice (examined from the host copy of
 * the occupied cells on the first call, then remembered by the handle).
 *   flags_out : bit 0 (DDA_SYM_ROT90_Z) set when the occupancy, materials
 *   included, is invariant under the rotation by +90 degrees about z
 *   ((x, y) -> (-y, x); needs nx = ny), e.g. every sphere lattice.
 */
#define DDA_SYM_ROT90_Z 1
int dda_symmetry(dda_t h, int* flags_out);

/*
 * dda_mueller_plane_sym -- the 16 Mueller elements in the xz plane from ONE
 * solution, the x-polarised one for incidence along +z (Sec. 3.1 uses the
 * symmetry of the sphere to get all results from one polarisation state).
 * For a lattice invariant under R = rotation by +90 degrees about z, the
 * y-polarised solution is P_y(r) = R P_x(R^-1 r), so its amplitude is
 * F_y(n) = R F_x(R^-1 n); the library evaluates F_x at n = (sin t, 0, cos t)
 * and at R^-1 n = (0, -sin t, cos t) on the device and proceeds as
 * dda_mueller_plane_full.  Holds for every polarizability prescription here
 * (for incidence along z both polarisations have the same alpha).
 *   P_dev : device [3][N_occ] complex128, the x-polarised solution.
 *   M_out_host : n_theta x 16.   F_out_host : optional, n_theta x 2 x 3
 *   complex (F_x then F_y per angle) or NULL.
 * DDA_ERR_ARG when the lattice lacks the symmetry (dda_symmetry) or on bad
 * arguments.  Synchronises the stream.
 */
int dda_mueller_plane_sym(dda_t h, int pol_prescription, const void* P_dev, int n_theta,
                          const double* theta_deg_host, double* M_out_host, double* F_out_host);

/*
 * dda_orientation_average -- scattering averaged over particle orientations
 * (Sec. 2: averaging over the Euler angles alpha, beta, gamma; alpha by
 * scattering planes of one solution, beta and gamma by independent
 * solutions).  Orientation R = Rz(alpha) Ry(beta) Rz(gamma) (z-y-z) takes the
 * particle frame to the laboratory, incidence along laboratory z.  For each
 * (beta, gamma) node the library solves the two polarisations (incidence
 * R^T z, polarisations R^T x and R^T y) as two right-hand sides, evaluates
 * the far field in n_alpha scattering planes of azimuth 2 pi k / n_alpha
 * (amplitudes along theta_hat and phi_hat of each plane, polarisations
 * combined as cos(phi) e_x + sin(phi) e_y and -sin(phi) e_x + cos(phi) e_y)
 * and accumulates the Mueller matrix and the cross sections for unpolarised
 * light.  Quadrature, fixed: Gauss-Legendre in cos(beta) (n_beta nodes),
 * uniform gamma (n_gamma) and alpha (n_alpha) nodes; no Romberg adaptivity.
 *   opts : solver options as in dda_solve; opts->pol must not be DDA_LDR
 *          (its polarizability depends on the incident polarisation, so the
 *          field of a rotated polarisation is not a combination of the two
 *          solutions): DDA_ERR_ARG.
 *   theta_deg_host : n_theta scattering angles.
 *   q_avg_host : 2 doubles = <Q_ext>, <Q_abs>.
 *   M_avg_host : n_theta x 16 doubles, the averaged Mueller matrix.
 *   info_host  : optional, 2 * n_beta * n_gamma entries (node (ib, ig),
 *                polarisation r at 2 (ib n_gamma + ig) + r).
 * The D-matrix must be built for opts->prec.  Allocates 2 x 3 N_occ
 * complex128 of device memory for the duration of the call.  Returns DDA_OK,
 * or the first non-OK solver status (the averages are still written).
 */
int dda_orientation_average(dda_t h, const dda_solve_opts* opts, int n_alpha, int n_beta,
                            int n_gamma, int n_theta, const double* theta_deg_host,
                            double* q_avg_host, double* M_avg_host, dda_solve_info* info_host);

/*
 * dda_farfield_noalloc -- the scattering amplitude F(n) of dda_scatter for
 * one polarization vector, computed without allocating any device memory.
 * (The paper has no counterpart: this is an interface for callers that cannot
 * let a library call cudaMalloc -- code running under CUDA stream capture,
 * processes whose device memory comes from their own allocator or is fixed
 * at start-up.)
 *   P_dev    : device [3][N_occ] complex128 polarization (one RHS), read only.
 *   n_dir    : number of directions, >= 1.
 *   dirs_dev : device [n_dir][3] doubles, unit directions n.
 *   F_dev    : device [n_dir][3] complex128 (re, im) output,
 *              F(n) = -i kd^3 (I - n n) sum_j P_j exp(-i kd n.r_j).
 * Working memory is one fixed 8 MiB array in device global memory that the
 * library image carries (every GPU that loads the library holds it until the
 * process exits); a request needing more than that (about n_dir *
 * (nx+ny+nz) * 16 bytes plus the partial sums) returns DDA_ERR_ARG with the
 * size in dda_last_error.  The first call on a device looks up the array's
 * address with that device current: make it before any stream capture.  The
 * handle's device must be the current device (this call does not switch
 * devices, so that a capture in progress is left alone): DDA_ERR_ARG if not.  All
 * calls share the array, so calls that overlap on the GPU race; the array
 * keeps the last call's contents, which no call depends on.  Asynchronous on
 * the handle's stream; calls no cudaMalloc or cudaFree.
 */
int dda_farfield_noalloc(dda_t h, const void* P_dev, int n_dir, const double* dirs_dev,
                         void* F_dev);

/*
 * Learned right preconditioner (no counterpart in the paper, which traces the
 * slow convergence for large m to the system itself, Sec. 4, and names
 * better preconditioning as the way forward, Sec. 5).  A 3D convolutional
 * network N maps a residual r of Eq. (3) to an approximation of the error
 * A^-1 r: features are the 2x2x2 averages of (Re, Im) of the three components
 * of r / rms(r) and the occupied fraction at half resolution; a three-level
 * encoder-decoder of 3x3x3 convolutions with ReLU (7-16-32-160-160 channels,
 * 1,033,430 parameters, BF16 weights in the products, FP32 master weights,
 * activations and accumulation) returns six channels that each dipole
 * reads from its half-resolution cell, times rms(r), and adds to r
 * (N(r) = r + correction: identity plus what was learned).  Training, inference
 * and the solver run in the library's own kernels; every reduction has a
 * fixed order (deterministic).
 */
typedef struct dda_pcnet* dda_pcnet_t;

/* dda_pcnet_create -- a new network on the current device, He-normal weights
 * from a seeded generator (the last layer scaled by 0.1), zero biases.
 * Errors: DDA_ERR_ARG (out NULL), DDA_ERR_CUDA, DDA_ERR_OOM. */
int dda_pcnet_create(dda_pcnet_t* out, unsigned long long seed);
int dda_pcnet_free(dda_pcnet_t net);                        /* NULL ok */
int dda_pcnet_params(dda_pcnet_t net, long long* n);        /* parameter count */
const char* dda_pcnet_last_error(dda_pcnet_t net);
/* weights and biases as one host array of dda_pcnet_params floats, layer by
 * layer ([cout][cin][k][k][k] weights, then [cout] biases); set_weights also
 * resets the optimiser state. */
int dda_pcnet_get_weights(dda_pcnet_t net, float* host);
int dda_pcnet_set_weights(dda_pcnet_t net, const float* host);
/* gradients of the last training step, same layout (host) */
int dda_pcnet_get_grads(dda_pcnet_t net, float* host);

/* dda_pcnet_apply -- z = N(v) on the lattice of handle h (same device).
 * v_dev, z_dev: device [3][N_occ] complex128 (caller-owned, may not alias).
 * Asynchronous on the handle's stream; the network keeps activation memory
 * for the largest lattice it has seen. */
int dda_pcnet_apply(dda_pcnet_t net, dda_t h, const void* v_dev, void* z_dev);

/* dda_pcnet_train_step -- one Adam step (lr, betas 0.9 / 0.999) on the pair
 * (r, e) of the handle's lattice: loss = |N(r) - e|^2 / |e|^2 over the
 * dipoles.  z_dev (device [3][N_occ] complex128) receives N(r) before the
 * step; *loss_out (host, may be NULL) the loss.  Synchronises the stream.
 * DDA_ERR_NONFINITE for a non-finite loss. */
int dda_pcnet_train_step(dda_pcnet_t net, dda_t h, const void* r_dev, const void* e_dev,
                         void* z_dev, float lr, double* loss_out);

/* dda_pcnet_pair -- a training pair from two solutions of the same
 * right-hand side: e = x* - x_k with x = P / beta (beta of the given
 * incidence), and r = A e (the residual of x_k), with the exact product
 * (double-float where available, else FP64).  P_star, P_k: device [3][N_occ]
 * complex128 in; r_out, e_out: device [3][N_occ] complex128 out.
 * Synchronises the stream. */
int dda_pcnet_pair(dda_t h, int pol_prescription, const double* prop_host, const double* pol_host,
                   const void* P_star, const void* P_k, void* r_out, void* e_out);

/*
 * dda_solve_pc -- one right-hand side of Eq. (3) by flexible Bi-CGSTAB with
 * the network as right preconditioner (net = NULL: plain Bi-CGSTAB with
 * the same kernels), complex128 vectors and the exact product: double-float
 * when the handle has the double-float D-matrix (a DDA_FP32_REFINED build on
 * a grid with register-resident passes), else FP64.  Convergence is declared
 * on the true residual ||b - A x|| / ||b|| < opts->tol; when the
 * preconditioned iteration has not improved its residual by 1 % in 50
 * iterations (or breaks down) the solve continues from its current x without
 * the network.  Uses opts->pol, tol, maxiter (iterations; two products each).
 *   prop_host, pol_host : one incidence (3 and 6 doubles).
 *   P_dev    : device [3][N_occ] complex128, the polarizations (out).
 *   res_hist : optional host [hist_len] recurrence residuals per iteration.
 *   info     : one entry; info->outer is the iteration at which the network
 *              was dropped (0: it never was); matvecs counts the products.
 * Allocates 10 x 3 N_occ complex128 for the call.  Synchronises the stream.
 */
int dda_solve_pc(dda_t h, dda_pcnet_t net, const dda_solve_opts* opts, const double* prop_host,
                 const double* pol_host, void* P_dev, double* res_hist, int hist_len,
                 dda_solve_info* info);

/*
 * dda_trace -- per-kernel timing (the paper reports only whole-run times,
 * Fig. 3; this is the library's own tracing).  enable != 0 starts recording a
 * CUDA event pair around each launch of the product passes P1..P5, the
 * D-matrix build and the far-field kernels on the handle's stream, and
 * resets the totals; 0 stops.  Adds two event records per traced launch.
 */
int dda_trace(dda_t h, int enable);

/*
 * dda_trace_read -- totals since dda_trace(h, 1), after waiting for the
 * recorded events.  For k < min(max_n, *n_out): names_out + 32*k receives the
 * kernel name (NUL-terminated), ms_out[k] the summed duration in ms and
 * count_out[k] the number of launches.  *n_out = number of entries.  Entry 0
 * is "all_launches": ms 0, count = every kernel launch this library made (in
 * any handle) since dda_trace(h, 1).
 */
int dda_trace_read(dda_t h, int max_n, char* names_out, double* ms_out, long long* count_out,
                   int* n_out);

/* Queries. */
int dda_n_occ(dda_t h, long long* n_occ);
int dda_kd(dda_t h, double* kd);
int dda_grid(dda_t h, int* grid3);              /* padded (M_x, M_y, M_z)            */
int dda_positions(dda_t h, int* ijk_host);      /* [N_occ][3] lattice indices (ix,iy,iz) */
const char* dda_last_error(dda_t h);            /* never NULL; "" if no error        */
int dda_free(dda_t h);                          /* releases all handle memory (device
                                                   buffers go to the cache of
                                                   dda_release_cached_memory); NULL ok */

/*
 * dda_release_cached_memory -- returns to the CUDA driver the device memory
 * the library keeps for reuse.  Device buffers a handle frees (at dda_free,
 * or when a buffer grows) go to a per-process cache keyed by device and size,
 * so that the next handle of a lattice of the same size allocates without
 * cudaMalloc or a device-synchronising cudaFree; each cached block carries an
 * event of the stream that last used it and is reused only after that event.
 * At most 4 GiB stay cached; the cache of a device is also emptied when a
 * cudaMalloc of the library runs out of memory.  Call this to hand the memory
 * back to other users of the GPU (e.g. PyTorch's allocator).  Thread-safe;
 * blocks whose stream work is still pending are waited for before release.
 * Memory held by live handles is not affected.  Returns DDA_OK.
 */
int dda_release_cached_memory(void);

/*
 * dda_set_memory_limit -- caps the device memory held by the library's live
 * handles (all devices together) at `bytes` (0 = no cap, the default).  An
 * allocation that would pass the cap fails as if the device were out of
 * memory: the entry point returns DDA_ERR_OOM with the handle left usable
 * (a product or solve that needs more memory can be retried after the cap
 * is raised or other handles are freed).  For services that share a GPU and
 * give each library a memory budget.  Setting a nonzero cap also releases
 * the cache of freed blocks (dda_release_cached_memory).  Thread-safe;
 * returns DDA_OK.
 */
int dda_set_memory_limit(unsigned long long bytes);

/*
 * dda_memory_in_use -- bytes of device memory held by live handles and by
 * the cache of freed blocks (all devices).  DDA_ERR_ARG on a null pointer.
 */
int dda_memory_in_use(unsigned long long* live_bytes, unsigned long long* cached_bytes);

#ifdef __cplusplus
}
#endif
#endif /* DDA_H */
