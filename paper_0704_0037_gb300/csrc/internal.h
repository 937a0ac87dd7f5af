// Internal declarations of the DDA library (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dda.h"
#include "common.cuh"
#include "fft.cuh"

namespace dda {

// Per-kernel CUDA-event timing (dda_trace).  Kernels are identified by a
// small fixed table of names; event pairs are resolved at sync points.
enum TraceId {
  TR_P1_C64, TR_P2_C64, TR_P3_C64, TR_P4_C64, TR_P5_C64,
  TR_P1_C128, TR_P2_C128, TR_P3_C128, TR_P4_C128, TR_P5_C128,
  TR_DB_GREEN, TR_DB_LINES, TR_DB_OCTANT, TR_FARFIELD, TR_QSUMS, TR_P1_DF, TR_P2_DF,
  TR_P3_DF, TR_P4_DF, TR_P5_DF, TR_QMR_K1, TR_QMR_K2, TR_QMR_SCALARS, TR_COUNT
};
struct Tracer {
  bool on = false;
  struct Rec { int id; cudaEvent_t a, b; };
  std::vector<cudaEvent_t> pool;
  std::vector<Rec> pending;
  cudaEvent_t open = nullptr;
  double ms[TR_COUNT] = {};
  long long cnt[TR_COUNT] = {};
  long long launch_base = 0;
};
const char* trace_name(int id);
void tr_begin(Tracer* t, cudaStream_t st);
void tr_end(Tracer* t, cudaStream_t st, int id);
void tr_flush(Tracer* t);
void tr_reset(Tracer* t);
void tr_destroy(Tracer* t);

// Padded-grid geometry and the per-axis FFT plans.
struct Geom {
  int nx, ny, nz;          // lattice box
  int Mx, My, Mz;          // padded grid, M >= 2n - 1, 7-smooth
  int nrows;               // ny * nz rows along x
  long long n_occ;         // occupied dipoles
  FftPlan px, py, pz;      // plans for lengths Mx, My, Mz
  Tracer* tr = nullptr;    // per-kernel timing, owned by the handle
  int engine = 0;          // 0: register-resident passes where available; 1: Stockham only
  // tile variants of the register-resident y forward, z and y inverse
  // passes per arithmetic (0 complex64, 1 complex128, 2 double-float): -1
  // not yet chosen (the autotuner picks at the D-matrix build), else the
  // variant of FastArgs::var_*
  int tiles[3][3] = {{-1, -1, -1}, {-1, -1, -1}, {-1, -1, -1}};
  long long oct() const { return (long long)(Mx / 2 + 1) * (My / 2 + 1) * (Mz / 2 + 1); }
  long long b1() const { return 3LL * nrows * Mx; }          // [3][nz][ny][Mx]
  long long b2() const { return 3LL * nz * My * Mx; }        // [3][nz][My][Mx]
};

// Lattice description on the device: occupied dipoles of row r = iz*ny + iy
// are row_off[r] .. row_off[r+1]-1 (x-fastest order), at x = xi[i].
struct LatticeDev {
  const long long* row_off;
  const uint16_t* xi;
  const uint8_t* mat;
  // The rows that hold dipoles lie, in each z plane, within the span
  // yr[2 z] <= y <= yr[2 z + 1] of its occupied rows (an empty plane has
  // yr = {1, 0}); arow lists the nact rows of all spans in increasing order
  // and aoff[i] = row_off[arow[i]] (aoff[nact] = n_occ).  The register-resident
  // x passes transform only these rows and the y forward pass reads only
  // them (nullptr: every row).
  const int* arow = nullptr;
  const long long* aoff = nullptr;
  const int* yr = nullptr;
  int nact = 0;
};

// Layout of the D-matrix octant: interleaved by point for complex64 (its six
// 8-byte entries are three 16-byte loads), planar by component for the wider
// types (six 16-byte loads either way; planar reads measured faster there).
template <typename R> constexpr bool kOctInterleaved = sizeof(R) == 4;

// Per-precision workspace of the FFT product.
template <typename R>
struct Work {
  cpx<R>* B1 = nullptr;     // after the x pass
  cpx<R>* B2 = nullptr;     // after the y pass (z pass in place)
  cpx<R>* tw = nullptr;     // twiddles: [Mx] then [My] then [Mz], exp(-2 pi i m / M)
  cpx<R>* D = nullptr;      // octant of FFT(G)/(Mx My Mz): complex64 interleaved
                            // [Mz/2+1][My/2+1][Mx/2+1][6] (xx, xy, xz, yy, yz, zz of a point
                            // together), the wider types [6][Mz/2+1][My/2+1][Mx/2+1]
  cpx<R>* beta = nullptr;   // [nrhs][n_mat][3]
  bool have_D = false;
  int cap = 0;              // right-hand sides B1 and B2 hold
  int cap_beta = 0;         // entries of beta (double-float tables only)
};

// Device memory of the library (devmem.cu): blocks come from a cache of
// freed blocks of (nearly) the same size when one is free, else cudaMalloc;
// dev_free puts a block back with an event recorded on st (the stream that
// last used it).
cudaError_t dev_malloc_raw(void** p, size_t bytes);
cudaError_t dev_free(void* p, cudaStream_t st);
template <typename T> inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_raw(reinterpret_cast<void**>(p), bytes);
}

// Grow the product buffers of w to hold min(want, what fits) right-hand
// sides (api.cu); at least one.
template <typename R> int ensure_work_cap(dda_t h, Work<R>& w, int want);

// Launch helpers (matvec.cu)
// y = A x for nrhs right-hand sides ([nrhs][3][n_occ]), in chunks of w.cap
// right-hand sides per launch.  With dotp != null the last pass also writes
// per-block partials of x^T y when it can: *dot_nb = their count per
// right-hand side (those of right-hand side r start at dotp + 2 r *dot_nb),
// else 0.  skip (device, nrhs ints, or null): right-hand sides with a nonzero
// entry are left untouched.
template <typename R>
cudaError_t launch_matvec(const Geom& g, const LatticeDev& lat, Work<R>& w, const cpx<R>* beta,
                          int n_mat, const cpx<R>* x, cpx<R>* y, int nrhs, bool adjoint,
                          cudaStream_t st, double* dotp = nullptr, int* dot_nb = nullptr,
                          const int* skip = nullptr);

template <typename R>
cudaError_t launch_lines(const Geom& g, const cpx<R>* in, cpx<R>* out, const FftPlan& p,
                         const cpx<R>* tw, bool inverse, int n_in, int n_out, int nt, int n_outer,
                         int n_batch, bool contig, long long in_sm, long long in_st,
                         long long in_so, long long in_sb, long long out_sm, long long out_st,
                         long long out_so, long long out_sb, cudaStream_t st,
                         const int* skip = nullptr);

// y = A x in double-float arithmetic for complex128 vectors x, y
// ([nrhs][3][n_occ]); register-resident passes only (cudaErrorNotSupported
// when an axis has no split).  beta: complex128 [nrhs][n_mat][3], converted
// into w.beta; skip as launch_matvec.
cudaError_t launch_matvec_df(const Geom& g, const LatticeDev& lat, Work<df>& w, const c128* beta,
                             int n_mat, const c128* x, c128* y, int nrhs, cudaStream_t st,
                             const int* skip = nullptr);

// Autotuner of the tile variants of the register-resident y forward, z and
// y inverse passes (Geom::tiles[kind], kind 0 complex64 / 1 complex128 /
// 2 double-float): each variant of each pass timed with CUDA events on the
// handle's own buffers (one warm-up and three timed launches of one
// right-hand side), the faster kept; entries already >= 0 are left alone.
// Choices are cached per device and grid shape.  Needs w's buffers and D.
template <typename R>
cudaError_t tune_tiles(Geom& g, const LatticeDev& lat, Work<R>& w, cudaStream_t st);

FftPlan make_plan(int M);
int smooth_size(int lo);

}  // namespace dda

// The handle.
struct dda_ctx {
  long long uid = 0;        // unique in the process (caches keyed by handle use it, not the address)
  int sym_flags = -1;       // DDA_SYM_* of the lattice (-1: not yet examined)
  int device = 0;           // CUDA device current at dda_init_lattice
  bool d64_from_df = false; // w64.D not yet derived from the double-float octant
  dda::Geom g{};
  int n_mat = 0;
  std::vector<double> m;          // 2*n_mat
  double kd = 0;
  cudaStream_t stream = nullptr;
  std::vector<long long> row_off_h;
  std::vector<uint16_t> xi_h;
  std::vector<uint8_t> mat_h;     // material index of each occupied dipole
  long long* d_row_off = nullptr;
  uint16_t* d_xi = nullptr;
  uint8_t* d_mat = nullptr;
  dda::Work<double> w64;
  dda::Work<float> w32;
  dda::Work<dda::df> wdf;         // double-float D-matrix and buffers (FP32_REFINED residuals)
  dda::Tracer tracer;
  int beta_nrhs = 0;              // RHS count of the current beta tables
  int beta_cap = 0;               // RHS capacity of the beta allocations
  int beta_presc = -1;
  std::string err;
  // solver scratch (krylov.cu)
  void* sv = nullptr;             // solver vectors, grown on demand
  size_t sv_bytes = 0;
  double* d_part = nullptr;       // reduction partials
  double* d_mvpart = nullptr;     // per-block x^T y partials of the product's last pass
  void* bm = nullptr;             // batched-solver state (krylov.cu)
  void* d_scal = nullptr;         // device scalar state
  void* h_scal = nullptr;         // pinned host mirror
  // scatter scratch
  double* d_tab = nullptr;
  size_t tab_bytes = 0;
  double* d_fpart = nullptr;
  size_t fpart_bytes = 0;
  void* d_coll = nullptr;         // y-collapsed polarization + its lattice
  size_t coll_bytes = 0;
  void* d_dscratch = nullptr;     // D-matrix build scratch kept between builds (small grids)
  size_t dscratch_bytes = 0;
  void* d_ptab = nullptr;         // incident-wave phase per axis (right-hand sides), complex128
  int* d_arow = nullptr;          // rows within each plane's span of occupied rows
  long long* d_aoff = nullptr;    // their dipole offsets (+ n_occ)
  int* d_yr = nullptr;            // per z plane: first and last occupied row
  int nact = 0;
  dda::LatticeDev lat() const { return {d_row_off, d_xi, d_mat, d_arow, d_aoff, d_yr, nact}; }
};

int dda_fail(dda_t h, int code, const std::string& msg);
int dda_cuda_fail(dda_t h, cudaError_t e, const char* where);

#define DDA_CK(h, call)                                      \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return dda_cuda_fail(h, e_, #call); \
  } while (0)

// beta tables on the device (api.cu)
int dda_beta_internal(dda_t h, int presc, int nrhs, const double* prop, const double* pol);
// D-matrix (dmatrix.cu)
int dda_build_D_internal(dda_t h, bool want32);
// solvers (krylov.cu)
// the FP64 octant of a double-float build, derived on first use (dmatrix.cu)
int ensure_d64(dda_t h);
// all right-hand sides at once (QMR-CS only); frees with batch_free (krylov.cu)
int dda_solve_batch_internal(dda_t h, const dda_solve_opts* o, int nrhs, const double* prop,
                             const double* pol, void* P_dev, dda_solve_info* info);
void batch_free(dda_t h);
// incident plane wave of one right-hand side: propagation a, polarisation e
// (complex, re/im pairs), and b = beta e exp(i kd a.r) on the handle's stream
namespace dda {
struct Wave { double a[3]; double e[6]; };
int launch_rhs(dda_t h, c128* b, const c128* beta, const Wave& wv, cudaStream_t st);
}  // namespace dda
// bytes of the host image of a batched QMR-CS solve (krylov.cu)
long long dda_checkpoint_bytes_internal(dda_t h, int prec, int nrhs);
// ||b - A x|| / ||b|| per right-hand side with x = P / beta, native FP64 product
int dda_residual_internal(dda_t h, int presc, int nrhs, const double* prop, const double* pol,
                          const void* P_dev, double* res);
int dda_solve_internal(dda_t h, const dda_solve_opts* o, int nrhs, const double* prop,
                       const double* pol, void* P_dev, double* hist, int hist_len,
                       dda_solve_info* info);
// the 16 Mueller elements (row-major) of amplitudes S = {S1, S2, S3, S4} (api.cu)
void mueller_from_S(const dda::c128 S[4], double* m);
// scatter (scatter.cu)
int dda_scatter_internal(dda_t h, int presc, const void* P_dev, int nrhs, const double* prop,
                         const double* pol, int n_dir, const double* dirs, const double* w,
                         double* F_out, double* q_out);

namespace dda {
// Process-wide count of kernel launches made by this library (dda_trace_read
// reports the increase since tracing was enabled).
void count_launch();
void count_launches(long long n);   // n kernels of a replayed CUDA graph (may be negative)
long long launch_total();
}  // namespace dda

namespace dda {
// Far-field kernels (scatter.cu), shared with the allocation-free entry point.
constexpr int kFarfieldDB = 4;   // directions per block of k_farfield
__global__ void k_phase_tab(const double* dirs, int n_dir, double kd, int nx, int ny, int nz,
                            c128* tab);
__global__ void __launch_bounds__(256) k_farfield(const c128* P, LatticeDev lat, const c128* tab,
                                                  int n_dir, int nx, int ny, int nz, int nrows,
                                                  long long n_occ, int rows_per_chunk,
                                                  double* part);
__global__ void k_farfield_fin(const double* part, int n_chunks, int n_dir, const double* dirs,
                               double kd, double* F);
}  // namespace dda

namespace dda {
// Register-resident product passes for padded lengths with a compile-time
// split M = M1 * M2 (fastfft.cuh).  fast_supported(M) tells whether a length
// has one; fast_pass returns cudaErrorNotSupported otherwise.
// FP_XFULL: whole contiguous lines, nrows rows: rows y < ny of planes of My
// rows.  FP_SFULL: whole strided lines, nrows lines of element stride Mx in
// nz groups, msign as fk_yfwd (D-matrix build).
enum FastPass { FP_XFWD, FP_YFWD, FP_ZCONV, FP_YINV, FP_XINV, FP_XFULL, FP_SFULL };
struct FastArgs {
  const void* in;        // pass input (B1, B2, or x for FP_XFWD)
  void* out;             // pass output (B1, B2, or y for FP_XINV); FP_ZCONV: B2 in place
  const void* x;         // FP_XINV: the product's input vector
  const void* beta;      // [n_mat][3] for this right-hand side
  const void* D;         // FP_ZCONV: octant of FFT(G)
  const void* tw;        // twiddles of this axis, exp(-2 pi i m / M)
  LatticeDev lat;
  long long n_occ;
  int nrows, ny, nz, Mx, My;
  bool adj;
  int msign;
  double* dotp;          // FP_XINV: per-block partials of x^T y (re, im), or null
  cudaStream_t st;
  // right-hand sides in one launch: vectors [nrhs][3][n_occ], buffers
  // [nrhs][3][...], beta of right-hand side r at beta + r * bstride; a
  // right-hand side with skip[r] != 0 is left untouched (null: none skipped)
  int nrhs = 1;
  int bstride = 0;
  const int* skip = nullptr;
  // FP_SFULL: element offset between the outer groups of lines (0: M times
  // the element stride, i.e. whole line sets one after another)
  long long ostride = 0;
  // tile variants of FP_YFWD, FP_ZCONV, FP_YINV (0: default lines per block,
  // 1: half as many; the same product bit for bit)
  int var_yf = 0, var_z = 0, var_yi = 0;
  // launch the passes as programmatic dependents (fast_pdl)
  bool pdl = false;
};
// Whether the product passes launch as programmatic dependents: for the
// complex64 and double-float arithmetic on grids of up to 2^23 points over
// all right-hand sides, where a pass is a few microseconds and the launch
// latency it hides is a large part of it.  On larger grids the attribute
// measured slower for the memory-bound complex64 passes (a standalone
// product 0.507 -> 0.542 ms at 270^3, 3.85 -> 4.13 ms at 512^3).
inline bool fast_pdl(bool fp64, long long Mx, long long My, long long Mz, int nrhs) {
  return !fp64 && Mx * My * Mz * nrhs <= (1LL << 23);
}
// rows per block of the x passes: 16 for complex64 lines shorter than 1000
// points, 4 for the longer ones, 8 for the double-width arithmetic
inline int fast_x_rows(bool fp32, int Mx) { return fp32 ? (Mx < 1000 ? 16 : 4) : 8; }
// number of (re, im) partials FP_XINV writes to dotp for nrows rows
inline int fast_xinv_blocks(int nrows, bool fp32, int Mx) {
  const int t = fast_x_rows(fp32, Mx);
  return 3 * ((nrows + t - 1) / t);
}
// the most partials any arithmetic and length writes for nrows rows (the
// size of the buffers that receive them)
inline int fast_xinv_blocks_max(int nrows) { return 3 * ((nrows + 3) / 4); }
bool fast_supported(int M);          // complex64, complex128 and double-float passes
bool fast_supported_c64(int M);      // complex64 passes (also 512 and 1080)
cudaError_t fast_pass_512_c64(int pass, const FastArgs& a);
cudaError_t fast_pass_1080_c64(int pass, const FastArgs& a);
template <typename R> cudaError_t fast_pass(int M, int pass, const FastArgs& a);
template <typename R> cudaError_t fast_pass_270(int pass, const FastArgs& a);
template <typename R> cudaError_t fast_pass_256(int pass, const FastArgs& a);
template <typename R> cudaError_t fast_pass_small(int M, int pass, const FastArgs& a);
template <typename R> cudaError_t fast_pass_mid(int M, int pass, const FastArgs& a);
cudaError_t fast_pass_mid_df(int M, int pass, const FastArgs& a);
// padded length of an axis: the smallest compiled length >= lo when it is at
// most 1.35 times the smallest 7-smooth one (engine DDA_ENGINE_AUTO), else
// the smallest 7-smooth length (api.cu)
int padded_length(int lo, int engine);
// double-float passes (fast_df_*.cu); fast_pass<df> dispatches to them
cudaError_t fast_pass_270_df(int pass, const FastArgs& a);
cudaError_t fast_pass_256_df(int pass, const FastArgs& a);
cudaError_t fast_pass_small_df(int M, int pass, const FastArgs& a);
template <> cudaError_t fast_pass<df>(int M, int pass, const FastArgs& a);
}  // namespace dda

namespace dda {
// Makes device dev current for the lifetime of the guard and puts the calling
// thread's current device back afterwards, so that every entry point runs on
// the handle's device whatever device the caller had selected.
struct DeviceGuard {
  int prev = -1;
  int dev;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int d) : dev(d) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
    if (prev != dev) err = cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};
// Number of multiprocessors of the current device (queried once per device);
// grid sizes of the grid-stride kernels are multiples of it.
int num_sms();
}  // namespace dda

// Entry-point prologue: a null handle is an argument error; otherwise the
// handle's device is made current until the entry point returns.
#define DDA_ON_DEVICE(h)                                                        \
  if (!(h)) return DDA_ERR_ARG;                                                 \
  dda::DeviceGuard dda_dev_guard_(h->device);                                   \
  if (dda_dev_guard_.err != cudaSuccess)                                        \
    return dda_cuda_fail(h, dda_dev_guard_.err, "cudaSetDevice(handle's device)")

namespace dda {
// Launch with programmatic stream serialization when pdl is set: the kernel
// may be scheduled while the previous kernel on st finishes, so it must call
// pdl_wait() (common.cuh) before reading what earlier work on st wrote.  The
// QMR sweeps use it, and the complex64 and double-float product passes on the
// grids fast_pdl selects (a 16^3 sphere's FP32-refined solve 1.68 -> 1.24 ms,
// its FP64 solve 2.36 -> 2.20 ms); the complex128 product passes measured
// slower with it (the FP64 solve 2.36 -> 3.37 ms) and launch plainly.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Kernel attributes set once per (kernel, device) instead of before every
// launch: the dynamic shared-memory limit (raised when a larger size is
// needed) and the maximum shared-memory carveout.
cudaError_t ensure_smem(const void* func, size_t bytes);
cudaError_t ensure_carveout_max(const void* func);
}  // namespace dda
