// pp_internal.h -- plan and kernel-argument structures shared by the host code and the kernels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "pp_fft.cuh"
#include "pittpack_gb.h"

namespace pp {

// Per-axis transform family (Table "Summary of the appropriate Fourier transformations",
// plus the type-IV pair for an axis with a Dirichlet face at one end and Neumann at the other).
enum AxisKind { AX_P = 0, AX_NN = 1, AX_DD = 2, AX_DN = 3, AX_ND = 4 };

// Line transform kinds.
enum LineKind {
  LK_R2C = 0,   // real N -> N/2+1 complex, forward DFT (periodic)
  LK_C2R = 1,   // N/2+1 complex -> real N, unnormalised Hermitian synthesis
  LK_C2C_F = 2, // complex N -> complex N, forward
  LK_C2C_I = 3, // complex N -> complex N, unnormalised inverse
  LK_DCT2 = 4,  // Neumann forward  ("DCT10")
  LK_DCT3 = 5,  // Neumann inverse  ("DCT01"), Y0 + 2 sum_{k>0} Yk cos(...)
  LK_DST2 = 6,  // Dirichlet forward ("DST10")
  LK_DST3 = 7,  // Dirichlet inverse ("DST01"), (-1)^n Y_{N-1} + 2 sum_{k<N-1} Yk sin(...)
  LK_DCT4 = 8,  // Neumann-low / Dirichlet-high, self-inverse up to 2/N
  LK_DST4 = 9,  // Dirichlet-low / Neumann-high, self-inverse up to 2/N
};

// Arguments of one batched line-transform launch.  All offsets and strides are in
// "real" storage units of the respective array (a complex element is 2 consecutive reals).
struct LineArgs {
  const void* in;
  void* out;
  int N;              // line length (reals for real kinds, complex count for C2C)
  int kind;           // LineKind
  int nlines;         // total lines of the launch
  int lpc;            // lines per CTA
  int ldm;            // shared-memory stride of one line (complex elements)
  int lines_per_plane;
  int parts;          // 2: a complex column split into re/im real lines
  long long in_plane, out_plane;
  int in_line, in_pos;          // input: stride between consecutive lines / positions (reals)
  long long out_line, out_pos;  // output: stride between consecutive lines / positions (reals)
  int ntiles;         // tiles of the launch (x: lpc rows; y: one plane x tx columns)
  int vec_ok;         // x lines: both arrays 32-byte aligned (vectorised pre/post allowed)
  int vec_y;          // y tiles: rows contiguous and 16-byte aligned, lpc a multiple of the vector width
  int tx, ncols, nblk;  // y: columns per tile, columns per plane, column blocks per plane
  const void* tw;     // stage twiddles w_M^j, j < M (complex, arithmetic type)
  const void* aux;    // pre/post twiddles (complex, arithmetic type), layout per kind
  FftPlan fp;
  FastDiv fd_kpre;    // number of pre-processing items per line (M; M/2 + 1 for Hermitian pairs)
  FastDiv fd_kpost;   // number of post-processing items per line
  FastDiv fd_lpc;     // lines per CTA
  FastDiv fd_lpp;     // lines per plane
  FastDiv fd_parts;   // 1 or 2
  FastDiv fd_nblk;    // column blocks per plane
  FastDiv fd_gpc;     // y: groups of vector-width adjacent lines per CTA
};
constexpr int kMaxLpc = 512;  // lines per CTA (bounds the per-line bases in shared memory)
constexpr int kHostChunks = 8;  // plane chunks of a host-buffer solve (copies overlap transforms)

// Complex FFT lengths with kernels compiled for the length: powers of two 8..1024 and 3 x 2^k
// 24..768.  Their stage twiddles are stored per stage in butterfly order (fft_lines_ct); other
// lengths keep w_M^j, j < M.
constexpr int kCtMin = 8, kCtMax = 1024;
inline bool ct_length(int M) {
  const bool p2 = M >= kCtMin && M <= kCtMax && (M & (M - 1)) == 0;
  const int t = M / 3;
  const bool p3 = M % 3 == 0 && t >= 8 && t <= 256 && (t & (t - 1)) == 0;
  return p2 || p3;
}

// Per-mode z-solve descriptor (tables computed on the host in FP64).  The multipliers (table
// prefix, winf, wlast) are stored as w_k, or for ZF_NEAR1 modes as 1 + w_k (pp_zmul.cuh).
struct ZMode {
  int woff, wlen;     // prefix of Thomas multipliers w_k in the w table
  int qoff, qlen;     // periodic z: prefix of q = A'^{-1} e_0
  float winf[2];      // converged multiplier (hi, lo)
  float wlast[2];     // multiplier of the last row
  float gam[2];       // periodic: gamma
  float igam[2];      // periodic: 1/gamma
  float dsm[2];       // periodic: 1 / (1 + z_0 + z_{n-1}/gamma)
  int flags;          // ZF_* bits
  int pad;
};
enum { ZF_PERIODIC = 1, ZF_SINGULAR = 2, ZF_NEAR1 = 4 };
// a mode whose converged multiplier has 1 + w below this stores 1 + w_k: the rounding of a stored
// w acts like a relative error of about 2^-48 / (1 + w) on the mode's solution, 2^-45 at the bound
constexpr double kNear1 = 0.125;

struct ZArgs {
  void* data;             // spectral array, in place
  long long plane;        // reals per z-plane
  int nz;
  int cplx;               // 1: consecutive real pairs share a mode
  long long nreal;        // reals per plane (including row padding)
  int row_reals;          // reals per spectral row (padded)
  int row_valid;          // reals of a row that carry modes
  int row_modes;          // modes per row
  FastDiv fd_row;
  const ZMode* modes;
  const float2* wtab;     // (hi, lo) multipliers
  const float2* qtab;     // (hi, lo) periodic end-solution prefix
  float scale[2];         // dz^2 * inverse-transform weights (hi, lo)
  int transpose;          // 1: solve with the transposed factorisation (adjoint)
  // range status (plan-owned words: [0] status bits, [1] largest |scaled input|, [2] largest |output|
  // (FP32 bits), [3] count of finished blocks); the last block of a launch compares the maxima
  // with dmin / umax and sets kStatusRange in [0]
  void* ck;               // checkpoints of the double-float sweeps ([nz/8 rounded up][nreal] pairs),
                          // or NULL for the two-sweep kernel
  unsigned* rstat;
  float dmin;             // 2^-100: below it the double-float low parts are subnormal
  float umax;             // 2^124 / (nx ny): above it the inverse transforms may overflow FP32
  int only_singular;      // 1: solve the singular mode's column only (after a partitioned solve)
};
// status bits of a plan's device status word
constexpr unsigned kStatusRange = 1u;

// Diagonal solve of periodic z by transform (pp_zfft.cu), in place on the z-transformed spectrum.
struct ZDiagArgs {
  void* data;          // spectral array [nz][plane] (spill type)
  long long plane;     // reals per z-plane
  long long nreal;     // reals per plane carrying lines (even: complex lines of real pairs)
  int nz;
  const float2* lam;   // per real slot: lambda_x/dx^2 + lambda_y/dy^2 of its mode (hi, lo)
  const float2* zeig;  // per kz: (2 cos(2 pi kz/nz) - 2)/dz^2 (hi, lo)
  float scale[2];      // w_x w_y / nz (hi, lo)
  int row_reals;       // reals per spectral row (padded)
  int row_valid;       // reals of a row that carry modes (even): later pairs are padding, skipped
  FastDiv fd_row;
  unsigned* rstat;     // range report (as ZArgs)
  float dmin, umax;
};
enum { ZM_SM = 0, ZM_FFT = 1 };  // periodic z: Sherman-Morrison sweeps / z transform
// partitioned z solve (pp_zpart.cu): chunk count and slots per CTA for rows-per-chunk M
bool zpart_shape(int nz, int M, int* G, int* lgG, int* P);
constexpr int kZSplitRows[3] = {8, 16, 32};  // compiled rows-per-chunk variants

}  // namespace pp

// Plan object behind the opaque C handle.
struct pp_plan {
  int nx, ny, nz;
  int bc[6];
  double dx, dy, dz;
  int dtype;        // pp_dtype
  int kx, ky;       // AxisKind
  int layout;       // 0: x periodic (complex after x); 1: y periodic only; 2: both real
  bool singular;
  // spectral sizes, in reals
  long long xrow;       // reals per row after the x transform
  long long xplane;     // reals per plane after the x transform
  long long splane;     // reals per plane of the fully transformed array
  size_t elem;          // bytes per spill real (8: df pair, 4: float)
  void* bufA;
  void* bufB;
  size_t buf_bytes;
  // tables
  void* d_tw_x; void* d_aux_x; void* d_tw_y; void* d_aux_y;
  pp::FftPlan fx, fy;
  pp::ZMode* d_modes;
  float2* d_wtab;
  float2* d_qtab;
  long long nmodes;
  double zscale;
  // launch shapes
  int threads_x[2], lpc_x[2], ldm_x;  // [0] forward, [1] inverse kernels
  int threads_y[2], lpc_y[2], ldm_y;
  // mixed-precision refinement scratch
  void* d_resid;       // residual / correction (FP64 I/O size)
  void* d_mean;        // kMeanParts partial sums + 1 mean (float2 each), singular refinement
  void* d_host_f;      // device staging for host-buffer solves
  void* d_host_u;
  cudaStream_t host_cs[2];  // copy streams of host-buffer solves (created on first use)
  cudaEvent_t host_ev[2 * pp::kHostChunks + 3];  // per-chunk copy / compute events, start, two joins
  unsigned* d_status;  // 4 words: status bits, two running maxima and a block counter (ZArgs::rstat)
  // periodic z by transform (zmethod == ZM_FFT): z-line DFT plan and twiddles, diagonal tables
  int zmethod;
  bool zfft_ok;         // periodic z with an nz the line kernels can transform
  pp::FftPlan fz;
  void* d_tw_z; void* d_aux_z;
  float2* d_zlam;       // per real slot of a plane
  float2* d_zeig;       // per kz
  int threads_z, lpc_z, ldm_z;
  // non-periodic z: 1 = Thomas sweeps, M = partitioned solve with M rows per chunk
  int zsplit;
  // created with autotune = 1 (launch shapes timed), and whether the autotuner also chose the z
  // algorithm (zsplit for non-periodic z, zmethod for periodic z); a batched graph may swap these
  // members to the library's shared-GPU settings (pp_solve_batched)
  bool tuned, z_tuned;
};

namespace pp {
// launchers (return cudaError_t of the launch)
// line stage over planes z0 .. z0+nzc-1 (nzc < 0: all); in / out point at plane 0
cudaError_t launch_lines(const pp_plan* p, int axis, int dir, int io_in, int io_out, const void* in, void* out,
                         cudaStream_t st, int z0 = 0, int nzc = -1);
cudaError_t launch_zsolve(const pp_plan* p, void* data, int transpose, cudaStream_t st);
// the Thomas sweeps of the singular mode alone (the plan's one pinned column)
cudaError_t launch_zsingular(const pp_plan* p, void* data, cudaStream_t st);
// periodic z by transform: forward z DFT, diagonal solve, inverse z DFT (in place)
cudaError_t launch_zfft(const pp_plan* p, void* data, cudaStream_t st);
// refinement: r = f - A u0 (f FP64; u0, r FP32), u = u0 + d - shift (u FP64; u0, d FP32)
cudaError_t launch_residual(const pp_plan* p, const void* f, const void* u0, void* r, cudaStream_t st);
cudaError_t launch_add(const pp_plan* p, void* u, const void* u0, const void* d, const void* shift, cudaStream_t st);
// f -= coef * g on the cells next to face `face` (0..5 = x-,x+,y-,y+,z-,z+), in place
cudaError_t launch_fold_face(void* f, const void* g, int nx, int ny, int nz, int face, double coef, bool f32,
                             cudaStream_t st);
// n pseudo-random values in [-1, 1) (FP32 or FP64), timing input of the autotuner
cudaError_t launch_fill(void* x, long long n, bool f32, cudaStream_t st);
// mean of an FP32 grid: nparts block sums into `partials` (nparts float2), result (hi,lo) into `mean`
cudaError_t launch_mean(const pp_plan* p, const void* u, void* partials, int nparts, void* mean, cudaStream_t st);
constexpr int kMeanParts = 1024;
// the refined solve on caller-provided scratch (resid: 2 nx*ny*nz floats, u0 then the residual /
// correction; partials: kMeanParts float2; mean: one float2)
__attribute__((visibility("hidden"))) pp_status solve_refined_core(pp_plan* p, const void* f, void* u, void* resid,
                                                                  void* partials, void* mean, cudaStream_t st);
// record the calling thread's error detail (returned by pp_last_error_string) and return s
__attribute__((visibility("hidden"))) pp_status set_last_error(pp_status s, const char* msg);
}  // namespace pp
