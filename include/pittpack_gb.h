/*
 * pittpack_gb.h -- C ABI of the GB300 FFT/tridiagonal Poisson solver.
 *
 * The library solves the second-order, cell-centred 7-point discretisation of
 * Poisson's equation (Hasbestan & Senocak, arXiv 1909.05423, Sec. "Mathematical
 * Formulation"):
 *
 *   (u[i+1]-2u[i]+u[i-1])/dx^2 + (same in y)/dy^2 + (same in z)/dz^2 = f
 *
 * on an nx x ny x nz grid of cells, by the paper's direct method: forward line
 * transforms in x and y chosen per boundary condition (Sec. "Boundary
 * Conditions", table of forward/backward transforms), one tridiagonal system
 * along z per (kx,ky) pair with the diagonal shifted by the eigenvalues of
 * Table "Eigenvalues" (Sec. "Solution of the Resulting Tridiagonal Matrices";
 * Thomas algorithm, Sherman-Morrison for periodic z), and the inverse
 * transforms.  Everything runs on one GPU, on caller-owned device memory.
 *
 * Conventions
 *  - Grids are real arrays [nz][ny][nx], x fastest (C order), cell centres at
 *    ((i+1/2)dx, (j+1/2)dy, (k+1/2)dz).
 *  - Faces are ordered x-, x+, y-, y+, z-, z+.  Boundary conditions are
 *    homogeneous: periodic (must be given on both faces of an axis), Neumann
 *    (ghost u[-1] = u[0]) or Dirichlet with zero face value by linear
 *    extrapolation (ghost u[-1] = -u[0], Sec. "Dirichlet-type Boundary
 *    Condition").  Non-zero face values are folded into f by pp_fold_bc.
 *  - With no Dirichlet face the operator is singular (Sec. "Well-posedness");
 *    the library then returns the zero-mean u with A u = f - mean(f).
 *  - Sizes: nx and ny must be even and of the form 2^a 3^b 5^c 7^d (a >= 1;
 *    FFT radices 2, 3, 4, 5, 7, 8), 2 <= nx, ny <= 4096; nz >= 2 (periodic z:
 *    nz >= 3).  Anything else returns PP_ERR_UNSUPPORTED_SIZE.
 *  - All solve calls are asynchronous on the given CUDA stream (NULL = legacy
 *    default stream).  The returned status reports argument validation and
 *    launch errors; device-side errors are reported by pp_plan_status() after
 *    the stream has been synchronised.
 *  - Error detail for the calling thread: pp_last_error_string().
 *  - A plan may be used by one stream at a time (its workspace is shared by
 *    all of its calls).
 */
#ifndef PITTPACK_GB_H
#define PITTPACK_GB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* pp_stream_t; /* identical to cudaStream_t */

typedef enum { PP_BC_PERIODIC = 0, PP_BC_NEUMANN = 1, PP_BC_DIRICHLET = 2 } pp_bc;

typedef enum {
  PP_F64 = 0,         /* FP64 in/out; FP64-class (double-float, ~47-bit) transforms and z-solve */
  PP_MIXED_F64IO = 1, /* FP64 in/out; FP32 transforms; z-solve in double-float arithmetic */
  PP_MIXED_F32IO = 2  /* FP32 in/out; FP32 transforms; z-solve in double-float arithmetic */
} pp_dtype;

typedef enum {
  PP_OK = 0,
  PP_ERR_INVALID_ARG = 1,
  PP_ERR_UNSUPPORTED_SIZE = 2,
  PP_ERR_BC_PAIRING = 3,
  PP_ERR_OUT_OF_MEMORY = 4,
  PP_ERR_CUDA = 5,
  PP_ERR_TIMEOUT = 6,
  PP_ERR_INTERNAL = 7,
  PP_ERR_RANGE = 8 /* pp_plan_status only: values left the range of full accuracy (see there) */
} pp_status;

/* Optional plan settings; pass NULL for the defaults. */
typedef struct pp_plan_options {
  int threads_x;   /* CTA size of the x-line kernels (0 = automatic) */
  int threads_y;   /* CTA size of the y-line kernels (0 = automatic) */
  int lines_x;     /* lines per CTA, x kernels (0 = automatic) */
  int cols_y;      /* columns per CTA, y kernels (0 = automatic) */
  int autotune;    /* 1: time candidate CTA sizes / lines per CTA for each of the four line
                      kernels at plan creation and keep the fastest (results cached per device,
                      sizes, boundary set and dtype for the life of the process); 0: fixed
                      heuristics */
  int threads_x_inv; /* the same four settings for the inverse-transform kernels */
  int lines_x_inv;   /*   (0 = as the forward setting above)                      */
  int threads_y_inv;
  int cols_y_inv;
  int z_method;    /* periodic z only: 0 = automatic (Sherman-Morrison, or with autotune = 1 the
                      faster of the two, timed), 1 = Sherman-Morrison sweeps, 2 = DFT along z and a
                      diagonal solve (needs nz = 2^a 3^b 5^c 7^d <= 4096, else
                      PP_ERR_UNSUPPORTED_SIZE); ignored for non-periodic z */
  int z_split;     /* non-periodic z only: 0 = automatic (the Thomas sweeps, or with autotune = 1
                      the fastest of them and the partitioned solves, timed as a lone launch),
                      1 = Thomas sweeps, 8 / 16 / 32 = partitioned solve: every z line split into
                      chunks of that many rows, one thread per chunk, the chunk carries combined by
                      recursive doubling (log2 of the chunk count levels; see pp_plan_z_split).
                      Needs nz <= 512 x rows (else PP_ERR_UNSUPPORTED_SIZE); other values
                      PP_ERR_INVALID_ARG; ignored for periodic z and for the adjoint's transposed
                      solve, which run the sweeps */
  int reserved[1]; /* must be zero */
} pp_plan_options;

typedef struct pp_plan pp_plan;

/* Create a plan (Sec. "Mathematical Formulation"; user API of the paper's appendix:
 * grid size, per-face boundary conditions, spacings).
 *   out       : receives the plan handle (owned by the caller; free with pp_plan_destroy)
 *   nx,ny,nz  : cells per axis (see size rules above)
 *   bc        : 6 face conditions, order x-,x+,y-,y+,z-,z+
 *   dx,dy,dz  : cell sizes (> 0)
 *   dtype     : arithmetic / I/O mode
 *   opt       : NULL or launch-shape overrides
 * Allocates the plan's device workspace (two spectral buffers) and its coefficient
 * tables on the current device.  Errors: PP_ERR_INVALID_ARG, PP_ERR_UNSUPPORTED_SIZE,
 * PP_ERR_BC_PAIRING, PP_ERR_OUT_OF_MEMORY, PP_ERR_CUDA; *out is NULL on error. */
pp_status pp_plan_create(pp_plan** out, int nx, int ny, int nz, const pp_bc bc[6], double dx, double dy,
                         double dz, pp_dtype dtype, const pp_plan_options* opt);

/* Solve A u = f (Secs. "Boundary Conditions" to "Solution of the Resulting Tridiagonal
 * Matrices").  f_dev, u_dev: device arrays of nx*ny*nz doubles (PP_F64, PP_MIXED_F64IO)
 * or floats (PP_MIXED_F32IO), owned by the caller; u may alias f.  Asynchronous on
 * stream.  Errors: PP_ERR_INVALID_ARG (NULL plan/pointer), PP_ERR_CUDA (launch).
 * Range: the double-float arithmetic has FP32's exponent range.  Sources and solutions with
 * magnitudes between about 1e-25 and 1e30 (the transforms sum up to n values, the z solve
 * scales by dz^2 and the inverse weights) keep the full ~47-bit accuracy; a solve outside the
 * range of full accuracy sets PP_ERR_RANGE in pp_plan_status().  The problem is linear: scale f
 * by a power of two into that range and u back by the same factor. */
pp_status pp_solve(pp_plan* plan, const void* f_dev, void* u_dev, pp_stream_t stream);

/* Mixed precision with one residual-refinement step: u0 = solve(f) (FP32 transforms; u0 is kept in
 * FP32), r = f - A u0 (7-point stencil of Sec. "Mathematical Formulation"; the second
 * differences of u0 are formed exactly, then scaled by 1/h^2 and subtracted from f in double-float
 * arithmetic, so r is accurate to ~2^-46 |f|), delta = solve(r) with FP32 I/O, u = u0 + delta
 * (rounded once to FP64).  Measured against the exact discrete solution of manufactured problems:
 * 1e-13 to 6e-13 at 64^3, 2.5e-12 to 3.2e-12 at 512^3, 5e-12 to 6e-12 at 1024^3 (one step multiplies
 * the mixed error by the correction solve's relative accuracy, ~1e-6).  Only for PP_MIXED_F64IO plans (PP_ERR_INVALID_ARG otherwise).  u
 * must not alias f.  The first call on a plan allocates its scratch: u0 and r in FP32, 8 bytes per
 * cell. */
pp_status pp_solve_refined(pp_plan* plan, const void* f_dev, void* u_dev, pp_stream_t stream);

/* pp_solve_refined without any device allocation.  (The paper has no counterpart: it is an
 * addition for callers that cannot allocate device memory when they solve -- time-stepping
 * loops that must not allocate, or risk an out-of-memory error, in the middle of a run, and
 * applications whose own memory manager has reserved the GPU's memory.)
 * pp_solve_refined allocates a grid-sized residual buffer on its first call; this entry point
 * instead uses a fixed 16 MiB device array inside the library (held by every GPU that loads the
 * library until the process exits) plus the plan's own workspace.  Same arithmetic as
 * pp_solve_refined, step for step.
 *   plan   : a PP_MIXED_F64IO plan (created beforehand; creating a plan does allocate)
 *   f_dev  : input, nx*ny*nz doubles on the device; u_dev: output, same size, must not alias f
 * Limit: nx*ny*nz <= 2,097,152 cells (u0 and the residual of such a grid in FP32), else PP_ERR_UNSUPPORTED_SIZE with a
 * message; other errors as pp_solve_refined.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress), so make that first call before any stream
 * capture.  All calls share the one array and each call overwrites what it reads, so calls
 * that may overlap on the GPU (different streams, or different host threads) race: serialise
 * them.  Asynchronous on stream like pp_solve. */
pp_status pp_solve_refined_noalloc(pp_plan* plan, const void* f_dev, void* u_dev, pp_stream_t stream);

/* Faces with data (non-homogeneous boundary conditions): folds face values into a source so that
 * pp_solve then solves the problem with those faces.  The ghost rules are the paper's (Sec.
 * "Boundary Conditions": the Dirichlet ghost extrapolates linearly to the face value):
 *   Dirichlet face value g:                u_ghost = 2 g - u_inside,
 *   Neumann data q (outward normal derivative): u_ghost = u_inside + h q,
 * so the stencil becomes L_g u = A u + L_g(0), and L_g u = f is A u = f - L_g(0).  This call
 * writes f_out = f_in - L_g(0): on the cells next to a face with data it subtracts 2 g / h^2
 * (Dirichlet) or q / h (Neumann), h the spacing normal to the face (edge and corner cells get
 * the terms of all their faces).
 *   g      : 6 pointers, faces x-,x+,y-,y+,z-,z+; NULL = homogeneous face (no term).  Device
 *            arrays of the plan's I/O type: x faces [nz][ny], y faces [nz][nx], z faces [ny][nx]
 *            (the face's cells in the grid's order).  A periodic face must be NULL.
 *   f_in   : device grid (nx*ny*nz, I/O type); f_out: device grid, may alias f_in (then only the
 *            face cells are rewritten; otherwise f_in is copied first).
 * With no Dirichlet face the solve removes the mean of the folded source (the compatibility
 * condition of the Neumann data), as for homogeneous faces.  FP64 arithmetic.  Asynchronous
 * on stream.  Errors: PP_ERR_INVALID_ARG (NULL plan / grid, data on a periodic face),
 * PP_ERR_CUDA (launch). */
pp_status pp_fold_bc(pp_plan* plan, const void* f_in, void* f_out, const void* const g[6], pp_stream_t stream);

/* Solve n independent problems, plans[i] applied to (f[i] -> u[i]) -- grids of any sizes,
 * boundary sets and dtypes -- as ONE CUDA-graph launch on `stream`.  The first call with a
 * given (plans, f, u) list captures the n five-kernel pipelines into a graph and instantiates
 * it (host work, a few ms); later calls with the same lists replay the cached graph (up to 8
 * batches are cached; pp_plan_destroy evicts the graphs that use that plan).  Members run on
 * up to 32 concurrent graph branches (measured: 8 -> 32 took 64 uneven grids from 4.19 to 4.04 ms
 * FP64, 2.26 to 2.13 ms FP32); members that share a plan share its workspace and run
 * one after another on one branch.
 * Autotuned members (options.autotune = 1) carry the settings that were fastest for each plan
 * alone, which in a shared graph can lose to the default ones (measured: 64 uneven grids, 5.36
 * against 4.30 ms FP64).  So the first call over a list of plans that includes autotuned members
 * waits for `stream` to be idle, allocates scratch grids of the members' sizes for the duration
 * of the call, and times the graph with the members' own settings and with the default launch
 * shapes and z sweeps (Thomas; Sherman-Morrison for periodic z) for the autotuned members; the
 * faster is kept for that list of plans (the plans themselves keep their settings for pp_solve).
 * Without the scratch memory, or while `stream` is being captured into a graph, the members' own
 * settings are used.
 * Errors: PP_ERR_INVALID_ARG (n < 0, NULL arrays or members), PP_ERR_CUDA (capture/instantiate/
 * launch). */
pp_status pp_solve_batched(pp_plan* const* plans, const void* const* f, void* const* u, int n,
                           pp_stream_t stream);

/* Adjoint: g_f = S^T g, where S is the solution operator f -> u.  Runs the transposed
 * pipeline: the line transforms, whose unnormalised syntheses are the transposes of the analyses
 * up to the per-mode weights the z scale absorbs, around the transposed tridiagonal
 * factorisation (for non-periodic z).  For periodic z the Sherman-Morrison sweep is run as it is
 * (A' and its rank-one update are symmetric, so that solve is its own transpose), and so is the
 * z transform (its eigenvalues are even in kz).  A is symmetric for periodic, Neumann and
 * Dirichlet faces, so S^T = S.  Same argument rules as pp_solve. */
pp_status pp_solve_adjoint(pp_plan* plan, const void* g_dev, void* gf_dev, pp_stream_t stream);

/* pp_solve on HOST buffers: copies f to the device, solves, copies u back, and synchronises
 * stream before returning.  The copies run in up to 8 plane chunks on two copy streams owned
 * by the plan: the host->device copy of a chunk overlaps the x/y forward transforms of the
 * chunks before it, the device->host copy of a chunk the inverse transforms of the chunks
 * after it (the z solve needs every plane, so it sits between the two halves).  Device staging
 * buffers and the streams are created by the first call on a plan.  f_host, u_host:
 * nx*ny*nz elements of the plan's I/O type (pinned memory gives full copy bandwidth and
 * lets the copies overlap).  Calls on one plan must not overlap. */
pp_status pp_solve_host(pp_plan* plan, const void* f_host, void* u_host, pp_stream_t stream);

/* Run one stage of the pp_solve pipeline on its own (for per-kernel timing and profiling):
 *   stage 0: x-forward transform   f -> plan workspace A
 *   stage 1: y-forward transform   A -> B
 *   stage 2: z tridiagonal solves  B in place
 *   stage 3: y-inverse transform   B -> A
 *   stage 4: x-inverse transform   A -> u
 * Running stages 0..4 in order on one stream is exactly pp_solve(plan, f, u, stream).
 * f is read only by stage 0 and u written only by stage 4 (either may be NULL otherwise).
 * Errors: PP_ERR_INVALID_ARG (bad stage / NULL pointer), PP_ERR_CUDA (launch). */
pp_status pp_run_stage(pp_plan* plan, int stage, const void* f_dev, void* u_dev, pp_stream_t stream);

/* Release the plan and its device memory (synchronises the device first). NULL is a no-op. */
pp_status pp_plan_destroy(pp_plan* plan);

/* Device-side status of the plan's solves since the last call (PP_OK unless a kernel reported a
 * condition).  Call after synchronising the stream; reading clears it.
 *   PP_ERR_RANGE: in at least one solve (every launch of the z-solve decides on its own data) the
 *     largest scaled right-hand side entering the tridiagonal solves was below 2^-100 (the
 *     FP32-exponent arithmetic then loses accuracy, e.g. a unit-cube source of magnitude 1e-32 at
 *     32^3), or the largest z-solve output exceeded 2^124 / (nx ny) (the inverse transforms may
 *     overflow FP32's range, e.g. 1e37 at 32^3), or a non-finite value appeared.  The decision is
 *     made on the largest magnitudes only, so small values beside large ones raise nothing.  Sources
 *     whose every magnitude is below FP32's smallest subnormal (~1.4e-45) are read as zero.  The
 *     problem is linear: scale f by a power of two and u back. */
pp_status pp_plan_status(pp_plan* plan);

/* Bytes of device memory held by the plan (workspace + tables). */
size_t pp_plan_device_bytes(const pp_plan* plan);

/* Launch shapes the plan uses (heuristic or autotuned): out[8] receives threads per CTA and lines
 * per CTA of the x-forward, y-forward, y-inverse and x-inverse kernels, in that order (for the y
 * kernels, real lines: two per complex column when its parts are transformed separately).
 * Errors: PP_ERR_INVALID_ARG (NULL). */
pp_status pp_plan_launch_shapes(const pp_plan* plan, int out[8]);

/* How the plan solves along z: *out = 0 (non-periodic z: Thomas), 1 (periodic z: Sherman-Morrison
 * sweeps) or 2 (periodic z: DFT along z and a diagonal solve), as chosen by options.z_method or the
 * autotuner.  Errors: PP_ERR_INVALID_ARG (NULL). */
pp_status pp_plan_z_method(const pp_plan* plan, int* out);

/* The plan's non-periodic z solver: *out = 1 for the Thomas sweeps (one thread per mode runs the
 * forward elimination and the back substitution along the whole line), or M = 8, 16 or 32 for the
 * partitioned solve (Sec. "Solution of the Resulting Tridiagonal Matrices", with the sequential
 * sweep replaced as in the parallel alternatives of Sec. "Cyclic Reduction Technique"): each line
 * is cut into ceil(nz / M) chunks of M rows, every chunk runs both recurrences of the Thomas
 * factorisation from a zero carry, and the chunks' affine carry maps are combined by recursive
 * doubling, ceil(log2(nz / M)) levels.  Same multipliers and results as the sweeps up to rounding;
 * about three times their arithmetic per value, in exchange for nz / M times the threads.  Chosen
 * by options.z_split or the autotuner; periodic z reports 1.  Errors: PP_ERR_INVALID_ARG (NULL). */
pp_status pp_plan_z_split(const pp_plan* plan, int* out);

/* ---- Prototype, not used by the solver: a DFT stage on the tensor cores (tcgen05, TMEM). ----
 * Measures whether a small-radix DFT stage posed as a dense product beats the double-float FFT stage
 * (Sec. "Computational Complexity Analysis" counts the transforms as the dominant work).
 *
 * pp_proto_tc_gemm_check: D = A B^T for A 128 x 64 and B 64 x 64 (bf16 bit patterns, row-major,
 * device), D 128 x 64 FP32 (device), by one CTA with four tcgen05.mma; swap = 1 exchanges the two
 * core-matrix offsets in the shared-memory descriptors (a self-check of the operand layout: only one
 * order reproduces A B^T).  *err_dev (device int, zeroed by the caller) becomes 1 if the MMAs did not
 * complete within the kernel's wait limit.  Asynchronous on stream.  Errors: PP_ERR_INVALID_ARG
 * (NULL), PP_ERR_CUDA (launch). */
pp_status pp_proto_tc_gemm_check(const void* A_dev, const void* B_dev, void* D_dev, int swap, int* err_dev,
                                 pp_stream_t stream);

/* pp_proto_dft32_tc: forward DFTs Y_k = sum_n z_n exp(-2 pi i n k / 32) of `lines` lines of 32
 * complex points (re_dev, im_dev: FP64 [lines][32], device; outputs the same, not aliasing the
 * inputs), at double-float accuracy from bf16 products: every line scaled by a power of two and cut
 * into seven 7-bit slices, the 28 slice products of the levels kept accumulated exactly in FP32
 * tensor memory, the levels summed in double-float (Ozaki-style splitting).  The seven slices of
 * the real 64 x 64 DFT matrix are built on the host and kept on the device (first call per device,
 * synchronous).  *err_dev as above.  Asynchronous on stream otherwise.  Errors:
 * PP_ERR_INVALID_ARG (NULL, lines < 0), PP_ERR_OUT_OF_MEMORY (the table), PP_ERR_CUDA (launch). */
pp_status pp_proto_dft32_tc(const double* re_dev, const double* im_dev, double* out_re_dev, double* out_im_dev,
                            long long lines, int* err_dev, pp_stream_t stream);

/* Human-readable detail of the last error on the calling thread ("" if none). */
const char* pp_last_error_string(void);

/* Library version string. */
const char* pp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PITTPACK_GB_H */
