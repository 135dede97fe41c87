// pp_misc.cu -- residual and update kernels of the mixed-precision refinement step.
//
// r = f - A_h u0 with the cell-centred 7-point stencil (Sec. "Mathematical Formulation") and the
// face ghost rules (periodic wrap, Neumann u[-1] = u[0], homogeneous Dirichlet u[-1] = -u[0]);
// then u = u0 + delta with delta = solve(r).
//
// The first solve's u0 comes out of FP32 transforms and is kept as FP32 (its x-inverse writes FP32
// into the refinement scratch).  That makes the stencil's second differences exact: with u0 in FP32, (m - c) and (p - c) are each an exact sum of two
// FP32 numbers (TwoSum), and their sum is formed in double-float to ~2^-48 of the difference
// itself.  Only then are the three differences scaled by 1/h^2 and subtracted from f.  Formed the
// other way round (each neighbour scaled, the sum taken after), the second difference inherits an
// error of ~2^-48 |u| -- 1/(kappa h)^2 times its own size for a smooth u -- which bounded the
// refined solution near 2e-12 at 512^3; with exact differences the residual is accurate to
// ~2^-46 |f| and one step reaches ~1e-13.  r and delta are stored as FP32: r is the input of an
// FP32-transform solve, and delta is ~1e-7 of u.
#include <cstdint>

#include "pp_internal.h"

namespace pp {

struct ResArgs {
  const double* f;
  const float* u;  // u0, FP32
  float* r;
  int nx, ny, nz;
  int bc[6];
  float ix2[2], iy2[2], iz2[2];  // 1/h^2 as (hi, lo)
  FastDiv fd_ny;                 // row -> (k, j)
  FastDiv fd_chunks;             // block -> (row, chunk of the row)
  int iso;                       // dx == dy == dz: the three second differences share one scaling
};

// ghost value of a homogeneous face (1 = Neumann: copy; 2 = Dirichlet: negate)
__device__ __forceinline__ float ghost_or(int bc, float c) { return bc == 1 ? c : -c; }

// (m - c) + (p - c) for FP32 m, c, p: each difference exactly as an unevaluated pair (TwoSum), the
// two pairs summed in double-float (relative error ~2^-48 of the result).  The sums and products
// below use the unnormalised forms of pp_arith.cuh (hi + lo keeps the value; only the final
// rounding to FP32 needs it normalised).
__device__ __forceinline__ df second_difference(float m, float c, float p) {
  df d1, d2;
  two_sum(m, -c, d1.hi, d1.lo);
  two_sum(p, -c, d2.hi, d2.lo);
  return add_u(d1, d2);
}

__device__ __forceinline__ float u32(const float* u, long long i) { return __ldg(u + i); }
__device__ __forceinline__ float4 u128(const float* u, long long i) { return __ldg(reinterpret_cast<const float4*>(u + i)); }

// A_h u0 at one cell from its three second differences (exact pairs, see second_difference):
// scaled by 1/h^2 per axis and summed, or, with equal spacings, summed and scaled once.
__device__ __forceinline__ df stencil(const ResArgs& a, df sx, df sy, df sz) {
  if (a.iso) return mul_u(add_u(add_u(sx, sy), sz), df{a.ix2[0], a.ix2[1]});
  return add_u(add_u(mul_u(sx, df{a.ix2[0], a.ix2[1]}), mul_u(sy, df{a.iy2[0], a.iy2[1]})),
               mul_u(sz, df{a.iz2[0], a.iz2[1]}));
}
__device__ __forceinline__ float4 ghost4(int bc, float4 c) {
  return make_float4(ghost_or(bc, c.x), ghost_or(bc, c.y), ghost_or(bc, c.z), ghost_or(bc, c.w));
}

// Block b takes chunk b mod C of x-row b / C (C chunks of blockDim.x cells per row), so consecutive
// blocks walk the grid in memory order (the chunks of a row, then the next row): with the chunk in
// blockIdx.y the grid was read in C passes of one chunk of every row (1024^3: 6.72 ms).
__global__ void __launch_bounds__(256) k_residual(const ResArgs a) {
  const unsigned row = a.fd_chunks.div(blockIdx.x);
  const int i = (int)((blockIdx.x - row * a.fd_chunks.d) * blockDim.x + threadIdx.x);
  if (i >= a.nx) return;
  const int k = (int)a.fd_ny.div(row);
  const int j = (int)(row - (unsigned)k * (unsigned)a.ny);
  const long long nxy = (long long)a.nx * a.ny;
  const long long p = (long long)row * a.nx + i;
  const float* u = a.u;
  const float c = u32(u, p);
  float xm, xp, ym, yp, zm, zp;
  if (i > 0) xm = u32(u, p - 1);
  else xm = (a.bc[0] == 0) ? u32(u, p + a.nx - 1) : ghost_or(a.bc[0], c);
  if (i < a.nx - 1) xp = u32(u, p + 1);
  else xp = (a.bc[1] == 0) ? u32(u, p - (a.nx - 1)) : ghost_or(a.bc[1], c);
  if (j > 0) ym = u32(u, p - a.nx);
  else ym = (a.bc[2] == 0) ? u32(u, p + (long long)(a.ny - 1) * a.nx) : ghost_or(a.bc[2], c);
  if (j < a.ny - 1) yp = u32(u, p + a.nx);
  else yp = (a.bc[3] == 0) ? u32(u, p - (long long)(a.ny - 1) * a.nx) : ghost_or(a.bc[3], c);
  if (k > 0) zm = u32(u, p - nxy);
  else zm = (a.bc[4] == 0) ? u32(u, p + (long long)(a.nz - 1) * nxy) : ghost_or(a.bc[4], c);
  if (k < a.nz - 1) zp = u32(u, p + nxy);
  else zp = (a.bc[5] == 0) ? u32(u, p - (long long)(a.nz - 1) * nxy) : ghost_or(a.bc[5], c);
  const df lap = stencil(a, second_difference(xm, c, xp), second_difference(ym, c, yp), second_difference(zm, c, zp));
  const df r = add_u(df_from_double(__ldg(a.f + p)), -lap);
  a.r[p] = df_to_f32(r);
}

// The same residual for four consecutive cells of an x-row a thread (nx a multiple of 4, f 16-byte
// aligned): 16-byte loads of u0's rows and of f, and each exact x-difference formed once for the
// two cells that share it (five TwoSums instead of eight).  Same operations on the same operands
// as k_residual, so the same bits.
__global__ void __launch_bounds__(256) k_residual4(const ResArgs a) {
  const unsigned row = a.fd_chunks.div(blockIdx.x);
  const int i0 = 4 * (int)((blockIdx.x - row * a.fd_chunks.d) * blockDim.x + threadIdx.x);
  if (i0 >= a.nx) return;
  const int k = (int)a.fd_ny.div(row);
  const int j = (int)(row - (unsigned)k * (unsigned)a.ny);
  const long long nxy = (long long)a.nx * a.ny;
  const long long p = (long long)row * a.nx + i0;
  const float* u = a.u;
  const float4 c = u128(u, p);
  float xl, xr;
  if (i0 > 0) xl = u32(u, p - 1);
  else xl = (a.bc[0] == 0) ? u32(u, p + a.nx - 1) : ghost_or(a.bc[0], c.x);
  if (i0 + 4 < a.nx) xr = u32(u, p + 4);
  else xr = (a.bc[1] == 0) ? u32(u, p - (a.nx - 4)) : ghost_or(a.bc[1], c.w);
  float4 ym, yp, zm, zp;
  if (j > 0) ym = u128(u, p - a.nx);
  else ym = (a.bc[2] == 0) ? u128(u, p + (long long)(a.ny - 1) * a.nx) : ghost4(a.bc[2], c);
  if (j < a.ny - 1) yp = u128(u, p + a.nx);
  else yp = (a.bc[3] == 0) ? u128(u, p - (long long)(a.ny - 1) * a.nx) : ghost4(a.bc[3], c);
  if (k > 0) zm = u128(u, p - nxy);
  else zm = (a.bc[4] == 0) ? u128(u, p + (long long)(a.nz - 1) * nxy) : ghost4(a.bc[4], c);
  if (k < a.nz - 1) zp = u128(u, p + nxy);
  else zp = (a.bc[5] == 0) ? u128(u, p - (long long)(a.nz - 1) * nxy) : ghost4(a.bc[5], c);
  const double2 f01 = __ldg(reinterpret_cast<const double2*>(a.f + p));
  const double2 f23 = __ldg(reinterpret_cast<const double2*>(a.f + p + 2));
  // exact x-differences: d0 = xl - c.x, d1 = c.y - c.x, d2 = c.z - c.y, d3 = c.w - c.z, d4 = xr - c.w
  df d0, d1, d2, d3, d4;
  two_sum(xl, -c.x, d0.hi, d0.lo);
  two_sum(c.y, -c.x, d1.hi, d1.lo);
  two_sum(c.z, -c.y, d2.hi, d2.lo);
  two_sum(c.w, -c.z, d3.hi, d3.lo);
  two_sum(xr, -c.w, d4.hi, d4.lo);
  const float cv[4] = {c.x, c.y, c.z, c.w};
  const float ymv[4] = {ym.x, ym.y, ym.z, ym.w}, ypv[4] = {yp.x, yp.y, yp.z, yp.w};
  const float zmv[4] = {zm.x, zm.y, zm.z, zm.w}, zpv[4] = {zp.x, zp.y, zp.z, zp.w};
  const df sx[4] = {add_u(d0, d1), add_u(-d1, d2), add_u(-d2, d3), add_u(-d3, d4)};
  const double fv[4] = {f01.x, f01.y, f23.x, f23.y};
  float out[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const df lap = stencil(a, sx[q], second_difference(ymv[q], cv[q], ypv[q]), second_difference(zmv[q], cv[q], zpv[q]));
    out[q] = df_to_f32(add_u(df_from_double(fv[q]), -lap));
  }
  *reinterpret_cast<float4*>(a.r + p) = make_float4(out[0], out[1], out[2], out[3]);
}

// u = u0 + d (- shift, the mean of u0, when the problem is singular and the result must be
// mean-free); u0 and d are FP32, their sum is exact in double-float, rounded once to FP64.
__device__ __forceinline__ double add_value(float u0, float d, const float2* shift) {
  if (!shift) return __dadd_rn(double_from_f32(u0), double_from_f32(d));  // RN(u0 + d)
  df v;
  two_sum(u0, d, v.hi, v.lo);
  v = v - df{shift->x, shift->y};
  return __dadd_rn(double_from_f32(v.hi), double_from_f32(v.lo));
}
// Four values a thread (16-byte loads, two 16-byte stores): the kernel is bound by HBM and needs
// the loads in flight; the FP32 values are widened with integer operations, so each value costs the
// FP64 unit (1/67 of the FP32 rate) one add.  One value a thread with the FP64 unit's conversion
// took 4.33 ms at 1024^3 (two FP64 operations per value), with integer widening 5.18 ms (latency).
__global__ void __launch_bounds__(256) k_add4(double2* u, const float4* u0, const float4* d, long long n4,
                                              const float2* shift) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n4) return;
  const float4 a = __ldg(u0 + p), b = __ldg(d + p);
  u[2 * p] = make_double2(add_value(a.x, b.x, shift), add_value(a.y, b.y, shift));
  u[2 * p + 1] = make_double2(add_value(a.z, b.z, shift), add_value(a.w, b.w, shift));
}
// any size or alignment
__global__ void __launch_bounds__(256) k_add(double* u, const float* u0, const float* d, long long n,
                                             const float2* shift) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  df v;
  two_sum(__ldg(u0 + p), __ldg(d + p), v.hi, v.lo);
  if (shift) v = v - df{shift->x, shift->y};
  u[p] = df_to_double(v);
}

// Block partial sums of an FP32 grid in double-float arithmetic (first pass of the mean).
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads) k_partial_sum(const float* u, long long n, float2* part) {
  __shared__ df sh[kSumThreads];
  df acc = df{0.f, 0.f};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
    acc = acc + df{__ldg(u + p), 0.0f};
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = make_float2(sh[0].hi, sh[0].lo);
}

// Second pass: mean = (sum of partials) / n, one block.
__global__ void __launch_bounds__(kSumThreads) k_finish_mean(const float2* part, int nparts, float inv_n_hi,
                                                              float inv_n_lo, float2* mean) {
  __shared__ df sh[kSumThreads];
  df acc = df{0.f, 0.f};
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc = acc + df{part[i].x, part[i].y};
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    df m = sh[0] * df{inv_n_hi, inv_n_lo};
    *mean = make_float2(m.hi, m.lo);
  }
}

static void split_h(double v, float* o) {
  float h = (float)v;
  o[0] = h;
  o[1] = (float)(v - (double)h);
}

cudaError_t launch_residual(const pp_plan* p, const void* f, const void* u, void* r, cudaStream_t st) {
  ResArgs a;
  a.f = (const double*)f; a.u = (const float*)u; a.r = (float*)r;
  a.nx = p->nx; a.ny = p->ny; a.nz = p->nz;
  for (int i = 0; i < 6; i++) a.bc[i] = p->bc[i];
  split_h(1.0 / (p->dx * p->dx), a.ix2);
  split_h(1.0 / (p->dy * p->dy), a.iy2);
  split_h(1.0 / (p->dz * p->dz), a.iz2);
  a.fd_ny = FastDiv::make((unsigned)p->ny);
  a.iso = (p->dx == p->dy && p->dy == p->dz) ? 1 : 0;
  // four cells a thread where the rows allow 16-byte accesses (u0 and r are the library's scratch,
  // 16-byte aligned with nx ny nz a multiple of 4; f is the caller's)
  const bool vec = p->nx % 4 == 0 && (uintptr_t)f % 16 == 0 && (uintptr_t)u % 16 == 0 && (uintptr_t)r % 16 == 0;
  const int cells = vec ? p->nx / 4 : p->nx;  // threads per row
  const int threads = cells >= 256 ? 256 : (cells + 31) / 32 * 32;
  const unsigned chunks = (unsigned)((cells + threads - 1) / threads);
  a.fd_chunks = FastDiv::make(chunks);
  // rows x chunks ~ nx ny nz / 256 + ny nz stays below 2^31 for every plan (ny nz < 2^31, and
  // chunks > 1 only for nx > 256, where nx ny nz <= 2^36 bounds it by 2^29)
  const long long blocks = (long long)p->ny * p->nz * chunks;
  if (blocks >= (1LL << 31)) return cudaErrorInvalidConfiguration;
  if (vec) k_residual4<<<(unsigned)blocks, threads, 0, st>>>(a);
  else k_residual<<<(unsigned)blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mean(const pp_plan* p, const void* u, void* partials, int nparts, void* mean, cudaStream_t st) {
  long long n = (long long)p->nx * p->ny * p->nz;
  k_partial_sum<<<nparts, kSumThreads, 0, st>>>((const float*)u, n, (float2*)partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  float inv[2];
  split_h(1.0 / (double)n, inv);
  k_finish_mean<<<1, kSumThreads, 0, st>>>((const float2*)partials, nparts, inv[0], inv[1], (float2*)mean);
  return cudaGetLastError();
}

// Faces with data: f -= coef * g on the cells next to one face (coef = 2/h^2 Dirichlet, 1/h
// Neumann).  Face arrays are [a0][a1]: x faces (k, j), y faces (k, i), z faces (j, i).  One launch
// per face, in sequence on the stream, so edge and corner cells take every face's term.
__global__ void k_fold_face(void* f, const void* g, int nx, int ny, int nz, int face, double coef, int f32) {
  const int axis = face >> 1, hi = face & 1;
  const long long n1 = (axis == 0) ? ny : nx;
  const long long n0 = (axis == 2) ? ny : nz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n0 * n1) return;
  const int a0 = (int)(t / n1), a1 = (int)(t - (t / n1) * n1);
  int i, j, k;
  if (axis == 0) { k = a0; j = a1; i = hi ? nx - 1 : 0; }
  else if (axis == 1) { k = a0; i = a1; j = hi ? ny - 1 : 0; }
  else { j = a0; i = a1; k = hi ? nz - 1 : 0; }
  const long long p = ((long long)k * ny + j) * nx + i;
  if (f32) {
    float* fp = reinterpret_cast<float*>(f);
    const double v = __fma_rn(-coef, (double)reinterpret_cast<const float*>(g)[t], (double)fp[p]);
    fp[p] = __double2float_rn(v);
  } else {
    double* fp = reinterpret_cast<double*>(f);
    fp[p] = __fma_rn(-coef, reinterpret_cast<const double*>(g)[t], fp[p]);
  }
}

cudaError_t launch_fold_face(void* f, const void* g, int nx, int ny, int nz, int face, double coef, bool f32,
                             cudaStream_t st) {
  const int axis = face >> 1;
  const long long n = (long long)(axis == 2 ? ny : nz) * (axis == 0 ? ny : nx);
  k_fold_face<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(f, g, nx, ny, nz, face, coef, f32 ? 1 : 0);
  return cudaGetLastError();
}

// Timing input of the autotuner: values in [-1, 1) from an integer hash of the index (no
// statistical quality needed, only normal non-constant data).
__global__ void k_fill(void* x, long long n, int f32) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned h = (unsigned)i * 2654435761u;
  h ^= h >> 15;
  h *= 2246822519u;
  h ^= h >> 13;
  const float v = (float)(h >> 8) * (1.0f / 8388608.0f) - 1.0f;
  if (f32) reinterpret_cast<float*>(x)[i] = v;
  else reinterpret_cast<double*>(x)[i] = double_from_f32(v);
}

cudaError_t launch_fill(void* x, long long n, bool f32, cudaStream_t st) {
  k_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, n, f32 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_add(const pp_plan* p, void* u, const void* u0, const void* d, const void* shift, cudaStream_t st) {
  long long n = (long long)p->nx * p->ny * p->nz;
  const bool vec = n % 4 == 0 && ((uintptr_t)u | (uintptr_t)u0 | (uintptr_t)d) % 16 == 0;
  if (vec) {
    const long long n4 = n / 4;
    k_add4<<<(unsigned)((n4 + 255) / 256), 256, 0, st>>>((double2*)u, (const float4*)u0, (const float4*)d, n4,
                                                          (const float2*)shift);
  } else {
    k_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((double*)u, (const float*)u0, (const float*)d, n,
                                                        (const float2*)shift);
  }
  return cudaGetLastError();
}

}  // namespace pp
