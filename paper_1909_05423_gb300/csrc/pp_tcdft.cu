// pp_tcdft.cu -- prototype: a DFT stage on the 5th-generation tensor cores at FP64-class accuracy.
//
// Not used by the solver.  It measures whether a small-radix DFT stage posed as a dense matrix
// product can beat the double-float FFT stage of the line kernels (Sec. "Computational Complexity
// Analysis" counts the transforms as the dominant work; the tensor cores run bf16 products only).
//
// A line of N = 32 complex points z (double-float or FP64) is the real vector x = [Re z, Im z]
// (64 values), and its DFT Y_k = sum_n z_n exp(-2 pi i n k / N) the real product y = W x with
// W = [[C, S], [-S, C]], C = cos(2 pi n k / N), S = sin(2 pi n k / N).  With Ozaki's splitting
// (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", 2012):
//   - every line is scaled by a power of two to |x| < 1 and cut into seven slices of seven bits,
//     x = sum_i 2^(-7(i+1)) a_i with integer a_0 in [-128, 128] and a_i in [-64, 64] for i > 0
//     (rounded digits; all exact in bf16);
//   - W is cut the same way into b_j;
//   - each slice product a_i b_j^T is an integer matrix with entries below 2^14 * 64 = 2^20, so the
//     FP32 accumulators of the tensor cores sum it exactly, and so do the up-to-seven products of
//     one level l = i + j (below 2^23);
//   - y = sum_{l <= 6} 2^(-7(l+2)) acc_l, assembled in double-float.  The slicing remainders lie
//     below 2^-50 of the line's largest value; the dropped levels l >= 7 (products of digits of at
//     most 2^6 each, weight 2^-63) contribute ~2^-45 of it in the worst case, ~2^-48 typically.
// One CTA takes 128 lines (the MMA's M) and runs the 28 slice products as 112 tcgen05.mma of
// 128 x 64 x 16 (bf16 operands in shared memory, K-major, no swizzle; FP32 accumulators in TMEM,
// one 64-column accumulator per level, 448 columns), then reads the seven levels back with
// tcgen05.ld and assembles the outputs.
//
// Every wait is bounded: a CTA whose MMAs do not complete within the limit records an error code,
// frees its tensor memory and returns.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "pp_internal.h"

namespace pp {

namespace tc {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start, leading / stride byte offsets, version 1, no swizzle
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  unsigned long long d = 0;
  d |= (unsigned long long)((addr & 0x3ffffu) >> 4);
  d |= (unsigned long long)((lbo >> 4) & 0x3fffu) << 16;
  d |= (unsigned long long)((sbo >> 4) & 0x3fffu) << 32;
  d |= 1ull << 46;  // descriptor version
  return d;         // base offset 0, absolute LBO mode, layout type 0 (no swizzle)
}

// instruction descriptor, kind::f16: FP32 accumulator, bf16 A and B, both K-major, M x N
__host__ __device__ constexpr unsigned instr_desc(int M, int N) {
  return (1u << 4)                     // D format FP32
         | (1u << 7) | (1u << 10)      // A, B format bf16
         | ((unsigned)(N >> 3) << 17)  // N / 8
         | ((unsigned)(M >> 4) << 24); // M / 16
}

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned idesc,
                                         int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// bounded wait for the phase of the given parity; returns false when the limit ran out
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity, long long limit) {
  for (long long it = 0; it < limit; it++) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float* v) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// warp-wide TMEM allocation (the address lands in *slot) and release
__device__ __forceinline__ void tmem_alloc(unsigned* slot, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(unsigned taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Core-matrix layout of a K-major bf16 operand of R rows x 64 K values in shared memory: the 8 x 8
// core matrix (row group g, K group q) at byte 1024 g + 128 q, its rows 16 bytes apart.  Adjacent
// K groups are 128 bytes apart (the leading offset), adjacent row groups 1024 (the stride offset).
__device__ __forceinline__ int cm_off(int row, int k) { return (row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2; }

constexpr long long kWaitLimit = 1ll << 24;

}  // namespace tc

// ---------------------------------------------------------------- descriptor self-check
// D (128 x 64, FP32) = A (128 x 64, bf16, row-major) * B^T (B: 64 x 64, bf16, row-major = K-major),
// one CTA of 128 threads, four MMAs of K = 16.  swap = 1 exchanges the two offsets in the
// descriptors (the self-check tells which order the hardware reads).  err: 0, or 1 on a timeout.
__global__ void __launch_bounds__(128) k_tc_gemm_check(const uint16_t* __restrict__ A, const uint16_t* __restrict__ B,
                                                       float* __restrict__ D, int swap, int* err) {
  __shared__ __align__(1024) unsigned char sa[128 * 64 * 2];
  __shared__ __align__(1024) unsigned char sb[64 * 64 * 2];
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ unsigned tslot;
  const int t = (int)threadIdx.x;
  for (int i = t; i < 128 * 64; i += 128) {
    const int r = i >> 6, k = i & 63;
    *reinterpret_cast<uint16_t*>(sa + tc::cm_off(r, k)) = A[i];
  }
  for (int i = t; i < 64 * 64; i += 128) {
    const int r = i >> 6, k = i & 63;
    *reinterpret_cast<uint16_t*>(sb + tc::cm_off(r, k)) = B[i];
  }
  tc::fence_async_smem();
  const unsigned mb = tc::smem_u32(&mbar);
  if (t == 0) tc::mbar_init(mb, 1);
  if (t < 32) tc::tmem_alloc(&tslot, 64);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const unsigned tmem = tslot;
  if (t == 0) {
    const unsigned lbo = swap ? 1024u : 128u, sbo = swap ? 128u : 1024u;
    const unsigned idesc = tc::instr_desc(128, 64);
    for (int kk = 0; kk < 4; kk++) {
      const unsigned long long da = tc::smem_desc(tc::smem_u32(sa) + kk * 256, lbo, sbo);
      const unsigned long long db = tc::smem_desc(tc::smem_u32(sb) + kk * 256, lbo, sbo);
      tc::mma_bf16(tmem, da, db, idesc, kk > 0);
    }
    tc::mma_commit(mb);
  }
  const bool done = tc::mbar_wait(mb, 0, tc::kWaitLimit);
  tc::tc_fence_after();
  if (!done) {
    if (t == 0) atomicExch(err, 1);
  } else {
    const int w = t >> 5, lane = t & 31;
    const int row = 32 * w + lane;
    for (int c0 = 0; c0 < 64; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((unsigned)(32 * w) << 16) + (unsigned)c0, v);
      for (int i = 0; i < 16; i++) D[row * 64 + c0 + i] = v[i];
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (t < 32) tc::tmem_free(tmem, 64);
}

// ---------------------------------------------------------------- DFT-32 stage
constexpr int kTcLines = 128;         // lines per tile (the MMA's M)
constexpr int kTcSlices = 7;          // seven-bit slices per operand
constexpr int kTcLevels = 7;          // levels l = i + j kept, 0..6
constexpr int kTcASlice = kTcLines * 64 * 2;   // bytes of one A slice (128 x 64 bf16)
constexpr int kTcBSlice = 64 * 64 * 2;         // bytes of one W slice
constexpr int kTcSmem = kTcSlices * kTcASlice + kTcSlices * kTcBSlice + 64;

__device__ __forceinline__ uint16_t bf16_bits(float v) {  // v is an integer of at most 8 bits: exact
  return (uint16_t)(__float_as_uint(v) >> 16);
}

// dft32: W slices (7 x 64 x 64 bf16, row c = output c, K contiguous) in global memory; re/im of
// `lines` lines of 32 points in, out.  One persistent CTA of 128 threads per SM; thread t owns line
// t of the tile (and TMEM lane t).
__global__ void __launch_bounds__(128, 1) k_tc_dft32(const uint16_t* __restrict__ wsl, const double* __restrict__ re,
                                                     const double* __restrict__ im, double* __restrict__ ore,
                                                     double* __restrict__ oim, long long lines, int* err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* sa = tsm;                                 // 7 A slices
  unsigned char* sb = tsm + kTcSlices * kTcASlice;         // 7 W slices
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(sb + kTcSlices * kTcBSlice);
  unsigned* tslot = reinterpret_cast<unsigned*>(mbar + 1);
  const int t = (int)threadIdx.x;
  // W slices into the core-matrix layout, once per CTA
  for (int i = t; i < kTcSlices * 64 * 64; i += kTcLines) {
    const int sl = i >> 12, r = (i >> 6) & 63, k = i & 63;
    *reinterpret_cast<uint16_t*>(sb + sl * kTcBSlice + tc::cm_off(r, k)) = wsl[i];
  }
  const unsigned mb = tc::smem_u32(mbar);
  if (t == 0) tc::mbar_init(mb, 1);
  if (t < 32) tc::tmem_alloc(tslot, 512);
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const unsigned tmem = *tslot;
  const long long ntiles = (lines + kTcLines - 1) / kTcLines;
  unsigned phase = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long line = tile * kTcLines + t;
    const bool live = line < lines;
    // 1. the line, scaled by a power of two below 1 in magnitude, cut into seven 7-bit slices
    int emax = -1074;
    if (live) {
      for (int n = 0; n < 32; n++) {
        int e;
        frexp(re[line * 32 + n], &e); emax = max(emax, e);
        frexp(im[line * 32 + n], &e); emax = max(emax, e);
      }
    }
    const double sc = ldexp(1.0, -emax);  // |x sc| < 1
    for (int q = 0; q < 8; q++) {         // K groups of 8 values: q < 4 real parts, q >= 4 imaginary
      float hi[8], lo[8];
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const int k = q * 8 + u;
        const double v = live ? (k < 32 ? re[line * 32 + k] : im[line * 32 + k - 32]) * sc : 0.0;
        const df d = df_from_double(v);
        hi[u] = d.hi;
        lo[u] = d.lo;
      }
#pragma unroll
      for (int sl = 0; sl < kTcSlices; sl++) {
        const float w = __int_as_float((127 + 7 * (sl + 1)) << 23);    // 2^(7(sl+1))
        const float iw = __int_as_float((127 - 7 * (sl + 1)) << 23);   // 2^(-7(sl+1))
        uint32_t pk[4];
#pragma unroll
        for (int u = 0; u < 8; u++) {
          const float a = rintf(hi[u] * w);                 // the slice digit
          float s2, e2;
          two_sum(__fmaf_rn(-a, iw, hi[u]), lo[u], s2, e2);  // exact remainder (the FMA is exact), renormalised
          hi[u] = s2;
          lo[u] = e2;
          const uint32_t b = bf16_bits(a);
          if (u & 1) pk[u >> 1] |= b << 16;
          else pk[u >> 1] = b;
        }
        *reinterpret_cast<uint4*>(sa + sl * kTcASlice + tc::cm_off(t, q * 8)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    // 2. the 28 slice products of levels 0..6, accumulated per level in TMEM (64 columns each)
    if (t == 0) {
      const unsigned idesc = tc::instr_desc(kTcLines, 64);
      for (int l = 0; l < kTcLevels; l++) {
        bool first = true;
        for (int i = 0; i <= l; i++) {
          const int j = l - i;
          if (i >= kTcSlices || j >= kTcSlices) continue;
          for (int kk = 0; kk < 4; kk++) {
            const unsigned long long da =
                tc::smem_desc(tc::smem_u32(sa + i * kTcASlice) + kk * 256, 128u, 1024u);
            const unsigned long long db =
                tc::smem_desc(tc::smem_u32(sb + j * kTcBSlice) + kk * 256, 128u, 1024u);
            tc::mma_bf16(tmem + 64 * l, da, db, idesc, first ? 0 : 1);
            first = false;
          }
        }
      }
      tc::mma_commit(mb);
    }
    const bool done = tc::mbar_wait(mb, phase, tc::kWaitLimit);
    phase ^= 1u;
    if (__syncthreads_or(!done)) {
      if (t == 0) atomicExch(err, 1);
      break;
    }
    tc::tc_fence_after();
    // 3. y = 2^emax sum_l 2^(-7(l+2)) acc_l, summed from the smallest level up in double-float
    const unsigned lane_base = tmem + ((unsigned)(32 * (t >> 5)) << 16);
    for (int c0 = 0; c0 < 64; c0 += 16) {
      df y[16];
#pragma unroll
      for (int u = 0; u < 16; u++) y[u] = df{0.f, 0.f};
      for (int l = kTcLevels - 1; l >= 0; l--) {
        float v[16];
        tc::tmem_ld16(lane_base + (unsigned)(64 * l + c0), v);
        const float wl = __int_as_float((127 - 7 * (l + 2)) << 23);
#pragma unroll
        for (int u = 0; u < 16; u++) y[u] = y[u] + df{v[u] * wl, 0.f};
      }
      if (live) {
        double* dst = (c0 < 32) ? ore : oim;
        const int k0 = c0 & 31;
#pragma unroll
        for (int u = 0; u < 16; u++) dst[line * 32 + k0 + u] = ldexp(df_to_double(y[u]), emax);
      }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (t < 32) tc::tmem_free(tmem, 512);
}

// The seven 7-bit slices of the real 64 x 64 DFT matrix W = [[C, S], [-S, C]] of length 32
// (C_kn = cos(2 pi nk/32), S_kn = sin(2 pi nk/32), angles reduced to nk mod 32), as bf16 bit patterns
// [slice][row = output][K = input], built on the host in FP64 once per device and kept.
static const void* tc_w_slices(int dev) {
  static std::mutex mu;
  static const void* tab[64] = {};
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (tab[dev]) return tab[dev];
  std::vector<uint16_t> h((size_t)kTcSlices * 64 * 64);
  const double pi = 3.14159265358979323846;
  for (int r = 0; r < 64; r++) {
    for (int k = 0; k < 64; k++) {
      const int kk = r & 31, n = k & 31;           // output k (re / im), input n (re / im)
      const int m = (kk * n) & 31;
      const double c = std::cos(2.0 * pi * m / 32.0), sn = std::sin(2.0 * pi * m / 32.0);
      double w = (r < 32) ? (k < 32 ? c : sn) : (k < 32 ? -sn : c);
      for (int sl = 0; sl < kTcSlices; sl++) {
        const double sc = std::ldexp(1.0, 7 * (sl + 1));
        const double a = std::nearbyint(w * sc);
        w -= a / sc;                                // exact
        const float af = (float)a;
        uint32_t bits;
        std::memcpy(&bits, &af, 4);
        h[((size_t)sl * 64 + r) * 64 + k] = (uint16_t)(bits >> 16);
      }
    }
  }
  void* d = nullptr;
  if (cudaMalloc(&d, h.size() * 2) != cudaSuccess) return nullptr;
  if (cudaMemcpy(d, h.data(), h.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) { cudaFree(d); return nullptr; }
  tab[dev] = d;
  return d;
}

}  // namespace pp

extern "C" {
// Prototype entry points (declared in pittpack_gb.h): descriptor self-check.
pp_status pp_proto_tc_gemm_check(const void* A_dev, const void* B_dev, void* D_dev, int swap, int* err_dev,
                                 pp_stream_t stream) {
  if (!A_dev || !B_dev || !D_dev || !err_dev) return pp::set_last_error(PP_ERR_INVALID_ARG, "NULL pointer");
  pp::k_tc_gemm_check<<<1, 128, 0, (cudaStream_t)stream>>>(static_cast<const uint16_t*>(A_dev),
                                                           static_cast<const uint16_t*>(B_dev), static_cast<float*>(D_dev),
                                                           swap, err_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PP_OK : pp::set_last_error(PP_ERR_CUDA, cudaGetErrorString(e));
}

pp_status pp_proto_dft32_tc(const double* re_dev, const double* im_dev, double* out_re_dev, double* out_im_dev,
                            long long lines, int* err_dev, pp_stream_t stream) {
  if (!re_dev || !im_dev || !out_re_dev || !out_im_dev || !err_dev || lines < 0)
    return pp::set_last_error(PP_ERR_INVALID_ARG, "NULL pointer or negative line count");
  if (lines == 0) return PP_OK;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  const void* w_slices_dev = pp::tc_w_slices(dev);
  if (!w_slices_dev) return pp::set_last_error(PP_ERR_OUT_OF_MEMORY, "DFT-matrix slice table");
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaFuncSetAttribute(pp::k_tc_dft32, cudaFuncAttributeMaxDynamicSharedMemorySize, pp::kTcSmem);
  if (e != cudaSuccess) return pp::set_last_error(PP_ERR_CUDA, cudaGetErrorString(e));
  const long long ntiles = (lines + pp::kTcLines - 1) / pp::kTcLines;
  const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);
  pp::k_tc_dft32<<<grid, pp::kTcLines, pp::kTcSmem, (cudaStream_t)stream>>>(
      static_cast<const uint16_t*>(w_slices_dev), re_dev, im_dev, out_re_dev, out_im_dev, lines, err_dev);
  e = cudaGetLastError();
  return e == cudaSuccess ? PP_OK : pp::set_last_error(PP_ERR_CUDA, cudaGetErrorString(e));
}
}
