// pp_zfft.cu -- periodic z by a third transform: the diagonal solve between the forward and the
// inverse z-line DFTs.
//
// With periodic z the z system of every (kx,ky) pair is circulant, so a DFT along z
// diagonalises it (the alternative the paper names beside Sherman-Morrison for periodic
// directions, Sec. "Introduction": Fourier analysis in every periodic direction): mode
// (kx,ky,kz) has the eigenvalue
//     sigma = lambda_x/dx^2 + lambda_y/dy^2 + (2 cos(2 pi kz / nz) - 2) / dz^2,
// and U = w_x w_y / nz * F / sigma, with w_x w_y the x/y inverse weights and 1/nz the weight of
// the unnormalised inverse z DFT.  sigma = 0 only for the singular mode of a problem without
// Dirichlet faces, whose coefficient is set to zero: the zero-mean solution of A u = f - mean f.
// No term of sigma cancels another (all three are <= 0), so it is accurate to its last bits.
//
// The z lines are complex: for spectra of complex modes (x or y periodic) each mode's (re, im)
// pair is one line; for all-real spectra two adjacent real modes A, B travel as one complex line
// Z = X + i Y.  Their DFTs separate as X_k = (Z_k + conj Z_{N-k}) / 2, Y_k = (Z_k - conj Z_{N-k})
// / 2i, and with a = 1/sigma_A(k), b = 1/sigma_B(k) (sigma(k) = sigma(N-k)) the solved line is
//     Z'_k = p Z_k + q conj Z_{N-k},  Z'_{N-k} = p Z_{N-k} + q conj Z_k,  p = (a+b)/2, q = (a-b)/2;
// for complex modes a = b and q = 0.  One thread takes the pair (k, N-k) of one line.
// Arithmetic: double-float (pp_arith.cuh) on the plan's spill type.  The range report of
// pp_range.cuh covers the weighted inputs and the outputs.
#include "pp_range.cuh"

namespace pp {

__device__ __forceinline__ df zf_ld(const float2* p) { const float2 v = *p; return df{v.x, v.y}; }
__device__ __forceinline__ df zf_ld(const float* p) { return df{*p, 0.0f}; }
__device__ __forceinline__ void zf_st(float2* p, df v) { *p = make_float2(v.hi, v.lo); }
__device__ __forceinline__ void zf_st(float* p, df v) { *p = df_to_f32(v); }

// 1/sigma, or 0 for the singular mode
__device__ __forceinline__ df zf_inv(df lam_xy, df lam_z) {
  const df s = lam_xy + lam_z;
  if (s.hi == 0.0f) return df{0.0f, 0.0f};
  return df_rcp(s);
}

// grid: x over the complex lines of a plane, y = k in [0, nz/2]
template <class S>
__device__ __forceinline__ void zdiag_pair(const ZDiagArgs& a, float& dmax, float& umax) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.nreal / 2) return;
  // the padding pairs at the end of a spectral row hold no mode (and whatever the buffer held
  // before): they are neither solved nor seen by the range report
  const unsigned row = a.fd_row.div((unsigned)(2 * c));
  if ((int)(2 * c - (long long)row * a.row_reals) >= a.row_valid) return;
  const int k = (int)blockIdx.y;
  const int km = (k == 0) ? 0 : a.nz - k;
  S* base = reinterpret_cast<S*>(a.data) + 2 * c;
  S* zk = base + (long long)k * a.plane;
  S* zm = base + (long long)km * a.plane;
  const df lz = df{a.zeig[k].x, a.zeig[k].y};
  const df ia = zf_inv(df{a.lam[2 * c].x, a.lam[2 * c].y}, lz);
  const df ib = zf_inv(df{a.lam[2 * c + 1].x, a.lam[2 * c + 1].y}, lz);
  const df w = df{a.scale[0], a.scale[1]};
  const df p = df_half(ia + ib) * w, q = df_half(ia - ib) * w;
  const df kr = zf_ld(zk), ki = zf_ld(zk + 1), mr = zf_ld(zm), mi = zf_ld(zm + 1);
  track(dmax, kr.hi * w.hi); track(dmax, ki.hi * w.hi); track(dmax, mr.hi * w.hi); track(dmax, mi.hi * w.hi);
  // Z'_k = p Z_k + q conj Z_m,  Z'_m = p Z_m + q conj Z_k
  const df ok_r = p * kr + q * mr, ok_i = p * ki - q * mi;
  track(umax, ok_r.hi); track(umax, ok_i.hi);
  zf_st(zk, ok_r);
  zf_st(zk + 1, ok_i);
  if (km != k) {
    const df om_r = p * mr + q * kr, om_i = p * mi - q * ki;
    track(umax, om_r.hi); track(umax, om_i.hi);
    zf_st(zm, om_r);
    zf_st(zm + 1, om_i);
  }
}

template <class S>
__global__ void __launch_bounds__(256) k_zdiag(const ZDiagArgs a) {
  float dmax = 0.0f, umax = 0.0f;
  zdiag_pair<S>(a, dmax, umax);
  range_report(a.rstat, a.dmin, a.umax, gridDim.x * gridDim.y, dmax, umax);
}

cudaError_t launch_zdiag_impl(const ZDiagArgs& a, bool df_spill, cudaStream_t st) {
  const dim3 grid((unsigned)((a.nreal / 2 + 255) / 256), (unsigned)(a.nz / 2 + 1));
  if (df_spill) k_zdiag<float2><<<grid, 256, 0, st>>>(a);
  else k_zdiag<float><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace pp
