// Alg. RSVD step 1 (Sec. II.B): the Gaussian test matrix Omega.
//
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by (seed, stream),
// counter (e / 4, 0, 0, 0) for element e = c*n + r of the n x l matrix; the
// four 64-bit words of a block give four normals by the Box-Muller transform
// (words 0,1 -> cos, sin; words 2,3 -> cos, sin).  One thread per Philox
// block; stores are scattered by row (Omega is row-major n x l) but Omega is
// tiny next to A (n*l elements against m*n).
#include <cuda_bf16.h>

#include "common.cuh"

namespace rsvd {

namespace {

// Philox4x64 multipliers and Weyl key increments (SC'11).
constexpr unsigned long long kM0 = 0xD2E7470EE14C6C93ull;
constexpr unsigned long long kM1 = 0xCA5A826395121157ull;
constexpr unsigned long long kW0 = 0x9E3779B97F4A7C15ull;
constexpr unsigned long long kW1 = 0xBB67AE8584CAA73Bull;

__device__ __forceinline__ void philox4x64_10(unsigned long long x[4], unsigned long long k0,
                                              unsigned long long k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kW0;
      k1 += kW1;
    }
    const unsigned long long lo0 = kM0 * x[0];
    const unsigned long long hi0 = __umul64hi(kM0, x[0]);
    const unsigned long long lo1 = kM1 * x[2];
    const unsigned long long hi1 = __umul64hi(kM1, x[2]);
    const unsigned long long y0 = hi1 ^ x[1] ^ k0;
    const unsigned long long y2 = hi0 ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = lo1;
    x[2] = y2;
    x[3] = lo0;
  }
}

__device__ __forceinline__ double open_unit(unsigned long long w) {
  return ((double)(w >> 11) + 0.5) * 0x1.0p-53;
}

template <typename T>
__device__ __forceinline__ void omega_block(const OmegaJob<T>& J, long long blk, long long total) {
  unsigned long long x[4] = {(unsigned long long)blk, 0ull, 0ull, 0ull};
  philox4x64_10(x, J.seed, J.stream);
  double z[4];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const double ua = open_unit(x[2 * p]);
    const double ub = open_unit(x[2 * p + 1]);
    const double rad = sqrt(-2.0 * log(ua));
    double sn, cs;
    sincospi(2.0 * ub, &sn, &cs);
    z[2 * p] = rad * cs;
    z[2 * p + 1] = rad * sn;
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const long long e = 4 * blk + s;
    if (e < total) {
      const long long c = e / J.n;
      const long long r = e - c * J.n;
      if (J.transposed)
        J.out[c * J.ld + r] = (T)z[s];
      else
        J.out[r * J.ld + c] = (T)z[s];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) omega_kernel(const __grid_constant__ OmegaBatch<T> b) {
  const OmegaJob<T>& J = b.job[blockIdx.y];
  if (J.active && !*J.active) return;  // an inactive job (whole CTA / cluster, before any barrier)
  const long long total = (long long)J.n * J.l;
  const long long nblk = (total + 3) / 4;
  for (long long blk = (long long)blockIdx.x * blockDim.x + threadIdx.x; blk < nblk;
       blk += (long long)gridDim.x * blockDim.x)
    omega_block(J, blk, total);
}

}  // namespace

template <typename T>
cudaError_t launch_omega(const OmegaBatch<T>& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  long long maxblk = 0;
  for (int i = 0; i < b.count; ++i) {
    long long nb = ((long long)b.job[i].n * b.job[i].l + 3) / 4;
    if (nb > maxblk) maxblk = nb;
  }
  int gx = (int)((maxblk + 255) / 256);
  if (gx < 1) gx = 1;
  if (gx > 1024) gx = 1024;
  prof_begin(KC_OMEGA, s);
  omega_kernel<T><<<dim3(gx, b.count), 256, 0, s>>>(b);
  prof_end(KC_OMEGA, s);
  return cudaGetLastError();
}

cudaError_t launch_omega_f64_single(int n, int l, int ld, double* out, unsigned long long seed,
                                    unsigned long long stream, cudaStream_t s) {
  OmegaBatch<double> b;
  b.count = 1;
  b.job[0] = OmegaJob<double>{n, l, ld, out, seed, stream, 0};
  return launch_omega<double>(b, s);
}

template cudaError_t launch_omega<double>(const OmegaBatch<double>&, cudaStream_t);
template cudaError_t launch_omega<float>(const OmegaBatch<float>&, cudaStream_t);
template cudaError_t launch_omega<__nv_bfloat16>(const OmegaBatch<__nv_bfloat16>&, cudaStream_t);

}  // namespace rsvd
