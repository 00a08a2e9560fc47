// Layout and precision changes around the tensor-core products: both operands
// of tcgen05.mma are read K-major, so the tall-skinny samples (rows x l, FP32)
// are handed to it transposed (l x rows) in the operand precision, A^T is
// materialised once per call, and B^T (n x l, FP32) comes back as B (l x n,
// FP64) for the Jacobi SVD.  32 x 32 tiles through shared memory keep both the
// reads and the writes coalesced.
#include <cuda_bf16.h>

#include "common.cuh"

namespace rsvd {

namespace {

template <typename Tin, typename Tout>
__device__ __forceinline__ Tout cvt(Tin v) {
  return (Tout)v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<float, __nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, __nv_bfloat16>(__nv_bfloat16 v) {
  return v;
}

// out[c, r] = in[r, c] for r < rows, c < cols
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) transpose_kernel(const __grid_constant__ XposeBatch b) {
  const XposeJob& J = b.job[blockIdx.z];
  if (J.active && !*J.active) return;  // an inactive job (whole CTA / cluster, before any barrier)
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  if (r0 >= J.rows || c0 >= J.cols) return;
  __shared__ Tin tile[32][33];
  const Tin* in = (const Tin*)J.in;
  Tout* out = (Tout*)J.out;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + tx;
    if (r < J.rows && c < J.cols) tile[i][tx] = in[(size_t)r * J.ldin + c];
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + tx;
    if (r < J.rows && c < J.cols) out[(size_t)c * J.ldout + r] = cvt<Tin, Tout>(tile[tx][i]);
  }
}

// the high part of x in the operand precision, and the low part x - hi
__device__ __forceinline__ void split(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}
__device__ __forceinline__ void split(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);  // the 10 explicit mantissa bits TF32 keeps
  lo = x - hi;
}

// out[c, r] = hi(in[r, c]), out[fold + c, r] = lo(in[r, c])
template <typename Tout>
__global__ void __launch_bounds__(256) split_transpose_kernel(const __grid_constant__ XposeBatch b) {
  const XposeJob& J = b.job[blockIdx.z];
  if (J.active && !*J.active) return;  // an inactive job (whole CTA / cluster, before any barrier)
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  if (r0 >= J.rows || c0 >= J.cols) return;
  __shared__ float tile[32][33];
  const float* in = (const float*)J.in;
  Tout* out = (Tout*)J.out;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + tx;
    if (r < J.rows && c < J.cols) tile[i][tx] = in[(size_t)r * J.ldin + c];
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + tx;
    if (r < J.rows && c < J.cols) {
      Tout hi, lo;
      split(tile[tx][i], hi, lo);
      out[(size_t)c * J.ldout + r] = hi;
      out[(size_t)(J.fold + c) * J.ldout + r] = lo;
    }
  }
}

}  // namespace

template <typename Tout>
cudaError_t launch_split_transpose(const XposeBatch& b, int, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  int mr = 1, mc = 1;
  for (int i = 0; i < b.count; ++i) {
    mr = max(mr, b.job[i].rows);
    mc = max(mc, b.job[i].cols);
  }
  prof_begin(KC_CONVERT, s);
  split_transpose_kernel<Tout><<<dim3(ceil_div(mc, 32), ceil_div(mr, 32), b.count), 256, 0, s>>>(b);
  prof_end(KC_CONVERT, s);
  return cudaGetLastError();
}
template cudaError_t launch_split_transpose<__nv_bfloat16>(const XposeBatch&, int, cudaStream_t);
template cudaError_t launch_split_transpose<float>(const XposeBatch&, int, cudaStream_t);

template <typename Tin, typename Tout>
cudaError_t launch_transpose(const XposeBatch& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  int mr = 1, mc = 1;
  for (int i = 0; i < b.count; ++i) {
    mr = max(mr, b.job[i].rows);
    mc = max(mc, b.job[i].cols);
  }
  prof_begin(KC_CONVERT, s);
  transpose_kernel<Tin, Tout><<<dim3(ceil_div(mc, 32), ceil_div(mr, 32), b.count), 256, 0, s>>>(b);
  prof_end(KC_CONVERT, s);
  return cudaGetLastError();
}

template cudaError_t launch_transpose<__nv_bfloat16, __nv_bfloat16>(const XposeBatch&, cudaStream_t);
template cudaError_t launch_transpose<float, float>(const XposeBatch&, cudaStream_t);
template cudaError_t launch_transpose<float, __nv_bfloat16>(const XposeBatch&, cudaStream_t);
template cudaError_t launch_transpose<float, double>(const XposeBatch&, cudaStream_t);
template cudaError_t launch_transpose<double, double>(const XposeBatch&, cudaStream_t);
template cudaError_t launch_transpose<double, float>(const XposeBatch&, cudaStream_t);

}  // namespace rsvd
