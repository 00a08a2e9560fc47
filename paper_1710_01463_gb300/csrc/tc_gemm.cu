// Tensor-core GEMM for the mixed-precision products of Alg. RSVD (Sec. II.B):
//   C[M x N] (FP32, row-major, ldc) = A[M x K] * B[N x K]^T
// with A and B both K-major (row-major with K contiguous), BF16 operands
// (tcgen05.mma kind::f16) or FP32 operands read as TF32 (kind::tf32), FP32
// accumulation in tensor memory.
//
// One CTA computes one 128 x N tile (N = the sample width l rounded up to a
// multiple of 16, at most 256, so A is streamed exactly once per product).
// Warp 0 issues the TMA loads (128-byte swizzle) of A and B slices of 128
// bytes along K into an S-stage shared-memory ring, warp 1 allocates the
// accumulator in TMEM and issues the MMAs from one elected thread, releasing
// each stage with tcgen05.commit; warps 2-5 read the accumulator back with
// tcgen05.ld (one TMEM lane quarter each) and store it.  Every wait on an
// mbarrier is bounded; on a timeout the kernel records an error flag and
// finishes without further work.  No TMA multicast.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "tcgen05.cuh"

namespace rsvd {

namespace {

constexpr int kTcThreads = 192;
constexpr int kTcM = 128;

using namespace tc;

template <typename TIn>
__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(const __grid_constant__ TcBatch b, int stages,
                                                                int skip_loads) {
  const TcJob& J = b.job[blockIdx.y];
  const int m0 = blockIdx.x * kTcM;
  if (m0 >= J.M) return;  // whole CTA, before any barrier or TMEM use
  constexpr int BK = TcKind<TIn>::BK;
  constexpr int MMA_K = TcKind<TIn>::MMA_K;
  const int N = J.Npad;
  const uint32_t a_bytes = kTcM * 128;
  const uint32_t b_bytes = (uint32_t)N * 128;
  const uint32_t stage_bytes = (a_bytes + b_bytes + 1023) / 1024 * 1024;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) / 1024 * 1024);
  uint64_t* full = (uint64_t*)(smem + (size_t)stages * stage_bytes);
  uint64_t* empty = full + stages;
  uint64_t* done = empty + stages;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  __shared__ int err;
  __shared__ int keep_tmem;  // an in-flight copy or MMA could not be drained: leave TMEM allocated

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  uint32_t ncols = 32;
  while ((int)ncols < N) ncols <<= 1;

  if (threadIdx.x == 0) {
    err = 0;
    keep_tmem = 0;
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int nk = (J.K + BK - 1) / BK;

  if (warp == 0 && lane == 0 && !skip_loads) {
    // producer
    int issued = 0;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % stages;
      if (kt >= stages && !mbar_wait(&empty[s], ((kt / stages) & 1) ^ 1)) {
        atomicExch(&err, 1);
        break;
      }
      if (err) break;
      uint8_t* sa = smem + (size_t)s * stage_bytes;
      mbar_expect_tx(&full[s], a_bytes + b_bytes);
      tma_load_2d(sa, &J.ta, &full[s], kt * BK, m0);
      tma_load_2d(sa + a_bytes, &J.tb, &full[s], kt * BK, 0);
      issued = kt + 1;
    }
    // no load may still be writing shared memory when the CTA leaves: wait (bounded) for
    // the last load of every stage (already complete on the normal path)
    for (int kt = max(0, issued - stages); kt < issued; ++kt)
      if (!mbar_wait(&full[kt % stages], (kt / stages) & 1)) {
        atomicExch(&err, 1);
        keep_tmem = 1;
      }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t id = idesc<TIn>(kTcM, N);
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % stages;
      if (!mbar_wait(&full[s], (kt / stages) & 1)) {
        atomicExch(&err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(smem + (size_t)s * stage_bytes);
      const uint32_t sb = sa + a_bytes;
#pragma unroll
      for (int kk = 0; kk < BK / MMA_K; ++kk) {
        const uint32_t off = kk * MMA_K * (uint32_t)sizeof(TIn);  // 32 bytes per MMA step
        mma<TIn>(tmem, smem_desc(sa + off), smem_desc(sb + off), id, (kt | kk) != 0 ? 1u : 0u);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);
    // every MMA issued has completed before TMEM is released (bounded wait)
    if (!mbar_wait(done, 0)) {
      atomicExch(&err, 1);
      keep_tmem = 1;
    }
  } else if (warp >= 2) {
    // epilogue: TMEM lane quarter (warp % 4) holds rows 32 (warp % 4) .. + 31
    const int q = warp % 4;
    const bool ok = mbar_wait(done, 0);
    if (!ok) atomicExch(&err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + q * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
    const int cend = J.fold > 0 ? J.fold : N;
    for (int c0 = 0; c0 < cend; c0 += 16) {
      float v[16];
      ld16(tl + (uint32_t)c0, v);
      if (J.fold > 0) {  // hi and lo parts of the B operand: add the two halves
        float w[16];
        ld16(tl + (uint32_t)(J.fold + c0), w);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] += w[i];
      }
      if (ok && row < J.M) {
        float* dst = J.C + (size_t)row * J.ldc + c0;
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (c0 + i < J.N) dst[i] = v[i];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1 && !keep_tmem) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
  if (threadIdx.x == 0 && err && J.err) atomicExch(J.err, 1);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

}  // namespace

size_t tc_smem_bytes(int Npad, int stages) {
  const size_t stage = ((size_t)kTcM * 128 + (size_t)Npad * 128 + 1023) / 1024 * 1024;
  return 1024 + stage * stages + (2 * (size_t)stages + 1) * 8 + 16;
}

int tc_stages(int Npad) {
  int s = 8;
  while (s > 2 && tc_smem_bytes(Npad, s) > 200 * 1024) --s;
  return s;
}

// Tensor map of a row-major rows x cols matrix (cols contiguous) with a box of
// box_rows x (128 bytes of cols); 128-byte swizzle, zero fill out of bounds.
bool make_tmap(CUtensorMap* map, const void* base, int rows, int cols, int ld, int elem_bytes, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  if (((uintptr_t)base) % 16 || ((size_t)ld * elem_bytes) % 16) return false;
  const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)ld * elem_bytes};
  cuuint32_t box[2] = {(cuuint32_t)(128 / elem_bytes), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <typename TIn>
cudaError_t launch_tc_gemm(const TcBatch& b, cudaStream_t s, int skip_loads) {
  if (b.count <= 0) return cudaSuccess;
  int maxM = 1, maxN = 16;
  for (int i = 0; i < b.count; ++i) {
    maxM = max(maxM, b.job[i].M);
    maxN = max(maxN, b.job[i].Npad);
  }
  const int stages = tc_stages(maxN);
  const size_t smem = tc_smem_bytes(maxN, stages);
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<TIn>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  prof_begin(KC_TCGEMM, s);
  tc_gemm_kernel<TIn><<<dim3(ceil_div(maxM, kTcM), b.count), kTcThreads, smem, s>>>(b, stages, skip_loads);
  prof_end(KC_TCGEMM, s);
  return cudaGetLastError();
}

template cudaError_t launch_tc_gemm<__nv_bfloat16>(const TcBatch&, cudaStream_t, int);
template cudaError_t launch_tc_gemm<float>(const TcBatch&, cudaStream_t, int);

}  // namespace rsvd

extern "C" int rsvd_gemm_tc(int M, int N, int K, int prec, const void* A, int lda, const void* B, int ldb, float* C,
                            int ldc, int* err, int test_flags, void* cuda_stream) {
  using namespace rsvd;
  if (prec != RSVD_BF16 && prec != RSVD_TF32) return RSVD_ERR_PRECISION;
  if (M < 1 || N < 1 || N > 256 || K < 1 || lda < K || ldb < K || ldc < N) return RSVD_ERR_INVALID_SIZE;
  if (!A || !B || !C) return RSVD_ERR_NULL_POINTER;
  const int eb = prec == RSVD_BF16 ? 2 : 4;
  TcBatch b;
  b.count = 1;
  TcJob& J = b.job[0];
  J.Npad = (N + 15) / 16 * 16;
  if (!make_tmap(&J.ta, A, M, K, lda, eb, 128) || !make_tmap(&J.tb, B, N, K, ldb, eb, J.Npad))
    return RSVD_ERR_INVALID_SIZE;
  J.C = C;
  J.err = err;
  J.fold = 0;
  J.M = M;
  J.N = N;
  J.K = K;
  J.ldc = ldc;
  if (test_flags & ~1) return RSVD_ERR_INVALID_SIZE;
  const int skip = test_flags & 1;
  cudaError_t e = prec == RSVD_BF16 ? launch_tc_gemm<__nv_bfloat16>(b, (cudaStream_t)cuda_stream, skip)
                                    : launch_tc_gemm<float>(b, (cudaStream_t)cuda_stream, skip);
  if (e != cudaSuccess) {
    last_cuda_error() = e;
    return RSVD_ERR_LAUNCH;
  }
  return RSVD_OK;
}
