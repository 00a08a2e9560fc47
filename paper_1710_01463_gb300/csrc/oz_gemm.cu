// FP64 products C = P S on the tcgen05 tensor cores, for the products with A
// of Alg. RSVD (Sec. II.B) - the sketch A Omega, the power-iteration products
// A^T Q and A Z, and the projection (as B^T = A^T Q) - when K <= 1024.
//
// Exact slicing (an error-free splitting of each FP64 row into small
// integers, in the spirit of Ozaki's scheme): a row r of P with largest
// magnitude below 2^e_r is written as |x| = 2^(e_r - 54) n with a 54-bit
// integer n = floor(|x| 2^(54 - e_r)) read off the FP64 bit pattern, and n is
// cut into nine 6-bit pieces, x = 2^e_r sum_{i=1..9} p_i 2^-6i exactly (only
// the bits of x below 2^(e_r - 54) are dropped; integer operations only).
// Each p_i in [-63, 63] is exact in BF16.  With the columns of S sliced the
// same way (q_j, exponents f_c):
//
//   C[r][c] = 2^(e_r + f_c) sum_L 2^-6L T_L[r][c],   T_L = sum_{i+j=L} P_i S_j^T
//
// Every product p_i q_j is an integer below 2^12; over a chunk of at most 256
// values of K, |T_L| <= 9 * 256 * 63^2 < 2^24, so the tcgen05 BF16 MMA
// accumulates each level of a chunk exactly in FP32 in tensor memory, and the
// chunks are added in FP64.  Levels L = 2 .. 11 are kept (53 slice products).
// Error per entry, with 2^e_r <= 2 max|P_r| and 2^f_c <= 2 max|S_c|: the bits
// cut off by the slicing add at most 2 K 2^-53 max|P_r| max|S_c|, the dropped
// levels L >= 12 at most 0.25 K 2^-53 max|P_r| max|S_c| - the normwise class
// of an FP64 GEMM (K 2^-53 |P_r| |S_c|).  The ten level sums are combined in
// FP64 in the epilogue.
//
// One CTA computes a 128 x ntile tile (ntile <= 48).  Slice i of P (all of K,
// at most 64 KB) stays in shared memory, double-buffered, while every slice j
// of S that it pairs with streams through a ring of stages; each product goes
// to the TMEM accumulator of its level (ten levels x ntile <= 480 columns).
// Level L receives its last product with i = L - 1 (L <= 10) or i = 9, so the
// epilogue warps read level L back and add it in FP64 while the MMAs of later
// slices run.  A longer K runs chunk after chunk of 256 through the same
// accumulators: the first product of level L in the next chunk waits until
// the epilogue has read level L of this one (levels 2 .. 9 are read while the
// chunk still runs, so only levels 10 and 11 hold the next chunk up).  Warp 0
// issues the TMA loads, warp 1 (one elected thread) the MMAs, warps 2-5 the
// epilogue.  Every mbarrier wait is bounded; on a timeout the kernel records
// an error and finishes without further work.
#include "common.cuh"
#include "tcgen05.cuh"

namespace rsvd {

namespace {

using namespace tc;

constexpr int kOzThreads = 192;
constexpr int kOzM = 128;
constexpr int kOzBK = 64;     // BF16 elements of K per stage (128 bytes)
constexpr int kOzMmaK = 16;   // K per MMA
constexpr int kOzMaxNt = 48;  // columns per CTA (ten level accumulators fit 512 TMEM columns)
constexpr int kOzMaxKt = kOzMaxK / 64;    // K tiles of one P slice chunk
constexpr int kOzLevels = kOzSlices + 1;  // levels L = 2 .. 11

// ---------------------------------------------------------------- slicing
// One warp per row of the slice block: the row's exponent from the largest
// magnitude (integer maximum of the bit patterns), then the nine slices of
// every entry.  Rows of a block past `rows` and entries past K are zero; a
// row holding Inf or NaN gets NaN slices, so that the product is NaN there.
__global__ void __launch_bounds__(256) oz_split_kernel(const __grid_constant__ OzSplitBatch b) {
  const OzSplitJob& J = b.job[blockIdx.y];
  if (J.active && !*J.active) return;  // an inactive job (whole CTA / cluster, before any barrier)
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int r = blockIdx.x * (blockDim.x / 32) + warp;
  if (r >= J.rows_blk) return;
  const size_t blk = (size_t)J.rows_blk * J.Kp;
  __nv_bfloat16* S = J.S + (size_t)r * J.Kp;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  if (r >= J.rows) {
    for (int k = lane; k < J.Kp; k += 32)
#pragma unroll
      for (int i = 0; i < kOzSlices; ++i) S[i * blk + k] = zero;
    if (lane == 0) J.e[r] = 0;
    return;
  }
  auto at = [&](int k) { return J.xt ? J.X[(size_t)k * J.ldx + r] : J.X[(size_t)r * J.ldx + k]; };
  long long mx = 0;
  for (int k = lane; k < J.K; k += 32) mx = max(mx, __double_as_longlong(at(k)) & 0x7fffffffffffffffLL);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int emax = (int)((mx >> 52) & 0x7ff);
  const bool nonfinite = emax == 0x7ff;
  const int e = mx == 0 ? 0 : max(emax, 1) - 1022;  // every |x| of the row is below 2^e
  if (lane == 0) J.e[r] = nonfinite ? 0 : e;
  const __nv_bfloat16 nan = __float2bfloat16_rn(__int_as_float(0x7fc00000));
  for (int k = lane; k < J.Kp; k += 32) {
    long long n = 0;
    bool neg = false;
    if (k < J.K && mx != 0 && !nonfinite) {
      const long long bits = __double_as_longlong(at(k));
      neg = bits < 0;
      const int E = (int)((bits >> 52) & 0x7ff);
      const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | (E ? (1LL << 52) : 0LL);
      const int sh = max(E, 1) - 1021 - e;  // n = floor(|x| 2^(54 - e)) = mant 2^sh, sh <= 1
      n = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0LL);
    }
#pragma unroll
    for (int i = 0; i < kOzSlices; ++i) {
      const int p = (int)((n >> (48 - 6 * i)) & 63);
      S[i * blk + k] = nonfinite ? nan : __float2bfloat16_rn((float)(neg ? -p : p));
    }
  }
}

// ---------------------------------------------------------------- product
// Per K tile of 64 (128 bytes of every slice row): all nine slice tiles of S (ntile
// rows each) are loaded once and stay in shared memory (two buffers, alternating
// between K tiles), while the nine slice tiles of P (128 rows) stream through a ring;
// P tile i meets S tiles j = 1 .. 11 - i (at most 9), four MMAs of K = 16 each, into the
// TMEM accumulator of level i + j.  Every tile is loaded once per CTA.
constexpr int kOzPStages = 4;  // P tiles in flight

__global__ void __launch_bounds__(kOzThreads, 1) oz_gemm_kernel(const __grid_constant__ OzBatch b) {
  const OzJob& J = b.job[blockIdx.z];
  if (J.active && !*J.active) return;  // an inactive job (whole CTA / cluster, before any barrier)
  const int NT = b.ntile;
  const int m0 = blockIdx.x * kOzM, n0 = blockIdx.y * NT;
  if (m0 >= J.M || n0 >= J.N) return;  // whole CTA, before any barrier or TMEM use
  if (J.n_eff && n0 >= *J.n_eff) {     // a tile of exact zeros
    for (int e = threadIdx.x; e < kOzM * NT; e += kOzThreads) {
      const int r = m0 + e / NT, c = n0 + e % NT;
      if (r < J.M && c < J.N) J.C[J.trans_c ? (size_t)c * J.ldc + r : (size_t)r * J.ldc + c] = 0.0;
    }
    return;
  }
  const int nkt = (J.K + kOzBK - 1) / kOzBK;        // K tiles in all
  const int nc = (nkt + kOzMaxKt - 1) / kOzMaxKt;   // chunks of at most kOzMaxKt tiles (exact level sums)
  constexpr uint32_t kTileA = kOzM * 128;           // one K tile of a P slice: 128 rows x 128 bytes
  const uint32_t s_bytes = (uint32_t)NT * 128;
  const uint32_t s_tile = (s_bytes + 1023) / 1024 * 1024;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) / 1024 * 1024);
  uint8_t* pbuf = smem;                                          // [kOzPStages] P tiles
  uint8_t* sbuf = smem + (size_t)kOzPStages * kTileA;            // [2][kOzSlices] S tiles
  uint64_t* pfull = (uint64_t*)(sbuf + (size_t)2 * kOzSlices * s_tile);
  uint64_t* pempty = pfull + kOzPStages;
  uint64_t* sfull = pempty + kOzPStages;  // [2]
  uint64_t* sempty = sfull + 2;           // [2]
  uint64_t* cdone = sempty + 2;           // the chunk's MMAs are complete
  uint64_t* lread = cdone + 1;            // the epilogue has read the chunk's levels
  uint64_t* mdone = lread + 1;            // every MMA issued has completed
  uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
  __shared__ int err;
  __shared__ int keep_tmem;  // an in-flight copy or MMA could not be drained: leave TMEM allocated

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  constexpr uint32_t ncols = 512;

  if (threadIdx.x == 0) {
    err = 0;
    keep_tmem = 0;
    for (int t = 0; t < kOzPStages; ++t) {
      mbar_init(&pfull[t], 1);
      mbar_init(&pempty[t], 1);
    }
    for (int t = 0; t < 2; ++t) {
      mbar_init(&sfull[t], 1);
      mbar_init(&sempty[t], 1);
    }
    mbar_init(cdone, 1);
    mbar_init(lread, 4);  // one arrival per epilogue warp
    mbar_init(mdone, 1);
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
  volatile int* errv = &err;
  // slices are numbered 1 .. kOzSlices; products (i, j) with i + j <= kOzSlices + 2 are kept
  auto jmax = [](int i) { return min(kOzSlices, kOzSlices + 2 - i); };

  if (warp == 0 && lane == 0) {
    // producer: per K tile the nine S tiles (into the buffer of the tile's parity), then
    // the nine P tiles through the ring
    int pstep = 0;
    int last_s[2] = {-1, -1};  // last use issued of each S buffer
    for (int kt = 0; kt < nkt && !*errv; ++kt) {
      const int sb = kt & 1, su = kt >> 1;
      if (su > 0 && !mbar_wait(&sempty[sb], (su - 1) & 1)) {
        atomicExch(&err, 1);
        break;
      }
      mbar_expect_tx(&sfull[sb], (uint32_t)kOzSlices * s_bytes);
      last_s[sb] = su;
      for (int j = 1; j <= kOzSlices; ++j)
        tma_load_2d(sbuf + ((size_t)sb * kOzSlices + j - 1) * s_tile, &J.ts, &sfull[sb], kt * kOzBK,
                    (j - 1) * J.Npad + n0);
      for (int i = 1; i <= kOzSlices && !*errv; ++i, ++pstep) {
        const int ps = pstep % kOzPStages;
        if (pstep >= kOzPStages && !mbar_wait(&pempty[ps], ((pstep / kOzPStages) & 1) ^ 1)) {
          atomicExch(&err, 1);
          break;
        }
        mbar_expect_tx(&pfull[ps], kTileA);
        tma_load_2d(pbuf + (size_t)ps * kTileA, &J.tp, &pfull[ps], kt * kOzBK, (i - 1) * J.M + m0);
      }
    }
    // no load may still be writing shared memory when the CTA leaves: wait (bounded) for
    // the last load of every buffer and stage (already complete on the normal path)
    bool drained = true;
    for (int sb = 0; sb < 2; ++sb)
      if (last_s[sb] >= 0) drained = mbar_wait(&sfull[sb], last_s[sb] & 1) && drained;
    for (int st = max(0, pstep - kOzPStages); st < pstep; ++st)
      drained = mbar_wait(&pfull[st % kOzPStages], (st / kOzPStages) & 1) && drained;
    if (!drained) {
      atomicExch(&err, 1);
      keep_tmem = 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: product (i, j) accumulates into the TMEM columns of level i + j; the
    // first product of a level in a chunk (i = max(1, L - 9), first K tile, first MMA)
    // overwrites it
    const uint32_t id = idesc<__nv_bfloat16>(kOzM, NT);
    int pstep = 0;
    for (int c = 0; c < nc && !*errv; ++c) {
      if (c > 0) {  // the epilogue has read the previous chunk's levels
        if (!mbar_wait(lread, (c - 1) & 1)) {
          atomicExch(&err, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      const int kt0 = c * kOzMaxKt, nk = min(kOzMaxKt, nkt - kt0);
      for (int t = 0; t < nk && !*errv; ++t) {
        const int kt = kt0 + t, sb = kt & 1;
        if (!mbar_wait(&sfull[sb], (kt >> 1) & 1)) {
          atomicExch(&err, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t s0 = smem_u32(sbuf + (size_t)sb * kOzSlices * s_tile);
        for (int i = 1; i <= kOzSlices; ++i, ++pstep) {
          const int ps = pstep % kOzPStages;
          if (!mbar_wait(&pfull[ps], (pstep / kOzPStages) & 1)) {
            atomicExch(&err, 1);
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t pa = smem_u32(pbuf + (size_t)ps * kTileA);
          for (int j = 1; j <= jmax(i); ++j) {
            const int L = i + j;
            const uint32_t td = tmem + (uint32_t)((L - 2) * NT);
            const bool first = t == 0 && i == max(1, L - kOzSlices);
            const uint32_t sa = s0 + (uint32_t)(j - 1) * s_tile;
#pragma unroll
            for (int kk = 0; kk < kOzBK / kOzMmaK; ++kk) {
              const uint32_t off = kk * kOzMmaK * 2;  // 32 bytes per MMA step
              mma<__nv_bfloat16>(td, smem_desc(pa + off), smem_desc(sa + off), id, (first && kk == 0) ? 0u : 1u);
            }
          }
          mma_commit(&pempty[ps]);
        }
        mma_commit(&sempty[sb]);
      }
      mma_commit(cdone);
    }
    // every MMA issued has completed before TMEM is released (bounded wait)
    mma_commit(mdone);
    if (!mbar_wait(mdone, 0)) {
      atomicExch(&err, 1);
      keep_tmem = 1;
    }
  } else if (warp >= 2) {
    // epilogue: TMEM lane quarter (warp % 4) holds rows 32 (warp % 4) .. + 31; after each
    // chunk the ten levels are read and added in FP64 with their weights 2^-6L
    const int q = warp % 4;
    const int row = m0 + q * 32 + lane;
    double acc[kOzMaxNt];
#pragma unroll
    for (int cc = 0; cc < kOzMaxNt; ++cc) acc[cc] = 0.0;
    bool ok = true;
    for (int c = 0; c < nc && ok; ++c) {
      // warp-uniform: the level reads and the arrival below are warp-collective
      if (!__all_sync(0xffffffffu, mbar_wait(cdone, c & 1) ? 1 : 0)) {
        ok = false;
        atomicExch(&err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int L = 2; L <= kOzSlices + 2; ++L) {
        const double w = __longlong_as_double((long long)(1023 - 6 * L) << 52);  // 2^-6L
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((L - 2) * NT);
#pragma unroll
        for (int c0 = 0; c0 < kOzMaxNt; c0 += 16)
          if (c0 < NT) {
            float t[16];
            ld16(tl + (uint32_t)c0, t);
#pragma unroll
            for (int u = 0; u < 16; ++u) acc[c0 + u] = fma((double)t[u], w, acc[c0 + u]);
          }
      }
      // the levels may now be overwritten by the next chunk
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(lread);
    }
    if (ok && !*errv && row < J.M) {
      const int er = J.ep[row];
#pragma unroll
      for (int cc = 0; cc < kOzMaxNt; ++cc) {
        const int col = n0 + cc;
        if (cc < NT && col < J.N) {
          const double x = ldexp(acc[cc], er + J.es[col]);
          J.C[J.trans_c ? (size_t)col * J.ldc + row : (size_t)row * J.ldc + col] = x;
        }
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

size_t oz_smem_bytes(int ntile) {
  const size_t s_tile = ((size_t)ntile * 128 + 1023) / 1024 * 1024;
  return 1024 + (size_t)kOzPStages * kOzM * 128 + 2 * (size_t)kOzSlices * s_tile +
         (2 * (size_t)kOzPStages + 4 + 3) * 8 + 16;
}

}  // namespace

// columns per CTA: the fewest tiles of at most kOzMaxNt columns, as even as multiples of 16 allow
int oz_ntile(int Npad) {
  const int nt = (Npad + kOzMaxNt - 1) / kOzMaxNt;
  return ((Npad + nt - 1) / nt + 15) / 16 * 16;
}

cudaError_t launch_oz_split(const OzSplitBatch& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  int mr = 1;
  for (int i = 0; i < b.count; ++i) mr = max(mr, b.job[i].rows_blk);
  prof_begin(KC_OZSPLIT, s);
  oz_split_kernel<<<dim3(ceil_div(mr, 8), b.count), 256, 0, s>>>(b);
  prof_end(KC_OZSPLIT, s);
  return cudaGetLastError();
}

cudaError_t launch_oz_gemm(const OzBatch& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  int maxM = 1, maxN = 1;
  for (int i = 0; i < b.count; ++i) {
    maxM = max(maxM, b.job[i].M);
    maxN = max(maxN, b.job[i].N);
  }
  const size_t smem = oz_smem_bytes(b.ntile);
  cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  prof_begin(KC_OZGEMM, s);
  oz_gemm_kernel<<<dim3(ceil_div(maxM, kOzM), ceil_div(maxN, b.ntile), b.count), kOzThreads, smem, s>>>(b);
  prof_end(KC_OZGEMM, s);
  return cudaGetLastError();
}

}  // namespace rsvd

// C = A B^T in FP64 through the sliced tensor-core product (the verification
// entry point declared in rsvd.h).
extern "C" size_t rsvd_gemm_f64_tc_workspace_size(int M, int N, int K) {
  using namespace rsvd;
  if (M < 1 || N < 1 || K < 1) return 0;
  const size_t Kp = (size_t)(K + 7) / 8 * 8, Npad = (size_t)(N + 15) / 16 * 16;
  const size_t sa = align_up((size_t)kOzSlices * M * Kp * 2), sb = align_up((size_t)kOzSlices * Npad * Kp * 2);
  return sa + sb + align_up((size_t)M * 4) + align_up(Npad * 4);
}

extern "C" int rsvd_gemm_f64_tc(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                                int ldc, void* work, size_t work_bytes, int* err, void* cuda_stream) {
  using namespace rsvd;
  if (M < 1 || N < 1 || N > 256 || K < 1 || K > kOzMaxKTotal || lda < K || ldb < K || ldc < N)
    return RSVD_ERR_INVALID_SIZE;
  if (!A || !B || !C || !work) return RSVD_ERR_NULL_POINTER;
  if (work_bytes < rsvd_gemm_f64_tc_workspace_size(M, N, K)) return RSVD_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int Kp = (K + 7) / 8 * 8, Npad = (N + 15) / 16 * 16;
  char* w = (char*)work;
  __nv_bfloat16* SA = (__nv_bfloat16*)w;
  w += align_up((size_t)kOzSlices * M * Kp * 2);
  __nv_bfloat16* SB = (__nv_bfloat16*)w;
  w += align_up((size_t)kOzSlices * Npad * Kp * 2);
  int* eA = (int*)w;
  w += align_up((size_t)M * 4);
  int* eB = (int*)w;
  OzSplitBatch sp;
  sp.count = 2;
  sp.job[0] = OzSplitJob{A, M, K, lda, 0, M, Kp, SA, eA};
  sp.job[1] = OzSplitJob{B, N, K, ldb, 0, Npad, Kp, SB, eB};
  cudaError_t e = launch_oz_split(sp, s);
  if (e != cudaSuccess) {
    last_cuda_error() = e;
    return RSVD_ERR_LAUNCH;
  }
  OzBatch b;
  b.count = 1;
  b.ntile = oz_ntile(Npad);
  OzJob& J = b.job[0];
  if (!make_tmap(&J.tp, SA, kOzSlices * M, Kp, Kp, 2, 128) || !make_tmap(&J.ts, SB, kOzSlices * Npad, Kp, Kp, 2, b.ntile))
    return RSVD_ERR_INVALID_SIZE;
  J.C = C;
  J.ep = eA;
  J.es = eB;
  J.n_eff = nullptr;
  J.err = err;
  J.M = M;
  J.N = N;
  J.Npad = Npad;
  J.K = K;
  J.ldc = ldc;
  J.trans_c = 0;
  e = launch_oz_gemm(b, s);
  if (e != cudaSuccess) {
    last_cuda_error() = e;
    return RSVD_ERR_LAUNCH;
  }
  return RSVD_OK;
}
