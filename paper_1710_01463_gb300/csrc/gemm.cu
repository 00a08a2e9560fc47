// Batched tall-skinny GEMM C = op(A) op(X) for the products of Alg. RSVD
// (Sec. II.B): the sketch Y = A Omega, the power-iteration products A^T Q and
// A Z, the projection B = Q^T A, the change of basis Y R^-1 of CholeskyQR and
// the lift U = Q U~.
//
// SIMT kernel (FFMA for float, DFMA for double): on GB300 FP64 has no tensor
// core path, so the FP64 products are bound by the DFMA pipe.  Conflict-free
// shared reads and 16-wide coalesced stores through a stride-16 register-tile
// layout; register double-buffering of the next K slice overlaps the global
// loads with the FMAs.
#include <cstdio>
#include <map>
#include <mutex>

#include "common.cuh"

namespace rsvd {

namespace {

constexpr int NT = 256;  // threads per CTA (a 16 x 16 grid)

// BM x BN output tile, K slices of BK through shared memory (double
// buffered via registers), a TM x TN register tile per thread with a stride-16
// layout: BM / 16 x BN / 16 per thread, BK 16.
template <typename Tin, bool TA, int BM, int BK>
__device__ __forceinline__ void load_a(const Tin* __restrict__ A, int lda, int M, int K, int m0, int k0,
                                       Tin (&ra)[BM * BK / NT]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < BM * BK / NT; ++q) {
    const int idx = t + q * NT;
    int i, kk;
    if (!TA) {  // A is M x K: k fastest
      kk = idx % BK;
      i = idx / BK;
    } else {    // A is K x M: m fastest
      i = idx % BM;
      kk = idx / BM;
    }
    const int gi = m0 + i, gk = k0 + kk;
    Tin v = (Tin)0;
    if (gi < M && gk < K) v = TA ? A[(long long)gk * lda + gi] : A[(long long)gi * lda + gk];
    ra[q] = v;
  }
}

template <typename Tin, bool TA, int BM, int BK>
__device__ __forceinline__ void store_a(Tin (*As)[BM + 1], const Tin (&ra)[BM * BK / NT]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < BM * BK / NT; ++q) {
    const int idx = t + q * NT;
    int i, kk;
    if (!TA) {
      kk = idx % BK;
      i = idx / BK;
    } else {
      i = idx % BM;
      kk = idx / BM;
    }
    As[kk][i] = ra[q];
  }
}

template <typename Tin, bool TX, int BN, int BK>
__device__ __forceinline__ void load_x(const Tin* __restrict__ X, int ldx, int N, int K, int n0, int k0,
                                       Tin (&rx)[BN * BK / NT]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < BN * BK / NT; ++q) {
    const int idx = t + q * NT;
    int j, kk;
    if (!TX) {  // X is K x N: n fastest
      j = idx % BN;
      kk = idx / BN;
    } else {    // X is N x K: k fastest
      kk = idx % BK;
      j = idx / BK;
    }
    const int gj = n0 + j, gk = k0 + kk;
    Tin v = (Tin)0;
    if (gj < N && gk < K) v = TX ? X[(long long)gj * ldx + gk] : X[(long long)gk * ldx + gj];
    rx[q] = v;
  }
}

template <typename Tin, bool TX, int BN, int BK>
__device__ __forceinline__ void store_x(Tin (*Xs)[BN + 1], const Tin (&rx)[BN * BK / NT]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < BN * BK / NT; ++q) {
    const int idx = t + q * NT;
    int j, kk;
    if (!TX) {
      j = idx % BN;
      kk = idx / BN;
    } else {
      kk = idx % BK;
      j = idx / BK;
    }
    Xs[kk][j] = rx[q];
  }
}

template <typename Tin, typename Tout, bool TA, bool TX, int BM, int BN, int BK>
__global__ void __launch_bounds__(NT) gemm_kernel(const __grid_constant__ GemmBatch<Tin, Tout> b) {
  constexpr int TM = BM / 16, TN = BN / 16;
  const GemmJob<Tin, Tout>& J = b.job[blockIdx.z];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (m0 >= J.M || n0 >= J.N) return;
  if (J.gate && *J.gate != J.gate_val) return;
  if (J.active && !*J.active) return;
  if ((J.m_eff && m0 >= *J.m_eff) || (J.n_eff && n0 >= *J.n_eff)) {  // a tile of exact zeros
    if (!J.accumulate)
      for (int e = threadIdx.x; e < BM * BN; e += NT) {
        const int gi = m0 + e / BN, gj = n0 + e % BN;
        if (gi < J.M && gj < J.N) J.C[(long long)gi * J.ldc + gj] = (Tout)0;
      }
    return;
  }

  __shared__ Tin As[2][BK][BM + 1];
  __shared__ Tin Xs[2][BK][BN + 1];

  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  Tin acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = (Tin)0;

  Tin ra[BM * BK / NT], rx[BN * BK / NT];
  const int K = J.k_eff ? min(J.K, *J.k_eff) : J.K;
  load_a<Tin, TA, BM, BK>(J.A, J.lda, J.M, K, m0, 0, ra);
  load_x<Tin, TX, BN, BK>(J.X, J.ldx, J.N, K, n0, 0, rx);
  store_a<Tin, TA, BM, BK>(As[0], ra);
  store_x<Tin, TX, BN, BK>(Xs[0], rx);
  __syncthreads();

  const int nk = (K + BK - 1) / BK;
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < nk) {
      load_a<Tin, TA, BM, BK>(J.A, J.lda, J.M, K, m0, (kt + 1) * BK, ra);
      load_x<Tin, TX, BN, BK>(J.X, J.ldx, J.N, K, n0, (kt + 1) * BK, rx);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Tin av[TM], xv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) av[i] = As[cur][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) xv[j] = Xs[cur][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], xv[j], acc[i][j]);
    }
    if (kt + 1 < nk) {
      store_a<Tin, TA, BM, BK>(As[cur ^ 1], ra);
      store_x<Tin, TX, BN, BK>(Xs[cur ^ 1], rx);
    }
    __syncthreads();
  }

  double scale = 1.0;
  if (J.div) scale = 1.0 / *J.div;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gi = m0 + ty + 16 * i;
    if (gi >= J.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gj = n0 + tx + 16 * j;
      if (gj < J.N) {
        Tout v = J.div ? (Tout)((double)acc[i][j] * scale) : (Tout)acc[i][j];
        if (J.alpha != 1.0) v = (Tout)(J.alpha * (double)v);
        Tout* c = J.C + (long long)gi * J.ldc + gj;
        *c = J.accumulate ? (Tout)(*c + v) : v;
      }
    }
  }
}

// FP32 products with a 128 x 128 output tile per CTA and an 8 x 8 register tile per thread
// (rows ty * 4 + {0..3} and 64 + ty * 4 + {0..3}, columns likewise with tx), so that a
// thread reads its eight values of A and of X for one k as two 128-bit shared loads each:
// four shared loads per 64 FFMA (the stride-16 tiles above issue one scalar load per two
// FFMA and are bound by the shared-memory pipe for FP32).  K slices of 16 through shared
// memory, double-buffered via registers.
constexpr int kVM = 128, kVN = 128, kVK = 16, kVPad = 4;

template <bool TA, bool TX>
__global__ void __launch_bounds__(NT, 2) gemm_v_kernel(const __grid_constant__ GemmBatch<float, float> b) {
  const GemmJob<float, float>& J = b.job[blockIdx.z];
  const int m0 = blockIdx.y * kVM, n0 = blockIdx.x * kVN;
  if (m0 >= J.M || n0 >= J.N) return;
  if (J.gate && *J.gate != J.gate_val) return;
  if (J.active && !*J.active) return;
  if ((J.m_eff && m0 >= *J.m_eff) || (J.n_eff && n0 >= *J.n_eff)) {  // a tile of exact zeros
    if (!J.accumulate)
      for (int e = threadIdx.x; e < kVM * kVN; e += NT) {
        const int gi = m0 + e / kVN, gj = n0 + e % kVN;
        if (gi < J.M && gj < J.N) J.C[(long long)gi * J.ldc + gj] = 0.0f;
      }
    return;
  }
  __shared__ __align__(16) float As[2][kVK][kVM + kVPad];
  __shared__ __align__(16) float Xs[2][kVK][kVN + kVPad];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  float ra[kVM * kVK / NT], rx[kVN * kVK / NT];
  const int K = J.k_eff ? min(J.K, *J.k_eff) : J.K;
  load_a<float, TA, kVM, kVK>(J.A, J.lda, J.M, K, m0, 0, ra);
  load_x<float, TX, kVN, kVK>(J.X, J.ldx, J.N, K, n0, 0, rx);
  // the element orders of load_a / load_x (idx = t + q * NT)
  auto put = [&](int buf) {
#pragma unroll
    for (int q = 0; q < kVM * kVK / NT; ++q) {
      const int idx = threadIdx.x + q * NT;
      const int i = TA ? idx % kVM : idx / kVK, kk = TA ? idx / kVM : idx % kVK;
      As[buf][kk][i] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < kVN * kVK / NT; ++q) {
      const int idx = threadIdx.x + q * NT;
      const int j = TX ? idx / kVK : idx % kVN, kk = TX ? idx % kVK : idx / kVN;
      Xs[buf][kk][j] = rx[q];
    }
  };
  put(0);
  __syncthreads();
  const int nk = (K + kVK - 1) / kVK;
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < nk) {
      load_a<float, TA, kVM, kVK>(J.A, J.lda, J.M, K, m0, (kt + 1) * kVK, ra);
      load_x<float, TX, kVN, kVK>(J.X, J.ldx, J.N, K, n0, (kt + 1) * kVK, rx);
    }
#pragma unroll
    for (int kk = 0; kk < kVK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + ty * 4]);
      const float4 x0 = *reinterpret_cast<const float4*>(&Xs[cur][kk][tx * 4]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Xs[cur][kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], xv[j], acc[i][j]);
    }
    if (kt + 1 < nk) put(cur ^ 1);
    __syncthreads();
  }
  double scale = 1.0;
  if (J.div) scale = 1.0 / *J.div;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gi = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (gi >= J.M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gj = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
      if (gj < J.N) {
        float v = J.div ? (float)((double)acc[i][j] * scale) : acc[i][j];
        if (J.alpha != 1.0) v = (float)(J.alpha * (double)v);
        float* c = J.C + (long long)gi * J.ldc + gj;
        *c = J.accumulate ? *c + v : v;
      }
    }
  }
}

}  // namespace

template <typename Tin, typename Tout, bool TA, bool TX, int BM, int BN>
cudaError_t launch_tile(const GemmBatch<Tin, Tout>& b, cudaStream_t s) {
  int tm = 1, tn = 1;
  for (int i = 0; i < b.count; ++i) {
    tm = max(tm, ceil_div(b.job[i].M, BM));
    tn = max(tn, ceil_div(b.job[i].N, BN));
  }
  prof_begin(KC_GEMM, s);
  gemm_kernel<Tin, Tout, TA, TX, BM, BN, 16><<<dim3(tn, tm, b.count), NT, 0, s>>>(b);
  prof_end(KC_GEMM, s);
  return cudaGetLastError();
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 1;
  }
  return n;
}

template <bool TA, bool TX>
cudaError_t launch_v_tile(const GemmBatch<float, float>& b, cudaStream_t s) {
  int tm = 1, tn = 1;
  for (int i = 0; i < b.count; ++i) {
    tm = max(tm, ceil_div(b.job[i].M, kVM));
    tn = max(tn, ceil_div(b.job[i].N, kVN));
  }
  prof_begin(KC_GEMM, s);
  gemm_v_kernel<TA, TX><<<dim3(tn, tm, b.count), NT, 0, s>>>(b);
  prof_end(KC_GEMM, s);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- autotuner
// Host cache of measured tile choices, keyed by the launch's shape class: operand and
// output types, transposes, batch size and the largest M, N, K of the batch (rounded up
// to multiples of 16).  With tuning enabled (rsvd_autotune_enable), a launch whose class
// is not cached yet - on a stream that is not being captured, with no job accumulating
// into or overwriting an operand - runs every candidate tile twice under CUDA events
// (synchronising the host), caches the fastest and then runs it; cached choices are used
// whether tuning is enabled or not (also inside a graph capture).  The cache is the
// library's only host state besides the side streams; it can be written to and read
// from a text file.
struct TuneKey {
  int tin, tout, ta, tx, count, M, N, K;
  bool operator<(const TuneKey& o) const {
    const int a[8] = {tin, tout, ta, tx, count, M, N, K}, b[8] = {o.tin, o.tout, o.ta, o.tx, o.count, o.M, o.N, o.K};
    for (int i = 0; i < 8; ++i)
      if (a[i] != b[i]) return a[i] < b[i];
    return false;
  }
};
struct Tuner {
  std::mutex mu;
  std::map<TuneKey, int> best;
  bool on = false;
  long long tuned = 0;  // launches timed so far
};
Tuner& tuner() {
  static Tuner t;
  return t;
}

template <typename Tin, typename Tout, bool TA, bool TX>
cudaError_t launch_choice(const GemmBatch<Tin, Tout>& b, int c, cudaStream_t s) {
  switch (c) {
    case 1: return launch_tile<Tin, Tout, TA, TX, 64, 48>(b, s);
    case 2: return launch_tile<Tin, Tout, TA, TX, 48, 64>(b, s);
    case 3:
      if constexpr (sizeof(Tin) == 8) return launch_tile<Tin, Tout, TA, TX, 48, 32>(b, s);
      if constexpr (sizeof(Tin) == 4 && sizeof(Tout) == 4) return launch_v_tile<TA, TX>(b, s);
      break;
    case 4: if constexpr (sizeof(Tin) == 8) return launch_tile<Tin, Tout, TA, TX, 32, 48>(b, s); break;
    case 5: if constexpr (sizeof(Tin) == 8) return launch_tile<Tin, Tout, TA, TX, 32, 32>(b, s); break;
    default: break;
  }
  return launch_tile<Tin, Tout, TA, TX, 64, 64>(b, s);
}

// Tile shape per launch.  The FMA loop of every shape keeps the SM's FP64 pipe
// busy, so an FP64 launch takes about as long as its most loaded SM:
// ceil(tiles / SMs) x tile area.  Small batches of narrow products (the sample
// widths l are not multiples of 64) waste most of that on idle SMs with 64-wide
// tiles, so FP64 launches also consider 32-row and 32-column tiles.  FP32
// tiles of 32 would be bound by shared-memory loads (FFMA issues 64 times
// faster than DFMA); FP32 picks the shape with the fewest padded outputs.
template <typename Tin, typename Tout, bool TA, bool TX>
cudaError_t launch_gemm(const GemmBatch<Tin, Tout>& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  constexpr bool f64 = sizeof(Tin) == 8;
  constexpr bool v32 = sizeof(Tin) == 4 && sizeof(Tout) == 4;  // the 128 x 128 FP32 tile is choice 3
  constexpr int ns = f64 ? 6 : (v32 ? 4 : 3);
  const int bm[6] = {64, 64, 48, f64 ? 48 : 128, 32, 32}, bn[6] = {64, 48, 64, f64 ? 32 : 128, 48, 32};
  long long cost[6];
  const long long sms = sm_count();
  int kmax = 0;
  for (int i = 0; i < b.count; ++i) kmax = max(kmax, b.job[i].K);
  for (int t = 0; t < ns; ++t) {
    long long tiles = 0, padded = 0;
    for (int i = 0; i < b.count; ++i) {
      const long long tm = ceil_div(b.job[i].M, bm[t]), tn = ceil_div(b.job[i].N, bn[t]);
      tiles += tm * tn;
      padded += tm * bm[t] * tn * bn[t];
    }
    cost[t] = f64 ? (tiles + sms - 1) / sms * bm[t] * bn[t] : padded;
    if (!f64 && t == 3) {
      // about 2.5x the FFMA rate of the stride-16 tiles per output, once the GPU holds two
      // such CTAs per SM and the K loop is long enough to amortise the tile's set-up
      const double fill = std::max(1.0, (double)(2 * sms) / (double)std::max(tiles, 1LL));
      cost[t] = kmax >= 256 ? (long long)(0.4 * fill * (double)padded) : (1LL << 62);
    }
  }
  int best = 0;
  for (int t = 1; t < ns; ++t)
    if (cost[t] < cost[best]) best = t;
  // measured choice of this shape class, when cached (or tuned now)
  TuneKey key{(int)sizeof(Tin), (int)sizeof(Tout), TA ? 1 : 0, TX ? 1 : 0, b.count, 0, 0, 0};
  bool safe = true;
  for (int i = 0; i < b.count; ++i) {
    key.M = max(key.M, (b.job[i].M + 15) / 16 * 16);
    key.N = max(key.N, (b.job[i].N + 15) / 16 * 16);
    key.K = max(key.K, (b.job[i].K + 15) / 16 * 16);
    const void* C = b.job[i].C;
    if (b.job[i].accumulate || C == (const void*)b.job[i].A || C == (const void*)b.job[i].X) safe = false;
  }
  Tuner& T = tuner();
  bool tune = false;
  {
    std::lock_guard<std::mutex> lock(T.mu);
    auto it = T.best.find(key);
    if (it != T.best.end()) return launch_choice<Tin, Tout, TA, TX>(b, it->second, s);
    tune = T.on && safe;
  }
  if (tune) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) tune = false;
  }
  if (tune) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
      float tbest = 1e30f;
      int cbest = best;
      bool ok = true;
      for (int t = 0; t < ns && ok; ++t) {
        float tt = 0.f;
        for (int rep = 0; rep < 2 && ok; ++rep) {  // the first run warms the caches
          ok = cudaEventRecord(e0, s) == cudaSuccess && launch_choice<Tin, Tout, TA, TX>(b, t, s) == cudaSuccess &&
               cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
               cudaEventElapsedTime(&tt, e0, e1) == cudaSuccess;
        }
        if (ok && tt < tbest) {
          tbest = tt;
          cbest = t;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (ok) {
        std::lock_guard<std::mutex> lock(T.mu);
        T.best[key] = cbest;
        T.tuned += 1;
        best = cbest;
      }
    }
  }
  return launch_choice<Tin, Tout, TA, TX>(b, best, s);
}

#define INST(Tin, Tout)                                                                           \
  template cudaError_t launch_gemm<Tin, Tout, false, false>(const GemmBatch<Tin, Tout>&, cudaStream_t); \
  template cudaError_t launch_gemm<Tin, Tout, true, false>(const GemmBatch<Tin, Tout>&, cudaStream_t);  \
  template cudaError_t launch_gemm<Tin, Tout, false, true>(const GemmBatch<Tin, Tout>&, cudaStream_t);
INST(double, double)
INST(float, float)
INST(float, double)
#undef INST

}  // namespace rsvd

// ---------------------------------------------------------------- autotuner entry points
extern "C" int rsvd_autotune_enable(int on) {
  rsvd::Tuner& T = rsvd::tuner();
  std::lock_guard<std::mutex> lock(T.mu);
  T.on = on != 0;
  return RSVD_OK;
}

extern "C" int rsvd_autotune_entries(void) {
  rsvd::Tuner& T = rsvd::tuner();
  std::lock_guard<std::mutex> lock(T.mu);
  return (int)T.best.size();
}

extern "C" int rsvd_autotune_clear(void) {
  rsvd::Tuner& T = rsvd::tuner();
  std::lock_guard<std::mutex> lock(T.mu);
  T.best.clear();
  return RSVD_OK;
}

extern "C" int rsvd_autotune_save(const char* path) {
  if (!path) return RSVD_ERR_NULL_POINTER;
  rsvd::Tuner& T = rsvd::tuner();
  std::lock_guard<std::mutex> lock(T.mu);
  FILE* f = std::fopen(path, "w");
  if (!f) return RSVD_ERR_INVALID_SIZE;
  std::fprintf(f, "# librsvd gemm tiles: tin tout ta tx count M N K choice\n");
  for (const auto& kv : T.best) {
    const rsvd::TuneKey& k = kv.first;
    std::fprintf(f, "%d %d %d %d %d %d %d %d %d\n", k.tin, k.tout, k.ta, k.tx, k.count, k.M, k.N, k.K, kv.second);
  }
  std::fclose(f);
  return RSVD_OK;
}

extern "C" int rsvd_autotune_load(const char* path) {
  if (!path) return RSVD_ERR_NULL_POINTER;
  FILE* f = std::fopen(path, "r");
  if (!f) return RSVD_ERR_INVALID_SIZE;
  rsvd::Tuner& T = rsvd::tuner();
  std::lock_guard<std::mutex> lock(T.mu);
  char line[256];
  int n = 0;
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    rsvd::TuneKey k;
    int c = 0;
    if (std::sscanf(line, "%d %d %d %d %d %d %d %d %d", &k.tin, &k.tout, &k.ta, &k.tx, &k.count, &k.M, &k.N, &k.K,
                    &c) == 9 &&
        c >= 0 && c < 6 && (c < 3 || k.tin == 8 || (c == 3 && k.tout == 4))) {
      T.best[k] = c;
      ++n;
    }
  }
  std::fclose(f);
  return n;
}
