// Orthonormalisation of a sample Y (rows x l): Alg. RSVD steps 2-3 (Sec. II.B)
// re-orthonormalise after every product with A or A^T.
//
// Primary path: CholeskyQR2 (Yamamoto, Nakatsukasa, Yanagisawa, Fukaya 2015).
//   G = Y^T Y (FP64 accumulation, deterministic two-stage reduction),
//   G = R^T R (FP64 Cholesky, upper R with positive diagonal),
//   Q1 = Y R^-1, then once more on Q1.  Q R equals the unique thin QR with
//   R_ii > 0 in exact arithmetic.
// A pivot below 1e-14 of its diagonal entry (Y numerically rank deficient, or
// conditioned beyond what two CholeskyQR passes can repair) sets a per-matrix
// flag; the remaining CholeskyQR launches skip that matrix and a Householder QR
// (FP64, one CTA per matrix) orthonormalises the ORIGINAL sample instead,
// again with R_ii >= 0.  The fallback is counted in rsvd_info.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace rsvd {

namespace {

constexpr double kPivotTol = 1e-14;

// ---------------------------------------------------------------- prep
template <typename T>
__global__ void __launch_bounds__(256) prep_kernel(const __grid_constant__ PrepBatch<T> b) {
  const PrepJob<T>& J = b.job[blockIdx.y];
  if (J.active && !*J.active) return;  // an inactive job (whole CTA / cluster, before any barrier)
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    J.info->status = RSVD_OK;
    J.info->path = J.exact ? RSVD_PATH_EXACT : 0;
    J.info->chol_fallbacks = 0;
    J.info->jacobi_sweeps = 0;
    J.info->l = J.l;
    J.info->rotations = 0;
    J.info->qr_columns = 0;
    J.info->qr_kflop = 0;
    J.info->jacobi_pairs = 0;
    J.info->cg_iterations = 0;
    J.flag[0] = 0;
    J.flag[1] = 0;
    J.flag[2] = J.l;  // columns of Q that carry the sampled range
  }
  if (!J.exact) return;
  // Q = I (m x l, l = m) and B = A (l x n, FP64)
  const long long tq = (long long)J.m * J.l;
  const long long tb = (long long)J.l * J.n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tq + tb;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < tq) {
      const long long r = e / J.l, c = e - r * J.l;
      J.Y[e] = (T)(r == c ? 1 : 0);
    } else {
      const long long f = e - tq;
      const long long r = f / J.n, c = f - r * J.n;
      J.Bm[f] = (double)J.A[r * J.lda + c];
    }
  }
}

// ---------------------------------------------------------------- Gram
__device__ __forceinline__ void tilepair(int idx, int T, int& ti, int& tj) {
  ti = 0;
  while (idx >= T - ti) {
    idx -= T - ti;
    ++ti;
  }
  tj = ti + idx;
}

// A sample whose Q is kept to its effective columns (trunc_q) after an earlier
// Householder QR of the same matrix ended early has exact zero columns beyond
// them: its Gram matrix is singular and CholeskyQR2 would break down, so it
// goes to Householder QR directly
template <typename T>
__device__ __forceinline__ bool known_deficient(const OrthJob<T>& J) {
  return J.trunc_q && J.rank_eff && *J.rank_eff < J.l;
}

// partial G over one chunk of rows for one kGramTile x kGramTile tile (ti <= tj),
// one output per thread.  16-wide tiles: the FMA loop is FP64-bound at any
// tile size, so the small tile loses nothing and pads less (l = 80 computes
// 15 x 256 outputs instead of 6 x 1024; l = 138, 45 x 256 instead of 15 x 1024).
template <typename T>
__global__ void __launch_bounds__(256) gram_kernel(const __grid_constant__ OrthBatch<T> b, int gated, int src1) {
  static_assert(kGramTile == 16, "one output per thread of a 16 x 16 tile");
  const OrthJob<T>& J = b.job[blockIdx.z];
  if (J.active && !*J.active) return;  // an inactive job (whole CTA / cluster, before any barrier)
  if (J.hh_first || (gated && *J.flag != 0) || known_deficient(J)) return;
  const int l = J.l;
  const int nt = (l + kGramTile - 1) / kGramTile;
  if ((int)blockIdx.x >= nt * (nt + 1) / 2) return;
  const int nchunk = (J.rows + kGramChunk - 1) / kGramChunk;
  const int c = blockIdx.y;
  if (c >= nchunk) return;
  int ti, tj;
  tilepair(blockIdx.x, nt, ti, tj);
  const T* Y = src1 ? J.Y1 : J.Y;

  constexpr int kRows = 32;  // rows of Y staged per step
  __shared__ double Si[kRows][kGramTile + 1], Sj[kRows][kGramTile + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc = 0.0;
  const int r_begin = c * kGramChunk;
  const int r_end = min(J.rows, r_begin + kGramChunk);
  for (int r0 = r_begin; r0 < r_end; r0 += kRows) {
    for (int e = threadIdx.x; e < kRows * kGramTile; e += 256) {
      const int rr = e / kGramTile, cc = e % kGramTile;
      const int r = r0 + rr;
      const int ci = ti * kGramTile + cc, cj = tj * kGramTile + cc;
      Si[rr][cc] = (r < r_end && ci < l) ? (double)Y[(long long)r * l + ci] : 0.0;
      Sj[rr][cc] = (r < r_end && cj < l) ? (double)Y[(long long)r * l + cj] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < kRows; ++rr) acc = fma(Si[rr][ty], Sj[rr][tx], acc);
    __syncthreads();
  }
  const int i = ti * kGramTile + ty, j = tj * kGramTile + tx;
  if (i < l && j < l) J.part[((long long)c * l + i) * l + j] = acc;
}

template <typename T>
__global__ void __launch_bounds__(256) gram_reduce_kernel(const __grid_constant__ OrthBatch<T> b, int gated) {
  const OrthJob<T>& J = b.job[blockIdx.y];
  if (J.active && !*J.active) return;  // an inactive job (whole CTA / cluster, before any barrier)
  if (J.hh_first || (gated && *J.flag != 0) || known_deficient(J)) return;
  const int l = J.l;
  const int nchunk = (J.rows + kGramChunk - 1) / kGramChunk;
  const long long tot = (long long)l * l;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / l), j = (int)(e % l);
    if (i > j) continue;
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += J.part[((long long)c * l + i) * l + j];
    J.G[(long long)i * l + j] = s;
    J.G[(long long)j * l + i] = s;
  }
}

// ---------------------------------------------------------------- Cholesky + R^-1
// One CTA per matrix.  R (upper, R^T R = G) is built in shared memory when l is
// small enough, else in place in G.  Breakdown (a pivot that is not above
// kPivotTol times its original diagonal entry) sets the flag; the matrix then
// takes the Householder path.  Right-looking: per column j, one lane forms the
// pivot, the scaled row j is staged, and the trailing upper triangle is updated
// with rows spread over warps and columns over lanes (no index division).
// R^-1 then overwrites R column by column (X[0:j, j] = -X[0:j, 0:j] R[0:j, j] /
// R_jj), a team of four lanes per row, and is written out with zeros below
// the diagonal.
template <typename T>
__global__ void __launch_bounds__(512) cholinv_kernel(const __grid_constant__ OrthBatch<T> b, int pass, int use_smem) {
  const OrthJob<T>& J = b.job[blockIdx.x];
  if (J.active && !*J.active) return;  // an inactive job (whole CTA / cluster, before any barrier)
  if (pass == 0 && (J.hh_first || known_deficient(J))) {
    if (threadIdx.x == 0) *J.flag = 1;
    return;
  }
  if (pass == 1 && *J.flag != 0) return;
  extern __shared__ double sm[];
  const int l = J.l;
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32, nw = blockDim.x / 32;
  double* diag0 = sm;
  double* srow = sm + l;  // scaled row j of R
  double* R = use_smem ? sm + 2 * l : J.G;
  __shared__ int bad;
  __shared__ double inv_rjj;
  if (tid == 0) bad = 0;
  if (use_smem)
    for (int e = tid; e < l * l; e += blockDim.x) R[e] = J.G[e];
  for (int i = tid; i < l; i += blockDim.x) diag0[i] = J.G[(long long)i * l + i];
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    if (tid == 0) {
      // pivot test on bit patterns (d > tol diag0 >= +0; d itself may have gone
      // negative by cancellation, which the signed compare rejects), and one
      // reciprocal square root for both R_jj and its inverse
      const double d = R[j * l + j];
      if (!(__double_as_longlong(d) > __double_as_longlong(kPivotTol * diag0[j])) ||
          !(__double_as_longlong(diag0[j]) > 0)) {
        bad = 1;
      } else {
        const double ir = rsqrt(d);
        R[j * l + j] = d * ir;
        inv_rjj = ir;
        srow[j] = ir;  // kept for the inverse below (srow[c] for c > j is written later in this column)
      }
    }
    __syncthreads();
    if (bad) break;
    for (int c = j + 1 + tid; c < l; c += blockDim.x) srow[c] = R[j * l + c] * inv_rjj;
    __syncthreads();
    for (int c = j + 1 + tid; c < l; c += blockDim.x) R[j * l + c] = srow[c];
    for (int r = j + 1 + warp; r < l; r += nw) {
      const double sr = srow[r];
      for (int c = r + lane; c < l; c += 32) R[r * l + c] = fma(-sr, srow[c], R[r * l + c]);
    }
    __syncthreads();
  }
  if (pass == 0 && tid == 0) *J.flag = bad;  // every orthonormalisation starts afresh
  if (bad) {
    if (tid == 0) *J.flag = 1;
    return;
  }
  if (pass == 1 && J.rank_eff && tid == 0) *J.rank_eff = l;  // CholeskyQR2 succeeded: full column rank
  // X = R^-1 in place: column j needs X[0:j, 0:j] (done) and R[0:j, j] (still R);
  // the new column is staged in srow until every read of the old one is done
  constexpr int kTeam = 4;
  const int team = tid / kTeam, tl = tid % kTeam, nteam = blockDim.x / kTeam;
  for (int j = 0; j < l; ++j) {
    const double xjj = srow[j];  // 1 / R_jj from the factorization (srow[i], i < j, is reused below)
    for (int i0 = 0; i0 < j; i0 += nteam) {  // team-uniform trip count: the shuffles see full teams
      const int i = i0 + team;
      double s = 0.0, s1 = 0.0;  // two chains per lane
      if (i < j) {
        int t = i + tl;
        for (; t + kTeam < j; t += 2 * kTeam) {
          s = fma(R[i * l + t], R[t * l + j], s);
          s1 = fma(R[i * l + t + kTeam], R[(t + kTeam) * l + j], s1);
        }
        if (t < j) s = fma(R[i * l + t], R[t * l + j], s);
      }
      s += s1;
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (i < j && tl == 0) srow[i] = -s * xjj;
    }
    __syncthreads();  // every read of column j is done
    for (int i = tid; i < j; i += blockDim.x) R[i * l + j] = srow[i];
    if (tid == 0) R[j * l + j] = xjj;
    __syncthreads();
  }
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int i = e / l, jcol = e - i * l;
    J.Rinv[e] = (T)(i <= jcol ? R[e] : 0.0);
  }
}

// CTA size of cholinv_kernel: small factors synchronise fewer warps per column
inline int chol_threads(int l) { return l <= 64 ? 128 : (l <= 128 ? 256 : 512); }

// ---------------------------------------------------------------- Householder QR
// Householder QR of Y (rows x l) by one thread-block CLUSTER per matrix: the
// rows are split across the CTAs (FP64 slices in shared memory, or in global
// scratch when they do not fit).  For column j every CTA forms the partial
// ||x||^2 and x_0 of its rows, the cluster sums them through distributed
// shared memory (same rank order everywhere -> identical reflectors), each CTA
// scales its part of v_j, forms the partial products v_j^T Y[:, c] of its
// rows, and after a second exchange applies the reflector to its rows.  Q is
// then accumulated backwards, Q = H_0 ... H_{l-1} [I; 0], one exchange per
// reflector, and written back into Y with column signs making R_ii >= 0.
// Runs for matrices whose flag is set (CholeskyQR2 breakdown, or the
// Householder-first policy of nearly square samples).
constexpr int kHhThreads = 512;
constexpr int kHhTeam = 8;  // lanes per column in the partial products and their exchange

// Algorithmic work of a Householder QR of a rows x c sample stopped after r
// reflectors, with the explicit Q formed on qc columns (kflop, rounded): the
// standard counts sum_{j<r} 4 (rows - j)(x - j) for x = c and x = qc
__device__ __forceinline__ int hh_kflop(int rows, int c, int qc, int r) {
  auto f = [&](double x) {
    return 4.0 * rows * x * r - 2.0 * ((double)rows + x) * r * (double)r + 4.0 / 3.0 * r * (double)r * r;
  };
  return (int)((f(c) + f(qc)) * 1e-3 + 0.5);
}

struct HLayout {
  int rs;  // rows per CTA
};

__host__ __device__ inline size_t hh_small_doubles(int l) { return (size_t)l + 2 * (size_t)l + 2 * 2 + 2 + (size_t)l; }

template <typename T>
__global__ void __launch_bounds__(kHhThreads) householder_kernel(const __grid_constant__ OrthBatch<T> b, int csize,
                                                                  int use_global) {
  cg::cluster_group cluster = cg::this_cluster();
  const OrthJob<T>& J = b.job[blockIdx.y];
  if (J.active && !*J.active) return;  // an inactive job (whole CTA / cluster, before any barrier)
  if (!J.hh_first && *J.flag == 0) return;  // cluster-uniform: one matrix per cluster
  const int C = csize;
  const int rank = (int)cluster.block_rank();
  const int rows = J.rows, l = J.l;
  const int rs = (rows + C - 1) / C;
  const int r0 = rank * rs;
  const int nr = max(0, min(rows, r0 + rs) - r0);
  extern __shared__ double sm[];
  double* alpha = sm;            // l
  double* pd = alpha + l;        // [2][l] partial dot products
  double* pn = pd + 2 * l;       // [2][2] partial (||x||^2, x_0)
  double* sc = pn + 4;           // [2] reduced (||x||^2, x_0)
  double* dsum = sc + 2;         // l reduced dot products
  double* Ys;
  double* Qs;
  if (use_global) {
    Ys = J.hw + (size_t)rank * rs * l;
    Qs = J.hq + (size_t)rank * rs * l;
  } else {
    Ys = sm + hh_small_doubles(l);
    Qs = Ys + (size_t)rs * l;
  }
  const int tid = threadIdx.x;
  const int team = tid / kHhTeam, tl = tid % kHhTeam, nteam = kHhThreads / kHhTeam;
  const unsigned tmask = 0xffu << ((tid % 32) / kHhTeam * kHhTeam);
  for (int e = tid; e < nr * l; e += kHhThreads) Ys[e] = (double)J.Y[(size_t)r0 * l + e];
  __shared__ double red[kHhThreads / 32][2];
  __syncthreads();

  for (int j = 0; j < l; ++j) {
    // phase 1: partial ||x||^2 and x_0 over own rows r >= j
    double a = 0.0, x0 = 0.0;
    for (int rr = tid; rr < nr; rr += kHhThreads) {
      const int r = r0 + rr;
      if (r >= j) {
        const double v = Ys[rr * l + j];
        a = fma(v, v, a);
        if (r == j) x0 = v;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      x0 += __shfl_xor_sync(0xffffffffu, x0, o);
    }
    if (tid % 32 == 0) {
      red[tid / 32][0] = a;
      red[tid / 32][1] = x0;
    }
    __syncthreads();
    if (tid == 0) {
      double s0 = 0.0, s1 = 0.0;
      for (int w = 0; w < kHhThreads / 32; ++w) {
        s0 += red[w][0];
        s1 += red[w][1];
      }
      pn[(j & 1) * 2 + 0] = s0;
      pn[(j & 1) * 2 + 1] = s1;
    }
    cluster.sync();
    if (tid < 32) {
      double s0 = 0.0, s1 = 0.0;
      if (tid < C) {
        const double* rp = cluster.map_shared_rank(pn, tid);
        s0 = rp[(j & 1) * 2 + 0];
        s1 = rp[(j & 1) * 2 + 1];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      }
      if (tid == 0) {  // the reflector's scalars, once (FP64 sqrt / divide are costly on this part)
        const double nrm2 = s0, xj0 = s1;
        double al0 = 0.0, inv0 = 0.0;
        if (nrm2 > 0.0) {
          al0 = xj0 >= 0.0 ? -sqrt(nrm2) : sqrt(nrm2);
          const double v0 = xj0 - al0;
          const double vn2 = nrm2 - xj0 * xj0 + v0 * v0;
          inv0 = vn2 > 0.0 ? 1.0 / sqrt(vn2) : 0.0;
        }
        alpha[j] = al0;
        sc[0] = inv0;
        sc[1] = xj0;
      }
    }
    __syncthreads();
    const double xj = sc[1], al = alpha[j], inv = sc[0];
    for (int rr = tid; rr < nr; rr += kHhThreads) {
      const int r = r0 + rr;
      if (r >= j) Ys[rr * l + j] = (r == j ? (xj - al) : Ys[rr * l + j]) * inv;
    }
    __syncthreads();
    // phase 2: partial v^T Y[:, c] for c > j
    double* pdj = pd + (j & 1) * l;
    for (int c = j + 1 + team; c < l; c += nteam) {
      double d = 0.0;
      for (int rr = max(0, j - r0) + tl; rr < nr; rr += kHhTeam) d = fma(Ys[rr * l + j], Ys[rr * l + c], d);
#pragma unroll
      for (int o = kHhTeam / 2; o > 0; o >>= 1) d += __shfl_xor_sync(tmask, d, o, kHhTeam);
      if (tl == 0) pdj[c] = d;
    }
    cluster.sync();
    for (int c = j + 1 + team; c < l; c += nteam) {
      double d = 0.0;
      for (int r = tl; r < C; r += kHhTeam) d += cluster.map_shared_rank(pdj, r)[c];
#pragma unroll
      for (int o = kHhTeam / 2; o > 0; o >>= 1) d += __shfl_xor_sync(tmask, d, o, kHhTeam);
      if (tl == 0) dsum[c] = d;
    }
    __syncthreads();
    const int w = l - j - 1;
    for (int e = tid; e < nr * w; e += kHhThreads) {
      const int rr = e / w, c = j + 1 + e % w;
      if (r0 + rr >= j) Ys[rr * l + c] = fma(-2.0 * Ys[rr * l + j], dsum[c], Ys[rr * l + c]);
    }
    __syncthreads();
  }
  cluster.sync();  // every remote read of pd / pn is done before they are reused below
  for (int e = tid; e < nr * l; e += kHhThreads) {
    const int rr = e / l, c = e % l;
    Qs[e] = (r0 + rr == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = l - 1; j >= 0; --j) {
    double* pdj = pd + (j & 1) * l;
    for (int c = j + team; c < l; c += nteam) {
      double d = 0.0;
      for (int rr = max(0, j - r0) + tl; rr < nr; rr += kHhTeam) d = fma(Ys[rr * l + j], Qs[rr * l + c], d);
#pragma unroll
      for (int o = kHhTeam / 2; o > 0; o >>= 1) d += __shfl_xor_sync(tmask, d, o, kHhTeam);
      if (tl == 0) pdj[c] = d;
    }
    cluster.sync();
    for (int c = j + team; c < l; c += nteam) {
      double d = 0.0;
      for (int r = tl; r < C; r += kHhTeam) d += cluster.map_shared_rank(pdj, r)[c];
#pragma unroll
      for (int o = kHhTeam / 2; o > 0; o >>= 1) d += __shfl_xor_sync(tmask, d, o, kHhTeam);
      if (tl == 0) dsum[c] = d;
    }
    __syncthreads();
    const int w = l - j;
    for (int e = tid; e < nr * w; e += kHhThreads) {
      const int rr = e / w, c = j + e % w;
      if (r0 + rr >= j) Qs[rr * l + c] = fma(-2.0 * Ys[rr * l + j], dsum[c], Qs[rr * l + c]);
    }
    __syncthreads();
  }
  for (int e = tid; e < nr * l; e += kHhThreads) {
    const int c = e % l;
    const double sg = alpha[c] < 0.0 ? -1.0 : 1.0;
    J.Y[(size_t)r0 * l + e] = (T)(sg * Qs[e]);
  }
  if (rank == 0 && tid == 0) {
    if (!J.hh_first) atomicAdd(&J.info->chol_fallbacks, 1);
    atomicOr(&J.info->path, RSVD_PATH_HOUSEHOLDER);
    J.info->qr_columns = l;
    atomicAdd(&J.info->qr_kflop, hh_kflop(rows, l, l, l));
    if (J.trunc_q && J.rank_eff) *J.rank_eff = l;
  }
  cluster.sync();  // no CTA leaves while others may read its shared memory
}

// ---------------------------------------------------------------- blocked Householder QR
// Same factorization as householder_kernel, blocked by panels of kNb columns
// (compact WY form, H_j0 ... H_j1-1 = I - V T V^T): the cluster factors the
// panel together, each CTA on its own rows (two cluster barriers per column:
// one CTA factoring the panel alone was bound by its SM's FP64 issue, 82% of
// the kernel's cycles), then every CTA applies I - V T^T V^T to its rows of
// the trailing columns: partial products V^T Y per CTA, each CTA sums and
// transforms one slice of the columns, and the slices are exchanged.  Q is
// accumulated backwards panel by panel the same way.
constexpr int kNb = 16;
constexpr int kPanelMaxCluster = 8;  // the blocked kernel runs on portable cluster sizes
// shared memory of the blocked kernel: up to about 110 KB two CTAs share an SM;
// above, one CTA per SM, which still beats the column kernel by far
constexpr size_t kPanelSmemMax = 218 * 1024;  // with the kernel's 6 KB of static shared memory, within 227 KB

struct PanelLayout {
  size_t ys, vo, wp, ws, alpha, total;  // shared-memory offsets in doubles
};

constexpr int kProdStride = 33;  // per-lane products of the panel columns, padded against bank conflicts

// Shared memory: own rows of Y (then Q), own rows of the current panel's V,
// one V^T Y buffer (partials, then the sums and T^T W; it also holds the
// panel's per-lane products while the panel is factored) and the reflector
// scalars.  The V and T of all panels are kept in the matrix's global scratch
// (hw and hq, L2-resident) for the accumulation of Q: with only the current
// panel of V in shared memory and one V^T Y buffer, two CTAs of 384- and
// 512-row samples fit an SM.  A CTA holds at most 64 rows (two per lane of a
// column's warp).  The static shared memory is kept small: two CTAs of the
// 256-row TEBD samples share an SM.
__host__ __device__ inline PanelLayout panel_layout(int rows, int l, int csize) {
  const int rs = (rows + csize - 1) / csize;
  PanelLayout L;
  size_t o = 0;
  L.ys = o; o += (size_t)rs * l;
  L.vo = o; o += (size_t)rs * kNb;
  // the summed V^T Y (Ws) shares the partials' buffer (Wb): a CTA writes sums only
  // into its own column slice, which no other CTA reads as partials, and the gather
  // of the other slices follows the barrier after which no partial is read
  L.wp = o;
  L.ws = o;
  const size_t wbuf = (size_t)kNb * l, prod = (size_t)kNb * kProdStride;
  o += wbuf > prod ? wbuf : prod;
  L.alpha = o; o += (size_t)l;
  L.total = o;
  return L;
}

// sum over own rows rr0 .. nr-1 of a[rr * lda] * b[rr * ldb] (a column of the
// panel's V times a column of Y), four independent chains: a dependent FP64 FMA
// costs about 64 cycles on this part
__device__ __forceinline__ double dot_rows2(const double* a, int lda, const double* b, int ldb, int rr0, int nr) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int rr = rr0;
  for (; rr + 3 < nr; rr += 4) {
    s0 = fma(a[rr * lda], b[rr * ldb], s0);
    s1 = fma(a[(rr + 1) * lda], b[(rr + 1) * ldb], s1);
    s2 = fma(a[(rr + 2) * lda], b[(rr + 2) * ldb], s2);
    s3 = fma(a[(rr + 3) * lda], b[(rr + 3) * ldb], s3);
  }
  for (; rr < nr; ++rr) s0 = fma(a[rr * lda], b[rr * ldb], s0);
  return (s0 + s1) + (s2 + s3);
}

// sum over jj < nb of v[jj] * w[jj * ld] (a row of V times a column of M), two chains
__device__ __forceinline__ double dot_panel(const double* v, const double* w, int ld, int nb) {
  double s0 = 0.0, s1 = 0.0;
  int jj = 0;
  for (; jj + 1 < nb; jj += 2) {
    s0 = fma(v[jj], w[jj * ld], s0);
    s1 = fma(v[jj + 1], w[(jj + 1) * ld], s1);
  }
  if (jj < nb) s0 = fma(v[jj], w[jj * ld], s0);
  return s0 + s1;
}

// After every CTA of the cluster has written its partial V^T Y for columns
// c0 .. c0 + wcols - 1 into Wb (kNb x l rows), forms W = the sum of the
// partials and M = T^T W (kTW = false, trailing update) or M = T W (kTW =
// true, accumulation of Q), and leaves all of M in every CTA's Ws.  Each CTA
// sums and transforms its own slice of the columns only (no FP64 work is
// repeated across the cluster) and then gathers the other slices.  Called by
// every CTA of the cluster (it contains a cluster barrier).
// Sum of the C partials v[q * stride], q < C, by a fixed pairwise tree of exactly C - 1
// FP64 additions (every CTA of the cluster gets the same bits)
__device__ __forceinline__ double panel_tree_sum(const double* v, int stride, int C) {
  double p[kPanelMaxCluster];
#pragma unroll
  for (int q = 0; q < kPanelMaxCluster; ++q) p[q] = q < C ? v[q * stride] : 0.0;
  switch (C) {  // cluster-uniform
    case 1: return p[0];
    case 2: return p[0] + p[1];
    case 3: return (p[0] + p[1]) + p[2];
    case 4: return (p[0] + p[1]) + (p[2] + p[3]);
    case 5: return ((p[0] + p[1]) + (p[2] + p[3])) + p[4];
    case 6: return ((p[0] + p[1]) + (p[2] + p[3])) + (p[4] + p[5]);
    case 7: return ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + p[6]);
    default: return ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
  }
}

template <bool kTW>
__device__ void cluster_sum_apply_t(cg::cluster_group& cluster, int rank, int C, const double* Wb, double* Ws,
                                    const double (*Ts)[kNb], int nb, int l, int c0, int wcols) {
  const int tid = threadIdx.x;
  const int cw = (wcols + C - 1) / C;
  const int cb = c0 + rank * cw, w = max(0, min(c0 + wcols, cb + cw) - cb);
  for (int e = tid; e < nb * w; e += kHhThreads) {
    const int jj = e / w, c = cb + e % w;
    double pv[kPanelMaxCluster];  // every remote load in flight at once, summed by a fixed tree
#pragma unroll
    for (int r = 0; r < kPanelMaxCluster; ++r) pv[r] = r < C ? cluster.map_shared_rank(Wb, r)[jj * l + c] : 0.0;
    Ws[jj * l + c] = panel_tree_sum(pv, 1, C);
  }
  __syncthreads();
  double mreg[(kNb * 256 + kHhThreads - 1) / kHhThreads];
  int cnt = 0;
  for (int e = tid; e < nb * w; e += kHhThreads, ++cnt) {
    const int jj = e / w, c = cb + e % w;
    double m0 = 0.0, m1 = 0.0;  // two chains: a dependent FP64 FMA costs about 64 cycles
    if (kTW) {
      int ii = jj;
      for (; ii + 1 < nb; ii += 2) {
        m0 = fma(Ts[jj][ii], Ws[ii * l + c], m0);
        m1 = fma(Ts[jj][ii + 1], Ws[(ii + 1) * l + c], m1);
      }
      if (ii < nb) m0 = fma(Ts[jj][ii], Ws[ii * l + c], m0);
    } else {
      int ii = 0;
      for (; ii + 1 <= jj; ii += 2) {
        m0 = fma(Ts[ii][jj], Ws[ii * l + c], m0);
        m1 = fma(Ts[ii + 1][jj], Ws[(ii + 1) * l + c], m1);
      }
      if (ii <= jj) m0 = fma(Ts[ii][jj], Ws[ii * l + c], m0);
    }
    mreg[cnt] = m0 + m1;
  }
  __syncthreads();
  cnt = 0;
  for (int e = tid; e < nb * w; e += kHhThreads, ++cnt) {
    const int jj = e / w, c = cb + e % w;
    Ws[jj * l + c] = mreg[cnt];
  }
  cluster.sync();  // every slice of M is complete
  for (int e = tid; e < nb * wcols; e += kHhThreads) {
    const int jj = e / wcols, c = c0 + e % wcols;
    const int owner = (c - c0) / cw;
    if (owner != rank) Ws[jj * l + c] = cluster.map_shared_rank(Ws, owner)[jj * l + c];
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kHhThreads, 2) householder_panel_kernel(const __grid_constant__ OrthBatch<T> b, int csize) {
  cg::cluster_group cluster = cg::this_cluster();
  const OrthJob<T>& J = b.job[blockIdx.y];
  if (J.active && !*J.active) return;  // an inactive job (whole CTA / cluster, before any barrier)
  if (!J.hh_first && *J.flag == 0) return;  // cluster-uniform
  const int C = csize;
  const int rank = (int)cluster.block_rank();
  const int rows = J.rows, l = J.l;
  // rows are dealt to the CTAs cyclically - CTA q holds rows q, q + C, q + 2C, ... - so
  // that every CTA keeps its share of the rows below the diagonal as the factorization
  // moves down (with contiguous blocks the first CTAs ran out of work in the trailing
  // updates and the formation of Q while the last ones carried all of theirs)
  const int nr = rank < rows ? (rows - rank + C - 1) / C : 0;
  const PanelLayout L = panel_layout(rows, l, C);
  extern __shared__ double sm[];
  double* Ys = sm + L.ys;      // own rows of Y, later of Q   (rs x l)
  double* Vo = sm + L.vo;      // own rows of the current panel's V (rs x kNb)
  double* Vg = J.hw;           // V of every panel, all rows (rows x l, global scratch)
  double* Wp = sm + L.wp;      // partial V^T Y               (kNb x l)
  double* Ws = sm + L.ws;      // summed V^T Y, then T^T W (kNb x l; the same buffer as Wp)
  double* alpha = sm + L.alpha;
  double* Tall = J.hq;         // T of every panel, npanel x kNb x kNb (global scratch)
  __shared__ double red[kHhThreads / 32][2];
  __shared__ double fin[kNb];
  __shared__ double Ts[kNb][kNb];  // T of the current panel
  __shared__ double sc[2];
  __shared__ double spart[2][kPanelMaxCluster][kNb];  // the cluster's partial products x_jj^T x_c
  __shared__ double xrowp[2][kNb];                     // the diagonal row's entries of the panel columns
  __shared__ double vbuf[64];                      // v on the own rows (rs <= 64)
  __shared__ double Gv[kNb][kNb];                  // V^T V of the panel (strictly upper part)
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32, nw = kHhThreads / 32;

  for (int e = tid; e < nr * l; e += kHhThreads) Ys[e] = (double)J.Y[(size_t)(rank + C * (e / l)) * l + e % l];
  // every CTA must apply the same column signs: columns left unfactored by an
  // early end keep alpha = 0 (sign +1) everywhere
  for (int c = tid; c < l; c += kHhThreads) alpha[c] = 0.0;
  __syncthreads();
  __shared__ double trail_part;  // this CTA's sum of squares of the trailing block
  __shared__ double trail_sum;
  __shared__ double fro0;
  // Without U (trunc_q), the columns of the sample at and beyond the previous
  // orthonormalisation's rank are exact zeros (the products skip them): the
  // factorization runs over the leading lc columns only.
  const int lc = (J.trunc_q && J.rank_eff) ? min(l, max(kNb, *J.rank_eff)) : l;
  const int npanel = (lc + kNb - 1) / kNb;
  int npanel_used = npanel;
  for (int p = 0; p < npanel; ++p) {
    const int j0 = p * kNb, nb = min(kNb, lc - j0);
    const int R = rows - j0;  // panel rows j0 .. rows-1
    double* Tp = Tall + (size_t)p * kNb * kNb;
    {  // sum of squares of the trailing block Y[j0:, j0:] over own rows
      double a = 0.0;
      for (int e = tid; e < nr * (lc - j0); e += kHhThreads) {
        const int rr = e / (lc - j0), c = j0 + e % (lc - j0);
        if (rank + C * rr >= j0) a = fma(Ys[rr * l + c], Ys[rr * l + c], a);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) red[warp][0] = a;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int q = 0; q < nw; ++q) t += red[q][0];
        trail_part = t;
      }
    }
    cluster.sync();  // trailing updates of the previous panel are complete everywhere
    if (tid == 0) {  // every remote load in flight at once, summed by a fixed tree
      double pv[kPanelMaxCluster];
#pragma unroll
      for (int r = 0; r < kPanelMaxCluster; ++r) pv[r] = r < C ? *cluster.map_shared_rank(&trail_part, r) : 0.0;
#pragma unroll
      for (int w2 = 1; w2 < kPanelMaxCluster; w2 <<= 1)
#pragma unroll
        for (int r = 0; r + w2 < kPanelMaxCluster; r += 2 * w2) pv[r] += pv[r + w2];
      trail_sum = pv[0];
      if (p == 0) fro0 = pv[0];
    }
    __syncthreads();
    // early end: the rest of Y is rounding noise.  The trailing block of a
    // numerically rank-deficient sample settles near 2^-52 ||Y||_F (the
    // rounding of the products and of the reflections); below 2^-51 ||Y||_F it
    // is dropped, which moves no singular value by more than 2^-51 sqrt(l)
    // sigma_1 (< 1e-14 sigma_1 for l <= 256).  The remaining columns of Q are
    // completed by the reflectors applied so far.
    if (p > 0 && !(trail_sum > fro0 * 0x1.0p-102)) {
      npanel_used = p;
      break;  // identical decision in every CTA of the cluster
    }
    {
      // The panel is factored by the whole cluster: warp c holds panel column c of
      // this CTA's own rows (lane and lane + 32), so the FP64 work of the reflections
      // is spread over the cluster's SMs.  Per column jj ONE cluster barrier: every CTA
      // forms the partial products x_jj^T x_c of the column with all panel columns over
      // its rows at and below the diagonal (c = jj gives ||x_jj||^2) and the CTA holding
      // the diagonal row sends that row's entries; after the barrier every CTA sums the
      // partials in the same fixed order and forms alpha, the reflector's scale and
      // v^T x_c = (x_jj^T x_c - alpha x_c[d]) / ||x_jj - alpha e_d|| (d the diagonal
      // row) - the same quantities as the reflector applied first, without a second
      // exchange.  For c < jj (columns holding earlier reflectors) this is v_c^T v_jj,
      // for T.  The exchange slots alternate between two buffers: a slot is rewritten
      // two columns later, after a barrier that every reader of its value has passed.
      static_assert(kHhThreads / 32 == kNb, "one warp per panel column");
      const int c = warp;
      const int rA = lane, rB = lane + 32;
      const bool inA = rA < nr, inB = rB < nr;
      const int gA = rank + C * rA, gB = rank + C * rB;
      double xA = (inA && c < nb) ? Ys[rA * l + j0 + c] : 0.0;
      double xB = (inB && c < nb) ? Ys[rB * l + j0 + c] : 0.0;
      for (int jj = 0; jj < nb; ++jj) {
        const int gd = j0 + jj;  // the diagonal row of column jj
        const int buf = jj & 1;
        if (c == jj) {  // column jj at and below the diagonal, for every warp's products
          vbuf[rA] = (inA && gA >= gd) ? xA : 0.0;
          vbuf[rB] = (inB && gB >= gd) ? xB : 0.0;
        }
        if (gd % C == rank && gd / C < nr && c < nb) {  // this CTA holds the diagonal row
          const int rd = gd / C;
          const double xd = __shfl_sync(0xffffffffu, rd < 32 ? xA : xB, rd & 31);
          if (lane < C) *cluster.map_shared_rank(&xrowp[buf][c], lane) = xd;  // lane q pushes to CTA q
        }
        __syncthreads();
        const double wA = vbuf[rA], wB = vbuf[rB];
        // each warp leaves its lanes' products, and warps 0-3 sum them, four columns per
        // warp, eight lanes per column (four products each, then three shuffle levels):
        // six FP64 instructions per warp.  A warp issues at most one FP64 instruction per
        // 64 cycles whatever its active lanes and independent work, so the sums are
        // spread over four warps rather than done in one (about 20 instructions)
        double (*prod)[kProdStride] = (double (*)[kProdStride])Wp;  // the V^T Y buffer is idle here
        prod[c][lane] = c < nb ? fma(xA, wA, xB * wB) : 0.0;
        __syncthreads();
        if (warp < kNb / 4) {
          const int cc = 4 * warp + (lane >> 3), h = (lane & 7) * 4;
          double sp = (prod[cc][h] + prod[cc][h + 1]) + (prod[cc][h + 2] + prod[cc][h + 3]);
          sp += __shfl_xor_sync(0xffffffffu, sp, 4);
          sp += __shfl_xor_sync(0xffffffffu, sp, 2);
          sp += __shfl_xor_sync(0xffffffffu, sp, 1);
          for (int q = lane & 7; q < C; q += 8) *cluster.map_shared_rank(&spart[buf][rank][cc], q) = sp;
        }
        cluster.sync();
        // one warp, lane c: the sum of column c's partials (a fixed tree over the
        // cluster), the reflector's scalars (redundantly in every lane: an FP64 warp
        // instruction costs the same with one active lane or sixteen), v^T x_c.  Sign
        // tests on the bit patterns (an FP64 compare-and-branch costs hundreds of
        // cycles on this part), and ||x|| = a rsqrt(a)
        if (warp == 0 && lane < kNb) {
          const double dc = panel_tree_sum(&spart[buf][0][lane], kNb, C);
          const double a = __shfl_sync(0x0000ffffu, dc, jj);  // ||x_jj||^2 below the diagonal
          const double x0 = xrowp[buf][jj];
          double al = 0.0, inv = 0.0;
          if (__double_as_longlong(a) > 0) {
            const double nx = a * rsqrt(a);
            al = __double_as_longlong(x0) >= 0 ? -nx : nx;
            const double vn2 = 2.0 * fma(fabs(x0), nx, a);  // ||x - alpha e||^2 = 2 (a + |x0| ||x||)
            inv = __double_as_longlong(vn2) > 0 ? rsqrt(vn2) : 0.0;
          }
          const double vtx = fma(-al, xrowp[buf][lane], dc) * inv;  // v^T x_lane
          fin[lane] = -2.0 * vtx;
          if (lane < jj) Gv[lane][jj] = vtx;  // v_lane^T v_jj, for T
          if (lane == jj) {
            sc[0] = inv;
            sc[1] = (x0 - al) * inv;  // v at the diagonal row
            alpha[gd] = al;
          }
        }
        __syncthreads();  // fin and the scalars complete
        // the unit reflector v on the own rows (zero above the diagonal), formed only in the
        // warps of columns jj .. nb-1 (warp-uniform: the columns before jj hold earlier
        // reflectors, and every FP64 warp instruction costs the SM's FP64 issue)
        if (c >= jj && c < nb) {
          const double vA = !inA ? 0.0 : gA == gd ? sc[1] : gA > gd ? wA * sc[0] : 0.0;
          const double vB = !inB ? 0.0 : gB == gd ? sc[1] : gB > gd ? wB * sc[0] : 0.0;
          if (c > jj) {
            xA = fma(fin[c], vA, xA);
            xB = fma(fin[c], vB, xB);
          } else {
            xA = vA;
            xB = vB;
          }
        }
      }
      // T of the panel (H_0 ... H_nb-1 = I - V T V^T, unit reflectors, tau = 2) by the
      // UT transform: T^-1 = I / 2 + strictly upper (V^T V); lane c solves for
      // column c by back substitution, T[c][c] = 2, T[i][c] = -2 sum_{j=i+1..c}
      // (V^T V)[i][j] T[j][c]
      if (warp == 0 && lane < kNb) {  // column cc of T in registers (fully unrolled, predicated)
        const int cc = lane;
        double tc[kNb];
#pragma unroll
        for (int i = 0; i < kNb; ++i) tc[i] = i == cc ? 2.0 : 0.0;
#pragma unroll
        for (int i = kNb - 2; i >= 0; --i) {
          double t4[4] = {0.0, 0.0, 0.0, 0.0};  // four chains: a dependent FP64 FMA costs about 64 cycles
#pragma unroll
          for (int j = i + 1; j < kNb; ++j) t4[(j - i) & 3] = fma(j <= cc ? Gv[i][j] : 0.0, tc[j], t4[(j - i) & 3]);
          if (i < cc) tc[i] = -2.0 * ((t4[0] + t4[1]) + (t4[2] + t4[3]));
        }
#pragma unroll
        for (int i = 0; i < kNb; ++i) Ts[i][cc] = cc < nb ? tc[i] : 0.0;
      }
      // the reflectors into this CTA's rows of V; T to the global copy that the
      // accumulation of Q reads back
      if (c < nb) {
        if (inA) {
          Vo[rA * kNb + c] = xA;
          Vg[(size_t)gA * l + j0 + c] = xA;
        }
        if (inB) {
          Vo[rB * kNb + c] = xB;
          Vg[(size_t)gB * l + j0 + c] = xB;
        }
      }
      __syncthreads();
      if (rank == 0 && tid < kNb * kNb) Tp[tid] = Ts[tid / kNb][tid % kNb];
    }
    cluster.sync();  // panel factored: V in place everywhere
    __syncthreads();
    // trailing update of columns j0 + nb .. l-1: Y <- Y - V T^T (V^T Y); V is
    // zero on the rows above j0, which neither contribute nor change
    const int c1 = j0 + nb, wcols = lc - c1;
    const int rr0 = max(0, min(nr, (j0 - rank + C - 1) / C));  // first own row at or below j0
    double* Wb = Wp;
    if (wcols > 0) {
      for (int e = tid; e < nb * wcols; e += kHhThreads) {
        const int jj = e / wcols, c = c1 + e % wcols;
        Wb[jj * l + c] = dot_rows2(Vo + jj, kNb, Ys + c, l, rr0, nr);
      }
    }
    cluster.sync();
    if (wcols > 0) {
      cluster_sum_apply_t<false>(cluster, rank, C, Wb, Ws, Ts, nb, l, c1, wcols);
      for (int e = tid; e < (nr - rr0) * wcols; e += kHhThreads) {
        const int rr = rr0 + e / wcols, c = c1 + e % wcols;
        Ys[rr * l + c] -= dot_panel(Vo + rr * kNb, Ws + c, l, nb);
      }
    }
    __syncthreads();
  }
  // Q = (I - V_0 T_0 V_0^T) ... (I - V_last T_last V_last^T) [I; 0], accumulated backwards.
  // With trunc_q and an early end, only the leading qc columns (those that
  // carry the sample's range) are formed; the others are written as zeros.
  const int qc = J.trunc_q ? min(lc, npanel_used * kNb) : l;
  cluster.sync();  // every remote read of Ys / Wp above is done
  for (int e = tid; e < nr * l; e += kHhThreads) {
    const int rr = e / l, c = e % l;
    Ys[e] = (rank + C * rr == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int p = npanel_used - 1; p >= 0; --p) {
    const int j0 = p * kNb, nb = min(kNb, lc - j0);
    const double* Tp = Tall + (size_t)p * kNb * kNb;
    const int wcols = qc - j0;
    const int rr0 = max(0, min(nr, (j0 - rank + C - 1) / C));  // rows above j0: V is zero there
    double* Wb = Wp;
    cluster.sync();  // the previous panel's remote reads of Wp are done
    if (tid < kNb * kNb) Ts[tid / kNb][tid % kNb] = Tp[tid];
    for (int e = tid; e < nr * kNb; e += kHhThreads) {  // this panel's V, own rows
      const int rr = e / kNb, c = e % kNb;
      Vo[e] = c < nb ? Vg[(size_t)(rank + C * rr) * l + j0 + c] : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < nb * wcols; e += kHhThreads) {
      const int jj = e / wcols, c = j0 + e % wcols;
      Wb[jj * l + c] = dot_rows2(Vo + jj, kNb, Ys + c, l, rr0, nr);
    }
    cluster.sync();
    cluster_sum_apply_t<true>(cluster, rank, C, Wb, Ws, Ts, nb, l, j0, wcols);
    for (int e = tid; e < (nr - rr0) * wcols; e += kHhThreads) {
      const int rr = rr0 + e / wcols, c = j0 + e % wcols;
      Ys[rr * l + c] -= dot_panel(Vo + rr * kNb, Ws + c, l, nb);
    }
    __syncthreads();
  }
  for (int e = tid; e < nr * l; e += kHhThreads) {
    const int c = e % l;
    const double sg = alpha[c] < 0.0 ? -1.0 : 1.0;
    J.Y[(size_t)(rank + C * (e / l)) * l + c] = c < qc ? (T)(sg * Ys[e]) : (T)0;
  }
  if (rank == 0 && tid == 0) {
    if (!J.hh_first) atomicAdd(&J.info->chol_fallbacks, 1);
    atomicOr(&J.info->path, RSVD_PATH_HOUSEHOLDER);
    J.info->qr_columns = min(l, npanel_used * kNb);
    atomicAdd(&J.info->qr_kflop, hh_kflop(rows, lc, qc, min(lc, npanel_used * kNb)));
    if (J.trunc_q && J.rank_eff) *J.rank_eff = qc;
  }
  cluster.sync();  // no CTA leaves while others may read its shared memory
}

}  // namespace

template <typename T>
cudaError_t launch_prep(const PrepBatch<T>& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  long long mx = 1;
  for (int i = 0; i < b.count; ++i)
    if (b.job[i].exact) mx = max(mx, (long long)b.job[i].m * b.job[i].l + (long long)b.job[i].l * b.job[i].n);
  int gx = (int)min(1024LL, (mx + 255) / 256);
  prof_begin(KC_PREP, s);
  prep_kernel<T><<<dim3(gx, b.count), 256, 0, s>>>(b);
  prof_end(KC_PREP, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cholqr2(const OrthBatch<T>& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  int maxl = 1, maxchunk = 1, maxtp = 1;
  long long maxll = 1;
  for (int i = 0; i < b.count; ++i) {
    const int l = b.job[i].l;
    maxl = max(maxl, l);
    maxll = max(maxll, (long long)l * l);
    maxchunk = max(maxchunk, ceil_div(b.job[i].rows, kGramChunk));
    const int nt = ceil_div(l, kGramTile);
    maxtp = max(maxtp, nt * (nt + 1) / 2);
  }
  // shared-memory Cholesky when R fits (l <= 160)
  const size_t smem_full = (size_t)(2 * maxl + (size_t)maxl * maxl) * sizeof(double);
  const int use_smem = smem_full <= 210 * 1024 ? 1 : 0;
  const size_t smem = use_smem ? smem_full : (size_t)2 * maxl * sizeof(double);
  cudaError_t e;
  e = cudaFuncSetAttribute(cholinv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int rgx = (int)min(1024LL, (maxll + 255) / 256);

  // pass 1: Y -> Y1 = Y R1^-1
  prof_begin(KC_GRAM, s);
  gram_kernel<T><<<dim3(maxtp, maxchunk, b.count), 256, 0, s>>>(b, 0, 0);
  gram_reduce_kernel<T><<<dim3(rgx, b.count), 256, 0, s>>>(b, 0);
  prof_end(KC_GRAM, s);
  prof_begin(KC_CHOL, s);
  cholinv_kernel<T><<<b.count, chol_threads(maxl), smem, s>>>(b, 0, use_smem);
  prof_end(KC_CHOL, s);
  {
    GemmBatch<T, T> g;
    g.count = b.count;
    for (int i = 0; i < b.count; ++i) {
      const OrthJob<T>& J = b.job[i];
      g.job[i] = GemmJob<T, T>{J.rows, J.l, J.l, J.l, J.l, J.l, J.Y, J.Rinv, J.Y1, nullptr, J.flag, 0};
      g.job[i].active = J.active;
    }
    e = launch_gemm<T, T, false, false>(g, s);
    if (e != cudaSuccess) return e;
  }
  // pass 2: Y1 -> Y = Y1 R2^-1
  prof_begin(KC_GRAM, s);
  gram_kernel<T><<<dim3(maxtp, maxchunk, b.count), 256, 0, s>>>(b, 1, 1);
  gram_reduce_kernel<T><<<dim3(rgx, b.count), 256, 0, s>>>(b, 1);
  prof_end(KC_GRAM, s);
  prof_begin(KC_CHOL, s);
  cholinv_kernel<T><<<b.count, chol_threads(maxl), smem, s>>>(b, 1, use_smem);
  prof_end(KC_CHOL, s);
  {
    GemmBatch<T, T> g;
    g.count = b.count;
    for (int i = 0; i < b.count; ++i) {
      const OrthJob<T>& J = b.job[i];
      g.job[i] = GemmJob<T, T>{J.rows, J.l, J.l, J.l, J.l, J.l, J.Y1, J.Rinv, J.Y, nullptr, J.flag, 0};
      g.job[i].active = J.active;
    }
    e = launch_gemm<T, T, false, false>(g, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// Householder QR of the matrices of b that are flagged (or Householder-first):
// the blocked kernel for matrices with l >= kNb whose shared-memory slices
// fit, the column kernel for the rest.
template <typename T>
cudaError_t launch_householder(const OrthBatch<T>& b, cudaStream_t s) {
  cudaError_t e;
  OrthBatch<T> pb, cb;
  pb.count = cb.count = 0;
  pb.max_chunks = cb.max_chunks = b.max_chunks;
  pb.max_tilepairs = cb.max_tilepairs = b.max_tilepairs;
  for (int i = 0; i < b.count; ++i) {
    const OrthJob<T>& J = b.job[i];
    const bool fits = panel_layout(J.rows, J.l, kPanelMaxCluster).total * sizeof(double) <= kPanelSmemMax;
    // at most 64 rows per CTA (two per lane of a column's warp) on clusters of kPanelMaxCluster
    if (J.l >= kNb && J.l <= 256 && J.rows <= 64 * kPanelMaxCluster && fits) pb.job[pb.count++] = J;
    else cb.job[cb.count++] = J;
  }
  if (pb.count > 0) {
    // spread over the SMs (at most 64 rows per CTA, at most kPanelMaxCluster CTAs, and
    // the shared-memory slices within budget)
    int cmin = 1;
    for (int i = 0; i < pb.count; ++i) {
      int c = max(1, ceil_div(pb.job[i].rows, 64));
      while (c < kPanelMaxCluster && panel_layout(pb.job[i].rows, pb.job[i].l, c).total * sizeof(double) > kPanelSmemMax)
        ++c;
      cmin = max(cmin, c);
    }
    const int pcs = spread_cluster(pb.count, min(cmin, kPanelMaxCluster), kPanelMaxCluster);
    size_t psmem = 0;
    for (int i = 0; i < pb.count; ++i)
      psmem = max(psmem, panel_layout(pb.job[i].rows, pb.job[i].l, pcs).total * sizeof(double));
    e = cudaFuncSetAttribute(householder_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pcs, pb.count, 1);
    cfg.blockDim = dim3(kHhThreads, 1, 1);
    cfg.dynamicSmemBytes = psmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = pcs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    prof_begin(KC_HOUSEHOLDER, s);
    e = cudaLaunchKernelEx(&cfg, householder_panel_kernel<T>, pb, pcs);
    prof_end(KC_HOUSEHOLDER, s);
    if (e != cudaSuccess) return e;
  }
  if (cb.count > 0) {
    const OrthBatch<T>& b2 = cb;
    int maxrows = 1;
    for (int i = 0; i < b2.count; ++i) maxrows = max(maxrows, b2.job[i].rows);
    int csize = min(8, max(1, ceil_div(maxrows, 32)));
    auto bytes = [&](int cs) {
      size_t mx = 0;
      for (int i = 0; i < b2.count; ++i) {
        const int rs = ceil_div(b2.job[i].rows, cs), l = b2.job[i].l;
        mx = max(mx, (hh_small_doubles(l) + 2 * (size_t)rs * l) * sizeof(double));
      }
      return mx;
    };
    if (bytes(csize) > 200 * 1024 && csize == 8 && bytes(16) <= 200 * 1024) csize = 16;
    const int use_global = bytes(csize) > 200 * 1024 ? 1 : 0;
    size_t hsmem = 0;
    if (use_global) {
      for (int i = 0; i < b2.count; ++i) hsmem = max(hsmem, hh_small_doubles(b2.job[i].l) * sizeof(double));
    } else {
      hsmem = bytes(csize);
    }
    e = cudaFuncSetAttribute(householder_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem);
    if (e != cudaSuccess) return e;
    if (csize > 8) {
      e = cudaFuncSetAttribute(householder_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize, b2.count, 1);
    cfg.blockDim = dim3(kHhThreads, 1, 1);
    cfg.dynamicSmemBytes = hsmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    prof_begin(KC_HOUSEHOLDER, s);
    e = cudaLaunchKernelEx(&cfg, householder_kernel<T>, b2, csize, use_global);
    prof_end(KC_HOUSEHOLDER, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// Orthonormalisation of a batch of samples (Alg. RSVD steps 2-3).  Nearly
// square samples go to Householder QR directly (hh_first), the others to
// CholeskyQR2 with Householder as the fallback on breakdown.  The two groups
// are independent: the Householder-first group runs on a side stream (forked
// from and joined back to s by events), concurrently with the CholeskyQR2
// group, whose short launches would otherwise leave the GPU idle.
template <typename T>
cudaError_t launch_orth(const OrthBatch<T>& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  OrthBatch<T> hb, cq;
  hb.count = cq.count = 0;
  hb.max_chunks = cq.max_chunks = b.max_chunks;
  hb.max_tilepairs = cq.max_tilepairs = b.max_tilepairs;
  for (int i = 0; i < b.count; ++i) {
    if (b.job[i].hh_first) hb.job[hb.count++] = b.job[i];
    else cq.job[cq.count++] = b.job[i];
  }
  cudaError_t e = cudaSuccess;
  SideStreams* fk = nullptr;
  if (hb.count > 0 && cq.count > 0 && !b.serial) {
    fk = side_streams();
    if (!fk) return cudaErrorUnknown;
    e = fork_side(fk, 1, s);
    if (e != cudaSuccess) return e;
  }
  if (hb.count > 0) {
    e = launch_householder<T>(hb, fk ? fk->stream[0] : s);
    if (e != cudaSuccess) return e;
  }
  if (cq.count > 0) {
    e = launch_cholqr2<T>(cq, s);
    if (e != cudaSuccess) return e;
    e = launch_householder<T>(cq, s);  // matrices whose Cholesky factorization broke down
    if (e != cudaSuccess) return e;
  }
  if (fk) e = join_side(fk, 1, s);
  return e;
}

template cudaError_t launch_prep<double>(const PrepBatch<double>&, cudaStream_t);
template cudaError_t launch_prep<float>(const PrepBatch<float>&, cudaStream_t);
template cudaError_t launch_orth<double>(const OrthBatch<double>&, cudaStream_t);
template cudaError_t launch_orth<float>(const OrthBatch<float>&, cudaStream_t);

}  // namespace rsvd
