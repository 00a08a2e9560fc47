// Backward of the rank-k truncated factorization A ~ U diag(s) V^T: given the
// cotangents (Ubar, sbar, Vbar) of the returned factors, form Abar.  The paper
// has no derivative; this is the differentiable form of its compression step.
//
// With F_ij = 1 / (s_j^2 - s_i^2) (i != j, retained block), P = I - U U^T and
// Q = I - V V^T:
//   Abar = U [ (F o (U^T Ubar - Ubar^T U)) S + diag(sbar) + S (F o (V^T Vbar - Vbar^T V)) ] V^T
//        + Z S V^T + U Z^T A + U S Y^T + A Y V^T,
//   z_i = (s_i^2 I - P A A^T P)^-1 P ubar_i,   y_i = (s_i^2 I - Q A^T A Q)^-1 Q vbar_i.
// The last four terms couple the retained triplets to the discarded part of A
// without forming it: each column is solved by conjugate gradients (the
// operator is symmetric positive definite on range(P) while s_i exceeds every
// discarded singular value), all k columns at once with their own shifts, the
// operator applied as GEMMs with A and A^T.  A column stops when its residual
// falls below tol times its right-hand side (device-side; no host sync).
#include <algorithm>

#include "common.cuh"

namespace rsvd {

namespace {

constexpr int kColTile = 32;
constexpr int kColRows = 8;  // warps per CTA in the column reductions

// out[c] = sum_r x[r, c] * y[r, c] for c < k; one CTA per 32 columns, fixed
// reduction order (deterministic).
template <typename T>
__global__ void __launch_bounds__(256) coldot_kernel(const __grid_constant__ BwBatch<T> b, int which) {
  const BwJob<T>& J = b.job[blockIdx.y];
  if (which != 2 && !J.flags[2]) return;  // the solve of this matrix has ended
  const int rows = J.rows, k = J.k;
  const int c = blockIdx.x * kColTile + (threadIdx.x % 32);
  const int w = threadIdx.x / 32;
  const T* x;
  const T* y;
  double* out;
  if (which == 0) { x = J.p; y = J.w; out = J.pw; }       // p . w
  else if (which == 1) { x = J.r; y = J.r; out = J.rho_new; }  // r . r
  else { x = J.r; y = J.r; out = J.rho0; }                 // initial residual
  double acc = 0.0;
  if (c < k)
    for (int r = w; r < rows; r += kColRows) acc = fma((double)x[(size_t)r * k + c], (double)y[(size_t)r * k + c], acc);
  __shared__ double red[kColRows][32];
  red[w][threadIdx.x % 32] = acc;
  __syncthreads();
  if (w == 0 && c < k) {
    double s = 0.0;
    for (int q = 0; q < kColRows; ++q) s += red[q][threadIdx.x % 32];
    out[c] = s;
  }
}

// w = s^2 p - t; (first pass) r = b, p = b, z = 0
template <typename T>
__global__ void __launch_bounds__(256) cg_apply_kernel(const __grid_constant__ BwBatch<T> b, int init) {
  const BwJob<T>& J = b.job[blockIdx.y];
  if (!init && !J.flags[2]) return;
  const size_t tot = (size_t)J.rows * J.k;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % J.k);
    if (init) {
      const T v = J.bvec[e];
      J.r[e] = v;
      J.p[e] = v;
      J.z[e] = (T)0;
    } else {
      const double s = J.s[c];
      J.w[e] = (T)(s * s * (double)J.p[e] - (double)J.t[e]);
    }
  }
}

// alpha = rho / pw; z += alpha p; r -= alpha w (active columns only)
template <typename T>
__global__ void __launch_bounds__(256) cg_update_zr_kernel(const __grid_constant__ BwBatch<T> b) {
  const BwJob<T>& J = b.job[blockIdx.y];
  if (!J.flags[2]) return;
  const size_t tot = (size_t)J.rows * J.k;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % J.k);
    if (!J.active[c]) continue;
    const double pw = J.pw[c];
    if (!(pw > 0.0)) continue;  // not positive definite along p: the column is frozen by cg_scalar_kernel
    const double al = J.rho[c] / pw;
    J.z[e] = (T)((double)J.z[e] + al * (double)J.p[e]);
    J.r[e] = (T)((double)J.r[e] - al * (double)J.w[e]);
  }
}

// per column: convergence / breakdown bookkeeping, beta = rho_new / rho
// (flags[0]: a column broke down; flags[1]: iterations in which a column was still active)
template <typename T>
__global__ void cg_scalar_kernel(const __grid_constant__ BwBatch<T> b, int init) {
  const BwJob<T>& J = b.job[blockIdx.x];
  if (init && threadIdx.x == 0) {
    J.flags[0] = 0;
    J.flags[1] = 0;
  }
  int had = 0;
  for (int c = threadIdx.x; c < J.k && !init; c += blockDim.x) had |= J.active[c];
  if (__syncthreads_or(had) && threadIdx.x == 0) J.flags[1] += 1;
  int still = 0;
  for (int c = threadIdx.x; c < J.k; c += blockDim.x) {
    if (init) {
      J.rho[c] = J.rho0[c];
      J.active[c] = J.rho0[c] > 0.0 ? 1 : 0;
      J.beta[c] = 0.0;
      continue;
    }
    if (!J.active[c]) {
      J.beta[c] = 0.0;
      continue;
    }
    if (!(J.pw[c] > 0.0)) {  // indefinite or breakdown: keep the last iterate
      J.active[c] = 0;
      atomicOr(J.flags, 1);
      J.beta[c] = 0.0;
      continue;
    }
    const double rn = J.rho_new[c];
    if (rn <= J.tol2 * J.rho0[c]) {
      J.active[c] = 0;
      J.beta[c] = 0.0;
    } else {
      J.beta[c] = rn / J.rho[c];
    }
    J.rho[c] = rn;
  }
  for (int c = threadIdx.x; c < J.k; c += blockDim.x) still |= J.active[c];
  // every launch of the next iteration reads this flag (stream order) and skips the
  // matrix once no column is left: the work ends with the slowest column
  const int any = __syncthreads_or(still);
  if (threadIdx.x == 0) J.flags[2] = any ? 1 : 0;
}

// p = r + beta p (active columns)
template <typename T>
__global__ void __launch_bounds__(256) cg_update_p_kernel(const __grid_constant__ BwBatch<T> b) {
  const BwJob<T>& J = b.job[blockIdx.y];
  if (!J.flags[2]) return;
  const size_t tot = (size_t)J.rows * J.k;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % J.k);
    if (!J.active[c]) continue;
    J.p[e] = (T)((double)J.r[e] + J.beta[c] * (double)J.p[e]);
  }
}

// core = (F o (X - X^T)) S + diag(sbar) + S (F o (Yv - Yv^T)), F_ij = 1/(s_j^2 - s_i^2)
template <typename T>
__global__ void __launch_bounds__(256) bw_core_kernel(const __grid_constant__ BwCoreBatch<T> b) {
  const BwCoreJob<T>& J = b.job[blockIdx.y];
  const int k = J.k;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
    const int i = e / k, j = e % k;
    double v = 0.0;
    if (i == j) {
      v = J.sbar ? J.sbar[i] : 0.0;
    } else {
      const double si = J.s[i], sj = J.s[j];
      const double f = 1.0 / (sj * sj - si * si);
      double a = 0.0;
      if (J.X) a += ((double)J.X[i * k + j] - (double)J.X[j * k + i]) * sj;
      if (J.Yv) a += si * ((double)J.Yv[i * k + j] - (double)J.Yv[j * k + i]);
      v = f * a;
    }
    J.core[e] = (T)v;
  }
}

// out[r, c] = s[c] in[r, c] (or a plain / transposed copy when s is null)
template <typename T>
__global__ void __launch_bounds__(256) colscale_kernel(const __grid_constant__ BwScaleBatch<T> b) {
  const BwScaleJob<T>& J = b.job[blockIdx.y];
  if (J.gate && !*J.gate) return;
  const size_t tot = (size_t)J.rows * J.k;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / J.k), c = (int)(e % J.k);
    const T v = J.transpose ? J.in[(size_t)c * J.ldin + r] : J.in[(size_t)r * J.ldin + c];
    J.out[e] = J.s ? (T)(J.s[c] * (double)v) : v;
  }
}

inline int grid_for(size_t tot) { return (int)std::min<size_t>(1024, (tot + 255) / 256); }

}  // namespace

template <typename T>
cudaError_t launch_bw_coldot(const BwBatch<T>& b, int which, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  int mk = 1;
  for (int i = 0; i < b.count; ++i) mk = max(mk, b.job[i].k);
  prof_begin(KC_BACKWARD, s);
  coldot_kernel<T><<<dim3(ceil_div(mk, kColTile), b.count), 256, 0, s>>>(b, which);
  prof_end(KC_BACKWARD, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bw_elementwise(const BwBatch<T>& b, int op, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  size_t mx = 1;
  for (int i = 0; i < b.count; ++i) mx = std::max(mx, (size_t)b.job[i].rows * b.job[i].k);
  const dim3 grid(grid_for(mx), b.count);
  prof_begin(KC_BACKWARD, s);
  switch (op) {
    case 0: cg_apply_kernel<T><<<grid, 256, 0, s>>>(b, 1); break;
    case 1: cg_apply_kernel<T><<<grid, 256, 0, s>>>(b, 0); break;
    case 2: cg_update_zr_kernel<T><<<grid, 256, 0, s>>>(b); break;
    case 3: cg_update_p_kernel<T><<<grid, 256, 0, s>>>(b); break;
    case 4: cg_scalar_kernel<T><<<b.count, 256, 0, s>>>(b, 1); break;
    case 5: cg_scalar_kernel<T><<<b.count, 256, 0, s>>>(b, 0); break;
    default: break;
  }
  prof_end(KC_BACKWARD, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bw_core(const BwCoreBatch<T>& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  int mk = 1;
  for (int i = 0; i < b.count; ++i) mk = max(mk, b.job[i].k);
  prof_begin(KC_BACKWARD, s);
  bw_core_kernel<T><<<dim3(grid_for((size_t)mk * mk), b.count), 256, 0, s>>>(b);
  prof_end(KC_BACKWARD, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bw_colscale(const BwScaleBatch<T>& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  size_t mx = 1;
  for (int i = 0; i < b.count; ++i) mx = std::max(mx, (size_t)b.job[i].rows * b.job[i].k);
  prof_begin(KC_BACKWARD, s);
  colscale_kernel<T><<<dim3(grid_for(mx), b.count), 256, 0, s>>>(b);
  prof_end(KC_BACKWARD, s);
  return cudaGetLastError();
}

#define INST(T)                                                                        \
  template cudaError_t launch_bw_coldot<T>(const BwBatch<T>&, int, cudaStream_t);      \
  template cudaError_t launch_bw_elementwise<T>(const BwBatch<T>&, int, cudaStream_t); \
  template cudaError_t launch_bw_core<T>(const BwCoreBatch<T>&, cudaStream_t);         \
  template cudaError_t launch_bw_colscale<T>(const BwScaleBatch<T>&, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace rsvd

// ---------------------------------------------------------------- host side
#include <cstring>
#include <vector>

namespace rsvd {
namespace {

constexpr size_t kBwAlign = 256;
inline size_t bw_align(size_t x) { return (x + kBwAlign - 1) / kBwAlign * kBwAlign; }

struct BwProb {
  int m, n, k;
  const void *A, *U, *Vt, *Ubar, *Vtbar;
  int lda, ldu, ldvt, ldub, ldvb, ldab;
  const double *S, *Sbar;
  void* Abar;
  rsvd_info* info;
  // workspace
  void *X, *Yv, *core, *T1, *p, *r, *w, *z, *t, *bvec, *G1, *t1, *tmp;
  double *pw, *rho, *rho_new, *rho0, *beta;
  int *active, *flags;
};

size_t bw_layout(BwProb* P, int m, int n, int k, size_t ts, char* base) {
  const int mx = std::max(m, n);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += bw_align(bytes);
    return base ? (void*)(base + o) : nullptr;
  };
  void* X = take((size_t)k * k * ts);
  void* Yv = take((size_t)k * k * ts);
  void* core = take((size_t)k * k * ts);
  void* T1 = take((size_t)mx * k * ts);
  void* p = take((size_t)mx * k * ts);
  void* r = take((size_t)mx * k * ts);
  void* w = take((size_t)mx * k * ts);
  void* z = take((size_t)mx * k * ts);
  void* t = take((size_t)mx * k * ts);
  void* bvec = take((size_t)mx * k * ts);
  void* G1 = take((size_t)k * k * ts);
  void* t1 = take((size_t)mx * k * ts);
  void* tmp = take((size_t)k * mx * ts);
  void* pw = take((size_t)k * 8);
  void* rho = take((size_t)k * 8);
  void* rho_new = take((size_t)k * 8);
  void* rho0 = take((size_t)k * 8);
  void* beta = take((size_t)k * 8);
  void* active = take((size_t)k * 4);
  void* flags = take(16);
  if (P) {
    P->X = X; P->Yv = Yv; P->core = core; P->T1 = T1; P->p = p; P->r = r; P->w = w; P->z = z; P->t = t;
    P->bvec = bvec; P->G1 = G1; P->t1 = t1; P->tmp = tmp;
    P->pw = (double*)pw; P->rho = (double*)rho; P->rho_new = (double*)rho_new; P->rho0 = (double*)rho0;
    P->beta = (double*)beta; P->active = (int*)active; P->flags = (int*)flags;
  }
  return off;
}

template <typename T>
struct InfoPtrs {
  rsvd_info* p[kMaxJobs];
};

template <typename T>
__global__ void bw_info_kernel(const __grid_constant__ BwBatch<T> b, const __grid_constant__ InfoPtrs<T> infos,
                               int first) {
  const BwJob<T>& J = b.job[blockIdx.x];
  rsvd_info* info = infos.p[blockIdx.x];
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < J.k; c += blockDim.x)
    if (J.active[c]) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (first) {
      info->status = RSVD_OK;
      info->path = 0;
      info->chol_fallbacks = 0;
      info->jacobi_sweeps = 0;
      info->l = J.k;
      info->rotations = 0;
      info->cg_iterations = 0;
    }
    info->cg_iterations += J.flags[1];
    if ((any || (*J.flags & 1)) && info->status == RSVD_OK) info->status = RSVD_WARN_CG;
  }
}

#define BW_TRY(x)                   \
  do {                              \
    cudaError_t e__ = (x);          \
    if (e__ != cudaSuccess) {       \
      last_cuda_error() = e__;      \
      return RSVD_ERR_LAUNCH;       \
    }                               \
  } while (0)

template <typename T>
int bw_chunk(std::vector<BwProb>& P, int max_iter, double tol, cudaStream_t s) {
  const int cnt = (int)P.size();
  using G = GemmJob<T, T>;
  auto gemm_batch = [&](auto fill, auto launch) {
    GemmBatch<T, T> g;
    g.count = 0;
    for (int i = 0; i < cnt; ++i) fill(P[i], g);
    return launch(g);
  };
  auto NN = [&](const GemmBatch<T, T>& g) { return launch_gemm<T, T, false, false>(g, s); };
  auto TN = [&](const GemmBatch<T, T>& g) { return launch_gemm<T, T, true, false>(g, s); };
  auto NT = [&](const GemmBatch<T, T>& g) { return launch_gemm<T, T, false, true>(g, s); };

  // X = U^T Ubar, Yv = V^T Vbar (= Vt Vtbar^T)
  BW_TRY(gemm_batch([&](BwProb& q, GemmBatch<T, T>& g) {
    if (q.Ubar) g.job[g.count++] = G{q.k, q.k, q.m, q.ldu, q.ldub, q.k, (const T*)q.U, (const T*)q.Ubar, (T*)q.X, nullptr, nullptr, 0};
  }, TN));
  BW_TRY(gemm_batch([&](BwProb& q, GemmBatch<T, T>& g) {
    if (q.Vtbar) g.job[g.count++] = G{q.k, q.k, q.n, q.ldvt, q.ldvb, q.k, (const T*)q.Vt, (const T*)q.Vtbar, (T*)q.Yv, nullptr, nullptr, 0};
  }, NT));
  {
    BwCoreBatch<T> b;
    b.count = cnt;
    for (int i = 0; i < cnt; ++i)
      b.job[i] = BwCoreJob<T>{P[i].k, P[i].Ubar ? (const T*)P[i].X : nullptr, P[i].Vtbar ? (const T*)P[i].Yv : nullptr,
                              P[i].S, P[i].Sbar, (T*)P[i].core};
    BW_TRY(launch_bw_core<T>(b, s));
  }
  // Abar = (U core) Vt
  BW_TRY(gemm_batch([&](BwProb& q, GemmBatch<T, T>& g) {
    g.job[g.count++] = G{q.m, q.k, q.k, q.ldu, q.k, q.k, (const T*)q.U, (const T*)q.core, (T*)q.T1, nullptr, nullptr, 0};
  }, NN));
  BW_TRY(gemm_batch([&](BwProb& q, GemmBatch<T, T>& g) {
    g.job[g.count++] = G{q.m, q.n, q.k, q.k, q.ldvt, q.ldab, (const T*)q.T1, (const T*)q.Vt, (T*)q.Abar, nullptr, nullptr, 0};
  }, NN));

  for (int side = 0; side < 2; ++side) {  // 0: left (Ubar, rows m), 1: right (Vbar, rows n)
    std::vector<int> sel;
    for (int i = 0; i < cnt; ++i)
      if (side == 0 ? P[i].Ubar != nullptr : P[i].Vtbar != nullptr) sel.push_back(i);
    BwBatch<T> bb;
    bb.count = (int)sel.size();
    for (int j = 0; j < bb.count; ++j) {
      BwProb& q = P[sel[j]];
      bb.job[j] = BwJob<T>{side == 0 ? q.m : q.n, q.k, (T*)q.p, (T*)q.r, (T*)q.w, (T*)q.z, (T*)q.t, (const T*)q.bvec,
                           q.S, q.pw, q.rho, q.rho_new, q.rho0, q.beta, q.active, q.flags, tol * tol};
    }
    if (bb.count == 0) continue;
    auto forsel = [&](auto fill, auto launch) {
      GemmBatch<T, T> g;
      g.count = 0;
      for (int j : sel) fill(P[j], g);
      return launch(g);
    };
    // right-hand sides: b = Ubar - U (U^T Ubar)  |  b = Vbar - V (V^T Vbar)
    {
      BwScaleBatch<T> sc;
      sc.count = bb.count;
      for (int j = 0; j < bb.count; ++j) {
        BwProb& q = P[sel[j]];
        sc.job[j] = side == 0 ? BwScaleJob<T>{q.m, q.k, (const T*)q.Ubar, q.ldub, nullptr, 0, (T*)q.bvec}
                              : BwScaleJob<T>{q.n, q.k, (const T*)q.Vtbar, q.ldvb, nullptr, 1, (T*)q.bvec};
      }
      BW_TRY(launch_bw_colscale<T>(sc, s));
    }
    if (side == 0) {
      BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {
        G j{q.m, q.k, q.k, q.ldu, q.k, q.k, (const T*)q.U, (const T*)q.X, (T*)q.bvec, nullptr, nullptr, 0};
        j.alpha = -1.0; j.accumulate = 1;
        g.job[g.count++] = j;
      }, NN));
    } else {
      BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {  // V (n x k) = Vt^T
        G j{q.n, q.k, q.k, q.ldvt, q.k, q.k, (const T*)q.Vt, (const T*)q.Yv, (T*)q.bvec, nullptr, nullptr, 0};
        j.alpha = -1.0; j.accumulate = 1;
        g.job[g.count++] = j;
      }, TN));
    }
    BW_TRY(launch_bw_elementwise<T>(bb, 0, s));  // r = p = b, z = 0
    BW_TRY(launch_bw_coldot<T>(bb, 2, s));       // rho0
    BW_TRY(launch_bw_elementwise<T>(bb, 4, s));  // init scalars
    // projection X -> X - U (U^T X) (side 0) or X - V (V^T X) (side 1), in place on `dst`
    auto project = [&](auto src_of) -> int {
      BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {
        if (side == 0) g.job[g.count++] = G{q.k, q.k, q.m, q.ldu, q.k, q.k, (const T*)q.U, src_of(q), (T*)q.G1, nullptr, q.flags + 2, 1};
        else g.job[g.count++] = G{q.k, q.k, q.n, q.ldvt, q.k, q.k, (const T*)q.Vt, src_of(q), (T*)q.G1, nullptr, q.flags + 2, 1};
      }, [&](const GemmBatch<T, T>& g) { return side == 0 ? TN(g) : NN(g); }));
      if (side == 0) {
        BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {
          G j{q.m, q.k, q.k, q.ldu, q.k, q.k, (const T*)q.U, (const T*)q.G1, (T*)src_of(q), nullptr, q.flags + 2, 1};
          j.alpha = -1.0; j.accumulate = 1;
          g.job[g.count++] = j;
        }, NN));
      } else {
        BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {
          G j{q.n, q.k, q.k, q.ldvt, q.k, q.k, (const T*)q.Vt, (const T*)q.G1, (T*)src_of(q), nullptr, q.flags + 2, 1};
          j.alpha = -1.0; j.accumulate = 1;
          g.job[g.count++] = j;
        }, TN));
      }
      return RSVD_OK;
    };
    for (int it = 0; it < max_iter; ++it) {
      {  // t = p (copy), then t <- P t
        BwScaleBatch<T> sc;
        sc.count = bb.count;
        for (int j = 0; j < bb.count; ++j) {
          BwProb& q = P[sel[j]];
          const int rows = side == 0 ? q.m : q.n;
          sc.job[j] = BwScaleJob<T>{rows, q.k, (const T*)q.p, q.k, nullptr, 0, (T*)q.t};
          sc.job[j].gate = q.flags + 2;
        }
        BW_TRY(launch_bw_colscale<T>(sc, s));
      }
      int rc = project([](BwProb& q) { return (const T*)q.t; });
      if (rc) return rc;
      if (side == 0) {  // t1 = A^T t (n x k), t = A t1 (m x k)
        BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {
          g.job[g.count++] = G{q.n, q.k, q.m, q.lda, q.k, q.k, (const T*)q.A, (const T*)q.t, (T*)q.t1, nullptr, q.flags + 2, 1};
        }, TN));
        BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {
          g.job[g.count++] = G{q.m, q.k, q.n, q.lda, q.k, q.k, (const T*)q.A, (const T*)q.t1, (T*)q.t, nullptr, q.flags + 2, 1};
        }, NN));
      } else {  // t1 = A t (m x k), t = A^T t1 (n x k)
        BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {
          g.job[g.count++] = G{q.m, q.k, q.n, q.lda, q.k, q.k, (const T*)q.A, (const T*)q.t, (T*)q.t1, nullptr, q.flags + 2, 1};
        }, NN));
        BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {
          g.job[g.count++] = G{q.n, q.k, q.m, q.lda, q.k, q.k, (const T*)q.A, (const T*)q.t1, (T*)q.t, nullptr, q.flags + 2, 1};
        }, TN));
      }
      rc = project([](BwProb& q) { return (const T*)q.t; });
      if (rc) return rc;
      BW_TRY(launch_bw_elementwise<T>(bb, 1, s));  // w = s^2 p - t
      BW_TRY(launch_bw_coldot<T>(bb, 0, s));       // pw
      BW_TRY(launch_bw_elementwise<T>(bb, 2, s));  // z, r
      BW_TRY(launch_bw_coldot<T>(bb, 1, s));       // rho_new
      BW_TRY(launch_bw_elementwise<T>(bb, 5, s));  // beta, freeze
      BW_TRY(launch_bw_elementwise<T>(bb, 3, s));  // p
    }
    {
      InfoPtrs<T> sp;
      for (int j = 0; j < bb.count; ++j) sp.p[j] = P[sel[j]].info;
      bw_info_kernel<T><<<bb.count, 256, 0, s>>>(bb, sp, 0);
      BW_TRY(cudaGetLastError());
    }
    if (side == 0) {
      // Abar += (Z S) Vt + U (Z^T A)
      {
        BwScaleBatch<T> sc;
        sc.count = bb.count;
        for (int j = 0; j < bb.count; ++j) {
          BwProb& q = P[sel[j]];
          sc.job[j] = BwScaleJob<T>{q.m, q.k, (const T*)q.z, q.k, q.S, 0, (T*)q.T1};
        }
        BW_TRY(launch_bw_colscale<T>(sc, s));
      }
      BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {
        G j{q.m, q.n, q.k, q.k, q.ldvt, q.ldab, (const T*)q.T1, (const T*)q.Vt, (T*)q.Abar, nullptr, nullptr, 0};
        j.accumulate = 1;
        g.job[g.count++] = j;
      }, NN));
      BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {  // tmp = Z^T A (k x n)
        g.job[g.count++] = G{q.k, q.n, q.m, q.k, q.lda, q.n, (const T*)q.z, (const T*)q.A, (T*)q.tmp, nullptr, nullptr, 0};
      }, TN));
      BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {
        G j{q.m, q.n, q.k, q.ldu, q.n, q.ldab, (const T*)q.U, (const T*)q.tmp, (T*)q.Abar, nullptr, nullptr, 0};
        j.accumulate = 1;
        g.job[g.count++] = j;
      }, NN));
    } else {
      // Abar += (U S) Y^T + (A Y) Vt
      {
        BwScaleBatch<T> sc;
        sc.count = bb.count;
        for (int j = 0; j < bb.count; ++j) {
          BwProb& q = P[sel[j]];
          sc.job[j] = BwScaleJob<T>{q.m, q.k, (const T*)q.U, q.ldu, q.S, 0, (T*)q.T1};
        }
        BW_TRY(launch_bw_colscale<T>(sc, s));
      }
      BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {
        G j{q.m, q.n, q.k, q.k, q.k, q.ldab, (const T*)q.T1, (const T*)q.z, (T*)q.Abar, nullptr, nullptr, 0};
        j.accumulate = 1;
        g.job[g.count++] = j;
      }, NT));
      BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {  // tmp = A Y (m x k)
        g.job[g.count++] = G{q.m, q.k, q.n, q.lda, q.k, q.k, (const T*)q.A, (const T*)q.z, (T*)q.tmp, nullptr, nullptr, 0};
      }, NN));
      BW_TRY(forsel([&](BwProb& q, GemmBatch<T, T>& g) {
        G j{q.m, q.n, q.k, q.k, q.ldvt, q.ldab, (const T*)q.tmp, (const T*)q.Vt, (T*)q.Abar, nullptr, nullptr, 0};
        j.accumulate = 1;
        g.job[g.count++] = j;
      }, NN));
    }
  }
  return RSVD_OK;
}

template <typename T>
__global__ void bw_info_init_kernel(const __grid_constant__ InfoPtrs<T> ip, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    rsvd_info* info = ip.p[i];
    info->status = RSVD_OK;
    info->path = 0;
    info->chol_fallbacks = 0;
    info->jacobi_sweeps = 0;
    info->l = 0;
    info->rotations = 0;
    info->qr_columns = 0;
    info->qr_kflop = 0;
    info->jacobi_pairs = 0;
    info->cg_iterations = 0;
  }
}

}  // namespace
}  // namespace rsvd

using namespace rsvd;

extern "C" int rsvd_backward_workspace_size(int batch, const int* m, const int* n, const int* k, int prec,
                                            size_t* bytes) {
  if (!m || !n || !k || !bytes) return RSVD_ERR_NULL_POINTER;
  if (batch < 1) return RSVD_ERR_INVALID_SIZE;
  if (prec != RSVD_F64 && prec != RSVD_F32) return RSVD_ERR_PRECISION;
  const size_t ts = prec == RSVD_F64 ? 8 : 4;
  size_t tot = 0;
  for (int b = 0; b < batch; ++b) {
    if (m[b] < 1 || n[b] < 1 || k[b] < 1 || k[b] > std::min(m[b], n[b])) return RSVD_ERR_INVALID_SIZE;
    tot += bw_layout(nullptr, m[b], n[b], k[b], ts, nullptr);
  }
  *bytes = tot;
  return RSVD_OK;
}

extern "C" int rsvd_truncate_backward_batched(int batch, const int* m, const int* n, const int* k, int prec,
                                              const void* const* A, const int* lda, const double* const* S,
                                              const void* const* U, const int* ldu, const void* const* Vt,
                                              const int* ldvt, const void* const* Ubar, const int* ldub,
                                              const double* const* Sbar, const void* const* Vtbar, const int* ldvb,
                                              void* const* Abar, const int* ldab, int max_iter, double tol,
                                              void* work, size_t work_bytes, rsvd_info* info, void* cuda_stream) {
  if (prec != RSVD_F64 && prec != RSVD_F32) return RSVD_ERR_PRECISION;
  if (batch < 1 || max_iter < 0 || !(tol >= 0.0)) return RSVD_ERR_INVALID_SIZE;
  if (!m || !n || !k || !A || !lda || !S || !U || !ldu || !Vt || !ldvt || !Abar || !ldab || !work || !info)
    return RSVD_ERR_NULL_POINTER;
  if ((Ubar && !ldub) || (Vtbar && !ldvb)) return RSVD_ERR_NULL_POINTER;
  if (((uintptr_t)work) % kBwAlign) return RSVD_ERR_WORKSPACE;
  const size_t ts = prec == RSVD_F64 ? 8 : 4;
  std::vector<BwProb> P(batch);
  size_t need = 0;
  for (int b = 0; b < batch; ++b) {
    if (m[b] < 1 || n[b] < 1 || k[b] < 1 || k[b] > std::min(m[b], n[b])) return RSVD_ERR_INVALID_SIZE;
    if (lda[b] < n[b] || ldu[b] < k[b] || ldvt[b] < n[b] || ldab[b] < n[b]) return RSVD_ERR_INVALID_SIZE;
    if ((Ubar && ldub[b] < k[b]) || (Vtbar && ldvb[b] < n[b])) return RSVD_ERR_INVALID_SIZE;
    if (!A[b] || !S[b] || !U[b] || !Vt[b] || !Abar[b]) return RSVD_ERR_NULL_POINTER;
    if ((Ubar && !Ubar[b]) || (Sbar && !Sbar[b]) || (Vtbar && !Vtbar[b])) return RSVD_ERR_NULL_POINTER;
    need += bw_layout(nullptr, m[b], n[b], k[b], ts, nullptr);
  }
  if (need > work_bytes) return RSVD_ERR_WORKSPACE;
  size_t off = 0;
  for (int b = 0; b < batch; ++b) {
    BwProb& q = P[b];
    std::memset(&q, 0, sizeof(BwProb));
    q.m = m[b]; q.n = n[b]; q.k = k[b];
    q.A = A[b]; q.lda = lda[b]; q.S = S[b];
    q.U = U[b]; q.ldu = ldu[b]; q.Vt = Vt[b]; q.ldvt = ldvt[b];
    q.Ubar = Ubar ? Ubar[b] : nullptr; q.ldub = Ubar ? ldub[b] : 0;
    q.Sbar = Sbar ? Sbar[b] : nullptr;
    q.Vtbar = Vtbar ? Vtbar[b] : nullptr; q.ldvb = Vtbar ? ldvb[b] : 0;
    q.Abar = Abar[b]; q.ldab = ldab[b];
    q.info = info + b;
    off += bw_layout(&q, q.m, q.n, q.k, ts, (char*)work + off);
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  for (size_t c0 = 0; c0 < P.size(); c0 += kMaxJobs) {
    std::vector<BwProb> chunk(P.begin() + c0, P.begin() + std::min(P.size(), c0 + kMaxJobs));
    InfoPtrs<double> ip;
    for (size_t i = 0; i < chunk.size(); ++i) ip.p[i] = chunk[i].info;
    bw_info_init_kernel<double><<<1, 64, 0, s>>>(ip, (int)chunk.size());
    if (cudaGetLastError() != cudaSuccess) return RSVD_ERR_LAUNCH;
    int rc = prec == RSVD_F64 ? bw_chunk<double>(chunk, max_iter, tol, s) : bw_chunk<float>(chunk, max_iter, tol, s);
    if (rc != RSVD_OK) return rc;
  }
  return RSVD_OK;
}
