// Small kernels around the factorization:
//  - sign canonicalisation of the singular vector pairs (u_i, v_i);
//  - the global post-selection of the chi largest singular values over the
//    blocks of a block-diagonal matrix (Sec. III.A);
//  - the two-site contraction and Schmidt-value update of a TEBD block update
//    (Sec. III.A, "block update (B)").
#include "common.cuh"

namespace rsvd {

namespace {

// ---------------------------------------------------------------- signs
// Flip (u_i, v_i) so that the largest-|.| entry of u_i is positive (lowest row
// index on ties).  One warp per column.
template <typename T>
__global__ void __launch_bounds__(256) sign_kernel(const __grid_constant__ SignBatch<T> b) {
  const SignJob<T>& J = b.job[blockIdx.y];
  if (J.active && !*J.active) return;  // an inactive job (whole CTA / cluster, before any barrier)
  const int lane = threadIdx.x % 32;
  const int col = blockIdx.x * 8 + threadIdx.x / 32;
  if (col >= J.k) return;
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int r = lane; r < J.m; r += 32) {
    const double v = fabs((double)J.U[(size_t)r * J.ldu + col]);
    if (v > best) {
      best = v;
      bi = r;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  if (bi >= J.m) return;
  const double lead = (double)J.U[(size_t)bi * J.ldu + col];
  __syncwarp();
  if (!(lead < 0.0)) return;
  for (int r = lane; r < J.m; r += 32) J.U[(size_t)r * J.ldu + col] = -J.U[(size_t)r * J.ldu + col];
  for (int c = lane; c < J.n; c += 32) J.Vt[(size_t)col * J.ldvt + c] = -J.Vt[(size_t)col * J.ldvt + c];
}

// ---------------------------------------------------------------- global top-chi
__device__ __forceinline__ double skey(double v) { return isfinite(v) ? v : -1.0; }

// number of entries of the descending array s[0..k) with key > v (gt) and >= v (ge)
__device__ __forceinline__ void count_desc(const double* s, int k, double v, int& gt, int& ge) {
  int lo = 0, hi = k;
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (skey(s[mid]) > v) lo = mid + 1; else hi = mid;
  }
  gt = lo;
  hi = k;
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (skey(s[mid]) >= v) lo = mid + 1; else hi = mid;
  }
  ge = lo;
}

__global__ void select_zero_kernel(int* k_out, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) k_out[i] = 0;
}

// candidate (b, i) is kept when fewer than chi candidates precede it in the
// order (value descending, then matrix index, then position)
__global__ void __launch_bounds__(256) select_kernel(const __grid_constant__ SelectBatch b) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= b.total) return;
  int bb = 0, off = 0;
  while (bb < b.count && g >= off + b.job[bb].k) {
    off += b.job[bb].k;
    ++bb;
  }
  const int i = g - off;
  // a matrix's count of values may be a device count (<= k): candidates beyond it are none
  auto kval = [&](int c) { return b.job[c].kdev ? min(*b.job[c].kdev, b.job[c].k) : b.job[c].k; };
  if (i >= kval(bb)) return;
  const double v = skey(b.job[bb].S[i]);
  int before = 0;
  for (int c = 0; c < b.count; ++c) {
    int gt, ge;
    count_desc(b.job[c].S, kval(c), v, gt, ge);
    before += gt;
    if (c < bb) before += ge - gt;
    else if (c == bb) before += i - gt;  // equal values at lower positions of the same matrix
  }
  if (before < b.chi) atomicMax(&b.k_out[bb], i + 1);
}

// ---------------------------------------------------------------- TEBD
// theta_B[(a,s1),(s2,c)] = sum_{t1,t2} G[(s1 s2),(t1 t2)] T2[(a,t1),(t2,c)],
// theta = lam[a] theta_B, and per-block partial sums of ||theta||_F^2.
constexpr int kTebdBlocks = 64;

__global__ void __launch_bounds__(256) tebd_theta_kernel(const __grid_constant__ TebdBatch b) {
  const TebdJob& J = b.job[blockIdx.y];
  const int d = J.d, Dl = J.Dl, Dr = J.Dr;
  const int rows = Dl * d, cols = d * Dr;
  const long long tot = (long long)rows * cols;
  double acc = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(e / cols), col = (int)(e % cols);
    const int a = row / d, s1 = row % d;
    const int s2 = col / Dr, c = col % Dr;
    double v = 0.0;
    for (int t1 = 0; t1 < d; ++t1)
      for (int t2 = 0; t2 < d; ++t2)
        v = fma(J.gate[(s1 * d + s2) * d * d + t1 * d + t2], J.T2[(long long)(a * d + t1) * cols + t2 * Dr + c], v);
    J.thetaB[e] = v;
    const double w = J.lam[a] * v;
    J.theta[e] = w;
    acc = fma(w, w, acc);
  }
  __shared__ double red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    J.fro2[blockIdx.x] = s;
  }
}

// lam <- S / ||S||, nrm <- ||S||, trunc_err <- 1 - ||S||^2 / ||theta||_F^2
__global__ void __launch_bounds__(256) tebd_finish_kernel(const __grid_constant__ TebdFinBatch b) {
  const TebdFinJob& J = b.job[blockIdx.x];
  __shared__ double red[8];
  __shared__ double nrm;
  double acc = 0.0;
  for (int r = threadIdx.x; r < J.k; r += blockDim.x) acc = fma(J.S[r], J.S[r], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    double f = 0.0;
    for (int q = 0; q < kTebdBlocks; ++q) f += J.fro2[q];
    nrm = sqrt(s);
    *J.nrm = nrm;
    double te = f > 0.0 ? 1.0 - s / f : 0.0;
    *J.trunc_err = te > 0.0 ? te : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < J.k; r += blockDim.x) J.lam[r] = nrm > 0.0 ? J.S[r] / nrm : 0.0;
}

// product update (Sec. III.A "product update (P)"): the K single-site operators
// of each side widen the bond to K Dm; consecutive threads take consecutive
// columns, so the reads of B_i (over b) and B_{i+1} (over c) are coalesced
__global__ void __launch_bounds__(256) tebd_product_kernel(const __grid_constant__ TebdProdBatch b) {
  const TebdProdJob& J = b.job[blockIdx.y];
  const int d = J.d, Dm = J.Dm, Dr = J.Dr;
  const int r = J.K * Dm, n = d * Dr;
  const long long nx = (long long)J.Dl * d * r, ny = (long long)r * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nx + ny; e += (long long)gridDim.x * blockDim.x) {
    if (e < nx) {
      const int row = (int)(e / r), col = (int)(e % r);
      const int a = row / d, s1 = row % d, k = col / Dm, c = col % Dm;
      const double* u = J.uL + ((size_t)k * d + s1) * d;
      const double* bi = J.Bi + (size_t)a * d * Dm + c;
      double v = 0.0;
      for (int t = 0; t < d; ++t) v = fma(u[t], bi[(size_t)t * Dm], v);
      J.XB[e] = v;
      J.X[e] = J.lam[a] * v;
    } else {
      const long long f = e - nx;
      const int row = (int)(f / n), col = (int)(f % n);
      const int k = row / Dm, bb = row % Dm, s2 = col / Dr, c = col % Dr;
      const double* u = J.uR + ((size_t)k * d + s2) * d;
      const double* bj = J.Bj + (size_t)bb * d * Dr + c;
      double v = 0.0;
      for (int t = 0; t < d; ++t) v = fma(u[t], bj[(size_t)t * Dr], v);
      J.Y[f] = v;
    }
  }
}

// ||X Y||_F^2 = trace((X^T X)(Y Y^T)) = sum_ij G1[i,j] G2[i,j] (G2 symmetric), as
// kTebdBlocks partial sums in the layout tebd_finish_kernel reads
__global__ void __launch_bounds__(256) tebd_gram_dot_kernel(const __grid_constant__ TebdGramDotBatch b) {
  const TebdGramDotJob& J = b.job[blockIdx.y];
  const long long tot = (long long)J.r * J.r;
  double acc0 = 0.0, acc1 = 0.0;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long st = (long long)gridDim.x * blockDim.x;
  for (; e + st < tot; e += 2 * st) {
    acc0 = fma(J.G1[e], J.G2[e], acc0);
    acc1 = fma(J.G1[e + st], J.G2[e + st], acc1);
  }
  if (e < tot) acc0 = fma(J.G1[e], J.G2[e], acc0);
  double acc = acc0 + acc1;
  __shared__ double red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    J.fro2[blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------- fixed-error RSVD
// kSqParts partial sums of x^2 over a rows x cols matrix (ld), two chains per thread
__global__ void __launch_bounds__(256) sq_sum_kernel(const double* X, int rows, int cols, int ld, double* part) {
  const long long tot = (long long)rows * cols;
  const long long st = (long long)gridDim.x * blockDim.x;
  double a0 = 0.0, a1 = 0.0;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e + st < tot; e += 2 * st) {
    const double x0 = X[(e / cols) * ld + e % cols], x1 = X[((e + st) / cols) * ld + (e + st) % cols];
    a0 = fma(x0, x0, a0);
    a1 = fma(x1, x1, a1);
  }
  if (e < tot) {
    const double x0 = X[(e / cols) * ld + e % cols];
    a0 = fma(x0, x0, a0);
  }
  double acc = a0 + a1;
  __shared__ double red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// One warp.  err2(k) = r2 + sum_{i >= k} sig_i^2 (0-based, sig sorted descending) is the
// squared error of the rank-k result; the smallest k in [1, k_trial] with
// err2(k) <= eps^2 fro2 is chosen, else k_trial with grow = 1.  Lane j sums a contiguous
// chunk of sig from its small end; the chunk totals of the lanes above j give its
// starting suffix, and walking its chunk downwards it meets err2(i + 1) before adding
// sig_i^2, so every k = 1 .. l is seen by exactly one lane.
__global__ void tol_rank_kernel(const double* sig, int l, int k_trial, const double* r2_part, const double* fro2_part,
                                double eps, TolResult* out) {
  const int lane = threadIdx.x;
  double r2 = 0.0, fro2 = 0.0;
  for (int i = lane; i < kSqParts; i += 32) {
    r2 += r2_part[i];
    fro2 += fro2_part[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    fro2 += __shfl_xor_sync(0xffffffffu, fro2, o);
  }
  const int c = (l + 31) / 32;
  const int i0 = min(l, lane * c), i1 = min(l, i0 + c);
  double own = 0.0;
  for (int i = i1 - 1; i >= i0; --i) own = fma(sig[i], sig[i], own);
  // sum of the chunk totals of the lanes above this one: an inclusive suffix scan, read
  // from the next lane (no subtraction, so the large head values do not round the tail)
  double suf = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double v = __shfl_down_sync(0xffffffffu, suf, o);
    if (lane + o < 32) suf += v;
  }
  double above = __shfl_down_sync(0xffffffffu, suf, 1);
  if (lane == 31) above = 0.0;
  const double thr = eps * eps * fro2;
  double run = r2 + above;
  int best = 0x7fffffff;
  double best_err2 = 0.0;
  for (int i = i1 - 1; i >= i0; --i) {
    const int k = i + 1;  // run == err2(k) here
    if (k <= k_trial && run <= thr) {
      best = k;
      best_err2 = run;
    }
    run = fma(sig[i], sig[i], run);
  }
  // smallest qualifying k over the warp (err2 is non-increasing in k)
  int kmin = best;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
  const int owner = __ffs(__ballot_sync(0xffffffffu, best == kmin)) - 1;
  const double e2 = __shfl_sync(0xffffffffu, best_err2, owner);
  // err2(k_trial) for the case that no k qualifies: from the lane whose walk met it
  double et = 0.0;
  {
    double r = r2 + above;
    for (int i = i1 - 1; i >= i0; --i) {
      if (i + 1 == k_trial) et = r;
      r = fma(sig[i], sig[i], r);
    }
  }
  const bool has_t = k_trial >= i0 + 1 && k_trial <= i1;
  const int tl = __ffs(__ballot_sync(0xffffffffu, has_t)) - 1;
  et = __shfl_sync(0xffffffffu, et, tl < 0 ? 0 : tl);
  if (lane == 0) {
    const bool found = kmin != 0x7fffffff;
    out->k = found ? kmin : k_trial;
    out->grow = found ? 0 : 1;
    const double ee = found ? e2 : et;
    out->err = fro2 > 0.0 ? sqrt(ee / fro2) : 0.0;
  }
}

}  // namespace

cudaError_t launch_sq_sum(const double* X, int rows, int cols, int ld, double* part, cudaStream_t s) {
  prof_begin(KC_TEBD, s);
  sq_sum_kernel<<<kSqParts, 256, 0, s>>>(X, rows, cols, ld, part);
  prof_end(KC_TEBD, s);
  return cudaGetLastError();
}

cudaError_t launch_tol_rank(const double* sig, int l, int k_trial, const double* r2_part, const double* fro2_part,
                            double eps, TolResult* out, cudaStream_t s) {
  prof_begin(KC_SELECT, s);
  tol_rank_kernel<<<1, 32, 0, s>>>(sig, l, k_trial, r2_part, fro2_part, eps, out);
  prof_end(KC_SELECT, s);
  return cudaGetLastError();
}

cudaError_t launch_tebd_product(const TebdProdBatch& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  long long mx = 1;
  for (int i = 0; i < b.count; ++i) {
    const TebdProdJob& J = b.job[i];
    const long long r = (long long)J.K * J.Dm;
    mx = max(mx, (long long)J.Dl * J.d * r + r * J.d * J.Dr);
  }
  const long long want = (mx + 255) / 256, cap = 2048LL / b.count + 1;  // about 2048 blocks in all
  const int gx = (int)(want < cap ? want : cap);
  prof_begin(KC_TEBD, s);
  tebd_product_kernel<<<dim3(gx, b.count), 256, 0, s>>>(b);
  prof_end(KC_TEBD, s);
  return cudaGetLastError();
}

cudaError_t launch_tebd_gram_dot(const TebdGramDotBatch& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  prof_begin(KC_TEBD, s);
  tebd_gram_dot_kernel<<<dim3(kTebdBlocks, b.count), 256, 0, s>>>(b);
  prof_end(KC_TEBD, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sign(const SignBatch<T>& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  int mk = 1;
  for (int i = 0; i < b.count; ++i) mk = max(mk, b.job[i].k);
  prof_begin(KC_SIGN, s);
  sign_kernel<T><<<dim3(ceil_div(mk, 8), b.count), 256, 0, s>>>(b);
  prof_end(KC_SIGN, s);
  return cudaGetLastError();
}

cudaError_t launch_select(const SelectBatch& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  prof_begin(KC_SELECT, s);
  select_zero_kernel<<<1, 256, 0, s>>>(b.k_out, b.count);
  if (b.total > 0) select_kernel<<<ceil_div(b.total, 256), 256, 0, s>>>(b);
  prof_end(KC_SELECT, s);
  return cudaGetLastError();
}

namespace {
// one warp per bond: Schmidt values are >= +0, so "nonzero" is a test of the bit pattern
__global__ void tebd_rank_kernel(const __grid_constant__ TebdRankBatch b) {
  const TebdRankJob& J = b.job[blockIdx.x];
  int c = 0;
  for (int j = threadIdx.x; j < J.D; j += 32) c += __double_as_longlong(J.lam[j]) > 0 ? 1 : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (threadIdx.x == 0) *J.out = c;
}
}  // namespace

cudaError_t launch_tebd_rank(const TebdRankBatch& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  prof_begin(KC_TEBD, s);
  tebd_rank_kernel<<<b.count, 32, 0, s>>>(b);
  prof_end(KC_TEBD, s);
  return cudaGetLastError();
}

cudaError_t launch_tebd_theta(const TebdBatch& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  prof_begin(KC_TEBD, s);
  tebd_theta_kernel<<<dim3(kTebdBlocks, b.count), 256, 0, s>>>(b);
  prof_end(KC_TEBD, s);
  return cudaGetLastError();
}

cudaError_t launch_tebd_finish(const TebdFinBatch& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  prof_begin(KC_TEBD, s);
  tebd_finish_kernel<<<b.count, 256, 0, s>>>(b);
  prof_end(KC_TEBD, s);
  return cudaGetLastError();
}

template cudaError_t launch_sign<double>(const SignBatch<double>&, cudaStream_t);
template cudaError_t launch_sign<float>(const SignBatch<float>&, cudaStream_t);


// ---------------------------------------------------------------- adaptive rounds on the device
namespace {
__global__ void adapt_init_kernel(const __grid_constant__ AdaptInitBatch b) {
  for (int i = threadIdx.x; i < b.count; i += blockDim.x) {
    b.active[i] = 1;
    b.kdev[i] = b.k[i];
  }
  if (threadIdx.x == 0) *b.rounds = 0;
}
// after a round's selection: a block that ran in it stays active when every one of its
// values was kept and its rank is below its cap (it may hold more above the cut), and its
// rank grows for the next round; the round is counted when any block ran in it
__global__ void adapt_decide_kernel(const __grid_constant__ AdaptDecideBatch b) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < b.count; i += blockDim.x) {
    if (!b.active[i]) continue;
    any = 1;
    const int grow = (b.k_out[i] == b.kdev[i] && b.kdev[i] < b.cap[i]) ? 1 : 0;
    b.active[i] = grow;
    if (grow) b.kdev[i] = b.next_k[i];
  }
  __syncthreads();
  if (threadIdx.x == 0 && any) *b.rounds += 1;
}
}  // namespace

cudaError_t launch_adapt_init(const AdaptInitBatch& b, cudaStream_t s) {
  prof_begin(KC_SELECT, s);
  adapt_init_kernel<<<1, 64, 0, s>>>(b);
  prof_end(KC_SELECT, s);
  return cudaGetLastError();
}

cudaError_t launch_adapt_decide(const AdaptDecideBatch& b, cudaStream_t s) {
  prof_begin(KC_SELECT, s);
  adapt_decide_kernel<<<1, 64, 0, s>>>(b);
  prof_end(KC_SELECT, s);
  return cudaGetLastError();
}

}  // namespace rsvd
