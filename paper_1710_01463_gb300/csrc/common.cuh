// Internal declarations shared by the translation units of librsvd.
// Kernel job descriptors are passed BY VALUE as kernel parameters (up to
// kMaxJobs per launch), so no descriptor array has to be copied to the device
// and every launch sequence can be captured in a CUDA graph.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/rsvd.h"

namespace rsvd {

constexpr int kMaxJobs = 64;       // jobs per launch (larger batches are chunked)
constexpr int kGramChunk = 256;    // rows of Y per Gram partial
constexpr int kGramTile = 16;      // Gram tile edge

// ---- batched GEMM: C = op(A) * op(X) [/ *div] ----------------------------
// op(A) is M x K, op(X) is K x N, C is M x N; all row-major.
// TA: op(A) = A^T with A stored K x M.  TX: op(X) = X^T with X stored N x K.
template <typename Tin, typename Tout>
struct GemmJob {
  int M, N, K;
  int lda, ldx, ldc;
  const Tin* A;
  const Tin* X;
  Tout* C;
  const double* div;   // optional: divide C by *div
  const int* gate;     // optional: run only if *gate == gate_val
  int gate_val;
  double alpha = 1.0;  // C = alpha op(A) op(X) (+ C when accumulate)
  int accumulate = 0;
  // optional device counts: rows m >= *m_eff / columns n >= *n_eff of C are
  // exact zeros (the operand's rows / columns there are zero) and are written
  // without the product
  const int* m_eff = nullptr;
  const int* n_eff = nullptr;
  // optional device count: the sum over k stops at *k_eff (op(A)'s columns and
  // op(X)'s rows beyond it are zero)
  const int* k_eff = nullptr;
  const int* active = nullptr;  // optional device flag: the job runs only while *active != 0
};

template <typename Tin, typename Tout>
struct GemmBatch {
  int count;
  int tiles_m, tiles_n;
  GemmJob<Tin, Tout> job[kMaxJobs];
};

// ---- Omega --------------------------------------------------------------
template <typename T>
struct OmegaJob {
  int n, l, ld;
  T* out;
  unsigned long long seed, stream;
  int transposed = 0;  // 1: write Omega^T (l x n, ld) instead of Omega (n x l, ld)
  const int* active = nullptr;  // optional device flag: the job runs only while *active != 0
};
template <typename T>
struct OmegaBatch {
  int count;
  OmegaJob<T> job[kMaxJobs];
};

// ---- orthonormalisation (CholeskyQR2 + Householder fallback) ------------
template <typename T>
struct OrthJob {
  int rows, l;
  T* Y;              // rows x l (ld = l), in: sample, out: Q
  T* Y1;             // rows x l scratch
  double* part;      // Gram partials, nchunk x l x l
  double* G;         // l x l
  T* Rinv;           // l x l
  double* hw;        // (rows + 16) x l FP64 scratch (Householder slices)
  double* hq;        // (rows + 16) x l FP64 scratch (Householder slices)
  int* flag;         // breakdown flag
  rsvd_info* info;
  int hh_first;      // 1: skip CholeskyQR2, use Householder QR directly
  // leading columns of Q that carry the sample's range (device); with trunc_q
  // a Householder QR that ends early forms only those columns (the rest of Q
  // is left zero) and records their number here
  int* rank_eff = nullptr;
  int trunc_q = 0;
  const int* active = nullptr;  // optional device flag: the job runs only while *active != 0
};
template <typename T>
struct OrthBatch {
  int count;
  int max_chunks;
  int max_tilepairs;
  int serial = 0;  // run the Householder-first and CholeskyQR2 groups one after another on the caller's stream
  OrthJob<T> job[kMaxJobs];
};

// ---- one-sided Jacobi SVD of B (l x n, FP64) -----------------------------
template <typename T>
struct JacobiJob {
  int l, n, k;
  const double* Bm;  // l x n input (ld = n)
  double* Bg;        // global slice storage when shared memory is too small (l x n)
  double* Pg;        // global slice storage for P (l x l)
  double* S;         // k outputs
  double* sig;       // l outputs (sorted)
  T* Vt;             // k x n (ldvt)
  int ldvt;
  T* Ps;             // k x l, rows of P in sorted order
  rsvd_info* info;
  int max_sweeps;
  int want_vt;
  int want_p = 1;                 // accumulate the rotations P (needed only for U~ = P^T)
  const int* pipe_err = nullptr;  // optional: nonzero when an earlier tensor-core pipeline wait timed out
  int no_exchange = 0;            // test of the failure path: no CTA sends its round partials
  const int* active = nullptr;    // optional device flag: the job runs only while *active != 0
};
template <typename T>
struct JacobiBatch {
  int count;
  int csize;         // CTAs per matrix (cluster size)
  int use_global;    // 1: slices live in global memory
  JacobiJob<T> job[kMaxJobs];
};

// ---- misc -----------------------------------------------------------------
template <typename T>
struct PrepJob {
  int m, n, l;
  int exact;         // 1: Q = I (written to Y), Bm = A
  const T* A;
  int lda;
  T* Y;
  double* Bm;
  int* flag;
  rsvd_info* info;
  const int* active = nullptr;  // optional device flag: the job runs only while *active != 0
};
template <typename T>
struct PrepBatch {
  int count;
  PrepJob<T> job[kMaxJobs];
};

template <typename T>
struct SignJob {
  int m, n, k;
  T* U;
  int ldu;
  T* Vt;
  int ldvt;
  const int* active = nullptr;  // optional device flag: the job runs only while *active != 0
};
template <typename T>
struct SignBatch {
  int count;
  SignJob<T> job[kMaxJobs];
};

struct SelectJob {
  const double* S;
  int k;                     // values of the matrix (the largest possible count with kdev)
  const int* kdev = nullptr; // optional device count of the matrix's values (<= k)
};
struct SelectBatch {
  int count;
  int chi;
  int total;
  int* k_out;
  SelectJob job[kMaxJobs];
};

// TEBD: theta = lam (row scale) * gate . (B_i B_{i+1}); T2 = B_i B_{i+1} from a GEMM.
struct TebdJob {
  int Dl, Dr, d;
  const double* T2;     // (Dl d) x (d Dr): T2[(a,t1),(t2,c)]
  const double* gate;   // d^2 x d^2
  const double* lam;    // Dl
  double* thetaB;       // (Dl d) x (d Dr)
  double* theta;        // (Dl d) x (d Dr)
  double* fro2;         // ||theta||_F^2 partial sums (one double, atomically accumulated)
};
struct TebdBatch {
  int count;
  TebdJob job[kMaxJobs];
};
// product update: XB[(a,s1),(k,b)] = sum_t uL[k][s1,t] Bi[a,t,b], X = lam[a] XB,
// Y[(k,b),(s2,c)] = sum_t uR[k][s2,t] Bj[b,t,c]
struct TebdProdJob {
  int Dl, Dm, Dr, d, K;
  const double* Bi;     // Dl x d x Dm
  const double* Bj;     // Dm x d x Dr
  const double* uL;     // K x d x d
  const double* uR;     // K x d x d
  const double* lam;    // Dl
  double* XB;           // (Dl d) x (K Dm)
  double* X;            // (Dl d) x (K Dm)
  double* Y;            // (K Dm) x (d Dr)
};
struct TebdProdBatch {
  int count;
  TebdProdJob job[kMaxJobs];
};
// fro2 partial sums of sum_ij G1[i,j] G2[i,j] (= ||X Y||_F^2 for G1 = X^T X, G2 = Y Y^T)
struct TebdGramDotJob {
  int r;
  const double* G1;
  const double* G2;
  double* fro2;
};
struct TebdGramDotBatch {
  int count;
  TebdGramDotJob job[kMaxJobs];
};
struct TebdFinJob {
  int k;
  const double* S;
  double* lam;          // k outputs
  double* nrm;          // ||S||
  const double* fro2;
  double* trunc_err;
};
struct TebdFinBatch {
  int count;
  TebdFinJob job[kMaxJobs];
};

// ---- backward (CG on the discarded space) ---------------------------------
template <typename T>
struct BwJob {
  int rows, k;
  T *p, *r, *w, *z, *t;     // rows x k (ld = k)
  const T* bvec;            // right-hand sides, rows x k
  const double* s;          // k singular values
  double *pw, *rho, *rho_new, *rho0, *beta;  // k each
  int* active;              // k
  int* flags;               // [0] bit 0: a column met a non-positive curvature; [1] iterations run;
                            // [2] some column is still active (the loop's launches skip when 0)
  double tol2;
};
template <typename T>
struct BwBatch {
  int count;
  BwJob<T> job[kMaxJobs];
};
template <typename T>
struct BwCoreJob {
  int k;
  const T* X;               // U^T Ubar (k x k) or nullptr
  const T* Yv;              // V^T Vbar (k x k) or nullptr
  const double* s;
  const double* sbar;       // or nullptr
  T* core;                  // k x k
};
template <typename T>
struct BwCoreBatch {
  int count;
  BwCoreJob<T> job[kMaxJobs];
};
template <typename T>
struct BwScaleJob {
  int rows, k;              // out is rows x k (ld = k)
  const T* in;
  int ldin;
  const double* s;          // nullptr: plain copy
  int transpose;            // 1: out[r, c] = in[c * ldin + r]
  T* out;
  const int* gate = nullptr;  // optional: run only if *gate != 0
};
template <typename T>
struct BwScaleBatch {
  int count;
  BwScaleJob<T> job[kMaxJobs];
};

// ---- transposes with precision change ------------------------------------
struct XposeJob {
  int rows, cols;      // of the input
  int ldin, ldout;
  const void* in;
  void* out;           // cols x rows
  int fold = 0;        // split transposes: row offset of the low parts
  const int* active = nullptr;  // optional device flag: the job runs only while *active != 0
};
struct XposeBatch {
  int count;
  XposeJob job[kMaxJobs];
};
template <typename Tin, typename Tout>
cudaError_t launch_transpose(const XposeBatch& b, cudaStream_t s);
// out (2 * fold rows): rows c = hi(in[:, c]), rows fold + c = in[:, c] - hi(in[:, c])
template <typename Tout>
cudaError_t launch_split_transpose(const XposeBatch& b, int fold_rows_of_job0_unused, cudaStream_t s);

// ---- tensor-core GEMM (tcgen05, TMA) --------------------------------------
// C[M x N] (FP32) = A[M x K] B[N x K]^T, both operands K-major (row-major).
constexpr int kMaxTcJobs = 16;
struct TcJob {
  CUtensorMap ta;  // A, box 128 rows x 128 bytes
  CUtensorMap tb;  // B, box Npad rows x 128 bytes
  float* C;
  int* err;        // optional: set to 1 when a wait timed out
  int M, N, Npad, K, ldc;
  int fold;        // > 0: B holds [B_hi; B_lo] with B_lo starting at row `fold`; C = acc[:, c] + acc[:, fold + c]
};
struct TcBatch {
  int count;
  TcJob job[kMaxTcJobs];
};
bool make_tmap(CUtensorMap* map, const void* base, int rows, int cols, int ld, int elem_bytes, int box_rows);

// FP64 products on the tensor cores by exact slicing (oz_gemm.cu): every FP64
// value x of a row r is 2^e_r * sum_{i=1..9} p_i 2^-6i + (truncation below
// 2^(e_r - 54)) with integer p_i in [-63, 63] held exactly in BF16; the slice
// products of one level L = i + j <= 11 are summed exactly in an FP32
// accumulator over a K chunk of at most 256 (|sum| <= 9 * 256 * 63^2 < 2^24)
// and the levels of all chunks in FP64.
constexpr int kOzSlices = 9;
constexpr int kOzMaxK = 256;       // K per exactly accumulated chunk
constexpr int kOzMaxKTotal = 1024; // K of one product (chunks of kOzMaxK)
constexpr int kMaxOzJobs = 32;
struct OzJob {
  CUtensorMap tp;    // slices of P: kOzSlices blocks of M rows, row length Kp, box 128 rows x 64
  CUtensorMap ts;    // slices of S^T: kOzSlices blocks of Npad rows, box ntile rows x 64
  double* C;         // C = P S: M x N (ldc), or its transpose N x M when trans_c
  const int* ep;     // M row exponents of P
  const int* es;     // N column exponents of S
  const int* n_eff;  // optional: columns >= *n_eff are exact zeros
  int* err;          // optional: set to 1 when a pipeline wait timed out
  int M, N, Npad, K, ldc, trans_c;
  const int* active = nullptr;  // optional device flag: the job runs only while *active != 0
};
struct OzBatch {
  int count;
  int ntile;  // columns per CTA (multiple of 16, at most 64)
  OzJob job[kMaxOzJobs];
};
// one row (or, with xt, one column) of X split into slices per job
struct OzSplitJob {
  const double* X;
  int rows, K, ldx, xt;  // xt: row r is column r of X (X is K x rows)
  int rows_blk, Kp;      // slice block: rows_blk rows (rows .. rows_blk-1 zero) of Kp entries (K .. Kp-1 zero)
  __nv_bfloat16* S;      // kOzSlices blocks of rows_blk x Kp
  int* e;                // rows_blk exponents (0 for zero rows)
  const int* active = nullptr;  // optional device flag: the job runs only while *active != 0
};
struct OzSplitBatch {
  int count;
  OzSplitJob job[kMaxJobs];
};
cudaError_t launch_oz_split(const OzSplitBatch& b, cudaStream_t s);
cudaError_t launch_oz_gemm(const OzBatch& b, cudaStream_t s);
int oz_ntile(int Npad);
size_t tc_smem_bytes(int Npad, int stages);
int tc_stages(int Npad);

// ---- optional per-kernel timing (CUDA events around launches) -------------
enum KernelClass {
  KC_PREP = 0, KC_OMEGA, KC_GEMM, KC_GRAM, KC_CHOL, KC_HOUSEHOLDER, KC_JACOBI, KC_SIGN, KC_SELECT, KC_TEBD,
  KC_BACKWARD, KC_TCGEMM, KC_CONVERT, KC_OZGEMM, KC_OZSPLIT, KC_COUNT
};
void prof_begin(int cls, cudaStream_t s);
void prof_end(int cls, cudaStream_t s);

// ---- launchers (defined in the .cu files) ---------------------------------
template <typename Tin, typename Tout, bool TA, bool TX>
cudaError_t launch_gemm(const GemmBatch<Tin, Tout>& b, cudaStream_t s);
template <typename T>
cudaError_t launch_omega(const OmegaBatch<T>& b, cudaStream_t s);
cudaError_t launch_omega_f64_single(int n, int l, int ld, double* out, unsigned long long seed,
                                    unsigned long long stream, cudaStream_t s);
template <typename T>
cudaError_t launch_prep(const PrepBatch<T>& b, cudaStream_t s);
template <typename T>
cudaError_t launch_orth(const OrthBatch<T>& b, cudaStream_t s);
template <typename T>
cudaError_t launch_jacobi(const JacobiBatch<T>& b, cudaStream_t s);
template <typename T>
cudaError_t launch_sign(const SignBatch<T>& b, cudaStream_t s);
cudaError_t launch_select(const SelectBatch& b, cudaStream_t s);
cudaError_t launch_tebd_theta(const TebdBatch& b, cudaStream_t s);
// number of nonzero Schmidt values of a bond (they are sorted, zeros last)
struct TebdRankJob {
  const double* lam;
  int D;
  int* out;
};
struct TebdRankBatch {
  int count;
  TebdRankJob job[kMaxJobs];
};
cudaError_t launch_tebd_rank(const TebdRankBatch& b, cudaStream_t s);
cudaError_t launch_tebd_finish(const TebdFinBatch& b, cudaStream_t s);
cudaError_t launch_tebd_product(const TebdProdBatch& b, cudaStream_t s);
// fixed-error RSVD: partial sums of squares of a rows x cols FP64 matrix (ld), and
// the rank decision from the sample (see misc.cu)
constexpr int kSqParts = 64;
cudaError_t launch_sq_sum(const double* X, int rows, int cols, int ld, double* part, cudaStream_t s);
struct TolResult {
  int k;       // chosen rank
  int grow;    // 1: no k <= k_trial reaches eps
  double err;  // ||A - Q B_k||_F / ||A||_F
};
cudaError_t launch_tol_rank(const double* sig, int l, int k_trial, const double* r2_part, const double* fro2_part,
                            double eps, TolResult* out, cudaStream_t s);
cudaError_t launch_tebd_gram_dot(const TebdGramDotBatch& b, cudaStream_t s);
template <typename TIn>
cudaError_t launch_tc_gemm(const TcBatch& b, cudaStream_t s, int skip_loads = 0);
template <typename T>
cudaError_t launch_bw_coldot(const BwBatch<T>& b, int which, cudaStream_t s);
template <typename T>
cudaError_t launch_bw_elementwise(const BwBatch<T>& b, int op, cudaStream_t s);
template <typename T>
cudaError_t launch_bw_core(const BwCoreBatch<T>& b, cudaStream_t s);
template <typename T>
cudaError_t launch_bw_colscale(const BwScaleBatch<T>& b, cudaStream_t s);

// device-side rounds of the adaptive sector ranks (misc.cu): the initial flags and ranks,
// and after each round's selection the next round's flags (a block stays active while all
// of its values were kept and its rank is below its cap; its rank then grows to next_k)
struct AdaptInitBatch {
  int count;
  int *active, *kdev, *rounds;
  int k[kMaxJobs];
};
struct AdaptDecideBatch {
  int count;
  int *active, *kdev, *rounds;
  const int* k_out;
  int cap[kMaxJobs], next_k[kMaxJobs];
};
cudaError_t launch_adapt_init(const AdaptInitBatch& b, cudaStream_t s);
cudaError_t launch_adapt_decide(const AdaptDecideBatch& b, cudaStream_t s);

// complex matrices through their real embedding (complex.cu): R(A) = [X -Y; Y X] from the
// interleaved complex A, and the complex factors from the real ones (phase rule applied)
template <typename T>
cudaError_t launch_realify(int m, int n, const T* A, int lda, T* R, cudaStream_t s);
template <typename T>
cudaError_t launch_complex_extract(int m, int n, int k, const double* Sr, const T* Ur, int ldur, const T* Vtr,
                                   int ldvr, double* S, T* U, int ldu, T* Vh, int ldvh, cudaStream_t s);

// last CUDA error seen by a launch of this library (per host thread)
cudaError_t& last_cuda_error();

// Side streams for independent groups of work within one call (streams.cu).
constexpr int kSideStreams = 4;
struct SideStreams {
  bool ready = false;
  void* ctx = nullptr;  // the CUDA context they were created in
  cudaStream_t stream[kSideStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kSideStreams] = {};
};
// Chunks of a large batch run concurrently on kChunkStreams chunk streams (set
// kChunkSet); chunk stream c's work forks onto side-stream set c, so that the groups
// of different chunks never share a side stream.  Set 0 also serves unchunked calls.
constexpr int kChunkStreams = 4;
constexpr int kChunkSet = kChunkStreams;
constexpr int kSideSets = kChunkStreams + 1;
SideStreams* side_set(int set);   // this thread's set `set` for the current device; null on failure
SideStreams* side_streams();      // the set chosen by select_side_set (0 unless a chunk runs)
void select_side_set(int set);    // per host thread
void* current_context();  // the calling thread's current CUDA context (driver handle), null if none
cudaError_t fork_side(SideStreams* ss, int n, cudaStream_t s);  // side streams 0..n-1 wait for s's work so far
cudaError_t join_side(SideStreams* ss, int n, cudaStream_t s);  // s waits for side streams 0..n-1

// number of SMs of the current device
int sm_count();
// Cluster size for a launch of `count` independent matrices, each split over c CTAs
// (cmin <= c <= cmax): the busiest SM of a launch with count * c CTAs placed one per SM
// before any SM takes a second carries ceil(count c / SMs) CTAs of 1/c of a matrix each;
// the smallest c that minimises that load is taken (fewer CTAs per cluster: cheaper
// barriers and fewer partials to exchange; measured faster than two CTAs per SM on the
// TEBD layers).  The choice depends on the batch, so a matrix's rounding (the order of its
// cluster sums) can differ between batches of different sizes.  `rep` is the work every
// CTA of a cluster repeats (in units of one whole matrix's divisible work): a CTA then
// carries rep + 1/c.
inline int spread_cluster(int count, int cmin, int cmax, double rep = 0.0) {
  const long long sms = sm_count();
  int best = cmax;
  double bl = 1e300;
  for (int c = cmin; c <= cmax; ++c) {
    const double load = (double)((count * (long long)c + sms - 1) / sms) * (rep + 1.0 / c);
    if (load < bl * (1.0 - 1e-12)) {
      bl = load;
      best = c;
    }
  }
  return best;
}

// shared-memory budget of the Jacobi kernel for given sizes (bytes), and the
// cluster size chosen for them
int jacobi_cluster_size(int l, int n);
size_t jacobi_smem_bytes(int l, int n, int csize);
bool jacobi_fits_smem(int l, int n, int csize);

inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

constexpr size_t kAlign = 256;  // workspace buffer alignment
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace rsvd
