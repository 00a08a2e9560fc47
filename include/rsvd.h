/*
 * librsvd - randomized truncated SVD (RSVD) for tensor-network bond
 * compression on one GB300 (sm_103a).
 *
 * Method: Kohn, Tschirsich, Keck, Plenio, Tamascelli, Montangero,
 * "Probabilistic low-rank factorization accelerates tensor network simulations
 * of critical quantum many-body ground states", arXiv:1710.01463.
 *   - Alg. TSVD (Sec. II.A): the rank-chi truncated SVD that every call returns.
 *   - Alg. RSVD (Sec. II.B): Gaussian test matrix Omega, power iteration with
 *     re-orthonormalisation after every product, Q = orth(Y), B = Q^T A, small
 *     SVD of B, U = Q U~.
 *   - Sec. III.A: block-diagonal (symmetry-sector) matrices compressed block by
 *     block with a global post-selection of the chi largest singular values;
 *     TEBD "block update" of two neighbouring MPS tensors.
 *
 * Conventions shared by every entry point
 *   - Matrices are ROW-MAJOR with a leading dimension (elements between the
 *     starts of consecutive rows) >= the number of columns.
 *   - Every pointer to matrix / vector data is a DEVICE pointer unless stated
 *     otherwise; arrays of per-matrix sizes and of device pointers passed to
 *     the batched calls are HOST arrays.
 *   - The caller owns every buffer, including the workspace (size from the
 *     *_workspace_size queries).  The library allocates no device memory and
 *     keeps no state between calls.  Inputs are never written.
 *   - Every call is asynchronous on the given CUDA stream (a cudaStream_t,
 *     passed as void*; NULL = legacy default stream).  The return value covers
 *     only the host-side argument checks; conditions found on the device are
 *     written to the caller's rsvd_info records (device memory), readable after
 *     the caller synchronises the stream.
 *   - Singular values are returned in descending order, FP64.  Singular vector
 *     pairs (u_i, v_i) are sign-normalised: the entry of u_i with the largest
 *     magnitude is positive (lowest row index on ties).
 *   - l = min(k + p, m, n) columns are sampled (the paper's l; k is its chi).
 *   - The Gaussian test matrix of matrix b of a call uses the Philox4x64-10 key
 *     (seed, stream + b); see rsvd_gaussian.
 */
#ifndef RSVD_H
#define RSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define RSVD_OK                 0
#define RSVD_ERR_INVALID_SIZE  -1   /* m, n, k, l, batch or a leading dimension out of range */
#define RSVD_ERR_NULL_POINTER  -2   /* a required pointer is NULL */
#define RSVD_ERR_PRECISION     -3   /* precision not supported by this entry point */
#define RSVD_ERR_WORKSPACE     -4   /* workspace smaller than the size query returned */
#define RSVD_ERR_LAUNCH        -5   /* a CUDA launch failed (message via rsvd_status_string) */
#define RSVD_ERR_NONFINITE     -6   /* device: NaN or Inf met in the input (info.status) */
#define RSVD_ERR_TIMEOUT       -8   /* device: a tensor-core pipeline wait timed out (info.status) */
#define RSVD_ERR_SCRATCH_LIMIT -7   /* rsvd_truncate_noalloc: the matrix needs more scratch than its fixed array */
#define RSVD_WARN_NOCONV        1   /* device: the Jacobi SVD hit its sweep cap (info.status) */
#define RSVD_WARN_CG            2   /* device (backward): a conjugate-gradient column did not converge (info.status) */

/* rsvd_params.flags.  By default the FP64 products with A (the sketch, the
 * power iteration and the projection) of matrices with m, n <= 1024 and
 * l <= 256 run on the tensor cores by exact slicing (see rsvd_gemm_f64_tc:
 * FP64-class error); RSVD_FLAG_F64_SIMT computes them with FP64 FMAs instead. */
#define RSVD_FLAG_F64_SIMT      1
/* Alg. TSVD (Sec. II.A) on the same engine, the comparator that the paper's speedup
 * tau = T_TSVD / T_RSVD is defined against (Sec. IV): no sampling - B = A (all m rows,
 * m <= 1024), the one-sided Jacobi SVD of A itself (for n >= 3m on the m x m factor of
 * an orthonormalisation of A^T), then truncation to k; p and q are ignored.  Honoured
 * by rsvd_truncate, rsvd_truncate_batched (RSVD_F64 / RSVD_F32; RSVD_ERR_PRECISION for
 * the tensor-core precisions) and tebd_bond_update; the other entry points return
 * RSVD_ERR_INVALID_SIZE. */
#define RSVD_FLAG_FULL_SVD      2
/* Measurement aid: the independent groups of work of a call (Householder-first and
 * CholeskyQR2 orthonormalisations, Jacobi SVDs of different cluster sizes, the chunks of
 * a large batch) run one after another on the caller's stream instead of concurrently on
 * side streams, so that the kernels' durations add up to the call's time.  Same results
 * bit for bit. */
#define RSVD_FLAG_SERIAL        4
/* Test of a failure path, not for production use: the CTAs of the Jacobi SVD's
 * thread-block clusters send none of their round partials, so every exchange wait
 * runs out (after about 0.13 s), the cluster leaves the iteration together and
 * info.status reports RSVD_ERR_TIMEOUT (the results are invalid; nothing faults or
 * hangs, and the context stays usable).  Honoured by rsvd_truncate and
 * rsvd_truncate_batched. */
#define RSVD_FLAG_TEST_NO_EXCHANGE (1 << 30)

/* Paths recorded in rsvd_info.path (bit set). */
#define RSVD_PATH_EXACT         1   /* m <= l and m <= 16: Q = I, B = A (the sample covers the range) */
#define RSVD_PATH_HOUSEHOLDER   2   /* CholeskyQR2 broke down at least once; Householder QR used */

/* Arithmetic of the products with A (the sketch, the power iteration and the
 * projection).  The Gram matrix, the Cholesky factor and the SVD of B are
 * always computed in FP64.  With RSVD_TF32 / RSVD_BF16 the samples are FP32,
 * U and V^T are float, and the call needs l <= 256, m > l, a 16-byte aligned
 * A and lda * element size a multiple of 16 bytes (else RSVD_ERR_INVALID_SIZE). */
typedef enum {
  RSVD_F64 = 0,   /* A, U, V^T are double; every product in FP64 */
  RSVD_F32 = 1,   /* A, U, V^T are float; products in FP32 (FFMA) */
  RSVD_TF32 = 2,  /* A float; products with A on tensor cores as TF32, FP32 accumulation */
  RSVD_BF16 = 3   /* A bfloat16; products with A on tensor cores in BF16, FP32 accumulation */
} rsvd_prec;

typedef struct {
  int k;            /* target rank chi (>= 1, <= min(m, n)); batched calls may override per matrix */
  int p;            /* oversampling (>= 0); l = min(k + p, m, n) */
  int q;            /* power iterations (>= 0); 2q + 1 orthonormalisations */
  int prec;         /* rsvd_prec */
  uint64_t seed;    /* Philox key word 0 */
  uint64_t stream;  /* Philox key word 1 of the first matrix; matrix b uses stream + b */
  int max_sweeps;   /* Jacobi sweep cap (0 = default 40) */
  int flags;        /* 0, or RSVD_FLAG_F64_SIMT / RSVD_FLAG_FULL_SVD / RSVD_FLAG_SERIAL
                       (RSVD_FLAG_TEST_NO_EXCHANGE: tests only) */
} rsvd_params;

/* Device-written record, one per matrix. */
typedef struct {
  int status;          /* RSVD_OK, RSVD_WARN_NOCONV or RSVD_ERR_NONFINITE */
  int path;            /* RSVD_PATH_* bits */
  int chol_fallbacks;  /* orthonormalisations that fell back to Householder QR (CholeskyQR2 broke
                          down, or the sample was known to be rank deficient) */
  int jacobi_sweeps;   /* sweeps of the one-sided Jacobi SVD of B */
  int l;               /* sample width used */
  int rotations;       /* plane rotations applied by the Jacobi SVD (all sweeps) */
  int qr_columns;      /* columns the last Householder QR factored before its trailing block
                          fell to rounding level (l when it ran to the end; 0 if none ran):
                          a numerical-rank estimate of the sample, rounded up to 16 */
  int qr_kflop;        /* algorithmic work of all Householder QRs of this matrix, in units of
                          1000 flops: per QR of a rows x c sample stopped after r reflectors,
                          with Q formed on qc columns, f(c) + f(qc), f(x) = 4 rows x r -
                          2 (rows + x) r^2 + 4 r^3 / 3 (the standard factorization and
                          explicit-Q counts) */
  int jacobi_pairs;    /* row pairs whose inner product the Jacobi SVD formed (all sweeps) */
  int cg_iterations;   /* rsvd_truncate_backward_batched: conjugate-gradient iterations in which
                          a column was still active (both sides); 0 elsewhere */
} rsvd_info;

/*
 * rsvd_gaussian - Alg. RSVD step 1 (Sec. II.B): the n-by-l standard normal
 * test matrix Omega, FP64, row-major with leading dimension ld >= l.
 * Element (r, c) has linear index e = c*n + r (columns nest as l grows); it is
 * slot e % 4 of the Philox4x64-10 block with counter (e / 4, 0, 0, 0) and key
 * (seed, stream), mapped to a normal by the Box-Muller transform
 * (u = ((w >> 11) + 1/2) 2^-53; slots 0/1 = cos/sin of words 0,1; 2/3 of words 2,3).
 * Errors: RSVD_ERR_INVALID_SIZE (n < 1, l < 1, ld < l), RSVD_ERR_NULL_POINTER.
 */
int rsvd_gaussian(int n, int l, uint64_t seed, uint64_t stream, double* omega, int ld, void* cuda_stream);

/*
 * rsvd_workspace_size - bytes of device workspace rsvd_truncate needs for an
 * m-by-n matrix with parameters p (256-byte aligned base required).
 */
int rsvd_workspace_size(int m, int n, const rsvd_params* p, size_t* bytes);

/*
 * rsvd_truncate - Alg. RSVD (Sec. II.B) returning the rank-k truncated SVD
 * A ~ U diag(S) V^T of one m-by-n matrix.
 *   A    [in]  device, m x n, lda >= n; double (RSVD_F64), float (RSVD_F32,
 *              RSVD_TF32) or bfloat16 (RSVD_BF16)
 *   S    [out] device, k doubles, descending
 *   U    [out] device, m x k, ldu >= k, double for RSVD_F64 else float; orthonormal columns
 *   Vt   [out] device, k x n, ldvt >= n, type of U; orthonormal rows,
 *        except that rows of numerically negligible singular values
 *        (sigma_i <= 2^-52 sigma_1, below the rounding level of any FP64
 *        method) are orthogonal to the other rows but not to each other;
 *        a row whose singular value is exactly 0 is returned as 0
 *   work [tmp] device workspace of rsvd_workspace_size bytes, 256-byte aligned
 *   info [out] device, one rsvd_info
 * Errors: RSVD_ERR_INVALID_SIZE, RSVD_ERR_NULL_POINTER, RSVD_ERR_PRECISION,
 * RSVD_ERR_WORKSPACE (host checks, nothing launched); RSVD_ERR_LAUNCH.
 */
int rsvd_truncate(int m, int n, const void* A, int lda, const rsvd_params* p,
                  double* S, void* U, int ldu, void* Vt, int ldvt,
                  void* work, size_t work_bytes, rsvd_info* info, void* cuda_stream);

/*
 * rsvd_batched_workspace_size - workspace bytes of rsvd_truncate_batched for
 * `batch` matrices of sizes m[b] x n[b] at trial ranks k[b] (host arrays).
 */
int rsvd_batched_workspace_size(int batch, const int* m, const int* n, const int* k,
                                const rsvd_params* p, size_t* bytes);

/*
 * rsvd_truncate_batched - Alg. RSVD on `batch` independent matrices of
 * possibly different sizes, in one sequence of launches (Sec. III.A: the
 * blocks of a block-diagonal bond matrix, or the bonds of one TEBD layer).
 * All size / leading-dimension / pointer arrays are HOST arrays of length
 * batch; the pointers they hold are device pointers.  Matrix b is compressed
 * at trial rank k[b] with Philox stream p->stream + b; S[b] holds k[b]
 * doubles, U[b] is m[b] x k[b], Vt[b] is k[b] x n[b].
 * chi_global > 0: after the factorizations, the chi_global largest singular
 * values over all matrices are selected (ties: lower matrix index, then lower
 * position) and k_out[b] (DEVICE int array) receives how many of matrix b's
 * values are kept; the leading k_out[b] triplets of each matrix are the kept
 * ones.  chi_global == 0: k_out may be NULL; nothing is selected.
 * info: DEVICE array of `batch` records.
 * Batches above 64 matrices (16 for RSVD_BF16 / RSVD_TF32) are processed in
 * chunks that run concurrently on four chunk streams of the library, forked
 * from cuda_stream and joined back to it (so the call stays ordered on
 * cuda_stream and can be captured); RSVD_FLAG_SERIAL keeps the chunks in order
 * on cuda_stream, with bit-identical results.  The first chunked call from a
 * host thread on a device creates that thread's chunk streams and their
 * side streams (cudaStreamCreate, cudaEventCreate; no device memory).
 * Errors as rsvd_truncate.
 */
int rsvd_truncate_batched(int batch, const int* m, const int* n, const void* const* A, const int* lda,
                          const int* k, const rsvd_params* p,
                          double* const* S, void* const* U, const int* ldu, void* const* Vt, const int* ldvt,
                          int chi_global, int* k_out,
                          void* work, size_t work_bytes, rsvd_info* info, void* cuda_stream);

/*
 * tebd_workspace_size - workspace bytes of tebd_bond_update for up to nb
 * bonds of an MPS with bond dimensions D (host array, L + 1 entries).
 */
int tebd_workspace_size(int L, int d, const int* D, int nb, const rsvd_params* p, size_t* bytes);

/*
 * tebd_bond_update - TEBD "block update" (Sec. III.A) of nb independent bonds
 * of one Trotter layer, FP64, in place on a device-resident MPS.
 * MPS layout (right-canonical B tensors, Schmidt values on the virtual bonds):
 *   B    device, L tensors; tensor i is D[i] x d x D[i+1] (row-major, index
 *        order (a, s, b)) starting at B + i * tensor_stride doubles.
 *   lam  device, L + 1 vectors; vector j (D[j] entries) starts at
 *        lam + j * lam_stride doubles; lam[0] = lam[L] = {1}.
 *   D    HOST array of the L + 1 bond dimensions (D[0] = D[L] = 1).
 *   bond HOST array of the nb left sites i (0 <= i < L-1, pairwise |i-j| >= 2).
 *   gate device, nb gates, gate b is d^2 x d^2 row-major ((s1 s2), (t1 t2)) at
 *        gate + b * d^4.
 * Per bond i, with k = D[i+1]:
 *   theta_B = gate . (B[i] B[i+1]);  theta = lam[i] (row scaling) theta_B,
 *   reshaped (D[i] d) x (d D[i+2]);  (U, S, V^T) = RSVD(theta, k, p, q);
 *   B[i+1] <- V^T;  B[i] <- theta_B V / ||S||;  lam[i+1] <- S / ||S||;
 *   trunc_err[b] (device) <- 1 - ||S||^2 / ||theta||_F^2 (discarded weight).
 * Bond b uses Philox stream p->stream + bond[b].  p->prec must be RSVD_F64.
 * The contraction B[i] B[i+1] runs over the nonzero entries of lam[i+1] only
 * (sorted, zeros last): in right-canonical form B[i] = Gamma[i] lam[i+1], so
 * the columns of B[i] that belong to a zero Schmidt value are zero.
 * info: DEVICE array of nb records.
 * Errors: RSVD_ERR_INVALID_SIZE, RSVD_ERR_NULL_POINTER, RSVD_ERR_PRECISION,
 * RSVD_ERR_WORKSPACE, RSVD_ERR_LAUNCH.
 */
int tebd_bond_update(int L, int d, const int* D, int nb, const int* bond,
                     double* B, size_t tensor_stride, double* lam, size_t lam_stride,
                     const double* gate, const rsvd_params* p, double* trunc_err,
                     void* work, size_t work_bytes, rsvd_info* info, void* cuda_stream);

/*
 * tebd_product_workspace_size - workspace bytes of tebd_product_update for up
 * to nb bonds with K operator pairs per gate.
 */
int tebd_product_workspace_size(int L, int d, const int* D, int nb, int K, const rsvd_params* p, size_t* bytes);

/*
 * tebd_product_update - TEBD "product update" (Sec. III.A, P) of nb
 * independent bonds, FP64, in place on the MPS of tebd_bond_update (same B,
 * lam, D, bond layout and rules).  The gate of bond b is the sum of K
 * Kronecker products of single-site operators, sum_k uL[k] (x) uR[k]:
 *   uL, uR  device, nb x K x d x d row-major; operator k of bond b starts at
 *           uL + (b K + k) d^2, element [s, t] acting as s <- t.
 * Per bond i, with k = D[i+1] and r = K k:
 *   XB[(a,s1),(k',b)] = sum_t uL[k'][s1,t] B[i][a,t,b];  X = lam[i] (rows) XB
 *   Y[(k',b),(s2,c)]  = sum_t uR[k'][s2,t] B[i+1][b,t,c]
 *   theta = X Y ((D[i] d) x (d D[i+2]), never formed: every product of Alg.
 *   RSVD with theta is two products through an r x l buffer);
 *   (S, V^T) = RSVD(theta, k, p, q);  B[i+1] <- V^T;  B[i] <- XB (Y V) / ||S||;
 *   lam[i+1] <- S / ||S||;  trunc_err[b] <- 1 - ||S||^2 / ||theta||_F^2 with
 *   ||theta||_F^2 = trace((X^T X)(Y Y^T)).
 * Alg. RSVD of X Y equals Alg. RSVD of the paper's r x (d D[i+2]) matrix R Y
 * (X = Q_X R) with the same Omega: the samples differ by the isometry Q_X and
 * B = Q^T A is the same matrix.  Bond b uses Philox stream p->stream + bond[b].
 * Errors: RSVD_ERR_INVALID_SIZE, RSVD_ERR_NULL_POINTER, RSVD_ERR_PRECISION
 * (p->prec must be RSVD_F64), RSVD_ERR_WORKSPACE, RSVD_ERR_LAUNCH.
 */
int tebd_product_update(int L, int d, const int* D, int nb, const int* bond, double* B, size_t tensor_stride,
                        double* lam, size_t lam_stride, int K, const double* uL, const double* uR,
                        const rsvd_params* p, double* trunc_err, void* work, size_t work_bytes, rsvd_info* info,
                        void* cuda_stream);

/*
 * rsvd_factored_workspace_size - workspace bytes of rsvd_truncate_factored.
 */
int rsvd_factored_workspace_size(int m, int r, int n, const rsvd_params* p, size_t* bytes);

/*
 * rsvd_truncate_factored - Alg. RSVD of a matrix given as the product A = X Y
 * (Sec. II.A: A may be the contraction of two tensors), without forming A:
 * X (m x r, ldx) and Y (r x n, ldy) row-major device matrices of p->prec
 * (RSVD_F64 or RSVD_F32); every product with A or A^T is two products through
 * an r x l buffer (cost 2 (m + n) r l instead of 2 m n l).  Outputs as for
 * rsvd_truncate (S, U m x k, V^T k x n; same sign rule, Philox stream
 * p->stream).  The sampled path is taken for every m (no Q = I shortcut).
 * Errors: RSVD_ERR_INVALID_SIZE, RSVD_ERR_NULL_POINTER, RSVD_ERR_PRECISION,
 * RSVD_ERR_WORKSPACE, RSVD_ERR_LAUNCH.
 */
int rsvd_truncate_factored(int m, int r, int n, const void* X, int ldx, const void* Y, int ldy, const rsvd_params* p,
                           double* S, void* U, int ldu, void* Vt, int ldvt, void* work, size_t work_bytes,
                           rsvd_info* info, void* cuda_stream);

/*
 * rsvd_sectors_adaptive_workspace_size - workspace bytes of
 * rsvd_truncate_sectors_adaptive (ranks up to min(chi, m_b, n_b)).
 */
int rsvd_sectors_adaptive_workspace_size(int batch, const int* m, const int* n, int chi, const rsvd_params* p,
                                         size_t* bytes);

/*
 * rsvd_truncate_sectors_adaptive - block-wise Alg. RSVD of a block-diagonal
 * matrix with the global post-selection of the chi largest singular values
 * (Sec. III.A), with per-block trial ranks found adaptively instead of guessed
 * (the alternative route to the sector sizes that Sec. V proposes): after each
 * selection, a block all of whose k'_b values were kept while
 * k'_b < min(chi, m_b, n_b) may hold more values above the cut, so its trial
 * rank is doubled (capped there) and only that block is compressed again (same
 * Philox stream p->stream + b: its larger test matrix extends the previous
 * one); until no block of the last round is saturated (a block left out of a
 * round is not looked at again).  Each round ends with one device-to-host
 * read of the kept counts and a synchronisation of the stream.
 *   batch <= 64 blocks; A[b] (m_b x n_b, lda[b]) of p->prec (RSVD_F64 or
 *   RSVD_F32);  k_trial  HOST in/out: first guesses, on return the final trial
 *   ranks (an estimate for the next call);  S[b] (min(chi, m_b, n_b)), U[b]
 *   (ldu[b] >= that), Vt[b] as for rsvd_truncate_batched;  k_out  DEVICE
 *   int[batch], the kept counts;  rounds  HOST, the number of rounds.
 * Errors: RSVD_ERR_INVALID_SIZE, RSVD_ERR_NULL_POINTER, RSVD_ERR_PRECISION,
 * RSVD_ERR_WORKSPACE, RSVD_ERR_LAUNCH.
 */
int rsvd_truncate_sectors_adaptive(int batch, const int* m, const int* n, const void* const* A, const int* lda,
                                   int* k_trial, const rsvd_params* p, int chi, double* const* S, void* const* U,
                                   const int* ldu, void* const* Vt, const int* ldvt, int* k_out, int* rounds,
                                   void* work, size_t work_bytes, rsvd_info* info, void* cuda_stream);

/*
 * rsvd_complex_workspace_size - workspace bytes of rsvd_truncate_complex.
 */
int rsvd_complex_workspace_size(int m, int n, const rsvd_params* p, size_t* bytes);

/*
 * rsvd_truncate_complex - Alg. RSVD (Sec. II.B) of a complex m-by-n matrix (the paper
 * runs its simulations in complex double, Sec. IV): A ~ U diag(S) V^H with a real
 * Gaussian test matrix Omega (n x l, the one of rsvd_gaussian with key (seed, stream)),
 * every transpose a conjugate transpose, and the phase rule in place of the sign rule:
 * the entry of largest modulus of u_i (lowest row index on ties) is real and positive,
 * row i of V^H taking the conjugate phase so that u_i s_i v_i^H is unchanged.
 *   A   [in]  device, m x n complex, interleaved (re, im) pairs, row-major, lda >= n
 *             (complex elements); double (RSVD_F64) or float (RSVD_F32)
 *   S   [out] device, k doubles, descending
 *   U   [out] device, m x k complex (ldu >= k), orthonormal columns
 *   Vh  [out] device, k x n complex (ldvh >= n): V^H, orthonormal rows
 * Computed through the real embedding R(A) = [Re A, -Im A; Im A, Re A] (2m x 2n; the
 * same products, orthonormalisations and Jacobi SVD as rsvd_truncate, with the test
 * matrix diag(Omega, Omega)): its singular values are those of A twice, and its sampled
 * subspaces are the realifications of the complex algorithm's, so the results agree with
 * the complex algorithm in exact arithmetic.  Flags as rsvd_truncate
 * (RSVD_FLAG_FULL_SVD: Alg. TSVD of A on the same engine, m <= 512).
 * Errors: RSVD_ERR_INVALID_SIZE, RSVD_ERR_NULL_POINTER, RSVD_ERR_PRECISION (tensor-core
 * precisions), RSVD_ERR_WORKSPACE, RSVD_ERR_LAUNCH.
 */
int rsvd_truncate_complex(int m, int n, const void* A, int lda, const rsvd_params* p, double* S, void* U, int ldu,
                          void* Vh, int ldvh, void* work, size_t work_bytes, rsvd_info* info, void* cuda_stream);

/*
 * rsvd_truncate_sectors_adaptive_device - rsvd_truncate_sectors_adaptive with the rounds
 * decided on the device: no host synchronisation, so the whole call can be captured in a
 * CUDA graph (the batching form of a symmetry-sector bond).  Round r compresses, at the
 * scheduled rank min(k_first[b] 2^r, cap_b), every block that is still active; a block is
 * active in round 0 and stays active while all of its values were kept by the round's
 * global selection and its rank is below cap_b = min(chi, m_b, n_b).  Every launch of a
 * round is enqueued up front and each block's work is gated by its device flag (an
 * inactive block's launches return at once), so the results are those of
 * rsvd_truncate_sectors_adaptive up to the summation order (the cluster sizes follow the
 * number of blocks enqueued per round).
 *   k_first  HOST: first guesses;  k_out, k_final, rounds  DEVICE: the kept counts, the
 *   final trial ranks, the number of rounds in which a block was compressed.  S[b], U[b]
 *   and Vt[b] hold k_final[b] values and vectors (entries past it are not written).
 *   Workspace: rsvd_sectors_adaptive_workspace_size.  Other arguments as
 *   rsvd_truncate_sectors_adaptive.
 * Errors as rsvd_truncate_sectors_adaptive.
 */
int rsvd_truncate_sectors_adaptive_device(int batch, const int* m, const int* n, const void* const* A, const int* lda,
                                          const int* k_first, const rsvd_params* p, int chi, double* const* S,
                                          void* const* U, const int* ldu, void* const* Vt, const int* ldvt, int* k_out,
                                          int* k_final, int* rounds, void* work, size_t work_bytes, rsvd_info* info,
                                          void* cuda_stream);

/*
 * rsvd_tol_workspace_size - workspace bytes of rsvd_truncate_tol.
 */
int rsvd_tol_workspace_size(int m, int n, int k_max, const rsvd_params* p, size_t* bytes);

/*
 * rsvd_truncate_tol - fixed-error Alg. RSVD (the fixed-error form proposed in
 * Sec. V): the smallest rank k <= min(k_max, m, n) with
 * ||A - U diag(S) V^T||_F <= eps ||A||_F, FP64 (p->prec = RSVD_F64).
 * The error of the rank-k result Q B_k (B = Q^T A) is exact from the sample:
 * Q Q^T is an orthogonal projector, so ||A - Q B_k||_F^2 = ||A - Q B||_F^2 +
 * sum_{i>k} s_i(B)^2; the residual A - Q B is formed on the device.  Trial
 * ranks p->k, 2 p->k, 4 p->k, ... (capped), each a full Alg. RSVD with
 * l = min(k + p->p, m, n) and the same Philox stream, so the test matrix of a
 * larger trial extends the previous one.  Each trial ends with one
 * device-to-host read of the decision and a synchronisation of the stream.
 *   A   device, m x n row-major (lda);  S (k_max), U (m x k_max, ldu >=
 *       min(k_max, m, n)), Vt (k_max x n, ldvt): device outputs, of which the
 *       first *k_out singular values / columns of U / rows of V^T are the result.
 *   k_out, err_out  HOST: the rank and ||A - U S V^T||_F / ||A||_F (0 for
 *       A = 0).  When no k up to the cap reaches eps, k_out is the cap and
 *       err_out > eps (the return code is still RSVD_OK).
 *   info  device record of the last trial.
 * Errors: RSVD_ERR_INVALID_SIZE (also eps < 0 or NaN), RSVD_ERR_NULL_POINTER,
 * RSVD_ERR_PRECISION, RSVD_ERR_WORKSPACE, RSVD_ERR_LAUNCH.
 */
int rsvd_truncate_tol(int m, int n, const double* A, int lda, double eps, int k_max, const rsvd_params* p, double* S,
                      double* U, int ldu, double* Vt, int ldvt, int* k_out, double* err_out, void* work,
                      size_t work_bytes, rsvd_info* info, void* cuda_stream);

/*
 * rsvd_gemm_f64_tc - the FP64 tensor-core product of the FP64 path (exposed so
 * that it can be verified on its own): C = A B^T with A (M x K, lda), B (N x K,
 * ldb) and C (M x N, ldc) row-major FP64 device matrices, N <= 256, K <= 1024.
 * Every row of A and of B is split exactly into nine BF16 slices of 6-bit
 * integers relative to the row's power-of-two exponent (only bits below
 * 2^-54 of the row's largest magnitude are dropped); the slice products are
 * summed exactly by tcgen05.mma in FP32 tensor memory, level by level over
 * chunks of at most 256 values of K, and the levels of all chunks in FP64.
 * The FP64 path of rsvd_truncate / tebd_bond_update takes this product for
 * the products with A when m, n <= 1024 and l <= 256.  Error: at most about 2.3 K 2^-53 max|A_r| max|B_c| per
 * entry (the normwise class of an FP64 GEMM).  A row holding Inf or NaN gives
 * NaN.
 * work: device workspace of rsvd_gemm_f64_tc_workspace_size(M, N, K) bytes
 * (256-byte aligned).  err (device int, may be NULL) as for rsvd_gemm_tc.
 * Errors: RSVD_ERR_INVALID_SIZE, RSVD_ERR_NULL_POINTER, RSVD_ERR_WORKSPACE,
 * RSVD_ERR_LAUNCH.
 */
size_t rsvd_gemm_f64_tc_workspace_size(int M, int N, int K);
int rsvd_gemm_f64_tc(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                     void* work, size_t work_bytes, int* err, void* cuda_stream);

/*
 * rsvd_gemm_tc - the tensor-core product of the mixed-precision path (exposed
 * so that it can be verified on its own): C = A B^T with A (M x K, lda) and B
 * (N x K, ldb) row-major device matrices of bfloat16 (RSVD_BF16) or float read
 * as TF32 (RSVD_TF32), C (M x N, ldc) float.  tcgen05.mma with TMEM
 * accumulation, TMA-fed; N <= 256.  A, B must be 16-byte aligned with
 * lda * element size and ldb * element size multiples of 16 bytes.  err
 * (device int, may be NULL) is set to 1 if a pipeline wait timed out (every
 * wait gives up after about one second; the kernel then finishes and C is
 * invalid).  test_flags: 0, or 1 to issue no loads at all - the waits run out
 * and err reports it (a test of that failure path; nothing faults or hangs).
 * Errors: RSVD_ERR_PRECISION, RSVD_ERR_INVALID_SIZE (also for a layout TMA
 * cannot describe), RSVD_ERR_NULL_POINTER, RSVD_ERR_LAUNCH.
 */
int rsvd_gemm_tc(int M, int N, int K, int prec, const void* A, int lda, const void* B, int ldb, float* C, int ldc,
                 int* err, int test_flags, void* cuda_stream);

/*
 * rsvd_backward_workspace_size - workspace bytes of rsvd_truncate_backward_batched.
 */
int rsvd_backward_workspace_size(int batch, const int* m, const int* n, const int* k, int prec, size_t* bytes);

/*
 * rsvd_truncate_backward_batched - derivative of the rank-k truncated
 * factorization A ~ U diag(S) V^T (the differentiable form of the compression
 * step; the paper itself has no derivative).  Given the factors of each matrix
 * and the cotangents (Ubar, Sbar, Vbar) of a scalar loss with respect to them,
 * writes Abar = d loss / d A:
 *   Abar = U [ (F o (U^T Ubar - Ubar^T U)) S + diag(Sbar) + S (F o (V^T Vbar - Vbar^T V)) ] V^T
 *        + Z S V^T + U Z^T A + U S Y^T + A Y V^T,
 *   F_ij = 1 / (s_j^2 - s_i^2) (i != j, the retained block),
 *   z_i = (s_i^2 I - P A A^T P)^-1 P ubar_i,  y_i = (s_i^2 I - Q A^T A Q)^-1 Q vbar_i,
 *   P = I - U U^T, Q = I - V V^T.
 * The z / y terms carry the coupling to the discarded singular triplets without
 * forming them; they are solved by conjugate gradients on the device (all k
 * columns at once, up to max_iter iterations, a column stopping when its
 * residual is below tol times its right-hand side).  This equals the adjoint
 * of the full SVD with zero cotangents on the discarded triplets, and requires
 * the retained singular values to be distinct and above every discarded one.
 *   prec: RSVD_F64 (all double) or RSVD_F32 (A, U, Vt, cotangents and Abar float,
 *         products in FP32).
 *   A[b] m x n (lda), S[b] k doubles, U[b] m x k (ldu), Vt[b] k x n (ldvt): the
 *         factors (e.g. from rsvd_truncate_batched).
 *   Ubar, Sbar, Vtbar: HOST arrays of device pointers (m x k with ldub, k
 *         doubles, k x n with ldvb - the cotangent of Vt); a NULL array means a
 *         zero cotangent for every matrix.
 *   Abar[b] [out] m x n (ldab).
 *   info: DEVICE array of batch records; status RSVD_WARN_CG when a column did
 *         not converge or met non-positive curvature.
 * Errors: RSVD_ERR_INVALID_SIZE, RSVD_ERR_NULL_POINTER, RSVD_ERR_PRECISION,
 * RSVD_ERR_WORKSPACE, RSVD_ERR_LAUNCH.
 */
int rsvd_truncate_backward_batched(int batch, const int* m, const int* n, const int* k, int prec,
                                   const void* const* A, const int* lda, const double* const* S,
                                   const void* const* U, const int* ldu, const void* const* Vt, const int* ldvt,
                                   const void* const* Ubar, const int* ldub, const double* const* Sbar,
                                   const void* const* Vtbar, const int* ldvb,
                                   void* const* Abar, const int* ldab, int max_iter, double tol,
                                   void* work, size_t work_bytes, rsvd_info* info, void* cuda_stream);

/*
 * rsvd_truncate_noalloc - rsvd_truncate for callers that cannot allocate or
 * own a device workspace: code that runs where device allocation is forbidden
 * or unavailable after start-up (a host framework that owns and pre-reserves
 * all device memory, a real-time loop with a fixed memory budget, a plain C
 * caller without an allocator).  The paper has no counterpart; this is a
 * deployment variant of rsvd_truncate with identical arguments and results,
 * minus the workspace.
 *   Scratch: a fixed 16 MiB array inside the library's device image
 *   (rsvd_noalloc_scratch_bytes), present on every GPU that loads the library
 *   until the process exits.  FP64 products with A on the tensor cores need
 *   the slices of A and A^T (up to about 480 x 480 at l = 144 within 16 MiB);
 *   when they do not fit, the call takes the FP64-FMA products
 *   (RSVD_FLAG_F64_SIMT, the same factorization within the FP64 bar), which
 *   fit up to about 1280 x 1280 at l = 144.  A matrix that does not fit either
 *   way is rejected with RSVD_ERR_SCRATCH_LIMIT before anything is launched.
 *   No cudaMalloc, cudaFree or other allocating call is made.  The first call
 *   on a device looks up the array's device address (cudaGetSymbolAddress,
 *   with that device current) and caches it (looked up again after the
 *   device's context was replaced, e.g. by cudaDeviceReset); the first call
 *   from each host thread on a device also creates that thread's side streams
 *   and events for the call's independent groups of work (cudaStreamCreate,
 *   cudaEventCreate: no device memory).  Make the first call from every
 *   thread before any stream capture.
 *   All calls share the one array and it keeps the previous call's contents
 *   (every word a call reads it has written itself first): calls whose work
 *   overlaps on the GPU - different streams, or host threads issuing at once -
 *   race on it and must be serialised by the caller.
 * Errors: as rsvd_truncate, plus RSVD_ERR_SCRATCH_LIMIT.
 */
int rsvd_truncate_noalloc(int m, int n, const void* A, int lda, const rsvd_params* p,
                          double* S, void* U, int ldu, void* Vt, int ldvt,
                          rsvd_info* info, void* cuda_stream);

/* rsvd_noalloc_scratch_bytes - size of rsvd_truncate_noalloc's fixed scratch array. */
size_t rsvd_noalloc_scratch_bytes(void);

/*
 * Optional kernel timing (measurement aid, not part of the method).
 * rsvd_profile_enable(n): from now on, CUDA events are recorded on the
 * launching stream around each of up to n kernel launches of this library
 * (n <= 0 disables and releases the events).  Not thread-safe.
 * rsvd_profile_collect(ms, launches, nclass): waits for the recorded events,
 * adds each launch's duration (ms) and count to ms[c] / launches[c] for its
 * kernel class c < nclass (host arrays), clears the records and returns the
 * number of classes; classes are named by rsvd_profile_class_name.
 */
int rsvd_profile_enable(int max_launches);
int rsvd_profile_collect(double* ms, int* launches, int nclass);
const char* rsvd_profile_class_name(int cls);

/*
 * Tile autotuner of the batched SIMT products (FP64 and FP32 GEMMs of every entry
 * point; a measurement-driven choice, not part of the method).  The library keeps a
 * host cache of tile choices keyed by the launch's shape class (types, transposes,
 * batch size, largest M, N, K rounded up to 16).  rsvd_autotune_enable(1): from now
 * on a launch whose class is not cached yet times every candidate tile (CUDA events,
 * synchronising the host; never while its stream is being captured, and not for
 * products that accumulate into their output) and caches the fastest; (0) stops
 * tuning.  Cached choices are always used, inside graph captures too.  The choice
 * changes no result: every tile sums each output over K in the same order.
 * rsvd_autotune_entries: cached classes; rsvd_autotune_clear: empties the cache;
 * rsvd_autotune_save / _load: the cache as a text file (load returns the entries read,
 * or RSVD_ERR_INVALID_SIZE if the file cannot be opened).  Thread-safe.
 */
int rsvd_autotune_enable(int on);
int rsvd_autotune_entries(void);
int rsvd_autotune_clear(void);
int rsvd_autotune_save(const char* path);
int rsvd_autotune_load(const char* path);

/* rsvd_status_string - static description of a status code (never NULL). */
const char* rsvd_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* RSVD_H */
