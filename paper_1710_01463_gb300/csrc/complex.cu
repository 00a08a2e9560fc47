// Complex matrices (the paper's simulations run in complex double, Sec. IV) through
// their real embedding: A = X + iY (m x n) is mapped to the real 2m x 2n matrix
//
//   R(A) = [ X  -Y ]
//          [ Y   X ]
//
// whose singular values are those of A, each twice, and whose singular pairs
// (x, y) with R(A) y = s x are the realifications of complex pairs: A (y1 + i y2)
// = s (x1 + i x2).  Alg. RSVD of A with a real test matrix Omega is Alg. RSVD of
// R(A) with the test matrix diag(Omega, Omega): every product, conjugate
// transpose (R(A^H) = R(A)^T) and orthonormalisation of the complex algorithm
// maps to the real one, and the real bases span the realifications of the complex
// ones, so the sampled singular values agree in exact arithmetic.  The real engine
// (FP64 products on the tensor cores by exact slicing, CholeskyQR2 / Householder,
// the cluster Jacobi SVD) runs unchanged; these kernels only embed A and extract
// the complex factors: of each pair of equal singular values the first column of
// U and row of V^T give the complex u_i and v_i, with the phase rule applied.
#include "common.cuh"

namespace rsvd {

namespace {

// one thread per complex element: R[r][c] = X, R[r][n+c] = -Y, R[m+r][c] = Y, R[m+r][n+c] = X
template <typename T>
__global__ void __launch_bounds__(256) realify_kernel(int m, int n, const T* __restrict__ A, int lda,
                                                      T* __restrict__ R) {
  const long long tot = (long long)m * n;
  const long long ld = 2LL * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / n, c = e - r * n;
    const T x = A[2 * (r * lda + c)], y = A[2 * (r * lda + c) + 1];
    R[r * ld + c] = x;
    R[r * ld + n + c] = -y;
    R[(m + r) * ld + c] = y;
    R[(m + r) * ld + n + c] = x;
  }
}

// One block per retained triplet i: u = (column 2i of U_R, rows 0..m-1) + i (rows m..2m-1),
// v likewise from row 2i of V_R^T; the entry of largest modulus of u (lowest index on
// ties, moduli compared in FP64) is made real and positive, and V^H's row i takes the
// conjugate phase so that u_i s_i v_i^H is unchanged.
template <typename T>
__global__ void __launch_bounds__(256) complex_extract_kernel(int m, int n, const double* __restrict__ Sr,
                                                              const T* __restrict__ Ur, int ldur,
                                                              const T* __restrict__ Vtr, int ldvr, double* S, T* U,
                                                              int ldu, T* Vh, int ldvh) {
  const int i = blockIdx.x, c = 2 * i;
  __shared__ double bm[256];
  __shared__ int bj[256];
  double best = -1.0;
  int bidx = 0;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    const double a = (double)Ur[(size_t)r * ldur + c], b = (double)Ur[(size_t)(m + r) * ldur + c];
    const double v = a * a + b * b;
    if (v > best) {  // rows visited in increasing order: the first maximum is kept
      best = v;
      bidx = r;
    }
  }
  bm[threadIdx.x] = best;
  bj[threadIdx.x] = bidx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const double o = bm[threadIdx.x + w];
      const int oj = bj[threadIdx.x + w];
      if (o > bm[threadIdx.x] || (o == bm[threadIdx.x] && oj < bj[threadIdx.x])) {
        bm[threadIdx.x] = o;
        bj[threadIdx.x] = oj;
      }
    }
    __syncthreads();
  }
  const int j = bj[0];
  const double xr = (double)Ur[(size_t)j * ldur + c], xi = (double)Ur[(size_t)(m + j) * ldur + c];
  const double mod = sqrt(xr * xr + xi * xi);
  const double pr = mod > 0.0 ? xr / mod : 1.0, pi = mod > 0.0 ? xi / mod : 0.0;  // the phase of u_j
  for (int r = threadIdx.x; r < m; r += blockDim.x) {  // u / ph = u conj(ph)
    const double a = (double)Ur[(size_t)r * ldur + c], b = (double)Ur[(size_t)(m + r) * ldur + c];
    U[2 * ((size_t)r * ldu + i)] = (T)(a * pr + b * pi);
    U[2 * ((size_t)r * ldu + i) + 1] = (T)(b * pr - a * pi);
  }
  for (int q = threadIdx.x; q < n; q += blockDim.x) {  // conj(v) ph
    const double a = (double)Vtr[(size_t)c * ldvr + q], b = -(double)Vtr[(size_t)c * ldvr + n + q];
    Vh[2 * ((size_t)i * ldvh + q)] = (T)(a * pr - b * pi);
    Vh[2 * ((size_t)i * ldvh + q) + 1] = (T)(a * pi + b * pr);
  }
  if (threadIdx.x == 0) S[i] = Sr[c];
}

}  // namespace

template <typename T>
cudaError_t launch_realify(int m, int n, const T* A, int lda, T* R, cudaStream_t s) {
  const long long tot = (long long)m * n;
  const int gx = (int)std::min<long long>(4096, (tot + 255) / 256);
  prof_begin(KC_CONVERT, s);
  realify_kernel<T><<<gx, 256, 0, s>>>(m, n, A, lda, R);
  prof_end(KC_CONVERT, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_complex_extract(int m, int n, int k, const double* Sr, const T* Ur, int ldur, const T* Vtr,
                                   int ldvr, double* S, T* U, int ldu, T* Vh, int ldvh, cudaStream_t s) {
  prof_begin(KC_CONVERT, s);
  complex_extract_kernel<T><<<k, 256, 0, s>>>(m, n, Sr, Ur, ldur, Vtr, ldvr, S, U, ldu, Vh, ldvh);
  prof_end(KC_CONVERT, s);
  return cudaGetLastError();
}

template cudaError_t launch_realify<double>(int, int, const double*, int, double*, cudaStream_t);
template cudaError_t launch_realify<float>(int, int, const float*, int, float*, cudaStream_t);
template cudaError_t launch_complex_extract<double>(int, int, int, const double*, const double*, int, const double*,
                                                    int, double*, double*, int, double*, int, cudaStream_t);
template cudaError_t launch_complex_extract<float>(int, int, int, const double*, const float*, int, const float*, int,
                                                   double*, float*, int, float*, int, cudaStream_t);

}  // namespace rsvd
