// C ABI of librsvd (declarations and contracts in include/rsvd.h).
//
// Host side: argument checks, workspace layout, and the launch sequence of
// Alg. RSVD (Sec. II.B) for a batch of matrices.  Every step runs in the
// kernels of this library; the host only enqueues launches on the caller's
// stream and never synchronises, so a whole call can be captured in a CUDA
// graph.  Matrices of a batch are processed together, kMaxJobs per launch.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"

namespace rsvd {

cudaError_t& last_cuda_error() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}

namespace {

constexpr int kMaxSample = 1024;  // largest sample width l supported


struct Prob {
  int m, n, k, l;
  int exact;
  int want_u;
  const void* A;
  int lda;
  double* S;
  void* U;
  int ldu;
  void* Vt;
  int ldvt;
  unsigned long long seed, stream;
  rsvd_info* info;
  int max_sweeps;
  int no_exchange;  // RSVD_FLAG_TEST_NO_EXCHANGE
  int serial;       // RSVD_FLAG_SERIAL: independent groups one after another on the caller's stream
  int cplx;         // the real embedding of a complex matrix: Omega enters as diag(Omega, Omega)
  const int* active;  // device flag (null: always): every launch of this matrix runs only while it is set
  // workspace
  void *Y0, *Y1, *Z0, *Z1, *Rinv, *Ps;
  double *G, *part, *hw, *hq, *Bm, *Bg, *Pg, *sig;
  int* flag;
  int csize, use_global;
  // tensor-core path: A^T, Omega^T / Z^T, Q^T in the operand precision
  void *At, *WT, *QT;
  int ldAt, ldWT, ldQT;
  // wide B (n >= 3 l): B^T = Q_b R first, Jacobi on M = B Q_b (l x l)
  int wide;
  double *Bt, *Bt2, *Mb, *RinvD;
  void *Wb, *Qbt;
  // FP64 products with A on the tensor cores (exact slicing): slices of A
  // (m rows, K = n), of A^T (n rows, K = m) and of the thin operand's columns
  int oz;
  __nv_bfloat16 *SA, *SAt, *SS;
  int *eA, *eAt, *eS;
  int KpA, KpAt, KpS, Npad;
  // A given as the product X Y (X m x r, Y r x n; Sec. II.A): every product with A
  // is two products through W (r x l), and A itself is never formed
  int r;
  const void *Xf, *Yf;
  int ldxf, ldyf;
  void* Wf;
};

inline int pad8(int x) { return (x + 7) / 8 * 8; }

// B (l x n) is "wide" when n >= kWide10 / 10 * l (3 l: measured on TEBD bonds with n / l
// = 1.9, 2.8 and 3.7, only the last gains): its SVD then runs on the l x l
// factor M = B Q_b of an orthonormalisation B^T = Q_b R
constexpr int kWide10 = 30;

// Workspace of one matrix (bytes), with the buffer offsets when `p` is given.
// tc_bytes > 0 (the operand size of the tensor-core precisions) adds A^T
// (n x m), Omega^T / Z^T (l x n) and Q^T (l x m) with 8-element-aligned rows.
size_t layout(Prob* p, int m, int n, int k, int l, size_t tsize, char* base, int tc_bytes = 0, int oz = 0, int r = 0) {
  const int mx = std::max(m, n);
  const int nchunk = ceil_div(mx, kGramChunk);
  const int wide = 10 * n >= kWide10 * l ? 1 : 0;
  const int jn = wide ? l : n;  // columns of the matrix the Jacobi SVD works on
  const int cs = jacobi_cluster_size(l, jn);
  const int glob = jacobi_fits_smem(l, jn, cs) ? 0 : 1;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align_up(bytes);
    return base ? (void*)(base + o) : nullptr;
  };
  void* Y0 = take((size_t)m * l * tsize);
  void* Y1 = take((size_t)m * l * tsize);
  void* Z0 = take((size_t)n * l * tsize);
  void* Z1 = take((size_t)n * l * tsize);
  void* Rinv = take((size_t)l * l * tsize);
  void* Ps = take((size_t)std::max(k, 1) * l * tsize);
  void* G = take((size_t)l * l * 8);
  void* part = take((size_t)nchunk * l * l * 8);
  void* hw = take((size_t)(mx + 16) * l * 8);
  void* hq = take((size_t)(mx + 16) * l * 8);
  void* Bm = take((size_t)l * n * 8);
  void* Bg = take(glob ? (size_t)l * (jn + 16) * 8 : 0);
  void* Pg = take(glob ? (size_t)l * (l + 16) * 8 : 0);
  void* sig = take((size_t)l * 8);
  void* flag = take(sizeof(int) * 4);
  const size_t lop = 2 * (size_t)((l + 15) / 16 * 16);  // rows of a split (hi + lo) operand
  void* At = take(tc_bytes ? (size_t)n * pad8(m) * tc_bytes : 0);
  void* WT = take(tc_bytes ? lop * pad8(n) * tc_bytes : 0);
  void* QT = take(tc_bytes ? lop * pad8(m) * tc_bytes : 0);
  void* Bt = take(wide ? (size_t)n * l * 8 : 0);
  void* Bt2 = take(wide ? (size_t)n * l * 8 : 0);
  void* Mb = take(wide ? (size_t)l * l * 8 : 0);
  void* RinvD = take(wide ? (size_t)l * l * 8 : 0);
  void* Wb = take(wide ? (size_t)std::max(k, 1) * l * tsize : 0);
  void* Qbt = take(wide ? (size_t)l * n * tsize : 0);
  const int KpA = pad8(n), KpAt = pad8(m), KpS = pad8(std::max(m, n)), Npad = (l + 15) / 16 * 16;
  void* SA = take(oz ? (size_t)kOzSlices * m * KpA * 2 : 0);
  void* SAt = take(oz ? (size_t)kOzSlices * n * KpAt * 2 : 0);
  void* SS = take(oz ? (size_t)kOzSlices * Npad * KpS * 2 : 0);
  void* eA = take(oz ? (size_t)m * 4 : 0);
  void* eAt = take(oz ? (size_t)n * 4 : 0);
  void* eS = take(oz ? (size_t)Npad * 4 : 0);
  void* Wf = take(r ? (size_t)r * l * tsize : 0);
  if (p) {
    p->Wf = Wf;
    p->oz = oz;
    p->SA = (__nv_bfloat16*)SA; p->SAt = (__nv_bfloat16*)SAt; p->SS = (__nv_bfloat16*)SS;
    p->eA = (int*)eA; p->eAt = (int*)eAt; p->eS = (int*)eS;
    p->KpA = KpA; p->KpAt = KpAt; p->KpS = KpS; p->Npad = Npad;
    p->At = At; p->WT = WT; p->QT = QT;
    p->ldAt = pad8(m); p->ldWT = pad8(n); p->ldQT = pad8(m);
    p->Y0 = Y0; p->Y1 = Y1; p->Z0 = Z0; p->Z1 = Z1; p->Rinv = Rinv; p->Ps = Ps;
    p->G = (double*)G; p->part = (double*)part; p->hw = (double*)hw; p->hq = (double*)hq;
    p->Bm = (double*)Bm; p->Bg = (double*)Bg; p->Pg = (double*)Pg; p->sig = (double*)sig;
    p->flag = (int*)flag;
    p->csize = cs;
    p->use_global = glob;
    p->wide = wide;
    p->Bt = (double*)Bt; p->Bt2 = (double*)Bt2; p->Mb = (double*)Mb; p->RinvD = (double*)RinvD;
    p->Wb = Wb; p->Qbt = Qbt;
  }
  return off;
}

inline int sample_width(int m, int n, int k, int p) { return std::min(k + p, std::min(m, n)); }
// rows of B: the sample width, or all m rows for Alg. TSVD (RSVD_FLAG_FULL_SVD: B = A)
inline int b_rows(int m, int n, int k, const rsvd_params* p) {
  return (p->flags & RSVD_FLAG_FULL_SVD) ? m : sample_width(m, n, k, p->p);
}

// When the sample spans the whole column space (m <= l), a small matrix skips
// the sampling: Q = I, B = A.  Larger ones keep the sampled path with l = m:
// Q is then square orthogonal (B = Q^T A has A's singular values) and the
// power iteration aligns it with the left singular vectors, so the Jacobi SVD
// of B converges in a few sweeps over its numerically nonzero rows instead of
// many sweeps over all rows of A.
constexpr int kExactMaxRows = 16;
inline int use_exact_path(int m, int l) { return (m <= l && m <= kExactMaxRows) ? 1 : 0; }
inline int exact_of(int m, int l, const rsvd_params* p) {
  return (p->flags & RSVD_FLAG_FULL_SVD) ? 1 : use_exact_path(m, l);
}

// FP64 products with A on the tensor cores: K <= 1024 (K = n for A Z, m for
// A^T Y; exact level sums per chunk of 256) and the thin operand fits one CTA
// row (l <= 256)
inline int use_oz(int m, int n, int l, int exact, const rsvd_params* p) {
  return (p->prec == RSVD_F64 && !(p->flags & RSVD_FLAG_F64_SIMT) && !exact && m <= kOzMaxKTotal &&
          n <= kOzMaxKTotal && l <= 256)
             ? 1
             : 0;
}

#define RSVD_TRY(x)                              \
  do {                                           \
    cudaError_t err__ = (x);                     \
    if (err__ != cudaSuccess) {                  \
      last_cuda_error() = err__;                 \
      return RSVD_ERR_LAUNCH;                    \
    }                                            \
  } while (0)


template <typename T>
OrthBatch<T> orth_batch(const std::vector<Prob*>& ps, bool onY) {
  OrthBatch<T> b;
  b.count = (int)ps.size();
  b.max_chunks = 0;
  b.max_tilepairs = 0;
  b.serial = ps.empty() ? 0 : ps[0]->serial;
  for (size_t i = 0; i < ps.size(); ++i) {
    Prob& p = *ps[i];
    OrthJob<T>& J = b.job[i];
    J.rows = onY ? p.m : p.n;
    J.l = p.l;
    J.Y = (T*)(onY ? p.Y0 : p.Z0);
    J.Y1 = (T*)(onY ? p.Y1 : p.Z1);
    J.part = p.part;
    J.G = p.G;
    J.Rinv = (T*)p.Rinv;
    J.hw = p.hw;
    J.hq = p.hq;
    J.flag = p.flag;
    J.info = p.info;
    // nearly square samples: Householder QR directly (CholeskyQR2 has no flop
    // advantage there and such samples are often numerically rank deficient)
    J.hh_first = 3 * J.l > J.rows ? 1 : 0;
    // without U, Q only has to span the sampled range: a Householder QR that
    // ends early forms just its leading columns, and the later products skip
    // the rest (their operands are zero there)
    J.rank_eff = p.flag + 2;
    J.trunc_q = p.want_u ? 0 : 1;
    J.active = p.active;
  }
  return b;
}

// Rank-k SVD of B (l x n, FP64, in Bm) for every matrix: one-sided Jacobi on
// B itself, or - for wide B (n >= 3 l) - on the l x l matrix M = B Q_b where
// B^T = Q_b R is an FP64 orthonormalisation of B^T (same CholeskyQR2 /
// Householder machinery as the samples); then B = M Q_b^T and the rows of V^T
// are the Jacobi's normalised rows times Q_b^T.  Writes S, V^T and the sorted
// rotations Ps (U~ = Ps^T).
template <typename T>
int svd_of_B(std::vector<Prob>& probs, cudaStream_t s, bool tc_err) {
  const int cnt = (int)probs.size();
  std::vector<Prob*> wide;
  for (auto& p : probs)
    if (p.wide) wide.push_back(&p);
  // the wide matrices' preparation: Q_b = orth(B^T), M = B Q_b, Q_b^T
  auto wide_prep = [&]() -> int {
    if (wide.empty()) return RSVD_OK;
    const int wc = (int)wide.size();
    {  // B^T (n x l)
      XposeBatch x;
      x.count = wc;
      for (int i = 0; i < wc; ++i) {
        Prob& p = *wide[i];
        x.job[i] = XposeJob{p.l, p.n, p.n, p.l, p.Bm, p.Bt};
        x.job[i].active = p.active;
      }
      RSVD_TRY((launch_transpose<double, double>(x, s)));
    }
    {  // Q_b = orth(B^T) in FP64
      OrthBatch<double> ob;
      ob.count = wc;
      ob.max_chunks = 0;
      ob.max_tilepairs = 0;
      ob.serial = wide[0]->serial;
      for (int i = 0; i < wc; ++i) {
        Prob& p = *wide[i];
        OrthJob<double>& J = ob.job[i];
        J.rows = p.n; J.l = p.l; J.Y = p.Bt; J.Y1 = p.Bt2; J.part = p.part; J.G = p.G; J.Rinv = p.RinvD;
        J.hw = p.hw; J.hq = p.hq; J.flag = p.flag; J.info = p.info; J.hh_first = 3 * p.l > p.n ? 1 : 0;
        J.active = p.active;
      }
      RSVD_TRY(launch_orth<double>(ob, s));
    }
    {  // M = B Q_b (l x l)
      GemmBatch<double, double> g;
      g.count = wc;
      for (int i = 0; i < wc; ++i) {
        Prob& p = *wide[i];
        g.job[i] = GemmJob<double, double>{p.l, p.l, p.n, p.n, p.l, p.l, p.Bm, p.Bt, p.Mb, nullptr, nullptr, 0};
        g.job[i].active = p.active;
      }
      RSVD_TRY((launch_gemm<double, double, false, false>(g, s)));
    }
    {  // Q_b^T (l x n) in the output precision
      XposeBatch x;
      x.count = wc;
      for (int i = 0; i < wc; ++i) {
        Prob& p = *wide[i];
        x.job[i] = XposeJob{p.n, p.l, p.l, p.n, p.Bt, p.Qbt};
        x.job[i].active = p.active;
      }
      RSVD_TRY((launch_transpose<double, T>(x, s)));
    }
      return RSVD_OK;
  };
  // one launch per (cluster size, storage, wide or not) group; the groups are
  // independent and run concurrently (one after another on s with RSVD_FLAG_SERIAL: the
  // same groups, so the same results bit for bit)
  const bool serial = cnt > 0 && probs[0].serial;
  std::vector<int> done(cnt, 0);
  std::vector<JacobiBatch<T>> groups;
  std::vector<int> gwide;
  for (int i0 = 0; i0 < cnt; ++i0) {
    if (done[i0]) continue;
    groups.emplace_back();
    gwide.push_back(probs[i0].wide);
    JacobiBatch<T>& b = groups.back();
    b.count = 0;
    b.csize = probs[i0].csize;
    b.use_global = probs[i0].use_global;
    const int csize0 = b.csize;
    for (int i = i0; i < cnt; ++i) {
      Prob& p = probs[i];
      if (done[i] || p.csize != csize0 || p.use_global != b.use_global || p.wide != probs[i0].wide) continue;
      done[i] = 1;
      JacobiJob<T>& J = b.job[b.count++];
      J.l = p.l; J.n = p.wide ? p.l : p.n; J.k = p.k;
      J.Bm = p.wide ? p.Mb : p.Bm; J.Bg = p.Bg; J.Pg = p.Pg;
      J.S = p.S; J.sig = p.sig;
      J.Vt = p.wide ? (T*)p.Wb : (T*)p.Vt;
      J.ldvt = p.wide ? p.l : p.ldvt;
      J.Ps = (T*)p.Ps;
      J.info = p.info;
      J.max_sweeps = p.max_sweeps;
      J.want_vt = 1;
      J.want_p = p.want_u;
      J.pipe_err = tc_err ? p.flag + 1 : nullptr;
      J.no_exchange = p.no_exchange;
      J.active = p.active;
    }
    // spread the group over the SMs: a cluster size between the smallest whose slices fit
    // shared memory and one of at least 16 columns per CTA (at most 16 CTAs)
    if (!b.use_global && b.csize > 1) {
      int cmin = 16, cmax = 16;
      double rep = 0.0;
      for (int i = 0; i < b.count; ++i) {
        const int l = b.job[i].l, n = b.job[i].n;
        int c = 1;
        while (c < 16 && !jacobi_fits_smem(l, n, c)) ++c;
        cmin = i == 0 ? c : std::max(cmin, c);
        cmax = std::min(cmax, std::max(1, n / 16));
        // per round, in FP64 warp instructions: every CTA forms all l/2 pairs' rotation
        // scalars (about 40 per warp of pairs) and sums the team partials; the inner
        // products and the rotations (about 1.5 n per pair) are split over the CTAs
        const double np = (l + 1) / 2;
        rep = std::max(rep, (std::ceil(np / 32.0) * 40.0 + np / 4.0) / (np * n * 1.5 / 32.0));
      }
      if (cmin <= cmax) b.csize = spread_cluster(b.count, cmin, cmax, rep);
    }
  }
  const int ng = (int)groups.size();
  int nnarrow = 0;
  for (int g = 0; g < ng; ++g) nnarrow += gwide[g] ? 0 : 1;
  if (!wide.empty() && nnarrow > 0 && !serial) {
    // the SVDs of the matrices that need no preparation start at once on side streams
    // 1.., while the caller's stream prepares the wide matrices (whose orthonormalisation
    // may use side stream 0) and then runs their SVDs
    SideStreams* ss = side_streams();
    if (!ss) return RSVD_ERR_LAUNCH;
    RSVD_TRY(fork_side(ss, kSideStreams, s));
    int k = 0;
    for (int g = 0; g < ng; ++g)
      if (!gwide[g]) RSVD_TRY(launch_jacobi<T>(groups[g], ss->stream[1 + (k++) % (kSideStreams - 1)]));
    const int rc = wide_prep();
    if (rc != RSVD_OK) return rc;
    for (int g = 0; g < ng; ++g)
      if (gwide[g]) RSVD_TRY(launch_jacobi<T>(groups[g], s));
    RSVD_TRY(join_side(ss, kSideStreams, s));
  } else {
    const int rc = wide_prep();
    if (rc != RSVD_OK) return rc;
    // the first group on s and the others on side streams
    const int nside = serial ? 0 : std::min(ng - 1, kSideStreams);
    SideStreams* ss = nullptr;
    if (nside > 0) {
      ss = side_streams();
      if (!ss) return RSVD_ERR_LAUNCH;
      RSVD_TRY(fork_side(ss, nside, s));
    }
    for (int g = 0; g < ng; ++g)
      RSVD_TRY(launch_jacobi<T>(groups[g], (g == 0 || !ss) ? s : ss->stream[(g - 1) % kSideStreams]));
    if (ss) RSVD_TRY(join_side(ss, nside, s));
  }
  if (!wide.empty()) {  // V^T = W Q_b^T
    GemmBatch<T, T> g;
    g.count = 0;
    for (auto* pp : wide) {
      Prob& p = *pp;
      g.job[g.count++] = GemmJob<T, T>{p.k, p.n, p.l, p.l, p.n, p.ldvt, (const T*)p.Wb, (const T*)p.Qbt, (T*)p.Vt,
                                       nullptr, nullptr, 0};
      g.job[g.count - 1].active = p.active;
    }
    RSVD_TRY((launch_gemm<T, T, false, false>(g, s)));
  }
  return RSVD_OK;
}

// Alg. RSVD for up to kMaxJobs matrices of one precision.
template <typename T>
int run_chunk(std::vector<Prob>& probs, int q, cudaStream_t s) {
  const int cnt = (int)probs.size();
  std::vector<Prob*> rs;  // matrices on the randomized path
  for (auto& p : probs)
    if (!p.exact) rs.push_back(&p);

  {
    PrepBatch<T> b;
    b.count = cnt;
    for (int i = 0; i < cnt; ++i) {
      Prob& p = probs[i];
      b.job[i] = PrepJob<T>{p.m, p.n, p.l, p.exact, (const T*)p.A, p.lda, (T*)p.Y0, p.Bm, p.flag, p.info};
      b.job[i].active = p.active;
    }
    RSVD_TRY(launch_prep<T>(b, s));
  }
  if (!rs.empty()) {
    const int rc = (int)rs.size();
    {  // step 1: Omega (n x l) into Z0; for the real embedding of a complex matrix the
       // (n/2 x l/2) test matrix twice on the diagonal, zeros elsewhere
      OmegaBatch<T> b;
      b.count = 0;
      for (int i = 0; i < rc; ++i) {
        Prob& p = *rs[i];
        if (!p.cplx) {
          b.job[b.count++] = OmegaJob<T>{p.n, p.l, p.l, (T*)p.Z0, p.seed, p.stream};
          b.job[b.count - 1].active = p.active;
          continue;
        }
        RSVD_TRY(cudaMemsetAsync(p.Z0, 0, (size_t)p.n * p.l * sizeof(T), s));
        const int nc = p.n / 2, lc = p.l / 2;
        b.job[b.count++] = OmegaJob<T>{nc, lc, p.l, (T*)p.Z0, p.seed, p.stream};
        b.job[b.count - 1].active = p.active;
        b.job[b.count++] = OmegaJob<T>{nc, lc, p.l, (T*)p.Z0 + (size_t)nc * p.l + lc, p.seed, p.stream};
        b.job[b.count - 1].active = p.active;
        if (b.count + 2 > kMaxJobs) {
          RSVD_TRY(launch_omega<T>(b, s));
          b.count = 0;
        }
      }
      RSVD_TRY(launch_omega<T>(b, s));
    }
    // products with A: on the tensor cores by exact slicing for the eligible
    // matrices (the slices of A and A^T are made once per call), FP64 FMAs for
    // the others
    std::vector<Prob*> rsd, oz;
    for (auto* pp : rs) (pp->oz ? oz : rsd).push_back(pp);
    struct OzMaps {
      CUtensorMap tpA, tpAt, tsN, tsM;
    };
    std::vector<OzMaps> maps(oz.size());
    int ntile = 16;
    if (!oz.empty()) {
      int npad = 16;
      for (auto* pp : oz) npad = std::max(npad, pp->Npad);
      ntile = oz_ntile(npad);
      OzSplitBatch sb;
      sb.count = 0;
      for (size_t i = 0; i < oz.size(); ++i) {
        Prob& p = *oz[i];
        if (sb.count + 2 > kMaxJobs) {
          RSVD_TRY(launch_oz_split(sb, s));
          sb.count = 0;
        }
        sb.job[sb.count++] = OzSplitJob{(const double*)p.A, p.m, p.n, p.lda, 0, p.m, p.KpA, p.SA, p.eA};
        sb.job[sb.count - 1].active = p.active;
        sb.job[sb.count++] = OzSplitJob{(const double*)p.A, p.n, p.m, p.lda, 1, p.n, p.KpAt, p.SAt, p.eAt};
        sb.job[sb.count - 1].active = p.active;
        if (!make_tmap(&maps[i].tpA, p.SA, kOzSlices * p.m, p.n, p.KpA, 2, 128) ||
            !make_tmap(&maps[i].tpAt, p.SAt, kOzSlices * p.n, p.m, p.KpAt, 2, 128) ||
            !make_tmap(&maps[i].tsN, p.SS, kOzSlices * p.Npad, p.n, p.KpS, 2, ntile) ||
            !make_tmap(&maps[i].tsM, p.SS, kOzSlices * p.Npad, p.m, p.KpS, 2, ntile))
          return RSVD_ERR_LAUNCH;
      }
      RSVD_TRY(launch_oz_split(sb, s));
    }
    // C = P S with P = A (K = n) or A^T (K = m), S = the thin operand X (K x l,
    // ld l); C row-major (ldc = l) or, for B = Q^T A, written transposed
    enum { kAZ, kAtY, kQtA };
    auto oz_product = [&](int kind) -> int {
      OzSplitBatch sb;
      sb.count = 0;
      for (auto* pp : oz) {
        Prob& p = *pp;
        const bool onA = kind == kAZ;
        sb.job[sb.count++] = OzSplitJob{(const double*)(onA ? p.Z0 : p.Y0), p.l, onA ? p.n : p.m, p.l, 1, p.Npad,
                                        p.KpS, p.SS, p.eS};
        sb.job[sb.count - 1].active = p.active;
      }
      RSVD_TRY(launch_oz_split(sb, s));
      for (size_t c0 = 0; c0 < oz.size(); c0 += kMaxOzJobs) {
        OzBatch b;
        b.count = 0;
        b.ntile = ntile;
        for (size_t i = c0; i < std::min(oz.size(), c0 + kMaxOzJobs); ++i) {
          Prob& p = *oz[i];
          OzJob& J = b.job[b.count++];
          J.tp = kind == kAZ ? maps[i].tpA : maps[i].tpAt;
          J.ts = kind == kAZ ? maps[i].tsN : maps[i].tsM;
          J.ep = kind == kAZ ? p.eA : p.eAt;
          J.es = p.eS;
          J.M = kind == kAZ ? p.m : p.n;
          J.N = p.l;
          J.Npad = p.Npad;
          J.K = kind == kAZ ? p.n : p.m;
          J.C = kind == kAZ ? (double*)p.Y0 : kind == kAtY ? (double*)p.Z0 : p.Bm;
          J.ldc = kind == kQtA ? p.n : p.l;
          J.trans_c = kind == kQtA ? 1 : 0;
          J.n_eff = p.want_u ? nullptr : p.flag + 2;
          J.err = p.flag + 1;  // a timed-out pipeline wait is reported by the Jacobi SVD's status
          J.active = p.active;
        }
        RSVD_TRY(launch_oz_gemm(b, s));
      }
      return RSVD_OK;
    };
    // W = X^T Y0 (r x l) for the factored matrices: the first half of A^T Y0 and of Q^T A
    auto gemm_XtY = [&]() -> cudaError_t {
      GemmBatch<T, T> f;
      f.count = 0;
      for (auto* pp : rsd) {
        Prob& p = *pp;
        if (!p.r) continue;
        f.job[f.count] = GemmJob<T, T>{p.r, p.l, p.m, p.ldxf, p.l, p.l, (const T*)p.Xf, (const T*)p.Y0, (T*)p.Wf, nullptr, nullptr, 0};
        f.job[f.count].active = p.active;
        if (!p.want_u) f.job[f.count].n_eff = p.flag + 2;
        ++f.count;
      }
      return launch_gemm<T, T, true, false>(f, s);
    };
    auto gemm_AZ = [&]() -> cudaError_t {  // Y0 = A Z0 (factored: W = Y Z0, Y0 = X W)
      if (!oz.empty() && oz_product(kAZ) != RSVD_OK) return last_cuda_error();
      GemmBatch<T, T> g, f;
      g.count = f.count = 0;
      for (auto* pp : rsd) {
        Prob& p = *pp;
        if (p.r) {
          f.job[f.count] = GemmJob<T, T>{p.r, p.l, p.n, p.ldyf, p.l, p.l, (const T*)p.Yf, (const T*)p.Z0, (T*)p.Wf, nullptr, nullptr, 0};
          f.job[f.count].active = p.active;
          if (!p.want_u) f.job[f.count].n_eff = p.flag + 2;
          ++f.count;
          g.job[g.count] = GemmJob<T, T>{p.m, p.l, p.r, p.ldxf, p.l, p.l, (const T*)p.Xf, (const T*)p.Wf, (T*)p.Y0, nullptr, nullptr, 0};
          g.job[g.count].active = p.active;
        } else {
          g.job[g.count] = GemmJob<T, T>{p.m, p.l, p.n, p.lda, p.l, p.l, (const T*)p.A, (const T*)p.Z0, (T*)p.Y0, nullptr, nullptr, 0};
          g.job[g.count].active = p.active;
        }
        if (!p.want_u) g.job[g.count].n_eff = p.flag + 2;
        ++g.count;
      }
      cudaError_t e = launch_gemm<T, T, false, false>(f, s);
      if (e != cudaSuccess) return e;
      return launch_gemm<T, T, false, false>(g, s);
    };
    auto gemm_AtY = [&]() -> cudaError_t {  // Z0 = A^T Y0 (factored: Z0 = Y^T (X^T Y0))
      if (!oz.empty() && oz_product(kAtY) != RSVD_OK) return last_cuda_error();
      cudaError_t e = gemm_XtY();
      if (e != cudaSuccess) return e;
      GemmBatch<T, T> g;
      g.count = (int)rsd.size();
      for (int i = 0; i < g.count; ++i) {
        Prob& p = *rsd[i];
        if (p.r)
          g.job[i] = GemmJob<T, T>{p.n, p.l, p.r, p.ldyf, p.l, p.l, (const T*)p.Yf, (const T*)p.Wf, (T*)p.Z0, nullptr, nullptr, 0};
        else
          g.job[i] = GemmJob<T, T>{p.n, p.l, p.m, p.lda, p.l, p.l, (const T*)p.A, (const T*)p.Y0, (T*)p.Z0, nullptr, nullptr, 0};
        g.job[i].active = p.active;
        if (!p.want_u) g.job[i].n_eff = p.flag + 2;
      }
      return launch_gemm<T, T, true, false>(g, s);
    };
    // step 2: Y = A Omega, Q = orth(Y); then q times Z = orth(A^T Q), Q = orth(A Z)
    RSVD_TRY(gemm_AZ());
    RSVD_TRY(launch_orth<T>(orth_batch<T>(rs, true), s));
    for (int it = 0; it < q; ++it) {
      RSVD_TRY(gemm_AtY());
      RSVD_TRY(launch_orth<T>(orth_batch<T>(rs, false), s));
      RSVD_TRY(gemm_AZ());
      RSVD_TRY(launch_orth<T>(orth_batch<T>(rs, true), s));
    }
    {  // step 4: B = Q^T A (l x n) in FP64
      if (!oz.empty() && oz_product(kQtA) != RSVD_OK) return RSVD_ERR_LAUNCH;
      RSVD_TRY(gemm_XtY());  // factored: B = (X^T Q)^T Y
      GemmBatch<T, double> g;
      g.count = (int)rsd.size();
      for (int i = 0; i < g.count; ++i) {
        Prob& p = *rsd[i];
        if (p.r)
          g.job[i] = GemmJob<T, double>{p.l, p.n, p.r, p.l, p.ldyf, p.n, (const T*)p.Wf, (const T*)p.Yf, p.Bm, nullptr, nullptr, 0};
        else
          g.job[i] = GemmJob<T, double>{p.l, p.n, p.m, p.l, p.lda, p.n, (const T*)p.Y0, (const T*)p.A, p.Bm, nullptr, nullptr, 0};
        g.job[i].active = p.active;
        if (!p.want_u) g.job[i].m_eff = p.flag + 2;
      }
      RSVD_TRY((launch_gemm<T, double, true, false>(g, s)));
    }
  }
  // SVD of B (a timed-out wait of the tensor-core products is reported through its status)
  {
    bool any_oz = false;
    for (auto& pr : probs) any_oz = any_oz || (pr.oz && !pr.exact);
    int rc = svd_of_B<T>(probs, s, any_oz);
    if (rc != RSVD_OK) return rc;
  }
  // lift U = Q U~ and fix the signs
  {
    GemmBatch<T, T> g;
    g.count = 0;
    SignBatch<T> sb;
    sb.count = 0;
    for (int i = 0; i < cnt; ++i) {
      Prob& p = probs[i];
      if (!p.want_u) continue;
      g.job[g.count++] = GemmJob<T, T>{p.m, p.k, p.l, p.l, p.l, p.ldu, (const T*)p.Y0, (const T*)p.Ps, (T*)p.U, nullptr, nullptr, 0};
      g.job[g.count - 1].active = p.active;
      sb.job[sb.count++] = SignJob<T>{p.m, p.n, p.k, (T*)p.U, p.ldu, (T*)p.Vt, p.ldvt};
      sb.job[sb.count - 1].active = p.active;
    }
    RSVD_TRY((launch_gemm<T, T, false, true>(g, s)));
    RSVD_TRY(launch_sign<T>(sb, s));
  }
  return RSVD_OK;
}

// Alg. RSVD with the products of A on tensor cores (operands TIn = bf16 or
// float read as TF32, FP32 accumulation); orthonormalisation, SVD of B and the
// lift as in the FP32 path.
template <typename TIn>
int run_chunk_tc(std::vector<Prob>& probs, int q, cudaStream_t s) {
  const int cnt = (int)probs.size();
  const int eb = (int)sizeof(TIn);
  {
    PrepBatch<float> b;
    b.count = cnt;
    for (int i = 0; i < cnt; ++i) {
      Prob& p = probs[i];
      b.job[i] = PrepJob<float>{p.m, p.n, p.l, 0, nullptr, p.lda, (float*)p.Y0, p.Bm, p.flag, p.info};
    }
    RSVD_TRY(launch_prep<float>(b, s));
  }
  {  // A^T, once per call
    XposeBatch x;
    x.count = cnt;
    for (int i = 0; i < cnt; ++i) {
      Prob& p = probs[i];
      x.job[i] = XposeJob{p.m, p.n, p.lda, p.ldAt, p.A, p.At};
    }
    RSVD_TRY((launch_transpose<TIn, TIn>(x, s)));
  }
  // The thin operands (Omega, Z, Q) go to the tensor cores split into a high
  // and a low part in the operand precision, stacked as 2 lp rows (lp = l
  // rounded up to 16); the GEMM adds the two halves of its accumulator, so the
  // product carries the thin operand to about FP32 accuracy while A is read
  // once.  Samples wider than 128 columns use the plain (unsplit) operand.
  std::vector<int> lp(cnt), splitv(cnt);
  for (int i = 0; i < cnt; ++i) {
    lp[i] = (probs[i].l + 15) / 16 * 16;
    splitv[i] = 2 * lp[i] <= 256 ? 1 : 0;
  }
  {  // Omega (n x l, FP32) into Z0
    OmegaBatch<float> b;
    b.count = cnt;
    for (int i = 0; i < cnt; ++i) {
      Prob& p = probs[i];
      b.job[i] = OmegaJob<float>{p.n, p.l, p.l, (float*)p.Z0, p.seed, p.stream, 0};
    }
    RSVD_TRY(launch_omega<float>(b, s));
  }
  std::vector<Prob*> all;
  for (auto& p : probs) all.push_back(&p);
  // C (rows x l, FP32) = Aop (rows x K) * Bop (l x K)^T
  auto tc = [&](bool transposedA, bool fromQ, bool toZ) -> int {
    TcBatch b;
    b.count = 0;
    for (int i = 0; i < cnt; ++i) {
      Prob& p = probs[i];
      TcJob& J = b.job[b.count++];
      const int rows = transposedA ? p.n : p.m;
      const int K = transposedA ? p.m : p.n;
      const void* Aop = transposedA ? p.At : p.A;
      const int ldA = transposedA ? p.ldAt : p.lda;
      const void* Bop = fromQ ? p.QT : p.WT;
      const int ldB = fromQ ? p.ldQT : p.ldWT;
      J.fold = splitv[i] ? lp[i] : 0;
      J.Npad = splitv[i] ? 2 * lp[i] : lp[i];
      if (!make_tmap(&J.ta, Aop, rows, K, ldA, eb, 128) || !make_tmap(&J.tb, Bop, J.Npad, K, ldB, eb, J.Npad))
        return RSVD_ERR_INVALID_SIZE;
      J.C = (float*)(toZ ? p.Z0 : p.Y0);
      J.err = p.flag + 1;
      J.M = rows;
      J.N = p.l;
      J.K = K;
      J.ldc = p.l;
    }
    RSVD_TRY(launch_tc_gemm<TIn>(b, s));
    return RSVD_OK;
  };
  // thin operand: Q^T from Y0 (m x l) or Omega^T / Z^T from Z0 (n x l)
  auto xpose_to_op = [&](bool fromZ) -> int {
    XposeBatch xs, xp;
    xs.count = xp.count = 0;
    for (int i = 0; i < cnt; ++i) {
      Prob& p = probs[i];
      XposeJob j = fromZ ? XposeJob{p.n, p.l, p.l, p.ldWT, p.Z0, p.WT} : XposeJob{p.m, p.l, p.l, p.ldQT, p.Y0, p.QT};
      j.fold = lp[i];
      if (splitv[i]) xs.job[xs.count++] = j;
      else xp.job[xp.count++] = j;
    }
    RSVD_TRY(launch_split_transpose<TIn>(xs, 0, s));
    RSVD_TRY((launch_transpose<float, TIn>(xp, s)));
    return RSVD_OK;
  };
  int rc;
  if ((rc = xpose_to_op(true))) return rc;  // Omega^T
  if ((rc = tc(false, false, false))) return rc;  // Y = A Omega
  RSVD_TRY(launch_orth<float>(orth_batch<float>(all, true), s));
  for (int it = 0; it < q; ++it) {
    if ((rc = xpose_to_op(false))) return rc;
    if ((rc = tc(true, true, true))) return rc;   // Z = A^T Q
    RSVD_TRY(launch_orth<float>(orth_batch<float>(all, false), s));
    if ((rc = xpose_to_op(true))) return rc;
    if ((rc = tc(false, false, false))) return rc;  // Y = A Z
    RSVD_TRY(launch_orth<float>(orth_batch<float>(all, true), s));
  }
  if ((rc = xpose_to_op(false))) return rc;
  if ((rc = tc(true, true, true))) return rc;  // B^T = A^T Q (n x l)
  {
    XposeBatch x;
    x.count = cnt;
    for (int i = 0; i < cnt; ++i) {
      Prob& p = probs[i];
      x.job[i] = XposeJob{p.n, p.l, p.l, p.n, p.Z0, p.Bm};
    }
    RSVD_TRY((launch_transpose<float, double>(x, s)));
  }
  {
    int rc2 = svd_of_B<float>(probs, s, true);
    if (rc2 != RSVD_OK) return rc2;
  }
  {
    GemmBatch<float, float> g;
    g.count = 0;
    SignBatch<float> sb;
    sb.count = 0;
    for (auto& p : probs) {
      g.job[g.count++] = GemmJob<float, float>{p.m, p.k, p.l, p.l, p.l, p.ldu, (const float*)p.Y0, (const float*)p.Ps,
                                               (float*)p.U, nullptr, nullptr, 0};
      sb.job[sb.count++] = SignJob<float>{p.m, p.n, p.k, (float*)p.U, p.ldu, (float*)p.Vt, p.ldvt};
    }
    RSVD_TRY((launch_gemm<float, float, false, true>(g, s)));
    RSVD_TRY(launch_sign<float>(sb, s));
  }
  return RSVD_OK;
}

int check_params(const rsvd_params* p) {
  if (!p) return RSVD_ERR_NULL_POINTER;
  if (p->p < 0 || p->q < 0 || p->q > 64 || p->max_sweeps < 0 || (p->flags & ~(RSVD_FLAG_F64_SIMT | RSVD_FLAG_FULL_SVD | RSVD_FLAG_SERIAL | RSVD_FLAG_TEST_NO_EXCHANGE)) != 0)
    return RSVD_ERR_INVALID_SIZE;
  if (p->prec != RSVD_F64 && p->prec != RSVD_F32 && p->prec != RSVD_TF32 && p->prec != RSVD_BF16)
    return RSVD_ERR_PRECISION;
  return RSVD_OK;
}

size_t tsize_of(int prec) { return prec == RSVD_F64 ? 8 : 4; }
bool is_tc(int prec) { return prec == RSVD_TF32 || prec == RSVD_BF16; }
int tc_bytes_of(int prec) { return prec == RSVD_BF16 ? 2 : prec == RSVD_TF32 ? 4 : 0; }

int run_batched(std::vector<Prob>& probs, const rsvd_params* p, char* work, size_t work_bytes, cudaStream_t s) {
  const size_t ts = tsize_of(p->prec);
  const int tcb = tc_bytes_of(p->prec);
  size_t need = 0;
  for (auto& pr : probs)
    need += layout(nullptr, pr.m, pr.n, pr.k, pr.l, ts, nullptr, tcb, pr.r ? 0 : use_oz(pr.m, pr.n, pr.l, pr.exact, p), pr.r);
  if (need > work_bytes) return RSVD_ERR_WORKSPACE;
  size_t off = 0;
  for (auto& pr : probs) {
    off += layout(&pr, pr.m, pr.n, pr.k, pr.l, ts, work + off, tcb, pr.r ? 0 : use_oz(pr.m, pr.n, pr.l, pr.exact, p), pr.r);
  }
  const size_t step = is_tc(p->prec) ? (size_t)kMaxTcJobs : (size_t)kMaxJobs;
  const int nchunks = (int)((probs.size() + step - 1) / step);
  // the chunks of a large batch are independent (own workspace, own matrices): they run
  // concurrently on the chunk streams, forked from s and joined back to it, each chunk's
  // own groups on the side-stream set of its chunk stream; RSVD_FLAG_SERIAL keeps them
  // on s one after another
  const int nstreams = (nchunks > 1 && !(p->flags & RSVD_FLAG_SERIAL)) ? std::min(nchunks, kChunkStreams) : 0;
  SideStreams* cs = nullptr;
  if (nstreams > 0) {
    cs = side_set(kChunkSet);
    if (!cs) return RSVD_ERR_LAUNCH;
    RSVD_TRY(fork_side(cs, nstreams, s));
  }
  int rc = RSVD_OK;
  for (int c = 0; c < nchunks && rc == RSVD_OK; ++c) {
    const size_t c0 = (size_t)c * step;
    std::vector<Prob> chunk(probs.begin() + c0, probs.begin() + std::min(probs.size(), c0 + step));
    cudaStream_t cst = s;
    if (cs) {
      cst = cs->stream[c % nstreams];
      select_side_set(c % nstreams);
    }
    if (p->prec == RSVD_F64) rc = run_chunk<double>(chunk, p->q, cst);
    else if (p->prec == RSVD_F32) rc = run_chunk<float>(chunk, p->q, cst);
    else if (p->prec == RSVD_BF16) rc = run_chunk_tc<__nv_bfloat16>(chunk, p->q, cst);
    else rc = run_chunk_tc<float>(chunk, p->q, cst);
  }
  select_side_set(0);
  // joined on every path, so that s never runs ahead of work already enqueued
  if (cs) {
    const cudaError_t e = join_side(cs, nstreams, s);
    if (e != cudaSuccess && rc == RSVD_OK) {
      last_cuda_error() = e;
      rc = RSVD_ERR_LAUNCH;
    }
  }
  return rc;
}

}  // namespace
}  // namespace rsvd

using namespace rsvd;

extern "C" {

const char* rsvd_status_string(int status) {
  switch (status) {
    case RSVD_OK: return "ok";
    case RSVD_ERR_INVALID_SIZE: return "invalid size, rank or leading dimension";
    case RSVD_ERR_NULL_POINTER: return "required pointer is NULL";
    case RSVD_ERR_PRECISION: return "precision not supported";
    case RSVD_ERR_WORKSPACE: return "workspace too small";
    case RSVD_ERR_LAUNCH: return cudaGetErrorString(last_cuda_error());
    case RSVD_ERR_NONFINITE: return "non-finite value in the input";
    case RSVD_WARN_NOCONV: return "Jacobi SVD reached its sweep cap";
    case RSVD_WARN_CG: return "a conjugate-gradient column did not converge or met non-positive curvature";
    case RSVD_ERR_TIMEOUT: return "a device pipeline wait timed out (results invalid)";
    case RSVD_ERR_SCRATCH_LIMIT: return "matrix needs more scratch than the fixed no-allocation array holds";
    default: return "unknown status";
  }
}

int rsvd_gaussian(int n, int l, uint64_t seed, uint64_t stream, double* omega, int ld, void* cuda_stream) {
  if (n < 1 || l < 1 || ld < l) return RSVD_ERR_INVALID_SIZE;
  if (!omega) return RSVD_ERR_NULL_POINTER;
  RSVD_TRY(launch_omega_f64_single(n, l, ld, omega, seed, stream, (cudaStream_t)cuda_stream));
  return RSVD_OK;
}

int rsvd_batched_workspace_size(int batch, const int* m, const int* n, const int* k, const rsvd_params* p,
                                size_t* bytes) {
  int rc = check_params(p);
  if (rc) return rc;
  if (!m || !n || !k || !bytes) return RSVD_ERR_NULL_POINTER;
  if (batch < 1) return RSVD_ERR_INVALID_SIZE;
  size_t tot = 0;
  for (int b = 0; b < batch; ++b) {
    if (m[b] < 1 || n[b] < 1 || k[b] < 1 || k[b] > std::min(m[b], n[b])) return RSVD_ERR_INVALID_SIZE;
    const int l = b_rows(m[b], n[b], k[b], p);
    if (l > kMaxSample) return RSVD_ERR_INVALID_SIZE;
    if (is_tc(p->prec) && (l > 256 || m[b] <= l)) return RSVD_ERR_INVALID_SIZE;
    tot += layout(nullptr, m[b], n[b], k[b], l, tsize_of(p->prec), nullptr, tc_bytes_of(p->prec),
                  use_oz(m[b], n[b], l, exact_of(m[b], l, p), p));
  }
  *bytes = tot;
  return RSVD_OK;
}

int rsvd_workspace_size(int m, int n, const rsvd_params* p, size_t* bytes) {
  if (!p) return RSVD_ERR_NULL_POINTER;
  return rsvd_batched_workspace_size(1, &m, &n, &p->k, p, bytes);
}

int rsvd_truncate_batched(int batch, const int* m, const int* n, const void* const* A, const int* lda, const int* k,
                          const rsvd_params* p, double* const* S, void* const* U, const int* ldu, void* const* Vt,
                          const int* ldvt, int chi_global, int* k_out, void* work, size_t work_bytes, rsvd_info* info,
                          void* cuda_stream) {
  int rc = check_params(p);
  if (rc) return rc;
  if ((p->flags & RSVD_FLAG_FULL_SVD) && is_tc(p->prec)) return RSVD_ERR_PRECISION;
  if (batch < 1 || chi_global < 0) return RSVD_ERR_INVALID_SIZE;
  if (!m || !n || !A || !lda || !k || !S || !U || !ldu || !Vt || !ldvt || !work || !info) return RSVD_ERR_NULL_POINTER;
  if (chi_global > 0 && !k_out) return RSVD_ERR_NULL_POINTER;
  if (chi_global > 0 && batch > kMaxJobs) return RSVD_ERR_INVALID_SIZE;
  if (((uintptr_t)work) % kAlign) return RSVD_ERR_WORKSPACE;
  std::vector<Prob> probs(batch);
  int total_k = 0;
  for (int b = 0; b < batch; ++b) {
    if (m[b] < 1 || n[b] < 1 || k[b] < 1 || k[b] > std::min(m[b], n[b])) return RSVD_ERR_INVALID_SIZE;
    if (lda[b] < n[b] || ldu[b] < k[b] || ldvt[b] < n[b]) return RSVD_ERR_INVALID_SIZE;
    if (!A[b] || !S[b] || !U[b] || !Vt[b]) return RSVD_ERR_NULL_POINTER;
    Prob& pr = probs[b];
    std::memset(&pr, 0, sizeof(Prob));
    pr.m = m[b]; pr.n = n[b]; pr.k = k[b];
    pr.l = b_rows(m[b], n[b], k[b], p);
    if (pr.l > kMaxSample) return RSVD_ERR_INVALID_SIZE;
    if (is_tc(p->prec)) {
      // tensor-core operands: l <= 256, a sample narrower than A, TMA-describable rows
      const size_t eb = (size_t)tc_bytes_of(p->prec);
      if (pr.l > 256 || m[b] <= pr.l) return RSVD_ERR_INVALID_SIZE;
      if (((uintptr_t)A[b]) % 16 || ((size_t)lda[b] * eb) % 16) return RSVD_ERR_INVALID_SIZE;
    }
    pr.exact = exact_of(pr.m, pr.l, p);
    pr.want_u = 1;
    pr.A = A[b]; pr.lda = lda[b];
    pr.S = S[b]; pr.U = U[b]; pr.ldu = ldu[b]; pr.Vt = Vt[b]; pr.ldvt = ldvt[b];
    pr.seed = p->seed; pr.stream = p->stream + (uint64_t)b;
    pr.info = info + b;
    pr.max_sweeps = p->max_sweeps > 0 ? p->max_sweeps : 40;
    pr.serial = (p->flags & RSVD_FLAG_SERIAL) ? 1 : 0;
    pr.no_exchange = (p->flags & RSVD_FLAG_TEST_NO_EXCHANGE) ? 1 : 0;
    total_k += k[b];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  rc = run_batched(probs, p, (char*)work, work_bytes, s);
  if (rc) return rc;
  if (chi_global > 0) {
    SelectBatch sb;
    sb.count = batch;
    sb.chi = chi_global;
    sb.total = total_k;
    sb.k_out = k_out;
    for (int b = 0; b < batch; ++b) sb.job[b] = SelectJob{S[b], k[b]};
    RSVD_TRY(launch_select(sb, s));
  }
  return RSVD_OK;
}

int rsvd_sectors_adaptive_workspace_size(int batch, const int* m, const int* n, int chi, const rsvd_params* p,
                                         size_t* bytes) {
  if (!m || !n || !p || !bytes) return RSVD_ERR_NULL_POINTER;
  if (p->flags & RSVD_FLAG_FULL_SVD) return RSVD_ERR_INVALID_SIZE;
  if (batch < 1 || batch > kMaxJobs || chi < 1) return RSVD_ERR_INVALID_SIZE;
  std::vector<int> cap(batch);
  for (int b = 0; b < batch; ++b) cap[b] = std::min(chi, std::min(m[b], n[b]));
  int rc = rsvd_batched_workspace_size(batch, m, n, cap.data(), p, bytes);
  if (rc) return rc;
  *bytes += align_up(sizeof(int) * (2 * (size_t)batch + 1));  // the device rounds' state
  return RSVD_OK;
}

int rsvd_truncate_sectors_adaptive(int batch, const int* m, const int* n, const void* const* A, const int* lda,
                                   int* k_trial, const rsvd_params* p, int chi, double* const* S, void* const* U,
                                   const int* ldu, void* const* Vt, const int* ldvt, int* k_out, int* rounds,
                                   void* work, size_t work_bytes, rsvd_info* info, void* cuda_stream) {
  size_t need = 0;
  int rc = rsvd_sectors_adaptive_workspace_size(batch, m, n, chi, p, &need);
  if (rc) return rc;
  if (!A || !lda || !k_trial || !S || !U || !ldu || !Vt || !ldvt || !k_out || !rounds || !work || !info)
    return RSVD_ERR_NULL_POINTER;
  if (is_tc(p->prec)) return RSVD_ERR_PRECISION;
  if (((uintptr_t)work) % kAlign) return RSVD_ERR_WORKSPACE;
  if (need > work_bytes) return RSVD_ERR_WORKSPACE;
  std::vector<int> cap(batch), k(batch);
  for (int b = 0; b < batch; ++b) {
    cap[b] = std::min(chi, std::min(m[b], n[b]));
    if (lda[b] < n[b] || ldu[b] < cap[b] || ldvt[b] < n[b]) return RSVD_ERR_INVALID_SIZE;
    if (!A[b] || !S[b] || !U[b] || !Vt[b]) return RSVD_ERR_NULL_POINTER;
    k[b] = std::max(1, std::min(k_trial[b], cap[b]));
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  std::vector<int> todo(batch), kept(batch);
  for (int b = 0; b < batch; ++b) todo[b] = b;
  int r = 0;
  for (;;) {
    ++r;
    // Alg. RSVD of the blocks whose trial rank changed (all of them in the first round);
    // block b keeps Philox stream p->stream + b, so a larger trial extends its Omega
    std::vector<Prob> probs(todo.size());
    for (size_t t = 0; t < todo.size(); ++t) {
      const int b = todo[t];
      Prob& pr = probs[t];
      std::memset(&pr, 0, sizeof(Prob));
      pr.m = m[b]; pr.n = n[b]; pr.k = k[b];
      pr.l = sample_width(m[b], n[b], k[b], p->p);
      if (pr.l > kMaxSample) return RSVD_ERR_INVALID_SIZE;
      pr.exact = use_exact_path(pr.m, pr.l);
      pr.want_u = 1;
      pr.A = A[b]; pr.lda = lda[b];
      pr.S = S[b]; pr.U = U[b]; pr.ldu = ldu[b]; pr.Vt = Vt[b]; pr.ldvt = ldvt[b];
      pr.seed = p->seed; pr.stream = p->stream + (uint64_t)b;
      pr.info = info + b;
      pr.max_sweeps = p->max_sweeps > 0 ? p->max_sweeps : 40;
      pr.serial = (p->flags & RSVD_FLAG_SERIAL) ? 1 : 0;
    }
    rc = run_batched(probs, p, (char*)work, work_bytes, s);
    if (rc) return rc;
    // the chi largest over all blocks (Sec. III.A post-selection)
    SelectBatch sb;
    sb.count = batch;
    sb.chi = chi;
    sb.total = 0;
    sb.k_out = k_out;
    for (int b = 0; b < batch; ++b) {
      sb.job[b] = SelectJob{S[b], k[b]};
      sb.total += k[b];
    }
    RSVD_TRY(launch_select(sb, s));
    RSVD_TRY(cudaMemcpyAsync(kept.data(), k_out, sizeof(int) * batch, cudaMemcpyDeviceToHost, s));
    RSVD_TRY(cudaStreamSynchronize(s));
    // a block of this round all of whose values were kept may hold more above the cut:
    // double its rank (a block left out of a round is not looked at again)
    std::vector<int> ran;
    ran.swap(todo);
    for (int b : ran)
      if (kept[b] == k[b] && k[b] < cap[b]) {
        k[b] = std::min(2 * k[b], cap[b]);
        todo.push_back(b);
      }
    if (todo.empty()) break;
  }
  for (int b = 0; b < batch; ++b) k_trial[b] = k[b];
  *rounds = r;
  return RSVD_OK;
}

int rsvd_truncate_sectors_adaptive_device(int batch, const int* m, const int* n, const void* const* A, const int* lda,
                                          const int* k_first, const rsvd_params* p, int chi, double* const* S,
                                          void* const* U, const int* ldu, void* const* Vt, const int* ldvt, int* k_out,
                                          int* k_final, int* rounds, void* work, size_t work_bytes, rsvd_info* info,
                                          void* cuda_stream) {
  size_t need = 0;
  int rc = rsvd_sectors_adaptive_workspace_size(batch, m, n, chi, p, &need);
  if (rc) return rc;
  if (!A || !lda || !k_first || !S || !U || !ldu || !Vt || !ldvt || !k_out || !k_final || !rounds || !work || !info)
    return RSVD_ERR_NULL_POINTER;
  if (is_tc(p->prec)) return RSVD_ERR_PRECISION;
  if (((uintptr_t)work) % kAlign) return RSVD_ERR_WORKSPACE;
  if (need > work_bytes) return RSVD_ERR_WORKSPACE;
  std::vector<int> cap(batch), k0(batch);
  for (int b = 0; b < batch; ++b) {
    cap[b] = std::min(chi, std::min(m[b], n[b]));
    if (lda[b] < n[b] || ldu[b] < cap[b] || ldvt[b] < n[b]) return RSVD_ERR_INVALID_SIZE;
    if (!A[b] || !S[b] || !U[b] || !Vt[b]) return RSVD_ERR_NULL_POINTER;
    k0[b] = std::max(1, std::min(k_first[b], cap[b]));
  }
  // the device state after the factorizations' workspace: active[batch], then the rounds count
  const size_t state_off = need - align_up(sizeof(int) * (2 * (size_t)batch + 1));
  int* active = (int*)((char*)work + state_off);
  int* dround = active + batch;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  AdaptInitBatch ib;
  ib.count = batch;
  ib.active = active;
  ib.kdev = k_final;
  ib.rounds = dround;
  for (int b = 0; b < batch; ++b) ib.k[b] = k0[b];
  RSVD_TRY(launch_adapt_init(ib, s));
  // Round r compresses every block whose scheduled rank k0 2^r (capped) still grows, each
  // gated by its device flag; the selection and the decision of the next round's flags
  // stay on the device, so the whole sequence is enqueued at once (and capturable)
  std::vector<int> kr(k0);
  for (int r = 0;; ++r) {
    std::vector<Prob> probs;
    for (int b = 0; b < batch; ++b) {
      if (r > 0 && kr[b] >= cap[b]) continue;  // reached its cap in the schedule: never active again
      const int kb = r == 0 ? kr[b] : std::min(2 * kr[b], cap[b]);
      kr[b] = kb;
      probs.emplace_back();
      Prob& pr = probs.back();
      std::memset(&pr, 0, sizeof(Prob));
      pr.m = m[b]; pr.n = n[b]; pr.k = kb;
      pr.l = sample_width(m[b], n[b], kb, p->p);
      if (pr.l > kMaxSample) return RSVD_ERR_INVALID_SIZE;
      pr.exact = use_exact_path(pr.m, pr.l);
      pr.want_u = 1;
      pr.A = A[b]; pr.lda = lda[b];
      pr.S = S[b]; pr.U = U[b]; pr.ldu = ldu[b]; pr.Vt = Vt[b]; pr.ldvt = ldvt[b];
      pr.seed = p->seed; pr.stream = p->stream + (uint64_t)b;
      pr.info = info + b;
      pr.max_sweeps = p->max_sweeps > 0 ? p->max_sweeps : 40;
      pr.serial = (p->flags & RSVD_FLAG_SERIAL) ? 1 : 0;
      pr.active = active + b;
    }
    if (probs.empty()) break;
    rc = run_batched(probs, p, (char*)work, state_off, s);
    if (rc) return rc;
    SelectBatch sb;
    sb.count = batch;
    sb.chi = chi;
    sb.total = 0;
    sb.k_out = k_out;
    for (int b = 0; b < batch; ++b) {
      sb.job[b] = SelectJob{S[b], cap[b], k_final + b};
      sb.total += cap[b];
    }
    RSVD_TRY(launch_select(sb, s));
    AdaptDecideBatch db;
    db.count = batch;
    db.active = active;
    db.kdev = k_final;
    db.k_out = k_out;
    db.rounds = dround;
    for (int b = 0; b < batch; ++b) {
      db.cap[b] = cap[b];
      db.next_k[b] = std::min(2 * kr[b], cap[b]);
    }
    RSVD_TRY(launch_adapt_decide(db, s));
  }
  RSVD_TRY(cudaMemcpyAsync(rounds, dround, sizeof(int), cudaMemcpyDeviceToDevice, s));
  return RSVD_OK;
}

int rsvd_truncate(int m, int n, const void* A, int lda, const rsvd_params* p, double* S, void* U, int ldu, void* Vt,
                  int ldvt, void* work, size_t work_bytes, rsvd_info* info, void* cuda_stream) {
  if (!p) return RSVD_ERR_NULL_POINTER;
  const void* Aa[1] = {A};
  double* Sa[1] = {S};
  void* Ua[1] = {U};
  void* Va[1] = {Vt};
  return rsvd_truncate_batched(1, &m, &n, Aa, &lda, &p->k, p, Sa, Ua, &ldu, Va, &ldvt, 0, nullptr, work, work_bytes,
                               info, cuda_stream);
}

int rsvd_factored_workspace_size(int m, int r, int n, const rsvd_params* p, size_t* bytes) {
  int rc = check_params(p);
  if (rc) return rc;
  if (p->flags & RSVD_FLAG_FULL_SVD) return RSVD_ERR_INVALID_SIZE;
  if (!bytes) return RSVD_ERR_NULL_POINTER;
  if (p->prec != RSVD_F64 && p->prec != RSVD_F32) return RSVD_ERR_PRECISION;
  if (m < 1 || n < 1 || r < 1 || p->k < 1 || p->k > std::min(m, n)) return RSVD_ERR_INVALID_SIZE;
  const int l = sample_width(m, n, p->k, p->p);
  if (l > kMaxSample) return RSVD_ERR_INVALID_SIZE;
  *bytes = layout(nullptr, m, n, p->k, l, tsize_of(p->prec), nullptr, 0, 0, r);
  return RSVD_OK;
}

int rsvd_truncate_factored(int m, int r, int n, const void* X, int ldx, const void* Y, int ldy, const rsvd_params* p,
                           double* S, void* U, int ldu, void* Vt, int ldvt, void* work, size_t work_bytes,
                           rsvd_info* info, void* cuda_stream) {
  size_t need = 0;
  int rc = rsvd_factored_workspace_size(m, r, n, p, &need);
  if (rc) return rc;
  if (!X || !Y || !S || !U || !Vt || !work || !info) return RSVD_ERR_NULL_POINTER;
  if (ldx < r || ldy < n || ldu < p->k || ldvt < n) return RSVD_ERR_INVALID_SIZE;
  if (((uintptr_t)work) % kAlign) return RSVD_ERR_WORKSPACE;
  if (need > work_bytes) return RSVD_ERR_WORKSPACE;
  std::vector<Prob> probs(1);
  Prob& pr = probs[0];
  std::memset(&pr, 0, sizeof(Prob));
  pr.m = m; pr.n = n; pr.k = p->k;
  pr.l = sample_width(m, n, p->k, p->p);
  pr.exact = 0;  // A is never formed
  pr.want_u = 1;
  pr.r = r; pr.Xf = X; pr.ldxf = ldx; pr.Yf = Y; pr.ldyf = ldy;
  pr.S = S; pr.U = U; pr.ldu = ldu; pr.Vt = Vt; pr.ldvt = ldvt;
  pr.seed = p->seed; pr.stream = p->stream;
  pr.info = info;
  pr.max_sweeps = p->max_sweeps > 0 ? p->max_sweeps : 40;
    pr.serial = (p->flags & RSVD_FLAG_SERIAL) ? 1 : 0;
  return run_batched(probs, p, (char*)work, work_bytes, (cudaStream_t)cuda_stream);
}

// ---------------------------------------------------------------- fixed-error RSVD
namespace {
struct TolLayout {
  size_t rsvd, E, r2, fro2, res, total;
};
TolLayout tol_layout(int m, int n, int kcap, const rsvd_params* p) {
  TolLayout L;
  const int l = sample_width(m, n, kcap, p->p);
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t x = off;
    off += align_up(b);
    return x;
  };
  L.rsvd = take(layout(nullptr, m, n, kcap, l, 8, nullptr, 0, use_oz(m, n, l, use_exact_path(m, l), p)));
  L.E = take((size_t)m * n * 8);
  L.r2 = take(kSqParts * 8);
  L.fro2 = take(kSqParts * 8);
  L.res = take(sizeof(TolResult));
  L.total = off;
  return L;
}
}  // namespace

int rsvd_tol_workspace_size(int m, int n, int k_max, const rsvd_params* p, size_t* bytes) {
  int rc = check_params(p);
  if (rc) return rc;
  if (p->flags & RSVD_FLAG_FULL_SVD) return RSVD_ERR_INVALID_SIZE;
  if (!bytes) return RSVD_ERR_NULL_POINTER;
  if (p->prec != RSVD_F64) return RSVD_ERR_PRECISION;
  if (m < 1 || n < 1 || k_max < 1 || p->k < 1) return RSVD_ERR_INVALID_SIZE;
  const int kcap = std::min(k_max, std::min(m, n));
  if (sample_width(m, n, kcap, p->p) > kMaxSample) return RSVD_ERR_INVALID_SIZE;
  *bytes = tol_layout(m, n, kcap, p).total;
  return RSVD_OK;
}

int rsvd_truncate_tol(int m, int n, const double* A, int lda, double eps, int k_max, const rsvd_params* p, double* S,
                      double* U, int ldu, double* Vt, int ldvt, int* k_out, double* err_out, void* work,
                      size_t work_bytes, rsvd_info* info, void* cuda_stream) {
  size_t need = 0;
  int rc = rsvd_tol_workspace_size(m, n, k_max, p, &need);
  if (rc) return rc;
  if (!A || !S || !U || !Vt || !k_out || !err_out || !work || !info) return RSVD_ERR_NULL_POINTER;
  const int kcap = std::min(k_max, std::min(m, n));
  if (!(eps >= 0.0) || lda < n || ldu < kcap || ldvt < n) return RSVD_ERR_INVALID_SIZE;
  if (((uintptr_t)work) % kAlign) return RSVD_ERR_WORKSPACE;
  if (need > work_bytes) return RSVD_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  char* base = (char*)work;
  const TolLayout L = tol_layout(m, n, kcap, p);
  double* E = (double*)(base + L.E);
  double* r2p = (double*)(base + L.r2);
  double* fro2p = (double*)(base + L.fro2);
  TolResult* res = (TolResult*)(base + L.res);
  RSVD_TRY(launch_sq_sum(A, m, n, lda, fro2p, s));
  int kt = std::max(1, std::min(p->k, kcap));
  TolResult host{};
  for (;;) {
    rsvd_params pk = *p;
    pk.k = kt;
    std::vector<Prob> probs(1);
    Prob& pr = probs[0];
    std::memset(&pr, 0, sizeof(Prob));
    pr.m = m; pr.n = n; pr.k = kt;
    pr.l = sample_width(m, n, kt, p->p);
    pr.exact = use_exact_path(m, pr.l);
    pr.want_u = 1;
    pr.A = A; pr.lda = lda;
    pr.S = S; pr.U = U; pr.ldu = ldu; pr.Vt = Vt; pr.ldvt = ldvt;
    pr.seed = p->seed; pr.stream = p->stream;  // the same Philox stream: Omega's columns nest
    pr.info = info;
    pr.max_sweeps = p->max_sweeps > 0 ? p->max_sweeps : 40;
    pr.serial = (p->flags & RSVD_FLAG_SERIAL) ? 1 : 0;
    rc = run_batched(probs, &pk, base + L.rsvd, L.E - L.rsvd, s);
    if (rc) return rc;
    // E = A - Q B: the residual of the projection, ||E||_F^2 = ||(I - Q Q^T) A||_F^2
    RSVD_TRY(cudaMemcpy2DAsync(E, (size_t)n * 8, A, (size_t)lda * 8, (size_t)n * 8, m, cudaMemcpyDeviceToDevice, s));
    GemmBatch<double, double> g;
    g.count = 1;
    g.job[0] = GemmJob<double, double>{m, n, pr.l, pr.l, n, n, (const double*)pr.Y0, pr.Bm, E, nullptr, nullptr, 0};
    g.job[0].alpha = -1.0;
    g.job[0].accumulate = 1;
    RSVD_TRY((launch_gemm<double, double, false, false>(g, s)));
    RSVD_TRY(launch_sq_sum(E, m, n, n, r2p, s));
    RSVD_TRY(launch_tol_rank(pr.sig, pr.l, kt, r2p, fro2p, eps, res, s));
    RSVD_TRY(cudaMemcpyAsync(&host, res, sizeof(TolResult), cudaMemcpyDeviceToHost, s));
    RSVD_TRY(cudaStreamSynchronize(s));
    if (!host.grow || kt >= kcap) break;
    kt = std::min(2 * kt, kcap);
  }
  *k_out = host.k;
  *err_out = host.err;
  return RSVD_OK;
}

// ---------------------------------------------------------------- TEBD
namespace {
struct TebdLayout {
  size_t t2, thetaB, theta, S, nrm, fro2, keff, rsvd;
};
size_t tebd_bond_bytes(int m, int n, int k, int l, int oz, TebdLayout* o) {
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t x = off;
    off += align_up(b);
    return x;
  };
  TebdLayout L;
  L.t2 = take((size_t)m * n * 8);
  L.thetaB = take((size_t)m * n * 8);
  L.theta = take((size_t)m * n * 8);
  L.S = take((size_t)k * 8);
  L.nrm = take(8);
  L.fro2 = take(64 * 8);
  L.keff = take(sizeof(int));
  L.rsvd = off;
  off += layout(nullptr, m, n, k, l, 8, nullptr, 0, oz);
  if (o) *o = L;
  return off;
}
}  // namespace

int tebd_workspace_size(int L, int d, const int* D, int nb, const rsvd_params* p, size_t* bytes) {
  int rc = check_params(p);
  if (rc) return rc;
  if (!D || !bytes) return RSVD_ERR_NULL_POINTER;
  if (L < 2 || d < 1 || nb < 1) return RSVD_ERR_INVALID_SIZE;
  size_t mx = 0;
  for (int i = 0; i + 1 < L; ++i) {
    const int m = D[i] * d, n = d * D[i + 2], k = D[i + 1];
    if (k < 1 || k > std::min(m, n)) return RSVD_ERR_INVALID_SIZE;
    const int l = b_rows(m, n, k, p);
    if (l > kMaxSample) return RSVD_ERR_INVALID_SIZE;
    mx = std::max(mx, tebd_bond_bytes(m, n, k, l, use_oz(m, n, l, exact_of(m, l, p), p), nullptr));
  }
  *bytes = mx * (size_t)nb;
  return RSVD_OK;
}

int tebd_bond_update(int L, int d, const int* D, int nb, const int* bond, double* B, size_t tensor_stride, double* lam,
                     size_t lam_stride, const double* gate, const rsvd_params* p, double* trunc_err, void* work,
                     size_t work_bytes, rsvd_info* info, void* cuda_stream) {
  int rc = check_params(p);
  if (rc) return rc;
  if (p->prec != RSVD_F64) return RSVD_ERR_PRECISION;
  if (!D || !bond || !B || !lam || !gate || !trunc_err || !work || !info) return RSVD_ERR_NULL_POINTER;
  if (L < 2 || d < 1 || nb < 1 || nb > kMaxJobs) return RSVD_ERR_INVALID_SIZE;
  if (D[0] != 1 || D[L] != 1) return RSVD_ERR_INVALID_SIZE;
  if (((uintptr_t)work) % kAlign) return RSVD_ERR_WORKSPACE;
  for (int b = 0; b < nb; ++b) {
    const int i = bond[b];
    if (i < 0 || i + 1 >= L) return RSVD_ERR_INVALID_SIZE;
    for (int c = 0; c < b; ++c)
      if (std::abs(bond[c] - i) < 2) return RSVD_ERR_INVALID_SIZE;
    const int m = D[i] * d, n = d * D[i + 2], k = D[i + 1];
    if (k < 1 || k > std::min(m, n)) return RSVD_ERR_INVALID_SIZE;
    if (b_rows(m, n, k, p) > kMaxSample) return RSVD_ERR_INVALID_SIZE;
    if ((size_t)D[i] * d * D[i + 1] > tensor_stride || (size_t)D[i + 1] * d * D[i + 2] > tensor_stride) return RSVD_ERR_INVALID_SIZE;
    if ((size_t)D[i + 1] > lam_stride) return RSVD_ERR_INVALID_SIZE;
  }
  size_t per = 0;
  for (int i = 0; i + 1 < L; ++i) {
    const int m = D[i] * d, n = d * D[i + 2], k = D[i + 1];
    const int l = b_rows(m, n, k, p);
    per = std::max(per, tebd_bond_bytes(m, n, k, l, use_oz(m, n, l, exact_of(m, l, p), p), nullptr));
  }
  if (per * (size_t)nb > work_bytes) return RSVD_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  char* base = (char*)work;
  std::vector<TebdLayout> lay(nb);
  std::vector<Prob> probs(nb);
  GemmBatch<double, double> g2;
  g2.count = nb;
  TebdBatch tb;
  tb.count = nb;
  TebdRankBatch rb;
  rb.count = nb;
  for (int b = 0; b < nb; ++b) {
    const int i = bond[b];
    const int Dl = D[i], Dm = D[i + 1], Dr = D[i + 2];
    const int m = Dl * d, n = d * Dr, k = Dm;
    const int l = b_rows(m, n, k, p);
    char* wb = base + per * b;
    const int oz = use_oz(m, n, l, exact_of(m, l, p), p);
    tebd_bond_bytes(m, n, k, l, oz, &lay[b]);
    double* T2 = (double*)(wb + lay[b].t2);
    double* thB = (double*)(wb + lay[b].thetaB);
    double* th = (double*)(wb + lay[b].theta);
    double* Bi = B + tensor_stride * i;
    double* Bj = B + tensor_stride * (i + 1);
    // T2[(a,t1),(t2,c)] = sum_b B_i[(a,t1), b] B_{i+1}[b, (t2,c)]; b runs over the bond's
    // nonzero Schmidt values only (the rows of B_{i+1} and the columns of B_i of a zero
    // Schmidt value are zero: they were set so by the truncation and no later update of a
    // neighbouring bond fills them)
    g2.job[b] = GemmJob<double, double>{m, n, Dm, Dm, n, n, Bi, Bj, T2, nullptr, nullptr, 0};
    g2.job[b].k_eff = (const int*)(wb + lay[b].keff);
    rb.job[b] = TebdRankJob{lam + lam_stride * (i + 1), Dm, (int*)(wb + lay[b].keff)};
    tb.job[b] = TebdJob{Dl, Dr, d, T2, gate + (size_t)b * d * d * d * d, lam + lam_stride * i, thB, th,
                        (double*)(wb + lay[b].fro2)};
    Prob& pr = probs[b];
    std::memset(&pr, 0, sizeof(Prob));
    pr.m = m; pr.n = n; pr.k = k; pr.l = l;
    pr.exact = exact_of(m, l, p);
    pr.want_u = 0;
    pr.A = th; pr.lda = n;
    pr.S = (double*)(wb + lay[b].S);
    pr.U = nullptr; pr.ldu = k;
    pr.Vt = Bj; pr.ldvt = n;     // V^T is the new B_{i+1} (k x d D_r)
    pr.seed = p->seed; pr.stream = p->stream + (uint64_t)i;
    pr.info = info + b;
    pr.max_sweeps = p->max_sweeps > 0 ? p->max_sweeps : 40;
    pr.serial = (p->flags & RSVD_FLAG_SERIAL) ? 1 : 0;
    layout(&pr, m, n, k, l, 8, wb + lay[b].rsvd, 0, oz);
  }
  RSVD_TRY(launch_tebd_rank(rb, s));
  RSVD_TRY((launch_gemm<double, double, false, false>(g2, s)));
  RSVD_TRY(launch_tebd_theta(tb, s));
  rc = run_chunk<double>(probs, p->q, s);
  if (rc) return rc;
  TebdFinBatch fb;
  fb.count = nb;
  GemmBatch<double, double> g3;
  g3.count = nb;
  for (int b = 0; b < nb; ++b) {
    const int i = bond[b];
    char* wb = base + per * b;
    const int m = D[i] * d, n = d * D[i + 2], k = D[i + 1];
    double* nrm = (double*)(wb + lay[b].nrm);
    fb.job[b] = TebdFinJob{k, (double*)(wb + lay[b].S), lam + lam_stride * (i + 1), nrm,
                           (double*)(wb + lay[b].fro2), trunc_err + b};
    // B_i <- theta_B V / ||S||   (V^T now stored in B_{i+1})
    g3.job[b] = GemmJob<double, double>{m, k, n, n, n, k, (double*)(wb + lay[b].thetaB), B + tensor_stride * (i + 1),
                                        B + tensor_stride * i, nrm, nullptr, 0};
    // B = Q^T A has at most rank_eff nonzero rows, so V^T has at most that many
    // nonzero rows (zero singular values sort last): the columns of B_i beyond
    // them are exact zeros
    g3.job[b].n_eff = probs[b].flag + 2;
  }
  RSVD_TRY(launch_tebd_finish(fb, s));
  RSVD_TRY((launch_gemm<double, double, false, true>(g3, s)));
  return RSVD_OK;
}

namespace {
struct TebdProdLayout {
  size_t xb, x, y, g1, g2, S, nrm, fro2, rsvd;
};
size_t tebd_prod_bytes(int m, int n, int k, int l, int r, TebdProdLayout* o) {
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t x = off;
    off += align_up(b);
    return x;
  };
  TebdProdLayout L;
  L.xb = take((size_t)m * r * 8);
  L.x = take((size_t)m * r * 8);
  L.y = take((size_t)r * n * 8);
  L.g1 = take((size_t)r * r * 8);
  L.g2 = take((size_t)r * r * 8);
  L.S = take((size_t)k * 8);
  L.nrm = take(8);
  L.fro2 = take(64 * 8);
  L.rsvd = off;
  off += layout(nullptr, m, n, k, l, 8, nullptr, 0, 0, r);
  if (o) *o = L;
  return off;
}

// per-bond workspace of the product update over all bonds of the chain (0: invalid sizes)
size_t tebd_prod_per_bond(int L, int d, const int* D, int K, int pp) {
  size_t mx = 0;
  for (int i = 0; i + 1 < L; ++i) {
    const int m = D[i] * d, n = d * D[i + 2], k = D[i + 1];
    if (k < 1 || k > std::min(m, n)) return 0;
    const int l = sample_width(m, n, k, pp);
    if (l > kMaxSample) return 0;
    mx = std::max(mx, tebd_prod_bytes(m, n, k, l, K * k, nullptr));
  }
  return mx;
}
}  // namespace

int tebd_product_workspace_size(int L, int d, const int* D, int nb, int K, const rsvd_params* p, size_t* bytes) {
  int rc = check_params(p);
  if (rc) return rc;
  if (p->flags & RSVD_FLAG_FULL_SVD) return RSVD_ERR_INVALID_SIZE;
  if (!D || !bytes) return RSVD_ERR_NULL_POINTER;
  if (L < 2 || d < 1 || nb < 1 || K < 1) return RSVD_ERR_INVALID_SIZE;
  const size_t per = tebd_prod_per_bond(L, d, D, K, p->p);
  if (per == 0) return RSVD_ERR_INVALID_SIZE;
  *bytes = per * (size_t)nb;
  return RSVD_OK;
}

int tebd_product_update(int L, int d, const int* D, int nb, const int* bond, double* B, size_t tensor_stride,
                        double* lam, size_t lam_stride, int K, const double* uL, const double* uR,
                        const rsvd_params* p, double* trunc_err, void* work, size_t work_bytes, rsvd_info* info,
                        void* cuda_stream) {
  int rc = check_params(p);
  if (rc) return rc;
  if (p->flags & RSVD_FLAG_FULL_SVD) return RSVD_ERR_INVALID_SIZE;
  if (p->prec != RSVD_F64) return RSVD_ERR_PRECISION;
  if (!D || !bond || !B || !lam || !uL || !uR || !trunc_err || !work || !info) return RSVD_ERR_NULL_POINTER;
  if (L < 2 || d < 1 || nb < 1 || nb > kMaxJobs || K < 1) return RSVD_ERR_INVALID_SIZE;
  if (D[0] != 1 || D[L] != 1) return RSVD_ERR_INVALID_SIZE;
  if (((uintptr_t)work) % kAlign) return RSVD_ERR_WORKSPACE;
  for (int b = 0; b < nb; ++b) {
    const int i = bond[b];
    if (i < 0 || i + 1 >= L) return RSVD_ERR_INVALID_SIZE;
    for (int c = 0; c < b; ++c)
      if (std::abs(bond[c] - i) < 2) return RSVD_ERR_INVALID_SIZE;
    if ((size_t)D[i] * d * D[i + 1] > tensor_stride || (size_t)D[i + 1] * d * D[i + 2] > tensor_stride) return RSVD_ERR_INVALID_SIZE;
    if ((size_t)D[i + 1] > lam_stride) return RSVD_ERR_INVALID_SIZE;
  }
  const size_t per = tebd_prod_per_bond(L, d, D, K, p->p);
  if (per == 0) return RSVD_ERR_INVALID_SIZE;
  if (per * (size_t)nb > work_bytes) return RSVD_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  char* base = (char*)work;
  std::vector<TebdProdLayout> lay(nb);
  std::vector<Prob> probs(nb);
  TebdProdBatch tp;
  tp.count = nb;
  GemmBatch<double, double> g1, g2;
  g1.count = g2.count = nb;
  TebdGramDotBatch gd;
  gd.count = nb;
  for (int b = 0; b < nb; ++b) {
    const int i = bond[b];
    const int Dl = D[i], Dm = D[i + 1], Dr = D[i + 2];
    const int m = Dl * d, n = d * Dr, k = Dm, r = K * Dm;
    const int l = sample_width(m, n, k, p->p);
    char* wb = base + per * b;
    tebd_prod_bytes(m, n, k, l, r, &lay[b]);
    double* XB = (double*)(wb + lay[b].xb);
    double* X = (double*)(wb + lay[b].x);
    double* Y = (double*)(wb + lay[b].y);
    double* G1 = (double*)(wb + lay[b].g1);
    double* G2 = (double*)(wb + lay[b].g2);
    tp.job[b] = TebdProdJob{Dl, Dm, Dr, d, K, B + tensor_stride * i, B + tensor_stride * (i + 1),
                            uL + (size_t)b * K * d * d, uR + (size_t)b * K * d * d, lam + lam_stride * i, XB, X, Y};
    // ||theta||_F^2 = trace((X^T X)(Y Y^T)), theta = X Y never formed
    g1.job[b] = GemmJob<double, double>{r, r, m, r, r, r, X, X, G1, nullptr, nullptr, 0};
    g2.job[b] = GemmJob<double, double>{r, r, n, n, n, r, Y, Y, G2, nullptr, nullptr, 0};
    gd.job[b] = TebdGramDotJob{r, G1, G2, (double*)(wb + lay[b].fro2)};
    Prob& pr = probs[b];
    std::memset(&pr, 0, sizeof(Prob));
    pr.m = m; pr.n = n; pr.k = k; pr.l = l;
    pr.exact = 0;
    pr.want_u = 0;
    pr.r = r; pr.Xf = X; pr.ldxf = r; pr.Yf = Y; pr.ldyf = n;
    pr.S = (double*)(wb + lay[b].S);
    pr.U = nullptr; pr.ldu = k;
    pr.Vt = B + tensor_stride * (i + 1); pr.ldvt = n;  // V^T is the new B_{i+1}
    pr.seed = p->seed; pr.stream = p->stream + (uint64_t)i;
    pr.info = info + b;
    pr.max_sweeps = p->max_sweeps > 0 ? p->max_sweeps : 40;
    pr.serial = (p->flags & RSVD_FLAG_SERIAL) ? 1 : 0;
    layout(&pr, m, n, k, l, 8, wb + lay[b].rsvd, 0, 0, r);
  }
  RSVD_TRY(launch_tebd_product(tp, s));
  RSVD_TRY((launch_gemm<double, double, true, false>(g1, s)));
  RSVD_TRY((launch_gemm<double, double, false, true>(g2, s)));
  RSVD_TRY(launch_tebd_gram_dot(gd, s));
  rc = run_chunk<double>(probs, p->q, s);
  if (rc) return rc;
  TebdFinBatch fb;
  fb.count = nb;
  GemmBatch<double, double> g3, g4;
  g3.count = g4.count = nb;
  for (int b = 0; b < nb; ++b) {
    const int i = bond[b];
    char* wb = base + per * b;
    const int m = D[i] * d, n = d * D[i + 2], k = D[i + 1], r = K * k;
    double* nrm = (double*)(wb + lay[b].nrm);
    fb.job[b] = TebdFinJob{k, (double*)(wb + lay[b].S), lam + lam_stride * (i + 1), nrm,
                           (double*)(wb + lay[b].fro2), trunc_err + b};
    // B_i <- theta_B V / ||S|| = XB (Y V) / ||S||, V^T now in B_{i+1}; W = Y V (r x k) reuses
    // the factored products' r x l buffer
    double* Wv = (double*)probs[b].Wf;
    g3.job[b] = GemmJob<double, double>{r, k, n, n, n, k, (double*)(wb + lay[b].y), B + tensor_stride * (i + 1), Wv,
                                        nullptr, nullptr, 0};
    g3.job[b].n_eff = probs[b].flag + 2;
    g4.job[b] = GemmJob<double, double>{m, k, r, r, k, k, (double*)(wb + lay[b].xb), Wv, B + tensor_stride * i, nrm,
                                        nullptr, 0};
    g4.job[b].n_eff = probs[b].flag + 2;
  }
  RSVD_TRY(launch_tebd_finish(fb, s));
  RSVD_TRY((launch_gemm<double, double, false, true>(g3, s)));
  RSVD_TRY((launch_gemm<double, double, false, false>(g4, s)));
  return RSVD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- complex matrices
namespace rsvd {
namespace {
struct CplxLayout {
  size_t R, Ur, Vtr, Sr, rsvd, total;
};
// workspace of the complex call: R(A) (2m x 2n), the real factors (2m x 2k, 2k x 2n, 2k
// values) and the real call's workspace for R(A) at rank 2k, oversampling 2p
int cplx_layout(int m, int n, const rsvd_params* p, CplxLayout* L) {
  const size_t ts = tsize_of(p->prec);
  rsvd_params q = *p;
  q.k = 2 * p->k;
  q.p = 2 * p->p;
  size_t real = 0;
  const int m2 = 2 * m, n2 = 2 * n;
  int rc = rsvd_workspace_size(m2, n2, &q, &real);
  if (rc) return rc;
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t x = off;
    off += align_up(b);
    return x;
  };
  L->R = take((size_t)m2 * n2 * ts);
  L->Ur = take((size_t)m2 * q.k * ts);
  L->Vtr = take((size_t)q.k * n2 * ts);
  L->Sr = take((size_t)q.k * 8);
  L->rsvd = take(real);
  L->total = off;
  return RSVD_OK;
}
}  // namespace
}  // namespace rsvd

extern "C" int rsvd_complex_workspace_size(int m, int n, const rsvd_params* p, size_t* bytes) {
  using namespace rsvd;
  int rc = check_params(p);
  if (rc) return rc;
  if (!bytes) return RSVD_ERR_NULL_POINTER;
  if (p->prec != RSVD_F64 && p->prec != RSVD_F32) return RSVD_ERR_PRECISION;
  if (m < 1 || n < 1 || p->k < 1 || p->k > std::min(m, n)) return RSVD_ERR_INVALID_SIZE;
  CplxLayout L;
  rc = cplx_layout(m, n, p, &L);
  if (rc) return rc;
  *bytes = L.total;
  return RSVD_OK;
}

extern "C" int rsvd_truncate_complex(int m, int n, const void* A, int lda, const rsvd_params* p, double* S, void* U,
                                     int ldu, void* Vh, int ldvh, void* work, size_t work_bytes, rsvd_info* info,
                                     void* cuda_stream) {
  using namespace rsvd;
  size_t need = 0;
  int rc = rsvd_complex_workspace_size(m, n, p, &need);
  if (rc) return rc;
  if (!A || !S || !U || !Vh || !work || !info) return RSVD_ERR_NULL_POINTER;
  if (lda < n || ldu < p->k || ldvh < n) return RSVD_ERR_INVALID_SIZE;
  if (((uintptr_t)work) % kAlign) return RSVD_ERR_WORKSPACE;
  if (need > work_bytes) return RSVD_ERR_WORKSPACE;
  CplxLayout L;
  cplx_layout(m, n, p, &L);
  char* base = (char*)work;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const bool f64 = p->prec == RSVD_F64;
  RSVD_TRY(f64 ? launch_realify<double>(m, n, (const double*)A, lda, (double*)(base + L.R), s)
               : launch_realify<float>(m, n, (const float*)A, lda, (float*)(base + L.R), s));
  rsvd_params q = *p;
  q.k = 2 * p->k;
  q.p = 2 * p->p;
  std::vector<Prob> probs(1);
  Prob& pr = probs[0];
  std::memset(&pr, 0, sizeof(Prob));
  pr.m = 2 * m; pr.n = 2 * n; pr.k = q.k;
  pr.l = b_rows(pr.m, pr.n, pr.k, &q);  // 2 min(k + p, m, n), or 2m for Alg. TSVD
  pr.exact = exact_of(pr.m, pr.l, &q);
  pr.want_u = 1;
  pr.A = base + L.R; pr.lda = 2 * n;
  pr.S = (double*)(base + L.Sr);
  pr.U = base + L.Ur; pr.ldu = q.k;
  pr.Vt = base + L.Vtr; pr.ldvt = 2 * n;
  pr.seed = p->seed; pr.stream = p->stream;
  pr.info = info;
  pr.max_sweeps = p->max_sweeps > 0 ? p->max_sweeps : 40;
  pr.serial = (p->flags & RSVD_FLAG_SERIAL) ? 1 : 0;
  pr.no_exchange = (p->flags & RSVD_FLAG_TEST_NO_EXCHANGE) ? 1 : 0;
  pr.cplx = 1;
  rc = run_batched(probs, &q, base + L.rsvd, L.total - L.rsvd, s);
  if (rc) return rc;
  RSVD_TRY(f64 ? launch_complex_extract<double>(m, n, p->k, pr.S, (const double*)pr.U, q.k, (const double*)pr.Vt,
                                                2 * n, S, (double*)U, ldu, (double*)Vh, ldvh, s)
               : launch_complex_extract<float>(m, n, p->k, pr.S, (const float*)pr.U, q.k, (const float*)pr.Vt,
                                               2 * n, S, (float*)U, ldu, (float*)Vh, ldvh, s));
  return RSVD_OK;
}

// ---------------------------------------------------------------- no-allocation entry point
// Some callers cannot hand the library a workspace: code that runs where
// device allocation is forbidden or unavailable after start-up (a host
// framework that owns and pre-reserves all device memory, a real-time loop with
// a fixed memory budget, a plain C caller without any allocator).  For them,
// rsvd_truncate_noalloc runs the same computation as rsvd_truncate with its
// scratch in a fixed array that lives in this library's device image.
#include <mutex>

namespace rsvd {
namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB, held by every GPU that loads the library
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxScratchDevices = 64;
struct ScratchAddr {
  void* ctx;  // the context the address belongs to
  void* ptr;
};
ScratchAddr g_scratch_dev_ptr[kMaxScratchDevices] = {};
std::mutex g_scratch_mutex;

// Device address of g_static_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress once per device (with that device current) and cached;
// it is looked up again when the device's context was replaced (after a
// cudaDeviceReset the module, and the array, are loaded anew).  The same set-up
// creates this host thread's side streams and events for the call's independent
// groups of work, so that a first call made before any stream capture leaves
// nothing to create later on this thread.
int static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    last_cuda_error() = e;
    return RSVD_ERR_LAUNCH;
  }
  if (dev < 0 || dev >= kMaxScratchDevices) return RSVD_ERR_INVALID_SIZE;
  if (!side_streams()) {
    last_cuda_error() = cudaGetLastError();
    return RSVD_ERR_LAUNCH;
  }
  void* ctx = current_context();
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  ScratchAddr& a = g_scratch_dev_ptr[dev];
  if (!a.ptr || a.ctx != ctx) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      last_cuda_error() = e;
      return RSVD_ERR_LAUNCH;
    }
    a.ptr = ptr;
    a.ctx = ctx;
  }
  *out = a.ptr;
  return RSVD_OK;
}

}  // namespace
}  // namespace rsvd

extern "C" int rsvd_truncate_noalloc(int m, int n, const void* A, int lda, const rsvd_params* p, double* S, void* U,
                                     int ldu, void* Vt, int ldvt, rsvd_info* info, void* cuda_stream) {
  size_t need = 0;
  int rc = rsvd_workspace_size(m, n, p, &need);
  if (rc != RSVD_OK) return rc;
  rsvd_params q = *p;
  if (need > kStaticScratchBytes && p->prec == RSVD_F64 && !(p->flags & RSVD_FLAG_F64_SIMT)) {
    // the FP64 products' tensor-core slices of A and A^T do not fit: the products
    // with FP64 FMAs need none (the same factorization within the FP64 bar)
    q.flags |= RSVD_FLAG_F64_SIMT;
    rc = rsvd_workspace_size(m, n, &q, &need);
    if (rc != RSVD_OK) return rc;
  }
  if (need > kStaticScratchBytes) return RSVD_ERR_SCRATCH_LIMIT;
  void* scratch = nullptr;
  rc = static_scratch(&scratch);
  if (rc != RSVD_OK) return rc;
  return rsvd_truncate(m, n, A, lda, &q, S, U, ldu, Vt, ldvt, scratch, kStaticScratchBytes, info, cuda_stream);
}

extern "C" size_t rsvd_noalloc_scratch_bytes(void) { return kStaticScratchBytes; }
