// Small SVD of B = Q^T A (l x n, FP64): Alg. RSVD step 4 (Sec. II.B), the
// rank-k TSVD of B.  One-sided Jacobi (Hestenes; Demmel-Veselic) on the ROWS
// of B: plane rotations P B = W until the rows of W are mutually orthogonal;
// then sigma_i = ||w_i||, V~ rows = w_i / sigma_i and U~ = P^T (P is
// accumulated only when U is wanted: the TEBD bond update uses S and V only).
//
// GB300 layout: one thread-block CLUSTER per matrix.  The n columns of B (and
// the l columns of the rotation accumulator P) are split across the CTAs of
// the cluster and stay in each CTA's shared memory for the whole
// factorization.  Rows are paired by the round-robin (circle) ordering, l/2
// disjoint pairs per round.  Per round every CTA forms the partial inner
// products <b_i, b_j> of its column slice (teams of 4 lanes per pair), pushes
// them to every CTA of the cluster through distributed shared memory, one lane
// per pair sums them in rank order and forms the rotation - so all CTAs take
// bit-identical decisions, and the FP64 scalar work (square roots, divisions)
// occupies as few warps as possible - and teams of 8 lanes rotate their own
// slice.
//
// On this part a warp issues at most one FP64 instruction per 64 cycles, with
// any number of active lanes and whatever its independent work, and an SM
// about one per 16-19 cycles over all its warps (measured): the kernel's time
// follows its count of FP64 warp instructions, so sums over the cluster take
// exactly C - 1 additions.
//
// Row norms are recomputed exactly at the start of every sweep and updated by
// the rotation identities (alpha - t gamma, beta + t gamma) inside it.  A pair
// is rotated when |gamma| > tol sqrt(alpha beta), tol = n 2^-53.
// Deflation: at the start of every sweep, rows whose norm is at most 2^-52 of
// the largest row norm are set to zero - they are rounding noise of the
// computed B (a backward perturbation below eps ||B||) - and the round-robin
// ordering then runs over the remaining live rows only.  Zero rows give
// singular value 0 with a zero row of V^T.  The loop ends after a sweep
// without rotations, after a sweep whose rotations were all small enough that
// the next one would find every pair converged (see below), or at the sweep
// cap (status RSVD_WARN_NOCONV).
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace rsvd {

namespace {

constexpr int kJacobiThreads = 512;
constexpr int kMaxCluster = 16;  // cluster sizes up to 16 (non-portable above 8)
constexpr int kTeam = 8;     // lanes per row pair in the rotation phase
constexpr int kTeamDot = 4;  // lanes per row pair in the inner-product phase: two levels of shuffle
                             // additions per pair instead of three (an FP64 warp instruction holds
                             // the pipe for 16 cycles, so the reduction's additions cost as much
                             // as the products themselves with 8 lanes)
constexpr int kScalarThreads = 128;  // warps 0-3 form the rotation scalars, up to two per half of a round
// threads at the barrier of a half: its scalar warps (arrive) and the worker warps (wait)
constexpr int kWorkerThreads = kJacobiThreads - kScalarThreads;
constexpr size_t kSmemBudget = 220 * 1024;

// Round r of the circle ordering over lp (even) rows: pair s is (m, r) for s = 0 and
// ((r + s) mod m, (r - s) mod m) otherwise, m = lp - 1; 0 <= r, s < m, so each reduction is
// one conditional subtraction or addition
__device__ __forceinline__ void round_pair(int r, int s, int lp, int& i, int& j) {
  const int m = lp - 1;
  int a, bb;
  if (s == 0) {
    a = m;
    bb = r;
  } else {
    a = r + s;
    a -= a >= m ? m : 0;
    bb = r - s;
    bb += bb < 0 ? m : 0;
  }
  i = min(a, bb);
  j = max(a, bb);
}

struct JLayout {
  int nc, np, npairs, lp, cs;
};

__host__ __device__ inline JLayout jlayout(int l, int n, int csize) {
  JLayout L;
  L.nc = (n + csize - 1) / csize;
  L.np = (l + csize - 1) / csize;
  L.lp = l + (l & 1);
  L.npairs = L.lp / 2;
  L.cs = csize;
  return L;
}

__host__ __device__ inline size_t jsmem_small(int l, const JLayout& L) {
  // norms, nrm_part, gpart[2][cluster size][npairs] (every CTA's partial of every
  // pair, pushed), order (int, padded to doubles), the rotations' two update
  // coefficients [npairs] and flags (int, padded), the rows' scale factors and their
  // inverses [l each], the rotations' tangents and inner products [npairs each]
  return sizeof(double) * ((size_t)2 * l + (2 * (size_t)L.cs + 2) * L.npairs + (size_t)(l + 1) / 2 + 1 +
                           (size_t)(L.npairs + 1) / 2 + 1 + (size_t)2 * l + (size_t)2 * L.npairs);
}

// Sum over the CTAs of the cluster of v[i] in their shared memory: every
// remote load in flight at once, then a fixed pairwise tree (so every CTA gets
// the same bits, and the dependent FP64 adds are log2 C deep, not C).
__device__ __forceinline__ double cluster_tree_sum(cg::cluster_group& cluster, const double* v, int i, int C) {
  double pv[kMaxCluster];
#pragma unroll
  for (int r = 0; r < kMaxCluster; ++r) pv[r] = r < C ? cluster.map_shared_rank(v, r)[i] : 0.0;
#pragma unroll
  for (int w = 1; w < kMaxCluster; w <<= 1)
#pragma unroll
    for (int r = 0; r + w < kMaxCluster; r += 2 * w) pv[r] += pv[r + w];
  return pv[0];
}

// Sum of the C partials slot[q * stride], q < C, by a fixed pairwise tree over exactly C
// terms (C - 1 FP64 additions: each costs a whole warp instruction, about 64 cycles of its
// warp's issue, whatever its active lanes), so every CTA gets the same bits with log2 depth
__device__ __forceinline__ double tree_sum(const double* slot, int stride, int C) {
  double v[kMaxCluster];
#pragma unroll
  for (int q = 0; q < kMaxCluster; ++q) v[q] = q < C ? slot[q * stride] : 0.0;
  switch (C) {  // cluster-uniform
    case 1: return v[0];
    case 2: return v[0] + v[1];
    case 3: return (v[0] + v[1]) + v[2];
    case 4: return (v[0] + v[1]) + (v[2] + v[3]);
    case 5: return ((v[0] + v[1]) + (v[2] + v[3])) + v[4];
    case 6: return ((v[0] + v[1]) + (v[2] + v[3])) + (v[4] + v[5]);
    case 7: return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + v[6]);
    case 8: return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    default: break;
  }
#pragma unroll
  for (int w = 1; w < kMaxCluster; w <<= 1)
#pragma unroll
    for (int q = 0; q + w < kMaxCluster; q += 2 * w)
      if (q + w < C) v[q] += v[q + w];
  return v[0];
}

// Named barriers between the scalar warps (arrive) and the worker warps (sync): the
// workers wait until the scalars of a half are written; bar.arrive orders the arriving
// threads' shared-memory writes before the waiters' reads
// (ids 1 and 2 for halves A and B; id 0 is __syncthreads), over n threads: the half's
// scalar warps and the worker warps
__device__ __forceinline__ void half_sync(int h, int n) {
  __syncwarp();  // the barrier instructions are warp-aligned: reconverge first
  if (h == 0)
    asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
  else
    asm volatile("bar.sync 2, %0;" ::"r"(n) : "memory");
}
__device__ __forceinline__ void half_arrive(int h, int n) {
  __syncwarp();
  if (h == 0)
    asm volatile("bar.arrive 1, %0;" ::"r"(n) : "memory");
  else
    asm volatile("bar.arrive 2, %0;" ::"r"(n) : "memory");
}

// Point-to-point signals between the CTAs of a cluster: a value stored into
// another CTA's shared memory completes 8 bytes of that CTA's mbarrier, and the
// receiver waits on its own mbarrier (cluster-scope acquire).
__device__ __forceinline__ uint32_t cluster_addr(const void* p, int rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void push_f64(double* slot, uint64_t* bar, int rank, double v) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(cluster_addr(slot, rank)),
               "d"(v), "r"(cluster_addr(bar, rank))
               : "memory");
}
__device__ __forceinline__ void mb_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)) : "memory");
}
__device__ __forceinline__ void mb_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)),
               "r"(bytes)
               : "memory");
}
// gives up after about 2^28 cycles (0.13 s) and returns false
__device__ __forceinline__ bool mb_wait_cluster(uint64_t* bar, uint32_t parity) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1LL << 28)) return false;
  }
}

template <typename T>
__global__ void __launch_bounds__(kJacobiThreads, 2) jacobi_kernel(const __grid_constant__ JacobiBatch<T> b) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = b.csize;
  const int rank = (int)cluster.block_rank();
  const JacobiJob<T>& J = b.job[blockIdx.y];
  if (J.active && !*J.active) return;  // an inactive job (whole CTA / cluster, before any barrier)
  const int l = J.l, n = J.n;
  const JLayout L = jlayout(l, n, C);
  const int c0 = rank * L.nc, ncl = max(0, min(n, c0 + L.nc) - c0);
  const int p0 = rank * L.np, npl = max(0, min(l, p0 + L.np) - p0);

  extern __shared__ double sm[];
  double* norms = sm;
  double* nrm_part = norms + l;
  double* gpart = nrm_part + l;                 // [2][C][npairs]: the CTAs' partials, pushed
  int* order = (int*)(gpart + 2 * C * L.npairs);
  double* rcs = gpart + 2 * C * L.npairs + (l + 1) / 2 + 1;  // per pair of the round: the update
  double* rsn = rcs + L.npairs;                                // coefficients, rotate?
  int* rfl = (int*)(rsn + L.npairs);
  // Rows are stored scaled (fast Givens form): row i of the matrix is dsc[i] times the
  // stored row, so a rotation updates each element pair with two FMAs instead of four
  // multiplications and additions; isc = 1 / dsc.  The scales shrink by cos(theta) >= 1/sqrt(2)
  // per rotation and are folded back into the rows at every sweep head and every 64 rounds.
  double* dsc = rsn + L.npairs + (L.npairs + 1) / 2 + 1;
  double* isc = dsc + l;
  double* rtan = isc + l;           // per pair of the round: the tangent t and the inner product g,
  double* rgam = rtan + L.npairs;   // kept for the scale and norm updates after the coefficients
  double* Bs;
  double* Ps;
  if (b.use_global) {
    Bs = J.Bg + (size_t)rank * l * L.nc;
    Ps = J.Pg + (size_t)rank * l * L.np;
  } else {
    Bs = sm + jsmem_small(l, L) / sizeof(double);
    Ps = Bs + (size_t)l * L.nc;
  }
  __shared__ int rot_count;
  __shared__ int big_rot;  // a rotation of this sweep had |g| > thr sqrt(alpha beta)
  __shared__ int nonfinite;
  __shared__ int nlive;
  __shared__ double rowmax;
  int* live = order;  // live-row list during the sweeps; the sort order afterwards

  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  // the worker warps' teams (wid < 0 in the scalar warps, which never use them)
  const int wid = tid - kScalarThreads;
  const int team = wid / kTeam, tl = wid % kTeam, nteam = (kJacobiThreads - kScalarThreads) / kTeam;
  const int dteam = wid / kTeamDot, dl = wid % kTeamDot, ndteam = (kJacobiThreads - kScalarThreads) / kTeamDot;
  const unsigned dmask = 0xfu << ((tid % 32) / kTeamDot * kTeamDot);  // this inner-product team's lanes
  for (int e = tid; e < l * L.nc; e += kJacobiThreads) {
    const int i = e / L.nc, c = e % L.nc;
    Bs[e] = (c < ncl) ? J.Bm[(size_t)i * n + c0 + c] : 0.0;
  }
  const bool want_p = J.want_p != 0;
  if (want_p)
    for (int e = tid; e < l * L.np; e += kJacobiThreads) {
      const int i = e / L.np, c = e % L.np;
      Ps[e] = (c < npl && i == p0 + c) ? 1.0 : 0.0;
    }
  for (int i = tid; i < l; i += kJacobiThreads) {
    dsc[i] = 1.0;
    isc[i] = 1.0;
  }
  // fold the scale factors into the stored rows (every CTA at the same points: the
  // factors are identical across the cluster, as are all rotation decisions)
  auto rescale = [&]() {
    for (int e = tid; e < l * L.nc; e += kJacobiThreads) Bs[e] *= dsc[e / L.nc];
    if (want_p)
      for (int e = tid; e < l * L.np; e += kJacobiThreads) Ps[e] *= dsc[e / L.np];
    __syncthreads();
    for (int i = tid; i < l; i += kJacobiThreads) {
      dsc[i] = 1.0;
      isc[i] = 1.0;
    }
    __syncthreads();
  };
  __shared__ uint64_t mbR[2][2];  // round exchanges of even / odd global round number, halves A / B
  __shared__ int rerr;         // a round exchange timed out
  if (tid == 0) {
    nonfinite = 0;
    rerr = 0;
    mb_init(&mbR[0][0]);
    mb_init(&mbR[0][1]);
    mb_init(&mbR[1][0]);
    mb_init(&mbR[1][1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  uint32_t gr = 0;  // rounds done over all sweeps: the exchange buffer and mbarrier phase
  __syncthreads();

  const double tol = (double)max(n, 1) * 0x1.0p-53;
  const double tol2 = tol * tol;
  const double thr2 = tol2 * 1e8;  // (1e4 tol)^2
  const int max_sweeps = J.max_sweeps;
  int sweeps = 0;
  long long total_rot = 0;
  long long total_pairs = 0;  // inner products formed: nlive (nlive - 1) / 2 per sweep
  int myrot = 0;              // rotations of this sweep formed by this thread
  bool converged = false;
  for (;;) {
    if (sweeps > 0) rescale();
    // exact row norms of this sweep (four independent partial sums: a dependent
    // FP64 operation costs about 64 cycles on this part)
    for (int i = tid; i < l; i += kJacobiThreads) {
      const double* row = Bs + (size_t)i * L.nc;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int c = 0;
      for (; c + 3 < ncl; c += 4) {
        s0 = fma(row[c], row[c], s0);
        s1 = fma(row[c + 1], row[c + 1], s1);
        s2 = fma(row[c + 2], row[c + 2], s2);
        s3 = fma(row[c + 3], row[c + 3], s3);
      }
      for (; c < ncl; ++c) s0 = fma(row[c], row[c], s0);
      // a CTA whose round exchange timed out contributes +Inf to row 0: every CTA then
      // sees a non-finite norm after the same sum and leaves the iteration at the same
      // point (no CTA keeps sweeping, or pushing into the shared memory of one that left)
      nrm_part[i] = (i == 0 && rerr) ? __longlong_as_double(0x7ff0000000000000LL) : (s0 + s1) + (s2 + s3);
    }
    cluster.sync();
    for (int i = tid; i < l; i += kJacobiThreads) norms[i] = cluster_tree_sum(cluster, nrm_part, i, C);
    if (tid == 0) {
      rot_count = 0;
      big_rot = 0;
    }
    __syncthreads();
    // norms are >= +0, so finiteness, maxima and comparisons with non-negative
    // thresholds are integer operations on the bit patterns
    for (int i = tid; i < l; i += kJacobiThreads)
      if (((__double_as_longlong(norms[i]) >> 52) & 0x7ff) == 0x7ff) nonfinite = 1;
    __syncthreads();
    if (nonfinite) break;  // identical in every CTA of the cluster
    if (warp == 0) {
      long long mx = 0;
      for (int i = lane; i < l; i += 32) mx = max(mx, __double_as_longlong(norms[i]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) rowmax = __longlong_as_double(mx);
    }
    __syncthreads();
    {
      // (2^-52)^2 of the largest squared row norm
      const long long floor_bits = __double_as_longlong(rowmax * 0x1.0p-104);
      for (int e = tid; e < l * L.nc; e += kJacobiThreads)
        if (!(__double_as_longlong(norms[e / L.nc]) > floor_bits)) Bs[e] = 0.0;
      __syncthreads();
      for (int i = tid; i < l; i += kJacobiThreads)
        if (!(__double_as_longlong(norms[i]) > floor_bits)) norms[i] = 0.0;
      __syncthreads();  // every norm is final before the live list is built
      if (warp == 0) {  // live rows in index order, by ballots
        int nl = 0;
        for (int b0 = 0; b0 < l; b0 += 32) {
          const int i = b0 + lane;
          const bool lv = i < l && __double_as_longlong(norms[i]) > 0;
          const unsigned m = __ballot_sync(0xffffffffu, lv);
          if (lv) live[nl + __popc(m & ((1u << lane) - 1u))] = i;
          nl += __popc(m);
        }
        if (lane == 0) nlive = nl;
      }
      __syncthreads();
    }
    if (converged || sweeps >= max_sweeps) break;

    const int lpl = nlive + (nlive & 1);
    const int npl2 = lpl / 2;
    total_pairs += (long long)nlive * (nlive - 1) / 2;
    // the round's pairs in two halves, A = [0, hA) and B = [hA, npl2): the worker warps form
    // half A's inner products and send them, then half B's, while the scalar warps of
    // half A wait for A's partials and form its rotations; the workers then rotate half A
    // while the scalar warps of half B finish, and rotate half B last.  So the scalars'
    // dependent FP64 chains run beside the products and rotations of the other half
    // instead of holding the whole CTA
    // Half A is a whole number of warps of pairs where it can be, and each half has at
    // most two scalar warps (their lanes loop when a half holds more than 64 pairs): an
    // FP64 warp instruction costs its 16 pipe cycles whatever the active lanes, so a
    // warp with few pairs costs as much as a full one
    const int hA = npl2 >= 64 ? npl2 / 64 * 32 : (npl2 + 1) / 2;
    const int pw0 = min(2, (hA + 31) / 32), pw1 = min(2, (npl2 - hA + 31) / 32);
    for (int r = 0; r < lpl - 1; ++r, ++gr) {
      // after a timed-out exchange (rerr is uniform in the CTA after the round's last
      // __syncthreads) this CTA sends and waits no more; the sweep head then ends the
      // iteration in every CTA (see the row norms), so a CTA waits out at most one limit
      if (rerr) break;
      // this round's partials: slot [q][s] holds CTA q's partial of pair s, stored by
      // that CTA with st.async completing bytes on this CTA's mbarrier of the round's
      // parity and the pair's half; only the scalar warps wait for them, and every CTA
      // sums them in the same order.  A slot (and its mbarriers) of parity gr & 1 is
      // reused two rounds later: a CTA stores round gr + 2 only after receiving
      // everyone's round gr + 1, which each CTA sends after it has read its round gr
      // partials
      double* gp = gpart + (gr & 1) * C * L.npairs;
      uint64_t* mbA = &mbR[gr & 1][0];
      uint64_t* mbB = &mbR[gr & 1][1];
      if (tid == 0) {
        mb_expect(mbA, (uint32_t)C * hA * 8);
        mb_expect(mbB, (uint32_t)C * (npl2 - hA) * 8);
      }
      if (tid >= kScalarThreads) {
        // worker warps: inner products of half A, then of half B, pushed to every CTA
        for (int h = 0; h < 2; ++h) {
          const int s0 = h ? hA : 0, s1 = h ? npl2 : hA;
          uint64_t* mb = h ? mbB : mbA;
          for (int s = s0 + dteam; s < s1; s += ndteam) {
            int a, bq;
            round_pair(r, s, lpl, a, bq);
            double g0 = 0.0, g1 = 0.0;
            if (bq < nlive) {
              const double* xi = Bs + live[a] * L.nc;
              const double* xj = Bs + live[bq] * L.nc;
              int c = dl;
              for (; c + kTeamDot < ncl; c += 2 * kTeamDot) {
                g0 = fma(xi[c], xj[c], g0);
                g1 = fma(xi[c + kTeamDot], xj[c + kTeamDot], g1);
              }
              if (c < ncl) g0 = fma(xi[c], xj[c], g0);
            }
            double g = g0 + g1;
#pragma unroll
            for (int o = kTeamDot / 2; o > 0; o >>= 1) g += __shfl_xor_sync(dmask, g, o, kTeamDot);
            if (!J.no_exchange)
              for (int q = dl; q < C; q += kTeamDot) push_f64(&gp[rank * L.npairs + s], mb, q, g);
          }
        }
        // rotations of half A once its scalars are ready, then of half B
        for (int h = 0; h < 2; ++h) {
          half_sync(h, 32 * (h ? pw1 : pw0) + kWorkerThreads);
          const int s0 = h ? hA : 0, s1 = h ? npl2 : hA;
          for (int s = s0 + team; s < s1; s += nteam) {
            if (!rfl[s]) continue;  // team-uniform
            int a, bq;
            round_pair(r, s, lpl, a, bq);
            const int i = live[a], j = live[bq];
            const double ca = rcs[s], cb = rsn[s];
            for (int c = tl; c < ncl; c += kTeam) {
              const double x = Bs[i * L.nc + c], y = Bs[j * L.nc + c];
              Bs[i * L.nc + c] = fma(-ca, y, x);
              Bs[j * L.nc + c] = fma(cb, x, y);
            }
            for (int c = tl; want_p && c < npl; c += kTeam) {
              const double x = Ps[i * L.np + c], y = Ps[j * L.np + c];
              Ps[i * L.np + c] = fma(-ca, y, x);
              Ps[j * L.np + c] = fma(cb, x, y);
            }
          }
        }
      } else if (warp < pw0 + pw1) {
        // scalar warps: pw0 of them for half A, pw1 for half B; one lane per pair, every
        // CTA summing the partials in rank order, so all CTAs of the cluster take
        // bit-identical decisions
        const int h = warp < pw0 ? 0 : 1;
        const int s0 = h ? hA : 0, s1 = h ? npl2 : hA;
        const int nl = 32 * (h ? pw1 : pw0), sl = tid - (h ? 32 * pw0 : 0);
        if (s0 + sl < s1 && !mb_wait_cluster(h ? mbB : mbA, (gr >> 1) & 1)) atomicExch(&rerr, 1);
        for (int s = s0 + sl; s < s1; s += nl) {
          int a, bq;
          round_pair(r, s, lpl, a, bq);
          int rot = 0;
          double cs = 1.0, sn = 0.0;
          if (bq < nlive) {
            const int i = live[a], j = live[bq];
            const double al = norms[i], be = norms[j];
            const double di = dsc[i], dj = dsc[j];
            const double g = tree_sum(gp + s, L.npairs, C) * (di * dj);  // the inner product of the (unscaled) rows
            // al, be > 0 and g^2 > tol^2 al be, compared as bit patterns (all >= +0)
            if (__double_as_longlong(al) > 0 && __double_as_longlong(be) > 0 &&
                __double_as_longlong(g * g) > __double_as_longlong(tol2 * (al * be))) {
              rot = 1;
              // tangent of the annihilating angle, t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
              // zeta = (be - al) / (2g), formed in FP32 (a dependent FP64 chain of
              // square roots and divisions would hold the round for microseconds).
              // Any angle gives an exactly orthogonal rotation once cs, sn come from
              // the same t in FP64; the FP32 angle leaves |g| at about 1e-7 of its
              // value instead of 0, and the FP64 stopping test above decides
              // convergence, so the result keeps FP64 accuracy.
              // h and 2g are scaled by a power of two (from the exponent bits) into
              // FP32 range; live rows differ by at most 2^104 in squared norm
              // (deflation), so |zeta| < 1e29 and only zeta^2 needs the guard
              const double hd = be - al, g2 = 2.0 * g;
              const double mx = fmax(fabs(hd), fabs(g2));
              const long long ex = min(((__double_as_longlong(mx) >> 52) & 0x7ff) - 1023, 1022LL);
              const double sc = __longlong_as_double((1023 - ex) << 52);  // 2^-ex
              const float zf = (float)(hd * sc) / (float)(g2 * sc);
              const float tf = fabsf(zf) < 1e18f ? copysignf(1.0f, zf) / (fabsf(zf) + sqrtf(fmaf(zf, zf, 1.0f)))
                                                 : 0.5f / zf;
              const double t = (double)tf;
              // (c, c t) rotation in scaled form: x_i <- x_i - t (d_j / d_i) x_j,
              // x_j <- x_j + t (d_i / d_j) x_i, d_i, d_j <- c d_i, c d_j: the workers
              // need only the two coefficients; c and the new scales and norms follow
              // after the coefficients are published
              cs = t * dj * isc[i];
              sn = t * di * isc[j];
              rtan[s] = t;
              rgam[s] = g;
              if (__double_as_longlong(g * g) > __double_as_longlong(thr2 * (al * be))) big_rot = 1;
            }
          }
          rcs[s] = cs;
          rsn[s] = sn;
          rfl[s] = rot;
        }
        half_arrive(h, nl + kWorkerThreads);
        // the rotated rows' scales and norms for the next round (the rows of a round's
        // pairs are disjoint, and only this lane touches those of its pairs), while the
        // workers rotate
        for (int s = s0 + sl; s < s1; s += nl) {
          if (!rfl[s]) continue;
          int a, bq;
          round_pair(r, s, lpl, a, bq);
          const int i = live[a], j = live[bq];
          const double t = rtan[s], g = rgam[s];
          const double t2 = fma(t, t, 1.0);
          const double c = rsqrt(t2);
          const double tc = t2 * c;  // 1 / c
          dsc[i] *= c;
          dsc[j] *= c;
          isc[i] *= tc;
          isc[j] *= tc;
          norms[i] = fma(-t, g, norms[i]);
          norms[j] = fma(t, g, norms[j]);
          ++myrot;
        }
      }
      __syncthreads();
      if ((r & 63) == 63) rescale();  // the scales stay above 2^-32 between foldings
    }
    if (myrot) atomicAdd(&rot_count, myrot);
    myrot = 0;
    __syncthreads();
    ++sweeps;
    total_rot += rot_count;
    // A rotation leaves its pair's inner product at about 2e-7 of what it was
    // (FP32 angle); the other pairs it touches change to second order.  So
    // after a sweep whose rotations all had |g| <= thr sqrt(alpha beta),
    // thr = 1e4 tol, every pair is far below tol (about 2e-3 tol): the sweep
    // that would only confirm it is skipped (the norms are still recomputed
    // exactly before the singular values are taken).
    converged = (rot_count == 0) || (big_rot == 0);
  }
  // norms now hold the exact final row norms (computed at the loop head)
  double* sig = nrm_part;  // reuse: all remote reads of nrm_part finished before the last __syncthreads
  cluster.sync();          // make sure no CTA still reads this CTA's nrm_part
  for (int i = tid; i < l; i += kJacobiThreads) {
    const double v = sqrt(norms[i]);
    sig[i] = v;
    if (((__double_as_longlong(v) >> 52) & 0x7ff) == 0x7ff) nonfinite = 1;
  }
  __syncthreads();
  // descending order, lower index first on ties; the keys are the bit
  // patterns of the (non-negative) values, -1 for a non-finite one
  auto key = [&](int j) {
    const long long b = __double_as_longlong(sig[j]);
    return ((b >> 52) & 0x7ff) == 0x7ff ? -1LL : b;
  };
  for (int i = tid; i < l; i += kJacobiThreads) {
    const long long ki = key(i);
    int rk = 0;
    for (int j = 0; j < l; ++j) {
      const long long kj = key(j);
      rk += (kj > ki) || (kj == ki && j < i);
    }
    order[rk] = i;
  }
  __syncthreads();
  const int k = J.k;
  if (rank == 0) {
    for (int r = tid; r < l; r += kJacobiThreads) {
      const double v = sig[order[r]];
      J.sig[r] = v;
      if (r < k) J.S[r] = v;
    }
    if (tid == 0) {
      // a timed-out exchange in any CTA of the cluster (each CTA's flag is final: no
      // round runs after the cluster barrier above, and every CTA stays until the last one)
      int any_err = 0;
      for (int q = 0; q < C; ++q) any_err |= *cluster.map_shared_rank(&rerr, q);
      J.info->jacobi_sweeps = sweeps;
      J.info->rotations = (int)min(total_rot, (long long)0x7fffffff);
      J.info->jacobi_pairs = (int)min(total_pairs, (long long)0x7fffffff);
      if ((J.pipe_err && *J.pipe_err) || any_err)
        J.info->status = RSVD_ERR_TIMEOUT;
      else if (nonfinite)
        J.info->status = RSVD_ERR_NONFINITE;
      else if (!converged && J.info->status == RSVD_OK)
        J.info->status = RSVD_WARN_NOCONV;
    }
  }
  if (J.want_vt) {
    for (int e = tid; e < k * ncl; e += kJacobiThreads) {
      const int r = e / ncl, c = e % ncl;
      const int src = order[r];
      const double v = sig[src];
      J.Vt[(size_t)r * J.ldvt + c0 + c] = (T)(v > 0.0 ? Bs[src * L.nc + c] / v : 0.0);
    }
  }
  if (want_p)
    for (int e = tid; e < k * npl; e += kJacobiThreads) {
      const int r = e / npl, c = e % npl;
      J.Ps[(size_t)r * l + p0 + c] = (T)Ps[order[r] * L.np + c];
    }
  cluster.sync();  // no CTA leaves while others may still read its shared memory
}

}  // namespace

// One CTA per 32 columns, up to eight (sixteen when a slice of eight does not
// fit in shared memory).  Depends on the matrix alone, so no matrix's rounding
// depends on the rest of its batch.
int jacobi_cluster_size(int l, int n) {
  int c = n / 32;
  if (c < 1) c = 1;
  if (c > 8) c = 8;
  if (c == 8 && !jacobi_fits_smem(l, n, 8) && jacobi_fits_smem(l, n, 16)) c = 16;
  return c;
}

size_t jacobi_smem_bytes(int l, int n, int csize) {
  const JLayout L = jlayout(l, n, csize);
  return jsmem_small(l, L) + sizeof(double) * ((size_t)l * L.nc + (size_t)l * L.np);
}

bool jacobi_fits_smem(int l, int n, int csize) { return jacobi_smem_bytes(l, n, csize) <= kSmemBudget; }

template <typename T>
cudaError_t launch_jacobi(const JacobiBatch<T>& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  size_t smem = 0;
  for (int i = 0; i < b.count; ++i) {
    const int l = b.job[i].l, n = b.job[i].n;
    const size_t need = b.use_global ? jsmem_small(l, jlayout(l, n, b.csize)) : jacobi_smem_bytes(l, n, b.csize);
    smem = max(smem, need);
  }
  cudaError_t e = cudaFuncSetAttribute(jacobi_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (b.csize > 8) {
    e = cudaFuncSetAttribute(jacobi_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b.csize, b.count, 1);
  cfg.blockDim = dim3(kJacobiThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = b.csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  prof_begin(KC_JACOBI, s);
  e = cudaLaunchKernelEx(&cfg, jacobi_kernel<T>, b);
  prof_end(KC_JACOBI, s);
  return e;
}

template cudaError_t launch_jacobi<double>(const JacobiBatch<double>&, cudaStream_t);
template cudaError_t launch_jacobi<float>(const JacobiBatch<float>&, cudaStream_t);

}  // namespace rsvd
