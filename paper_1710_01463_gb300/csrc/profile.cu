// Optional timing of librsvd's kernels with CUDA events recorded around each
// launch on the launching stream (off by default; one host thread at a time).
#include <vector>

#include "common.cuh"

namespace rsvd {

namespace {

struct Rec {
  int cls;
  cudaEvent_t a, b;
};

struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<Rec> recs;
  int open_cls = -1;
  cudaEvent_t open_ev = nullptr;
};

Prof& prof() {
  static Prof p;
  return p;
}

const char* kNames[KC_COUNT] = {"prep", "omega", "gemm", "gram", "cholesky", "householder",
                                "jacobi", "sign", "select", "tebd", "backward", "tcgemm", "convert", "ozgemm", "ozsplit"};

}  // namespace

void prof_begin(int cls, cudaStream_t s) {
  Prof& P = prof();
  if (!P.on || P.used + 2 > P.pool.size()) return;
  P.open_cls = cls;
  P.open_ev = P.pool[P.used++];
  cudaEventRecord(P.open_ev, s);
}

void prof_end(int cls, cudaStream_t s) {
  Prof& P = prof();
  if (!P.on || P.open_cls != cls || P.open_ev == nullptr) return;
  cudaEvent_t e = P.pool[P.used++];
  cudaEventRecord(e, s);
  P.recs.push_back(Rec{cls, P.open_ev, e});
  P.open_cls = -1;
  P.open_ev = nullptr;
}

}  // namespace rsvd

using namespace rsvd;

extern "C" {

int rsvd_profile_enable(int max_launches) {
  Prof& P = prof();
  for (auto e : P.pool) cudaEventDestroy(e);
  P.pool.clear();
  P.recs.clear();
  P.used = 0;
  P.on = false;
  if (max_launches <= 0) return RSVD_OK;
  P.pool.resize((size_t)2 * max_launches);
  for (auto& e : P.pool)
    if (cudaEventCreate(&e) != cudaSuccess) return RSVD_ERR_LAUNCH;
  P.on = true;
  return RSVD_OK;
}

int rsvd_profile_collect(double* ms, int* launches, int nclass) {
  Prof& P = prof();
  if (!ms || !launches) return RSVD_ERR_NULL_POINTER;
  for (int c = 0; c < nclass; ++c) {
    ms[c] = 0.0;
    launches[c] = 0;
  }
  for (const Rec& r : P.recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return RSVD_ERR_LAUNCH;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return RSVD_ERR_LAUNCH;
    if (r.cls < nclass) {
      ms[r.cls] += t;
      launches[r.cls] += 1;
    }
  }
  P.recs.clear();
  P.used = 0;
  return KC_COUNT;
}

const char* rsvd_profile_class_name(int cls) {
  if (cls < 0 || cls >= KC_COUNT) return "unknown";
  return kNames[cls];
}

}  // extern "C"
