// Side streams for independent groups of work inside one library call: the
// groups are forked from the caller's stream by an event and joined back to it
// by one event per side stream, so the call stays ordered on the caller's
// stream (and capturable into a CUDA graph) while its groups overlap.
#include "common.cuh"

namespace rsvd {

void* current_context() {
  // cuCtxGetCurrent through the runtime's driver entry point (the library links the
  // runtime only)
  using Fn = int (*)(void**);
  static Fn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    fn = (Fn)p;
  }
  void* ctx = nullptr;
  return fn(&ctx) == 0 ? ctx : nullptr;
}

namespace {
thread_local int t_side_set = 0;  // the set that side_streams() returns (per host thread)
}

SideStreams* side_set(int set) {
  constexpr int kMaxDevices = 64;
  thread_local SideStreams ss[kMaxDevices][kSideSets];  // per host thread: concurrent callers never share events
  int dev = 0;
  if (set < 0 || set >= kSideSets) return nullptr;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  SideStreams& x = ss[dev][set];
  // created once per host thread, device and set, and again when the device's context
  // was replaced (cudaDeviceReset): handles of a destroyed context are not reused
  if (!x.ready || x.ctx != current_context()) {
    SideStreams y;
    if (cudaEventCreateWithFlags(&y.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    y.ctx = current_context();  // current now: the runtime made the device's context current
    for (int i = 0; i < kSideStreams; ++i)
      if (cudaStreamCreateWithFlags(&y.stream[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&y.join[i], cudaEventDisableTiming) != cudaSuccess)
        return nullptr;
    y.ready = true;
    x = y;
  }
  return &x;
}

SideStreams* side_streams() { return side_set(t_side_set); }

void select_side_set(int set) { t_side_set = set; }

cudaError_t fork_side(SideStreams* ss, int n, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(ss->fork, s);
  for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(ss->stream[i], ss->fork, 0);
  return e;
}

cudaError_t join_side(SideStreams* ss, int n, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    e = cudaEventRecord(ss->join[i], ss->stream[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ss->join[i], 0);
  }
  return e;
}

}  // namespace rsvd
