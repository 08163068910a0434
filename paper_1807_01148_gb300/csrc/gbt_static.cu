// sim_sssp_static: one shortest-path tree without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a framework owns the
// whole device memory pool, processes whose memory is capped by a supervisor, or
// plug-ins that must not change the device's allocation state.  This entry point
// gives them the trip-planning tree of sim_route for a caller-supplied graph: the
// caller passes every input and output buffer, and the working memory of the
// search (tentative distances, queue flags, near and far queues) lives in one
// file-scope __device__ array of fixed size that every GPU loading the library
// holds until the process exits.
//
// The search itself is the same near-far kernel sim_route runs per origin; its
// distance and flag words carry an epoch / round tag, so the array never needs
// clearing between calls: the distance words are filled with all-ones once, when
// a device is first used, and only the small per-call block (work counter, error
// word, cost sums) is cleared at the start of every call.
#include <algorithm>
#include <climits>
#include <mutex>

#include "gbt_internal.cuh"
#include "gbtraffic.h"

namespace gbt {
namespace {

constexpr size_t kN = SIM_SSSP_STATIC_MAX_NODES;

// persistent across calls (never cleared): epoch and round counters of the search
struct StaticPersist {
  unsigned cta_epoch;
  int32_t cta_round;
  int32_t pad[6];
};

// cleared at the start of every call
struct StaticCall {
  int32_t work;                 // origin counter of the search kernel
  int32_t origin;               // the single origin of this call
  int32_t err;                  // graph validation failures
  int32_t pad0;
  unsigned long long cost_sum;  // sum of link costs (bucket width)
  unsigned long long cost_max;
  Ctl ctl;                      // error word of the search kernel (unused without trips)
};

constexpr size_t kOffPersist = 0;
constexpr size_t kOffCall = 256;
constexpr size_t kOffDist = 1024;                        // 8 B x kN, epoch-tagged distances
constexpr size_t kOffQflag = kOffDist + 8 * kN;          // 4 B x kN each below
constexpr size_t kOffFflag = kOffQflag + 4 * kN;
constexpr size_t kOffQa = kOffFflag + 4 * kN;
constexpr size_t kOffQb = kOffQa + 4 * kN;
constexpr size_t kOffFa = kOffQb + 4 * kN;
constexpr size_t kOffFb = kOffFa + 4 * kN;
constexpr size_t kOffZeros = kOffFb + 4 * kN;            // kN + 1 zeros: "no trips at any node"
constexpr size_t kStaticBytes = kOffZeros + 4 * (kN + 1) + 256;
static_assert(sizeof(StaticPersist) <= kOffCall - kOffPersist, "persist block too large");
static_assert(sizeof(StaticCall) <= kOffDist - kOffCall, "call block too large");

// The working memory.  Zero at module load; only this file's host code takes its
// address, through cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_sssp_scratch[kStaticBytes];

// Device address of g_sssp_scratch per device ordinal (host-side name is only a stand-in).
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// The search tags distance words with an epoch and queue flags with a round number,
// both counted up for the life of the array.  Before either could wrap around (which
// would make stale words look current), the array is put back to its first-use state:
// distance words all-ones, flags zero, counters zero.  Both are read back after every
// call; the reset happens once either passes this bound (about a billion calls or
// rounds), far below the 2^31 where the comparisons would break.
constexpr unsigned kCounterResetAt = 1u << 30;

__global__ void k_static_check(int n, int m, const int32_t* out_start, const int32_t* out_link,
                               const int32_t* link_to, const int32_t* cost, StaticCall* call) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n || i < m; i += gridDim.x * blockDim.x) {
    if (i <= n) {
      const int a = out_start[i];
      bool ok = a >= 0 && a <= m && (i > 0 || a == 0) && (i < n || a == m);
      if (ok && i < n) ok = out_start[i + 1] >= a;
      if (!ok) atomicAdd(&call->err, 1);
    }
    if (i < m) {
      const int e = out_link[i];
      if (e < 0 || e >= m) {
        atomicAdd(&call->err, 1);
        continue;
      }
      const int v = link_to[e];
      const int c = cost[e];
      if (v < 0 || v >= n || c < 1 || c > 1000000) atomicAdd(&call->err, 1);
      if (c > 0) {
        atomicAdd(&call->cost_sum, (unsigned long long)c);
        atomicMax(&call->cost_max, (unsigned long long)c);
      }
    }
  }
}

__global__ void k_static_begin(StaticCall* call, int origin) {
  call->work = 0;
  call->origin = origin;
}

// The search kernel takes a new epoch each time it asks for work, including the last
// request that finds none, so the tree of this call carries the epoch before the
// counter's final value.
__global__ void k_static_dist_out(int n, const unsigned long long* dist, const StaticPersist* ps, int32_t* out) {
  const unsigned hi = 0xFFFFFFFFu - (ps->cta_epoch - 1u);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const unsigned long long k = dist[v];
    out[v] = (unsigned)(k >> 32) == hi ? (int32_t)(unsigned)k : INT32_MAX;
  }
}

int scratch_address(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SIM_ECUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sssp_scratch) != cudaSuccess || !p) return SIM_ECUDA;
    // A distance word compares as newer the smaller it is; the array starts at zero,
    // which would beat every real distance, so it is filled with all-ones once.
    unsigned char* b = static_cast<unsigned char*>(p);
    if (cudaMemset(b + kOffDist, 0xFF, 8 * kN) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
      return SIM_ECUDA;
    g_scratch_addr[dev] = b;
  }
  *out = g_scratch_addr[dev];
  return SIM_OK;
}

}  // namespace
}  // namespace gbt

using namespace gbt;

extern "C" int sim_sssp_static(int32_t n_nodes, int32_t n_links, const int32_t* out_start, const int32_t* out_link,
                               const int32_t* link_to, const int32_t* link_cost, int32_t origin, int32_t* dist_out,
                               void* stream) {
  if (n_nodes < 1 || n_nodes > (int32_t)kN || n_links < 0 || origin < 0 || origin >= n_nodes)
    return SIM_EINVAL;
  if (!out_start || !dist_out || (n_links > 0 && (!out_link || !link_to || !link_cost))) return SIM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != SIM_OK) return rc;
  StaticPersist* ps = reinterpret_cast<StaticPersist*>(base + kOffPersist);
  StaticCall* call = reinterpret_cast<StaticCall*>(base + kOffCall);

  if (cudaMemsetAsync(call, 0, sizeof(StaticCall), s) != cudaSuccess) return SIM_ECUDA;
  const int grid = (std::max(n_nodes + 1, n_links) + 255) / 256;
  k_static_check<<<grid < 1024 ? grid : 1024, 256, 0, s>>>(n_nodes, n_links, out_start, out_link, link_to, link_cost,
                                                           call);
  StaticCall hc;
  if (cudaMemcpyAsync(&hc, call, sizeof(StaticCall), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SIM_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SIM_ECUDA;
  if (hc.err) return SIM_EINVAL;
  if ((unsigned long long)n_nodes * hc.cost_max >= 2000000000ULL) return SIM_EINVAL;

  RouteDev R{};
  R.nn = n_nodes;
  R.nl = n_links;
  R.out_start = out_start;
  R.out_link = out_link;
  R.lto = link_to;
  R.cost = link_cost;
  R.origins = &call->origin;
  R.n_origins = 1;
  R.otrip_start = reinterpret_cast<const int32_t*>(base + kOffZeros);
  R.dist = reinterpret_cast<unsigned long long*>(base + kOffDist);
  R.qflag = reinterpret_cast<int32_t*>(base + kOffQflag);
  R.fflag = reinterpret_cast<int32_t*>(base + kOffFflag);
  R.qa = reinterpret_cast<int32_t*>(base + kOffQa);
  R.qb = reinterpret_cast<int32_t*>(base + kOffQb);
  R.fa = reinterpret_cast<int32_t*>(base + kOffFa);
  R.fb = reinterpret_cast<int32_t*>(base + kOffFb);
  R.cta_epoch = &ps->cta_epoch;
  R.cta_round = &ps->cta_round;
  R.work = &call->work;
  R.ctl = &call->ctl;
  R.delta = (int)std::max<unsigned long long>(1, n_links > 0 ? hc.cost_sum / (unsigned long long)n_links : 1);

  k_static_begin<<<1, 1, 0, s>>>(call, origin);
  launch_route(R, 1, s);
  const int g2 = (n_nodes + 255) / 256;
  k_static_dist_out<<<g2 < 1024 ? g2 : 1024, 256, 0, s>>>(n_nodes, R.dist, ps, dist_out);
  if (cudaGetLastError() != cudaSuccess) return SIM_ECUDA;
  StaticPersist hp;
  if (cudaMemcpyAsync(&hp, ps, sizeof(hp), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SIM_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SIM_ECUDA;
  if (hp.cta_epoch >= kCounterResetAt || (unsigned)hp.cta_round >= kCounterResetAt) {
    // back to the first-use state (see kCounterResetAt); this call's output is complete
    if (cudaMemsetAsync(base + kOffDist, 0xFF, 8 * kN, s) != cudaSuccess ||
        cudaMemsetAsync(base + kOffQflag, 0, 8 * kN, s) != cudaSuccess ||   // queue and far flags
        cudaMemsetAsync(ps, 0, sizeof(StaticPersist), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
      return SIM_ECUDA;
  }
  return SIM_OK;
}

// Test hook: set the persistent epoch and round counters (to check the reset above
// without a billion calls).  Same set-up and serialisation rules as sim_sssp_static.
extern "C" int sim_sssp_static_set_counters(uint32_t epoch, int32_t round, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != SIM_OK) return rc;
  StaticPersist hp{};
  hp.cta_epoch = epoch;
  hp.cta_round = round;
  if (cudaMemcpyAsync(base + kOffPersist, &hp, sizeof(hp), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SIM_ECUDA;
  return SIM_OK;
}
