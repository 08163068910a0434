// Trip planning on the GPU (Waddell et al., Sec. 6.3.1 and Sec. 6 "Simulation scale"):
// one shortest-path tree per distinct origin, shared by all trips from that origin
// (the paper replaces per-agent Dijkstra by per-source trees for a two-orders-of-
// magnitude speed-up), on integer decisecond link costs.
//
// Each CTA of a persistent grid takes origins from an atomic work counter and runs a
// near-far variant of delta-stepping (Meyer & Sanders 2003): nodes whose tentative
// distance is below the current threshold T are relaxed in synchronous rounds from a
// deduplicated near queue; farther improvements go to a deduplicated far pile, which
// is split when the near queue empties (T = smallest live far distance + delta).
// Distances are 64-bit words tagged with a per-CTA epoch, so no per-origin reset of
// the distance array is needed.  The tree is then read back for every trip of the
// origin by walking from the destination: at node v take the lowest-id in-link
// u -> v with dist[u] + c = dist[v] (a unique, canonical shortest path).  In the
// all-or-nothing mode (R.flow set) that walk adds one trip to every link of the path
// instead of storing it: the direction finding of Frank-Wolfe (Sec. 5.2).
#include <climits>

#include "gbt_internal.cuh"

namespace gbt {



__device__ __forceinline__ unsigned long long dkey(unsigned hi, int d) {
  return ((unsigned long long)hi << 32) | (unsigned)d;
}
__device__ __forceinline__ int dval(const unsigned long long* dist, int v, unsigned hi) {
  unsigned long long k = dist[v];
  return (unsigned)(k >> 32) == hi ? (int)(unsigned)k : INT_MAX;
}

__global__ void __launch_bounds__(256) k_sssp_route(RouteDev R) {
  __shared__ int sh_oi, sh_round, sh_nq, sh_nf, sh_min;
  __shared__ unsigned sh_epoch;
  const int tid = threadIdx.x, bd = blockDim.x;
  const size_t base = (size_t)blockIdx.x * (size_t)R.nn;
  unsigned long long* dist = R.dist + base;
  int* qflag = R.qflag + base;
  int* fflag = R.fflag + base;
  int* Q = R.qa + base;
  int* Qn = R.qb + base;
  int* F = R.fa + base;
  int* Fn = R.fb + base;
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      sh_oi = atomicAdd(R.work, 1);
      sh_epoch = ++R.cta_epoch[blockIdx.x];
    }
    __syncthreads();
    const int oi = sh_oi;
    if (oi >= R.n_origins) break;
    const unsigned ep = sh_epoch;
    const unsigned hi = 0xFFFFFFFFu - ep;
    const int o = R.origins[oi];
    if (tid == 0) {
      dist[o] = dkey(hi, 0);
      sh_round = ++R.cta_round[blockIdx.x];
      qflag[o] = sh_round;
      Q[0] = o;
      sh_nq = 0;
      sh_nf = 0;
    }
    __syncthreads();
    int nq = 1, nf = 0;
    int T = R.delta;
    for (;;) {
      // ---- relax the near bucket in rounds until it is empty
      while (nq > 0) {
        const int rnext = sh_round + 1;
        for (int k = tid; k < nq; k += bd) {
          const int u = Q[k];
          const int du = dval(dist, u, hi);
          for (int q = R.out_start[u]; q < R.out_start[u + 1]; q++) {
            const int e = R.out_link[q];
            const int v = R.lto[e];
            const int nd = du + R.cost[e];
            const unsigned long long nk = dkey(hi, nd);
            const unsigned long long old = atomicMin(&dist[v], nk);
            if (nk < old) {
              if (nd < T) {
                if (atomicExch(&qflag[v], rnext) != rnext) Qn[atomicAdd(&sh_nq, 1)] = v;
              } else {
                if (atomicExch(&fflag[v], (int)ep) != (int)ep) F[nf + atomicAdd(&sh_nf, 1)] = v;
              }
            }
          }
        }
        __syncthreads();
        nq = sh_nq;
        nf += sh_nf;
        int* tq = Q; Q = Qn; Qn = tq;
        __syncthreads();
        if (tid == 0) {
          sh_nq = 0;
          sh_nf = 0;
          sh_round = rnext;
        }
        __syncthreads();
      }
      // ---- split the far pile: smallest live distance opens the next bucket
      if (nf == 0) break;
      if (tid == 0) sh_min = INT_MAX;
      __syncthreads();
      for (int k = tid; k < nf; k += bd) {
        const int dv = dval(dist, F[k], hi);
        if (dv >= T) atomicMin(&sh_min, dv);
      }
      __syncthreads();
      const int mn = sh_min;
      if (mn == INT_MAX) break;
      const int Tprev = T;
      T = mn + R.delta;
      const int rnext = sh_round + 1;
      for (int k = tid; k < nf; k += bd) {
        const int v = F[k];
        const int dv = dval(dist, v, hi);
        if (dv < Tprev) {
          fflag[v] = 0;
        } else if (dv < T) {
          fflag[v] = 0;
          qflag[v] = rnext;
          Q[atomicAdd(&sh_nq, 1)] = v;
        } else {
          Fn[atomicAdd(&sh_nf, 1)] = v;
        }
      }
      __syncthreads();
      nq = sh_nq;
      nf = sh_nf;
      int* tf = F; F = Fn; Fn = tf;
      __syncthreads();
      if (tid == 0) {
        sh_nq = 0;
        sh_nf = 0;
        sh_round = rnext;
      }
      __syncthreads();
    }
    // round ids must never repeat within this CTA (they tag near-queue membership)
    if (tid == 0) R.cta_round[blockIdx.x] = sh_round;
    // ---- canonical routes of the trips from o
    for (int k = R.otrip_start[o] + tid; k < R.otrip_start[o + 1]; k += bd) {
      const int i = R.otrip_list[k];
      const int d = R.dest[i];
      if (dval(dist, d, hi) == INT_MAX) {
        atomicOr(&R.ctl->err, kErrUnreach);
        atomicExch(&R.ctl->err_info, i);
        if (!R.flow) {
          R.roff[i] = 0;
          R.rlen[i] = 0;
        }
        continue;
      }
      int n = 0, v = d;
      bool bad = false;
      while (v != o) {
        const int dvv = dval(dist, v, hi);
        int pick = -1;
        for (int q = R.in_start[v]; q < R.in_start[v + 1]; q++) {
          const int e = R.in_link[q];
          const int du = dval(dist, R.lfrom[e], hi);
          if (du != INT_MAX && du + R.cost[e] == dvv) {
            pick = e;
            break;
          }
        }
        if (pick < 0 || n >= R.nn) {
          bad = true;
          break;
        }
        if (R.flow) atomicAdd(&R.flow[pick], 1u);
        n++;
        v = R.lfrom[pick];
      }
      if (bad) {
        atomicOr(&R.ctl->err, kErrRoute);
        atomicExch(&R.ctl->err_info, i);
        if (!R.flow) {
          R.roff[i] = 0;
          R.rlen[i] = 0;
        }
        continue;
      }
      if (R.flow) continue;   // all-or-nothing: the path is counted, not stored
      const unsigned long long off = atomicAdd(&R.ctl->route_cursor, (unsigned long long)n);
      R.rlen[i] = n;
      if (off + (unsigned long long)n > R.cap) {
        R.roff[i] = 0;
        continue;   // the host grows the store to route_cursor and reruns
      }
      R.roff[i] = (int)off;
      v = d;
      for (int j = n - 1; j >= 0; j--) {
        const int dvv = dval(dist, v, hi);
        int pick = -1;
        for (int q = R.in_start[v]; q < R.in_start[v + 1]; q++) {
          const int e = R.in_link[q];
          const int du = dval(dist, R.lfrom[e], hi);
          if (du != INT_MAX && du + R.cost[e] == dvv) {
            pick = e;
            break;
          }
        }
        R.routes[off + j] = pick;
        v = R.lfrom[pick];
      }
    }
  }
}

void launch_route(const RouteDev& R, int n_cta, cudaStream_t s) {
  k_sssp_route<<<n_cta, 256, 0, s>>>(R);
}

// first link of every trip's route (departure-queue keys)
__global__ void k_first_links(const int32_t* roff, const int32_t* routes, int n, int32_t* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = routes[roff[i]];
}

void launch_first_links(const int32_t* roff, const int32_t* routes, int n, int32_t* out, cudaStream_t s) {
  int grid = (n + 255) / 256;
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  k_first_links<<<grid, 256, 0, s>>>(roff, routes, n, out);
}

// route of every trip copied to its new offset (compaction of the route store)
__global__ void k_compact_routes(const int32_t* roff, const int32_t* rlen, const int32_t* src,
                                 const int32_t* new_off, int32_t* dst, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t* a = src + roff[i];
    int32_t* b = dst + new_off[i];
    for (int k = 0; k < rlen[i]; k++) b[k] = a[k];
  }
}

void launch_compact_routes(const int32_t* roff, const int32_t* rlen, const int32_t* src, const int32_t* new_off,
                           int32_t* dst, int n, cudaStream_t s) {
  int grid = (n + 255) / 256;
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  k_compact_routes<<<grid, 256, 0, s>>>(roff, rlen, src, new_off, dst, n);
}

}  // namespace gbt
