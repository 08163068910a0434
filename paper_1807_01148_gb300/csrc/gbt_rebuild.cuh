// Phases of the occupancy rebuild (lane counts -> lane starts -> scatter -> rank in
// the lane segment), the per-edge sample, the step's counter update and the grid
// barrier of the persistent launch: shared by the per-kernel step (gbt_step.cu) and
// the persistent step (gbt_fused.cu).
#pragma once
#include "gbt_stepdev.cuh"

namespace gbt {

// The lane-start scan: each block pass covers kScanChunk lanes, kScanItems to each of
// its first kScanThreads threads, so every launch that runs it has at least
// kScanThreads threads per block (fewer would leave lane starts unwritten).
constexpr int kScanThreads = 256, kScanItems = 8, kScanChunk = kScanThreads * kScanItems;

// Lane segments longer than this are sorted by k_rank_long (one block per segment);
// the per-vehicle count of k_rank is quadratic in the segment length.
constexpr int kLongSeg = 64;

__device__ __forceinline__ int block_excl_scan(int val, int* smem_warp, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = val;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) smem_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int w = (lane < (int)(blockDim.x >> 5)) ? smem_warp[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    smem_warp[lane] = wi - w;   // exclusive warp offsets
    if (lane == 31) smem_warp[32] = wi;
  }
  __syncthreads();
  int res = smem_warp[warp] + inc - val;
  total = smem_warp[32];
  __syncthreads();
  return res;
}

// Per-chunk sums of the lane counts (chunks of kScanChunk lanes, one per block pass).
__device__ __forceinline__ void ph_scan_sum(const Dev& d) {
  __shared__ int sw[33];
  if (blockIdx.x == 0 && threadIdx.x == 0) d.ctl->n_long = 0;   // listed again by the scan
  const int nb = (d.n_lanes + kScanChunk - 1) / kScanChunk;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    int base = b * kScanChunk + threadIdx.x * kScanItems;
    int s = 0;
    if (threadIdx.x < kScanThreads && base + kScanItems <= d.n_lanes) {
      const int4 a0 = *reinterpret_cast<const int4*>(d.cnt + base);
      const int4 a1 = *reinterpret_cast<const int4*>(d.cnt + base + 4);
      s = ((a0.x + a0.y) + (a0.z + a0.w)) + ((a1.x + a1.y) + (a1.z + a1.w));
    } else {
#pragma unroll
      for (int k = 0; k < kScanItems; k++) {
        int i = base + k;
        if (i < d.n_lanes && threadIdx.x < kScanThreads) s += d.cnt[i];
      }
    }
    int tot;
    block_excl_scan(threadIdx.x < kScanThreads ? s : 0, sw, tot);
    if (threadIdx.x == 0) d.bsum[b] = tot;
  }
}

// Lane starts = chunk offset + exclusive scan inside the chunk; counts reset to zero.
// Each block sums the chunk totals before its chunk itself (a few hundred at most), so
// no separate pass over the chunk totals is needed; the block of the last chunk
// writes the total (the number of vehicles in the sorted buffer).
__device__ __forceinline__ void ph_scan_fin(const Dev& d) {
  __shared__ int sw[33];
  const int nb = (d.n_lanes + kScanChunk - 1) / kScanChunk;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    int before = 0;
    for (int i = threadIdx.x; i < b; i += blockDim.x) before += d.bsum[i];
    int tot_before;
    block_excl_scan(before, sw, tot_before);
    int base = b * kScanChunk + threadIdx.x * kScanItems;
    const bool lanes_of_thread = threadIdx.x < kScanThreads;
    int v[kScanItems];
    int s = 0;
    const bool full = lanes_of_thread && base + kScanItems <= d.n_lanes;
    if (full) {
      const int4 a0 = *reinterpret_cast<const int4*>(d.cnt + base);
      const int4 a1 = *reinterpret_cast<const int4*>(d.cnt + base + 4);
      v[0] = a0.x; v[1] = a0.y; v[2] = a0.z; v[3] = a0.w;
      v[4] = a1.x; v[5] = a1.y; v[6] = a1.z; v[7] = a1.w;
    } else {
#pragma unroll
      for (int k = 0; k < kScanItems; k++) {
        int i = base + k;
        v[k] = (lanes_of_thread && i < d.n_lanes) ? d.cnt[i] : 0;
      }
    }
#pragma unroll
    for (int k = 0; k < kScanItems; k++) s += v[k];
    int tot;
    int ex = block_excl_scan(s, sw, tot) + tot_before;
    // lanes whose segment the long-segment rank kernel sorts
#pragma unroll
    for (int k = 0; k < kScanItems; k++)
      if (v[k] > kLongSeg) d.long_list[atomicAdd(&d.ctl->n_long, 1)] = base + k;
    if (full) {
      int o[kScanItems];
#pragma unroll
      for (int k = 0; k < kScanItems; k++) {
        o[k] = ex;
        ex += v[k];
      }
      *reinterpret_cast<int4*>(d.lane_start + base) = make_int4(o[0], o[1], o[2], o[3]);
      *reinterpret_cast<int4*>(d.lane_start + base + 4) = make_int4(o[4], o[5], o[6], o[7]);
      *reinterpret_cast<int4*>(d.cnt + base) = make_int4(0, 0, 0, 0);
      *reinterpret_cast<int4*>(d.cnt + base + 4) = make_int4(0, 0, 0, 0);
    } else {
#pragma unroll
      for (int k = 0; k < kScanItems; k++) {
        int i = base + k;
        if (lanes_of_thread && i < d.n_lanes) {
          d.lane_start[i] = ex;
          d.cnt[i] = 0;
        }
        ex += v[k];
      }
    }
    if (b == nb - 1 && threadIdx.x == 0) {
      d.ctl->nB = tot_before + tot;
      d.lane_start[d.n_lanes] = tot_before + tot;
      d.ctl->n_elig = 0;
      d.ctl->chunk_next = 0;
      d.ctl->n_big = 0;
      const unsigned ep = d.ctl->occ_epoch + 1u;
      d.ctl->occ_epoch = ep ? ep : 1u;   // tag 0 marks never-written rear records
    }
  }
}

__device__ __forceinline__ void ph_scatter(const Dev& d) {
  const int nA = d.ctl->nA;
  GRID_STRIDE(s, nA) {
    // every load of the slot is issued before the test (slots below nA are allocated)
    const int e = d.A.link[s];
    const int g = d.A.gid[s], ai = d.aidx[s], vid = d.A.vid[s];
    const float x = d.A.x[s];
    if (e < 0) continue;
    const int p = d.lane_start[g] + ai;
    d.tx[p] = x;
    d.tvid[p] = vid;
    d.tsrc[p] = s;
    d.tg[p] = g;
  }
}

// The vehicle of scatter position p (buffer A slot src) lands at sorted position dst,
// rank r of its lane segment [s0, s1).
__device__ __forceinline__ void rank_emit(const Dev& d, int src, float xp, int vp, int g, int dst, int s1, bool first,
                                          int t, unsigned ep) {
  const int e = d.A.link[src], nxt = d.A.nxt[src], lane = d.A.lane[src], cur = d.A.cur[src];
  const float vv = d.A.v[src];
  d.B.x[dst] = xp;
  d.B.v[dst] = vv;
  d.B.vid[dst] = vp;
  d.B.link[dst] = e;
  d.B.nxt[dst] = nxt;
  d.B.cur[dst] = cur;
  d.B.lane[dst] = lane;
  d.B.mv[dst] = d.A.mv[src];
  if (first) d.rear[g] = RearRec{xp, vv, vp, ep};
  if (dst + 1 == s1) {
    d.fr[g] = FrontRec{xp, vv, vp, nxt};
    if (nxt >= 0) {
      const LinkRec& L = d.links[e];
      if (L.ctrl == kCtrlStop && d.holder[L.to] == -1 && (L.len - xp) <= d.stop_acq)
        atomicMin(&d.acq[L.to], epoch_key(t, rr_rank(L, t), lane));
    }
  }
}

template <bool SKIP_LONG>
__device__ __forceinline__ void ph_rank(const Dev& d) {
  const int nB = d.ctl->nB;
  const int t = (int)d.ctl->t;
  const unsigned ep = d.ctl->occ_epoch;
  GRID_STRIDE(p, nB) {
    const int g = d.tg[p];
    const int src = d.tsrc[p];
    const float xp = d.tx[p];
    const int vp = d.tvid[p];
    // the state to move does not depend on the rank: its loads overlap the count
    const int e = d.A.link[src], nxt = d.A.nxt[src], lane = d.A.lane[src], cur = d.A.cur[src];
    const float vv = d.A.v[src];
    const uint8_t mv = d.A.mv[src];
    const int s0 = d.lane_start[g], s1 = d.lane_start[g + 1];
    if (SKIP_LONG && s1 - s0 > kLongSeg) continue;
    int rank = 0;
    for (int q = s0; q < s1; q++) {
      const float xq = d.tx[q];
      rank += (xq < xp || (xq == xp && d.tvid[q] < vp)) ? 1 : 0;
    }
    const int dst = s0 + rank;
    d.B.x[dst] = xp;
    d.B.v[dst] = vv;
    d.B.vid[dst] = vp;
    d.B.link[dst] = e;
    d.B.nxt[dst] = nxt;
    d.B.cur[dst] = cur;
    d.B.lane[dst] = lane;
    d.B.mv[dst] = mv;
    if (rank == 0) d.rear[g] = RearRec{xp, vv, vp, ep};
    if (dst + 1 == s1) d.fr[g] = FrontRec{xp, vv, vp, nxt};
    if (dst + 1 == s1 && nxt >= 0) {
      const LinkRec& L = d.links[e];
      if (L.ctrl == kCtrlStop && d.holder[L.to] == -1 && (L.len - xp) <= d.stop_acq)
        atomicMin(&d.acq[L.to], epoch_key(t, rr_rank(L, t), lane));
    }
  }
}

// Sec. 6.4 per-edge sample of the state at step t (when t is a multiple of samp_every),
// one thread per link over its contiguous run of the sorted buffer (lanes in order,
// then position): utilisation = vehicles / (length * lanes / (vehicle length + s0)),
// speed = their mean speed, or the link's free-flow speed when it is empty.  Window w
// holds samples w * samp_per .. w * samp_per + samp_per - 1; its last sample writes
// the means over the samples taken since the outputs were cleared.
__device__ __forceinline__ void ph_edge_sample(const Dev& d) {
  const long long t = d.ctl->t;
  if (t % d.samp_every != 0) return;
  const long long k = t / d.samp_every;
  const long long w = k / d.samp_per;
  const bool closes = (k % d.samp_per) == d.samp_per - 1;
  const long long k0 = d.ctl->samp_k0;
  const long long from = w * d.samp_per > k0 ? w * d.samp_per : k0;
  const double taken = (double)(k - from + 1);
  GRID_STRIDE(e, d.n_links) {
    const LinkRec L = d.links[e];
    const int r0 = d.lane_start[L.lane_base], r1 = d.lane_start[L.lane_base + L.lanes];
    double vs = 0.0;
    for (int r = r0; r < r1; r++) vs += (double)d.B.v[r];
    const int n = r1 - r0;
    const double cap = ((double)L.len * (double)L.lanes) / ((double)d.vlen + (double)d.cls[L.cls].s0);
    const double u = d.acc_u[e] + (double)n / cap;
    const double sp = d.acc_s[e] + (n > 0 ? vs / (double)n : (double)L.v0);
    if (closes) {
      const size_t o = (size_t)w * (size_t)d.n_links + (size_t)e;
      d.out_u[o] = u / taken;
      d.out_s[o] = sp / taken;
      d.acc_u[e] = 0.0;
      d.acc_s[e] = 0.0;
    } else {
      d.acc_u[e] = u;
      d.acc_s[e] = sp;
    }
  }
  if (closes && blockIdx.x == 0 && threadIdx.x == 0) d.out_n[w] = (int32_t)(k - from + 1);
}

__host__ __device__ __forceinline__ bool outputs_on(const Dev& d) { return d.emis || d.tt_sum; }

__device__ __forceinline__ void ph_finish(const Dev& d) {
  Ctl* c = d.ctl;
  c->veh_steps += (unsigned long long)c->nB;
  c->lc_evals += (unsigned long long)c->n_elig;
  c->departed += (unsigned long long)c->n_ins;
  c->arrived += (unsigned long long)c->n_arr;
  c->active_last = c->nB;
  c->nA = c->nB + c->n_ins;
  c->n_ins = 0;
  c->n_arr = 0;
  c->n_elig = 0;
  c->t += 1;
}

}  // namespace gbt
