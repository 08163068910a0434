// Device helpers shared by the step kernels (gbt_step.cu) and the fused lane-front and
// chunk kernels (gbt_fused.cu): launch ordering, lane counts, stop and signal control
// (Sec. 6.3.2), Eq. 7 across a link end, and the bulk-copy / mbarrier primitives.
#pragma once
#include "gbt_internal.cuh"

namespace gbt {

#define GRID_STRIDE(i, n) for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)

// The step kernels are launched with programmatic stream serialization: a kernel's
// launch is prepared while the one before it in the stream runs, and the kernel waits
// here, before its first read, until that grid has completed and its writes are
// visible.  (Without such a launch the wait returns at once.)  No kernel triggers its
// dependents early: waiting blocks would hold registers and shared memory that the
// running kernel's blocks use (measured slower).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Arrival index of this vehicle in lane g's count for the next occupancy rebuild.
// Neighbouring threads mostly hold vehicles of the same lane (the sorted order), so
// the threads of a warp with equal g share one atomic; the order inside the group is
// arbitrary (the rebuild ranks by position and id).
__device__ __forceinline__ int count_in_lane(const Dev& d, int g) {
  const unsigned act = __activemask();
  const unsigned peers = __match_any_sync(act, g);
  const int ln = threadIdx.x & 31, lead = __ffs(peers) - 1;
  int base = 0;
  if (ln == lead) base = atomicAdd(&d.cnt[g], __popc(peers));
  base = __shfl_sync(peers, base, lead);
  return base + __popc(peers & ((1u << ln) - 1u));
}

// A step kernel returns at entry once a bounded wait of this step (or of an earlier
// one) ran out: the state is then undefined, the host reports SIM_ETIMEOUT and refuses
// to step until the state is reset, and no kernel works on partly computed scratch.
__device__ __forceinline__ bool step_timed_out(const Dev& d) {
  return (*(volatile int*)&d.ctl->err & kErrTimeout) != 0;
}

__device__ __forceinline__ bool is_holder(const Dev& d, const LinkRec& L, int t, int vid, int lane,
                                          bool front) {
  if (L.ctrl != kCtrlStop) return false;
  int h = d.holder[L.to];
  if (h == vid) return true;
  return h == -1 && front && d.acq[L.to] == epoch_key(t, rr_rank(L, t), lane);
}

__device__ __forceinline__ bool line_closed(const Dev& d, const LinkRec& L, int t, bool holder) {
  if (L.ctrl == kCtrlSignal) return !signal_green(L, t * d.dt_ds);
  if (L.ctrl == kCtrlStop) return !holder;
  return false;
}

// Eq. 7 parameters and desired speed of trip vid on link L: its class's, or with vehicle
// types (Sec. 6.3.5) the class's with a scaled by the type (a table built on the host)
// and v0 capped at the type's maximum speed.
template <bool TYPES>
__device__ __forceinline__ void veh_par(const Dev& d, const LinkRec& L, int vid, ClassPar& P, float& v0) {
  if (TYPES) {
    const int ty = d.vtype[vid];
    P = d.cls_ty[L.cls * d.n_vty + ty];
    v0 = fminf(L.v0, d.vty_vmax[ty]);
  } else {
    P = d.cls[L.cls];
    v0 = L.v0;
  }
}

// length of trip vid's vehicle
template <bool TYPES>
__device__ __forceinline__ float veh_len(const Dev& d, int vid) {
  return TYPES ? d.vty_len[d.vtype[vid]] : d.vlen;
}

// Acceleration of a vehicle with nothing ahead on its link e, considered in lane
// `lane`: leader = rearmost vehicle of the mapped lane of its next link (gap across
// the link end, to the leader's rear); a closed stop line is a standing obstacle
// (smaller acceleration).  P, v0: the vehicle's Eq. 7 parameters; ep: the epoch of the
// current rear records.  Optionally returns
// the mapped lane (*gt), whether it has a rearmost vehicle other than this one
// (*lead) and that vehicle's rear position (*room); next_rec: the next link's record
// when the caller has loaded it already.
template <bool TYPES>
__device__ __forceinline__ float acc_front(const Dev& d, unsigned ep, const LinkRec& L, const ClassPar& P, float v0,
                                           int vid, int nxt, int lane, float x, float v, bool closed,
                                           TapeForm* f = nullptr, int* gt = nullptr, bool* lead = nullptr,
                                           float* room = nullptr, const LinkRec* next_rec = nullptr) {
  if (nxt < 0) {
    if (f) *f = TapeForm{-1, 0.0f, 0.0f, kFormFree, 0, 0, 0};
    return idm_acc(P, v0, d.s_min, 0.0f, v, 0.0f, false);
  }
  const LinkRec Ln = next_rec ? *next_rec : d.links[nxt];
  const int m = lane < Ln.lanes - 1 ? lane : Ln.lanes - 1;
  const int g = Ln.lane_base + m;
  const RearRec r = d.rear[g];
  float a1;
  TapeForm f1;
  const bool has = r.tag == ep && r.vid != vid;
  if (gt) *gt = g;
  if (lead) *lead = has;
  if (has) {
    const float len_r = veh_len<TYPES>(d, r.vid);
    if (room) *room = r.x - len_r;
    float s = ((L.len - x) + r.x) - len_r;
    a1 = idm_acc(P, v0, d.s_min, s, v, r.v, true);
    if (f) f1 = TapeForm{r.vid, s, r.v, kFormNext, 0, 0, 0};
  } else {
    a1 = idm_acc(P, v0, d.s_min, 0.0f, v, 0.0f, false);
    if (f) f1 = TapeForm{-1, 0.0f, 0.0f, kFormFree, 0, 0, 0};
  }
  if (closed) {
    const float s2 = L.len - x;
    const float a2 = idm_acc(P, v0, d.s_min, s2, v, 0.0f, true);
    if (a2 < a1) {
      if (f) *f = TapeForm{-1, s2, 0.0f, kFormStop, 0, 0, 0};
      return a2;
    }
  }
  if (f) *f = f1;
  return a1;
}

__device__ __forceinline__ TapeRec* tape_slot(const Dev& d, int t, int vid) {
  return d.tape + (size_t)(t - (int)d.ctl->tape_t0) * (size_t)d.n_trips + (size_t)vid;
}

// Sec. 6.3.1: trip vid leaves link e in step t; it entered it in step enter[vid]
// (-1 when it was already on the link when the outputs were cleared).
__device__ __forceinline__ void note_exit(const Dev& d, int vid, int e, int t) {
  const int te = d.enter[vid];
  if (te >= 0) {
    atomicAdd(&d.tt_sum[e], (unsigned long long)(t - te));
    atomicAdd(&d.tt_n[e], 1);
  }
}

// ------------------------------------------------------------------ departures
// The head of each link's queue of due trips enters at x = 0, v = 0 in the allowed
// lane with the largest rear space (ties to the lowest lane) that received no
// vehicle from upstream in this step, if that space is at least s0 + vehicle length.
template <bool OUT, bool TYPES>
__device__ __forceinline__ void ph_insert(const Dev& d) {
  const int nq = d.n_qlinks;
  const int t = (int)d.ctl->t;
  const int nB = d.ctl->nB;
  GRID_STRIDE(i, nq) {
    const int e = d.qlinks[i];
    const int hd = d.q_head[e];
    if (hd >= d.q_end[e]) continue;
    const int h = d.q_items[hd];
    if ((long long)d.depart[h] > t) continue;
    const LinkRec L = d.links[e];
    const int off = d.roff[h], len = d.rlen[h];
    const int e2 = len >= 2 ? d.routes[off + 1] : (d.loop ? d.routes[off] : -1);
    const int mc = move_class(d, e, e2);
    const int M = lane_mask(mc, L.lanes);
    const unsigned ep = d.ctl->occ_epoch;
    int bl = -1;
    float brs = 0.0f;
    for (int l = 0; l < L.lanes; l++) {
      if (!((M >> l) & 1)) continue;
      const int g = L.lane_base + l;
      if (epoch_current(d.best[g], t)) continue;
      const RearRec r = d.rear[g];
      const float rs = r.tag == ep ? r.x - veh_len<TYPES>(d, r.vid) : INFINITY;
      if (bl < 0 || rs > brs) {
        bl = l;
        brs = rs;
      }
    }
    if (bl < 0) continue;
    const float need = d.cls[L.cls].s0 + veh_len<TYPES>(d, h);
    if (!(brs >= need)) continue;
    const int slot = nB + atomicAdd(&d.ctl->n_ins, 1);
    if (slot >= d.n_trips) { set_err(d, kErrSlot, slot); continue; }
    d.A.x[slot] = 0.0f;
    d.A.v[slot] = 0.0f;
    d.A.vid[slot] = h;
    d.A.link[slot] = e;
    d.A.nxt[slot] = e2;
    d.A.cur[slot] = 0;
    d.A.lane[slot] = bl;
    d.A.mv[slot] = (uint8_t)mc;
    d.adec[slot] = 0;
    d.A.gid[slot] = L.lane_base + bl;
    d.aidx[slot] = atomicAdd(&d.cnt[L.lane_base + bl], 1);
    d.status[h] = kActive;
    d.ins_step[h] = (int32_t)t;
    if (OUT && d.enter) d.enter[h] = t;
    d.q_head[e] = hd + 1;
  }
}


// ------------------------------------------------------------------ bulk-copy staging
// Default bound of the drain of issued copies after a timed-out wait.
constexpr long long kWaitLimit = kDefaultWaitCycles;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\tselp.u32 %0, 1, 0, P1;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P1;\n\tmbarrier.test_wait.parity.shared::cta.b64 P1, [%1], %2;\n\tselp.u32 %0, 1, 0, P1;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of bar for at most `limit` SM cycles (false when it runs out).
// The first probe does not suspend the thread, so that a limit shorter than a copy's
// latency runs out at once.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  if (mbar_test_wait(bar, parity)) return true;
  while (clock64() - t0 <= limit)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// bytes: a multiple of 16; src and dst 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

}  // namespace gbt
