// The per-vehicle part of one simulation step (Waddell et al., Sec. 6.3.2) in two
// kernels, after the occupancy rebuild has sorted the state at step t by (lane,
// position, id) into buffer B:
//
//   k_front  one thread per occupied lane: the lane's front vehicle, the only one whose
//            leader lies beyond its link (the rearmost vehicle of the mapped lane of its
//            next link) or is the stop line (signal phase, stop-sign holder).  Its
//            acceleration (Eq. 7) and the admission bid of a front whose move reaches
//            the link end are settled here, so that the bids of every approach to a
//            lane are complete before anyone crosses.
//   k_chunk  one block per chunk of whole links of B, staged in shared memory with
//            cp.async.bulk: own-lane Eq. 7 behind the next vehicle of the lane,
//            lane-change decisions (mandatory / discretionary with gap acceptance) with
//            every neighbour in the adjacent lanes read from the staged chunk,
//            simultaneous-change conflicts, the final ballistic move, admission,
//            transition and arrival -> the next state in buffer A with the lane counts
//            of the next rebuild; then the departures.
//
// A chunk holds the links whose first sorted position falls in [k T, (k+1) T) for a
// nominal size T, so the lanes of a link are never split and every read of a lane
// change or a conflict stays inside the block.  A chunk larger than the staging
// capacity (a link with more vehicles than that) runs the same code on B and on the
// per-position scratch arrays in global memory, or, on networks where such links carry
// most of the road, in k_chunk_big (a second launch with a larger staging area).
// Blocks take chunks from an atomic counter until none are left (one resident wave).
// The persistent launch at the end of this file runs the same phases (and the
// rebuild's) between grid barriers.
//
// Every decision reads the state at t only (B, the fronts' records, the rear records,
// the bids of this step) and is written to the state at t+1 (A), so the result does not
// depend on the order in which blocks run; ties are broken by vehicle id or by the
// rotating round-robin rank exactly as in the oracle.
#include "gbt_rebuild.cuh"

namespace gbt {

#ifndef GBT_CHUNK_T
#define GBT_CHUNK_T 256
#endif
#ifndef GBT_CHUNK_CAP
#define GBT_CHUNK_CAP 512
#endif
#ifndef GBT_CHUNK_THREADS
#define GBT_CHUNK_THREADS 128
#endif
#ifndef GBT_CHUNK_MINB
#define GBT_CHUNK_MINB 8
#endif
constexpr int kChunkT = GBT_CHUNK_T;         // nominal chunk size (positions)
constexpr int kChunkCap = GBT_CHUNK_CAP;     // staging capacity (positions)
constexpr int kChunkPad = kChunkCap + 32;    // staged arrays: capacity + 16-element alignment slack each side
constexpr int kChunkThreads = GBT_CHUNK_THREADS;
constexpr int kChunkMinBlocks = GBT_CHUNK_MINB;   // resident blocks per SM the register budget aims at
static_assert(kChunkCap % 16 == 0 && kChunkCap >= 2 * kChunkT, "chunk capacity");
#ifndef GBT_CHUNK_LINKS
#define GBT_CHUNK_LINKS 64
#endif
constexpr int kChunkLinks = GBT_CHUNK_LINKS;              // link records staged per chunk (more: read from global)
constexpr int kChunkLanes = 192;             // lane starts staged per chunk (more: read from global)
constexpr int kChunkClasses = 16;            // class parameters kept in shared memory (more: global)
constexpr uint8_t kFlagElig = 8;             // lane-change candidate (chunk-local flag)

// Shared-memory layout of one staged chunk (dynamic shared memory, 16-byte aligned
// arrays; the bulk copies start at a position rounded down to 16, lane starts at one
// rounded down to 4).
template <int CAP>
struct ChunkSmemT {
  static constexpr int kCap = CAP, kPad = CAP + 32;
  float x[kPad], v[kPad];
  int32_t vid[kPad], g[kPad], link[kPad], nxt[kPad], cur[kPad];
  float a[kPad], at[kPad], om[kPad];
  LinkRec lk[kChunkLinks];
  int32_t ls[kChunkLanes + 8];
  ClassPar cls[kChunkClasses];
  uint8_t mv[kPad], fl[kPad];
  int8_t it[kPad];
  int16_t list[CAP];
  uint64_t bar;
};
using ChunkSmem = ChunkSmemT<kChunkCap>;
constexpr size_t kChunkSmemBytes = sizeof(ChunkSmem);
// Chunks beyond kChunkCap (a link with more vehicles than that, as in a long standing
// queue) go to a second launch that stages up to kBigCap positions per block.
constexpr int kBigCap = 2048, kBigThreads = 256;
using ChunkSmemBig = ChunkSmemT<kBigCap>;
constexpr size_t kBigSmemBytes = sizeof(ChunkSmemBig);

// The arrays of a chunk, indexed by position - c0: staged copies in shared memory, or
// B and the per-position scratch in global memory for an oversized chunk; plus the
// chunk's link records [e_lo, e_lo + nlk) and lane starts [g_lo, g_lo + nls) when staged
// (nlk = nls = 0: read from global memory) and the class parameters.
struct ChunkView {
  const float* x;
  const float* v;
  const int32_t* vid;
  const int32_t* g;      // global lane id
  const int32_t* link;
  const int32_t* nxt;    // next link of the route (-1 on the last link)
  const int32_t* cur;    // route cursor
  const uint8_t* mv;     // movement class of link -> next link
  float* a;              // own-lane acceleration
  float* at;             // acceleration behind the target lane's leader (changers)
  float* om;             // free-road term 1 - (v / v0)^4 of Eq. 7
  uint8_t* fl;           // kFlagFront | kFlagHolder | kFlagCand | kFlagElig
  int8_t* it;            // lane-change intent
  const LinkRec* lk;
  const int32_t* ls;
  const ClassPar* cls;
  int e_lo, nlk, g_lo, nls;
};

__device__ __forceinline__ LinkRec view_link(const Dev& d, const ChunkView& V, int e) {
  const unsigned k = (unsigned)(e - V.e_lo);
  return k < (unsigned)V.nlk ? V.lk[k] : d.links[e];
}

__device__ __forceinline__ int view_lane_start(const Dev& d, const ChunkView& V, int g) {
  const unsigned k = (unsigned)(g - V.g_lo);
  return k < (unsigned)V.nls ? V.ls[k] : d.lane_start[g];
}

// Eq. 7 with the vehicle's free-road term om = 1 - (v / v0)^4 already computed (the same
// operations in the same order as idm_acc, so the same result).
__device__ __forceinline__ float idm_om(const ClassPar& P, float om, float s_min, float s, float v, float vl) {
  const float dv = v - vl;
  const float t1 = v * P.T;
  const float t2 = (v * dv) / P.sab2;
  const float dyn = t1 + t2;
  const float ss = P.s0 + fmaxf(0.0f, dyn);
  const float se = fmaxf(s, s_min);
  const float q = ss / se;
  const float q2 = q * q;
  return P.a * (om - q2);
}

__device__ __forceinline__ float free_term(float v, float v0) {
  const float r = v / v0;
  const float r2 = r * r;
  const float r4 = r2 * r2;
  return 1.0f - r4;
}

// Eq. 7 parameters and desired speed of trip vid on link L (vehicle types: veh_par).
template <bool TYPES>
__device__ __forceinline__ void view_par(const Dev& d, const ChunkView& V, const LinkRec& L, int vid, ClassPar& P,
                                         float& v0) {
  if (TYPES) {
    veh_par<true>(d, L, vid, P, v0);
  } else {
    P = V.cls[L.cls];
    v0 = L.v0;
  }
}

// First sorted position at or after b where a link begins (0 and nB at the ends).
__device__ __forceinline__ int chunk_cut(const Dev& d, int b, int nB) {
  if (b <= 0) return 0;
  if (b >= nB) return nB;
  const LinkRec& L = d.links[d.B.link[b]];
  const int s = d.lane_start[L.lane_base];
  return s == b ? b : d.lane_start[L.lane_base + L.lanes];
}

// ------------------------------------------------------------------ lane fronts
// Front of lane g: the last sorted position of the lane, whose record the occupancy
// rebuild wrote.  Same arithmetic as the front path of the own-lane step: holder of a
// stop-controlled node (Sec. 6.3.2, one vehicle at a time), closed stop line, Eq. 7
// behind the rearmost vehicle of the mapped lane of the next link or the stop line,
// and a bid for the target lane when the move reaches the end and lands behind that
// vehicle.
// split: chunks beyond kChunkCap go to the big-chunk launch (their entry in the chunk
// table is left empty, their record goes to the big-chunk list).
template <bool TYPES>
__device__ __forceinline__ void ph_front(const Dev& d, bool split) {
  const int t = (int)d.ctl->t;
  const unsigned ep = d.ctl->occ_epoch;
  GRID_STRIDE(g, d.n_lanes) {
    const int s0 = d.lane_start[g], s1 = d.lane_start[g + 1];
    if (s1 == s0) continue;
    const FrontRec f = d.fr[g];
    const int e = d.lane_link[g];
    const LinkRec L = d.links[e];
    LinkRec Lnx;
    if (f.nxt >= 0) Lnx = d.links[f.nxt];
    const int lane = g - L.lane_base;
    ClassPar P;
    float v0;
    veh_par<TYPES>(d, L, f.vid, P, v0);
    const bool hold = is_holder(d, L, t, f.vid, lane, true);
    const bool closed = f.nxt >= 0 && line_closed(d, L, t, hold);
    int gt = 0;
    bool lead = false;
    float room = 0.0f;
    const float a = acc_front<TYPES>(d, ep, L, P, v0, f.vid, f.nxt, lane, f.x, f.v, closed, nullptr, &gt, &lead,
                                     &room, &Lnx);
    float xo, vo;
    ballistic(f.x, f.v, a, d.dt, d.hdt2, xo, vo);
    uint8_t fl = hold ? kFlagHolder : 0;
    if (f.nxt >= 0 && !closed && xo >= L.len && (!lead || (xo - L.len) <= room)) {
      fl |= kFlagCand;
      atomicMin(&d.best[gt], epoch_key(t, rr_rank(L, t), lane));
      // the state after crossing, used if this bid wins (a bidding front never changes
      // lanes: its own-lane move reaches the link end, lane changers stay short of it)
      const int off = d.roff[f.vid], len = d.rlen[f.vid];
      const int cur = d.B.cur[s1 - 1];
      const int ncur = d.loop ? (cur + 1) % len : cur + 1;
      const int k2 = ncur + 1;
      const int nnxt = k2 < len ? d.routes[off + k2] : (d.loop ? d.routes[off + k2 % len] : -1);
      const int m = lane < Lnx.lanes - 1 ? lane : Lnx.lanes - 1;
      d.cr[g] = CrossRec{xo - L.len, vo, gt, ncur, nnxt, (uint8_t)move_class(d, f.nxt, nnxt), (uint8_t)m, 0, 0, {0, 0}};
    }
    // by sorted position, so that the chunk kernel stages them with the vehicle arrays
    d.a_own[s1 - 1] = a;
    d.flags[s1 - 1] = fl;
  }
  // the chunks of the chunk kernel: sorted positions, link and lane ranges
  const int nB = d.ctl->nB;
  const int n_chunks = (nB + kChunkT - 1) / kChunkT;
  // chunk k goes to thread T - 1 - k: the last threads of the grid, which have one lane
  // fewer than the first ones in the lane loop above
  const int T = gridDim.x * blockDim.x;
  for (int k = T - 1 - (int)(blockIdx.x * blockDim.x + threadIdx.x); k < n_chunks; k += T) {
    ChunkInfo c;
    c.c0 = chunk_cut(d, k * kChunkT, nB);
    c.c1 = chunk_cut(d, (k + 1) * kChunkT, nB);
    c.e_lo = c.e_hi = c.g_lo = c.g_hi = 0;
    if (c.c1 > c.c0) {
      c.e_lo = d.B.link[c.c0];
      c.e_hi = d.B.link[c.c1 - 1];
      c.g_lo = d.links[c.e_lo].lane_base;
      const LinkRec& Lh = d.links[c.e_hi];
      c.g_hi = Lh.lane_base + Lh.lanes;
    }
    if (split && c.c1 - c.c0 > kChunkCap) {
      d.big_chunks[atomicAdd(&d.ctl->n_big, 1)] = c;
      c.c1 = c.c0;
    }
    d.chunks[k] = c;
  }
}

template <bool TYPES>
__global__ void __launch_bounds__(256) k_front(Dev d) {
  griddep_wait();
  if (step_timed_out(d)) return;
  ph_front<TYPES>(d, d.chunk_split != 0);
}

// ------------------------------------------------------------------ chunks
// First view index q in [s0, s1) whose (x, vid) exceeds (x, vid).
__device__ __forceinline__ int view_upper(const ChunkView& V, int s0, int s1, float x, int vid) {
  int lo = s0, hi = s1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const float xm = V.x[mid];
    if (xm > x || (xm == x && V.vid[mid] > vid)) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// First view index q in [s0, s1) with x >= xb (positions ascend within a lane).
__device__ __forceinline__ int view_lower_x(const ChunkView& V, int s0, int s1, float xb) {
  int lo = s0, hi = s1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (V.x[mid] < xb) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Own-lane step of every vehicle of the chunk (fronts from k_front), tentative move,
// lane-change candidacy; returns the number of candidates (block-uniform).
template <bool FAST, bool TYPES>
__device__ __forceinline__ int chunk_own(const Dev& d, const ChunkView& V, int n, int16_t* list, int* s_cnt) {
  if (threadIdx.x == 0) *s_cnt = 0;
  __syncthreads();
  for (int i0 = 0; i0 < n; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    bool el = false;
    if (i < n) {
      const float x = V.x[i], v = V.v[i];
      const int g = V.g[i];
      const bool front = i + 1 == n || V.g[i + 1] != g;
      const LinkRec L = view_link(d, V, V.link[i]);
      const int vid = V.vid[i];
      ClassPar P;
      float v0;
      view_par<TYPES>(d, V, L, vid, P, v0);
      const float om = free_term(v, v0);
      float a;
      uint8_t fl;
      if (front) {   // the lane-front kernel's acceleration and flags, staged by position
        a = V.a[i];
        fl = V.fl[i] | kFlagFront;
      } else {
        const float sg = (V.x[i + 1] - x) - (TYPES ? veh_len<true>(d, V.vid[i + 1]) : d.vlen);
        a = idm_om(P, om, d.s_min, sg, v, V.v[i + 1]);
        // a stop-sign holder acquired the node within stop_acquire_m of the line and has
        // not moved back since (positions never decrease on a link): farther vehicles
        // cannot hold it, and skip the read
        fl = (L.ctrl == kCtrlStop && L.len - x <= d.stop_acq && d.holder[L.to] == vid) ? kFlagHolder : 0;
      }
      V.om[i] = om;
      float xo, vo;
      ballistic(x, v, a, d.dt, d.hdt2, xo, vo);
      el = L.lanes >= 2 && x >= d.zone && xo < L.len - d.zone;
      V.a[i] = a;
      V.fl[i] = fl | (el ? kFlagElig : 0);
      V.it[i] = 0;
    }
    if (FAST) {
      const unsigned m = __ballot_sync(0xffffffffu, el);
      const int ln = threadIdx.x & 31;
      int base = 0;
      if (ln == 0 && m) base = atomicAdd(s_cnt, __popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (el) list[base + __popc(m & ((1u << ln) - 1u))] = (int16_t)i;
    } else if (el) {
      atomicAdd(s_cnt, 1);
    }
  }
  __syncthreads();
  return *s_cnt;
}

// Lane-change decision of the candidate at view index i (position p = c0 + i) from the
// state at t: MOBIL incentive (Kesting, Treiber & Helbing 2007) for discretionary
// changes, mandatory changes toward the lanes of the next movement once within the
// drawn switch distance, gap acceptance = positive lead and lag gaps and both the
// changer's and the new follower's accelerations >= -b_safe.
template <bool TYPES>
__device__ __forceinline__ void chunk_decide_one(const Dev& d, const ChunkView& V, int i, int c0, int t,
                                                 unsigned ep) {
  const LinkRec L = view_link(d, V, V.link[i]);
  const float x = V.x[i], v = V.v[i];
  const int vid = V.vid[i], g = V.g[i];
  const int lane = g - L.lane_base;
  const int nxt = V.nxt[i];
  ClassPar P;
  float v0;
  view_par<TYPES>(d, V, L, vid, P, v0);
  const int M = lane_mask(V.mv[i], L.lanes);
  int dirs[2];
  int nd = 0;
  bool mand = false;
  if ((M >> lane) & 1) {
    if (lane + 1 < L.lanes && ((M >> (lane + 1)) & 1)) dirs[nd++] = 1;
    if (lane >= 1 && ((M >> (lane - 1)) & 1)) dirs[nd++] = -1;
  } else {
    const int ms = __ffs(M) - 1;
    const int dd = ms > lane ? 1 : -1;
    const int ncross = ms > lane ? ms - lane : lane - ms;
    const float thr = (d.lam * (float)ncross) * d.tau[mand_index(d.hseed[vid], V.cur[i])];
    mand = L.len - x <= thr;
    dirs[nd++] = dd;
  }
  const uint8_t flp = V.fl[i];
  const bool front = (flp & kFlagFront) != 0;
  const bool hold = (flp & kFlagHolder) != 0;
  const bool closed_self = nxt >= 0 && line_closed(d, L, t, hold);
  int chosen = 0;
  float chosen_inc = 0.0f, chosen_at = 0.0f;
  float dno = 0.0f;
  bool dno_known = false;
  for (int k = 0; k < nd; k++) {
    const int dd = dirs[k];
    const int l2 = lane + dd;
    const int g2 = L.lane_base + l2;
    const int s0 = view_lane_start(d, V, g2) - c0, s1 = view_lane_start(d, V, g2 + 1) - c0;
    const int up = view_upper(V, s0, s1, x, vid);
    const int Ln = up < s1 ? up : -1;
    const int Fn = up > s0 ? up - 1 : -1;
    float ac;
    if (Ln >= 0) {
      const float sl = (V.x[Ln] - x) - (TYPES ? veh_len<true>(d, V.vid[Ln]) : d.vlen);
      if (!(sl > 0.0f)) continue;
      ac = idm_om(P, V.om[i], d.s_min, sl, v, V.v[Ln]);
    } else {
      ac = acc_front<TYPES>(d, ep, L, P, v0, vid, nxt, l2, x, v, closed_self);
    }
    if (!(ac >= -d.mbsafe)) continue;
    float an = 0.0f;
    if (Fn >= 0) {
      const float sg = (x - V.x[Fn]) - veh_len<TYPES>(d, vid);
      if (!(sg > 0.0f)) continue;
      ClassPar PF = P;
      float v0F = v0;
      if (TYPES) veh_par<true>(d, L, V.vid[Fn], PF, v0F);
      an = idm_om(PF, V.om[Fn], d.s_min, sg, V.v[Fn], v);
      if (!(an >= -d.mbsafe)) continue;
    }
    if (mand) {
      chosen = dd;
      chosen_at = ac;
      break;
    }
    const float dc = ac - V.a[i];
    const float dn = Fn >= 0 ? an - V.a[Fn] : 0.0f;
    if (!dno_known) {   // the old follower's gain does not depend on the direction
      dno_known = true;
      if (i > 0 && V.g[i - 1] == g) {   // old follower F = i - 1
        const int F = i - 1;
        ClassPar PF = P;
        float v0F = v0;
        if (TYPES) veh_par<true>(d, L, V.vid[F], PF, v0F);
        float ao;
        if (!front) {
          const float sF = (V.x[i + 1] - V.x[F]) - (TYPES ? veh_len<true>(d, V.vid[i + 1]) : d.vlen);
          ao = idm_om(PF, V.om[F], d.s_min, sF, V.v[F], V.v[i + 1]);
        } else {
          const int vF = V.vid[F];
          const int nF = V.nxt[F];
          const bool holdF = L.len - V.x[F] <= d.stop_acq && is_holder(d, L, t, vF, lane, false);
          const bool closedF = nF >= 0 && line_closed(d, L, t, holdF);
          ao = acc_front<TYPES>(d, ep, L, PF, v0F, vF, nF, lane, V.x[F], V.v[F], closedF);
        }
        dno = ao - V.a[F];
      }
    }
    float inc = dc + d.mp * (dn + dno);
    if (dd < 0) inc = inc + d.mbias;
    if (!(inc > d.mathr)) continue;
    if (chosen == 0 || inc > chosen_inc) {
      chosen = dd;
      chosen_inc = inc;
      chosen_at = ac;
    }
  }
  V.it[i] = (int8_t)chosen;
  V.at[i] = chosen_at;
}

// Conflicts, final move, admission, transition, arrival of view index i -> slot c0 + i
// of buffer A, with its arrival index in the next rebuild's lane count.
template <bool OUT, bool TYPES>
__device__ __forceinline__ void chunk_move_one(const Dev& d, const ChunkView& V, int i, int c0, int t) {
  const int p = c0 + i;
  const int e = V.link[i];
  const LinkRec L = view_link(d, V, e);
  const float s0c = V.cls[L.cls].s0;
  const float x = V.x[i], v = V.v[i];
  const int vid = V.vid[i];
  const int lane = V.g[i] - L.lane_base;
  const int nxt = V.nxt[i], cur = V.cur[i];
  const uint8_t fl = V.fl[i];
  int change = V.it[i];
  const float a_own = V.a[i];
  const float a_chg = change ? V.at[i] : 0.0f;
  if (change != 0) {
    // cancelled by a lower-id vehicle changing into the same lane less than (vehicle
    // length + s0) away (the longer of the two lengths with vehicle types); such
    // vehicles sit in lanes tgt-1 and tgt+1 of the same link, inside the chunk
    // Only vehicles within the distance can cancel: each lane is sorted by position, so
    // the scan covers the window |x_q - x| <= 2 (longest length + s0) + 1 m found by a
    // binary search; every vehicle outside it fails the test below by a wide margin.
    const int tgt = lane + change;
    const float len_self = TYPES ? veh_len<true>(d, vid) : d.vlen;
    const float thr = d.vlen + s0c;
    const float win = 2.0f * ((TYPES ? d.vlen_max : d.vlen) + s0c) + 1.0f;
    bool cancel = false;
    for (int src = tgt - 1; src <= tgt + 1 && !cancel; src += 2) {
      if (src < 0 || src >= L.lanes) continue;
      const int gs = L.lane_base + src;
      const int q1 = view_lane_start(d, V, gs + 1) - c0;
      for (int q = view_lower_x(V, view_lane_start(d, V, gs) - c0, q1, x - win); q < q1 && V.x[q] <= x + win && !cancel;
           q++) {
        const int iq = V.it[q];
        if (iq == 0 || src + iq != tgt || V.vid[q] >= vid) continue;
        const float thr_q = TYPES ? fmaxf(len_self, veh_len<true>(d, V.vid[q])) + s0c : thr;
        if (fabsf(V.x[q] - x) < thr_q) cancel = true;
      }
    }
    if (cancel) change = 0;
  }
  const float acc = change ? a_chg : a_own;
  float x1, v1;
  ballistic(x, v, acc, d.dt, d.hdt2, x1, v1);
  if (OUT && d.emis) {
    // Eq. 8-9 at this step's speed and acceleration, over dt
    double2 q = d.emis[vid];
    q.x += (double)(fuel_rate(v, acc) * d.dt);
    q.y += (double)(co_rate(v) * d.dt);
    d.emis[vid] = q;
  }
  const bool hold = (fl & kFlagHolder) != 0;
  int nl = lane + change, nlink = e, ncur = cur, nnxt = nxt;
  int nmv = -1;   // movement class after a crossing (else unchanged)
  float nx = x1, nv = v1;
  bool crossed = false;
  int gcross = 0;   // lane id after a crossing
  if (x1 >= L.len) {
    if (nxt < 0) {
      d.A.link[p] = -1;
      if (OUT && d.tt_sum) note_exit(d, vid, e, t);
      d.status[vid] = kArrived;
      d.arr_step[vid] = (int32_t)t;
      atomicAdd(&d.ctl->n_arr, 1);
      return;
    }
    bool won = false;
    CrossRec c;
    if (fl & kFlagCand) {   // a bidding front: its crossing state is in the lane's record
      c = d.cr[V.g[i]];
      won = d.best[c.gt] == epoch_key(t, rr_rank(L, t), lane);
    }
    if (won) {
      gcross = c.gt;
      ncur = c.ncur;
      nnxt = c.nnxt;
      nlink = nxt;
      nl = c.m;
      nx = c.nx;
      nv = c.nv;
      crossed = true;
      nmv = c.nmv;
      if (OUT && d.tt_sum) {
        note_exit(d, vid, e, t);
        d.enter[vid] = t;
      }
    } else {
      nx = L.len;
      nv = 0.0f;
    }
  }
  if (hold) d.holder[L.to] = crossed ? -1 : vid;
  if (!crossed && (unsigned)nl >= L.lanes) {
    set_err(d, kErrLane, vid);
    d.A.link[p] = -1;
    return;
  }
  const int gn = crossed ? gcross : L.lane_base + nl;
  d.A.gid[p] = gn;
  d.aidx[p] = count_in_lane(d, gn);
  d.A.mv[p] = nmv >= 0 ? (uint8_t)nmv : V.mv[i];
  d.adec[p] = (int8_t)change;
  d.A.x[p] = nx;
  d.A.v[p] = nv;
  d.A.vid[p] = vid;
  d.A.link[p] = nlink;
  d.A.nxt[p] = nnxt;
  d.A.cur[p] = ncur;
  d.A.lane[p] = nl;
}

// One chunk: own-lane step, decisions, moves.
template <bool FAST, bool OUT, bool TYPES>
__device__ __forceinline__ void chunk_step(const Dev& d, const ChunkView& V, int c0, int n, int t, unsigned ep,
                                           int16_t* list, int* s_cnt) {
  const int nc = chunk_own<FAST, TYPES>(d, V, n, list, s_cnt);
  if (threadIdx.x == 0 && nc) atomicAdd(&d.ctl->n_elig, nc);
  if (FAST) {
    for (int j = threadIdx.x; j < nc; j += blockDim.x) chunk_decide_one<TYPES>(d, V, list[j], c0, t, ep);
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (V.fl[i] & kFlagElig) chunk_decide_one<TYPES>(d, V, i, c0, t, ep);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) chunk_move_one<OUT, TYPES>(d, V, i, c0, t);
  __syncthreads();   // the chunk's staged arrays are read before the next chunk refills them
}

// Which chunks a launch takes.  BIG = false: every chunk of the chunk table from the
// atomic counter (one beyond kChunkCap on global memory), then the departures.  BIG =
// true: the chunks the lane-front phase moved to the big-chunk list, by index, and no
// departures.  S: the block's staging area (dynamic shared memory).  Returns early
// (error word set) when a staging wait runs out.
// INS_FIRST: the departures before the chunks instead of after them (the persistent
// launch, where it is faster on sparse networks; the per-step kernel keeps them last,
// where every block's first chunk would wait for its share of the queue checks).
template <bool OUT, bool TYPES, bool BIG, typename SMT, bool INS_FIRST = false>
__device__ __forceinline__ void ph_chunk(const Dev& d, SMT& S) {
  constexpr int CAP = SMT::kCap;
  // the chunk being processed and the next one (taken by thread 0 while the current
  // chunk's copies are in flight), alternating between two slots
  __shared__ int s_k[2], s_cnt;
  __shared__ ChunkInfo s_info[2];
  // departures (appended after the sorted vehicles; they read only state of step t and
  // this step's admission bids, complete since the lane-front phase, and write slots and
  // counts that no chunk touches)
  if (INS_FIRST && !BIG && d.n_qlinks > 0) ph_insert<OUT, TYPES>(d);
  const int nB = d.ctl->nB;
  const int t = (int)d.ctl->t;
  const unsigned ep = d.ctl->occ_epoch;
  const int n_chunks = (nB + kChunkT - 1) / kChunkT;
  const bool cls_staged = !TYPES && d.n_cls <= kChunkClasses;
  if (cls_staged)
    for (int c = threadIdx.x; c < d.n_cls; c += blockDim.x) S.cls[c] = d.cls[c];
  if (threadIdx.x == 0) {
    mbar_init(&S.bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!BIG) {
      const int k = atomicAdd(&d.ctl->chunk_next, 1);
      s_k[0] = k;
      if (k < n_chunks) s_info[0] = d.chunks[k];
    }
  }
  __syncthreads();
  int slot = 0, kb = blockIdx.x;
  uint32_t phase = 0;
  for (;;) {
    ChunkInfo c;
    if (BIG) {   // the chunks the front phase listed as oversized
      if (kb >= d.ctl->n_big) break;
      c = d.big_chunks[kb];
      kb += gridDim.x;
    } else {
      const int k = s_k[slot];
      if (k >= n_chunks) break;
      c = s_info[slot];
      slot ^= 1;
      if (c.c1 - c.c0 <= 0) {   // empty, or left to the big-chunk launch
        if (threadIdx.x == 0) {
          const int k2 = atomicAdd(&d.ctl->chunk_next, 1);
          s_k[slot] = k2;
          if (k2 < n_chunks) s_info[slot] = d.chunks[k2];
        }
        __syncthreads();
        continue;
      }
    }
    const int c0 = c.c0, n = c.c1 - c.c0;
    const bool fast = n <= CAP;
    const int nlk = fast && c.e_hi - c.e_lo < kChunkLinks ? c.e_hi - c.e_lo + 1 : 0;
    const int g_la = c.g_lo & ~3;
    const int nls_a = ((c.g_hi + 1 - g_la) + 3) & ~3;   // lane starts g_la .. g_hi, a multiple of 4
    const int nls = fast && nls_a <= kChunkLanes ? nls_a : 0;
    const int c0a = c0 & ~15, c1a = (c.c1 + 15) & ~15;
    if (threadIdx.x == 0) {
      if (fast) {
        // stage [c0a, c1a) = [c0, c1) widened to multiples of 16 positions (the arrays
        // carry kSlotPad spare elements, so the widened copy stays inside them) with the
        // fronts' accelerations and flags, the link records of the chunk and its lane
        // starts
        const uint32_t cnt = (uint32_t)(c1a - c0a);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&S.bar, cnt * (8 * 4 + 2) + (uint32_t)nlk * (uint32_t)sizeof(LinkRec) + (uint32_t)nls * 4);
        bulk_g2s(S.x, d.B.x + c0a, cnt * 4, &S.bar);
        bulk_g2s(S.v, d.B.v + c0a, cnt * 4, &S.bar);
        bulk_g2s(S.vid, d.B.vid + c0a, cnt * 4, &S.bar);
        bulk_g2s(S.g, d.tg + c0a, cnt * 4, &S.bar);
        bulk_g2s(S.link, d.B.link + c0a, cnt * 4, &S.bar);
        bulk_g2s(S.nxt, d.B.nxt + c0a, cnt * 4, &S.bar);
        bulk_g2s(S.cur, d.B.cur + c0a, cnt * 4, &S.bar);
        bulk_g2s(S.a, d.a_own + c0a, cnt * 4, &S.bar);
        bulk_g2s(S.mv, d.B.mv + c0a, cnt, &S.bar);
        bulk_g2s(S.fl, d.flags + c0a, cnt, &S.bar);
        if (nlk) bulk_g2s(S.lk, d.links + c.e_lo, (uint32_t)nlk * (uint32_t)sizeof(LinkRec), &S.bar);
        if (nls) bulk_g2s(S.ls, d.lane_start + g_la, (uint32_t)nls * 4, &S.bar);
      }
      // the next chunk, into the other slot (read after this chunk's last barrier)
      if (!BIG) {
        const int k2 = atomicAdd(&d.ctl->chunk_next, 1);
        s_k[slot] = k2;
        if (k2 < n_chunks) s_info[slot] = d.chunks[k2];
      }
    }
    if (fast) {
      const bool ok = mbar_wait(&S.bar, phase, d.wait_limit);
      if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) {
          set_err(d, kErrTimeout, blockIdx.x);
          mbar_wait(&S.bar, phase, kWaitLimit);   // let the issued copies land
        }
        __syncthreads();
        return;
      }
      phase ^= 1u;
      const int o = c0 - c0a;
      const ChunkView V{S.x + o,   S.v + o,  S.vid + o, S.g + o,  S.link + o, S.nxt + o,  S.cur + o,
                        S.mv + o,  S.a + o,  S.at + o,  S.om + o, S.fl + o,   S.it + o,   S.lk,
                        S.ls,      cls_staged ? S.cls : d.cls,    c.e_lo,     nlk,        g_la,
                        nls};
      chunk_step<true, OUT, TYPES>(d, V, c0, n, t, ep, S.list, &s_cnt);
    } else {
      // oversized chunk: the same code on B and the per-position scratch (the own-lane
      // free terms in xo)
      const ChunkView V{d.B.x + c0,  d.B.v + c0,   d.B.vid + c0, d.tg + c0,     d.B.link + c0, d.B.nxt + c0,
                        d.B.cur + c0, d.B.mv + c0, d.a_own + c0, d.at + c0,     d.xo + c0,     d.flags + c0,
                        d.intent + c0, nullptr,    nullptr,      cls_staged ? S.cls : d.cls, 0, 0, 0, 0};
      chunk_step<false, OUT, TYPES>(d, V, c0, n, t, ep, S.list, &s_cnt);
    }
  }
  if (!INS_FIRST && !BIG && d.n_qlinks > 0) ph_insert<OUT, TYPES>(d);
}

template <bool OUT, bool TYPES>
__global__ void __launch_bounds__(kChunkThreads, kChunkMinBlocks) k_chunk(Dev d) {
  griddep_wait();
  if (step_timed_out(d)) return;
  extern __shared__ __align__(16) unsigned char chunk_smem[];
  ph_chunk<OUT, TYPES, false>(d, *reinterpret_cast<ChunkSmem*>(chunk_smem));
}

// The chunks beyond kChunkCap (launched after the chunk kernel when chunk_split).
template <bool OUT, bool TYPES>
__global__ void __launch_bounds__(kBigThreads, 2) k_chunk_big(Dev d) {
  griddep_wait();
  if (step_timed_out(d)) return;
  extern __shared__ __align__(16) unsigned char chunk_smem[];
  ph_chunk<OUT, TYPES, true>(d, *reinterpret_cast<ChunkSmemBig*>(chunk_smem));
}

// ------------------------------------------------------------------ persistent step
// All phases of n steps in one cooperative launch (the rebuild, the lane fronts, the
// chunks with the departures, the counters): every block runs each phase's share,
// then waits at a grid barrier.  The barrier's wait is bounded:
// after `limit` SM cycles (about a second by default) a block sets kErrTimeout in the
// error word and leaves; every waiting block also leaves as soon as it sees the flag,
// so the launch always ends and the host reports SIM_ETIMEOUT.
__device__ __forceinline__ bool grid_barrier(GridSync* gs, int* err, long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = &gs->gen;
    volatile int* verr = err;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&gs->count, 1u);
    if (arrived == gridDim.x - 1) {
      gs->count = 0;
      __threadfence();
      atomicAdd(&gs->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if ((*verr & kErrTimeout) || clock64() - t0 > limit) {
          atomicOr(err, kErrTimeout);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (*verr & kErrTimeout) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <bool OUT, bool TYPES>
__device__ __forceinline__ void persistent_steps(const Dev& d, GridSync* gs, int n_steps, long long limit,
                                                 ChunkSmem& S) {
  int* err = &d.ctl->err;
  for (int step = 0; step < n_steps; step++) {
    // the previous step's counter update (block 0) needs no barrier of its own: nothing
    // before this step's scatter reads what it writes
    ph_scan_sum(d);
    if (!grid_barrier(gs, err, limit)) return;
    ph_scan_fin(d);
    if (!grid_barrier(gs, err, limit)) return;
    ph_scatter(d);
    if (!grid_barrier(gs, err, limit)) return;
    ph_rank<false>(d);
    if (!grid_barrier(gs, err, limit)) return;
    // the edge sample and the lane fronts read the sorted state and write disjoint arrays
    if (d.acc_u) ph_edge_sample(d);
    ph_front<TYPES>(d, false);   // every chunk stays in the table
    if (!grid_barrier(gs, err, limit)) return;
    ph_chunk<OUT, TYPES, false, ChunkSmem, true>(d, S);
    if (!grid_barrier(gs, err, limit)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ph_finish(d);
  }
  // the last counter update is visible when the launch ends
}

__global__ void __launch_bounds__(1024, 1) k_persistent(Dev d, GridSync* gs, int n_steps, long long limit) {
  extern __shared__ __align__(16) unsigned char chunk_smem[];
  ChunkSmem& S = *reinterpret_cast<ChunkSmem*>(chunk_smem);
  const bool out = d.emis || d.tt_sum;
  if (d.vtype) {
    if (out) persistent_steps<true, true>(d, gs, n_steps, limit, S);
    else persistent_steps<false, true>(d, gs, n_steps, limit, S);
  } else {
    if (out) persistent_steps<true, false>(d, gs, n_steps, limit, S);
    else persistent_steps<false, false>(d, gs, n_steps, limit, S);
  }
}

// Largest co-resident grid of the persistent kernel for a block size (0 if none).
int persistent_max_blocks_per_sm(int threads) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent, threads, kChunkSmemBytes) != cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_persistent(const Dev& d, GridSync* gs, int blocks, int threads, int n_steps, long long limit,
                              cudaStream_t s) {
  Dev dd = d;
  void* args[] = {&dd, &gs, &n_steps, &limit};
  return cudaLaunchCooperativeKernel((const void*)k_persistent, dim3(blocks), dim3(threads), args, kChunkSmemBytes,
                                     s);
}

// ------------------------------------------------------------------ launch
template <typename K>
static int chunk_blocks(K kern) {
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kChunkSmemBytes) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
          cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kChunkThreads, kChunkSmemBytes) != cudaSuccess) return 0;
  return nb;
}

template <typename K>
static int chunk_big_blocks(K kern) {
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBigSmemBytes) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
          cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kBigThreads, kBigSmemBytes) != cudaSuccess) return 0;
  return nb;
}

// Entries of the chunk table for up to n_trips vehicles.
size_t chunk_table_size(int n_trips) { return (size_t)n_trips / kChunkT + 2; }

// Resident blocks per SM of the chunk kernel (plain / outputs x vehicle types); also
// raises the kernels' dynamic shared-memory limit.  Called once per handle.
void chunk_setup(int blocks_per_sm[8]) {
  blocks_per_sm[0] = chunk_blocks(k_chunk<false, false>);
  blocks_per_sm[1] = chunk_blocks(k_chunk<true, false>);
  blocks_per_sm[2] = chunk_blocks(k_chunk<false, true>);
  blocks_per_sm[3] = chunk_blocks(k_chunk<true, true>);
  blocks_per_sm[4] = chunk_big_blocks(k_chunk_big<false, false>);
  blocks_per_sm[5] = chunk_big_blocks(k_chunk_big<true, false>);
  blocks_per_sm[6] = chunk_big_blocks(k_chunk_big<false, true>);
  blocks_per_sm[7] = chunk_big_blocks(k_chunk_big<true, true>);
}

template <typename... KArgs, typename... Args>
static void launch_pdl2(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

// Resident 256-thread blocks per SM of the lane-front kernel (without / with vehicle
// types): its grid is one resident wave, every thread taking lanes in a grid stride (a
// partial second wave of blocks would take as long as the first).
void front_setup(int blocks_per_sm[2]) {
  blocks_per_sm[0] = blocks_per_sm[1] = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[0], k_front<false>, 256, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[1], k_front<true>, 256, 0);
}

void launch_front(const Dev& d, cudaStream_t s) {
  if (d.vtype) launch_pdl2(k_front<true>, d.front_grid[1], 256, 0, s, d);
  else launch_pdl2(k_front<false>, d.front_grid[0], 256, 0, s, d);
}

template <bool OUT, bool TYPES>
static void launch_chunk_v(const Dev& d, int v, cudaStream_t s) {
  launch_pdl2(k_chunk<OUT, TYPES>, d.chunk_grid[v], kChunkThreads, kChunkSmemBytes, s, d);
  if (d.chunk_split) launch_pdl2(k_chunk_big<OUT, TYPES>, d.chunk_grid[4 + v], kBigThreads, kBigSmemBytes, s, d);
}

// The chunk kernel, and the big-chunk kernel when the network has links that can hold
// more than kChunkCap vehicles (chunk_split; otherwise an oversized chunk, should one
// ever form, runs on global memory inside the chunk kernel: the same results either way).
void launch_chunk(const Dev& d, cudaStream_t s) {
  const bool out = d.emis || d.tt_sum;
  const int v = (out ? 1 : 0) + (d.vtype ? 2 : 0);
  switch (v) {
    case 0: launch_chunk_v<false, false>(d, v, s); break;
    case 1: launch_chunk_v<true, false>(d, v, s); break;
    case 2: launch_chunk_v<false, true>(d, v, s); break;
    default: launch_chunk_v<true, true>(d, v, s); break;
  }
}

// Whether the big-chunk launch is worth its place in the step: at least a quarter of
// the network's lane-metres lie on links that hold more than kChunkCap vehicles when
// their lanes are packed bumper to bumper with the shortest vehicle (lane_m[e]: lanes x
// length of link e).  Where such links are rare, their chunks run on global memory
// inside the chunk kernel, overlapped with the others, which costs less than a launch.
bool chunk_split_needed(const double* lane_m, int n_links, float vlen_min) {
  if (!(vlen_min > 0.0f)) return false;
  double all = 0.0, big = 0.0;
  for (int e = 0; e < n_links; e++) {
    all += lane_m[e];
    if (lane_m[e] / (double)vlen_min > (double)kChunkCap) big += lane_m[e];
  }
  return big >= 0.25 * all && big > 0.0;
}

}  // namespace gbt
