// One simulation step of the microsimulation hot path (Waddell et al., Sec. 6.3.2):
//
//   1. occupancy rebuild: counting pass by lane, exclusive scan, scatter, in-segment
//      rank by (position, vid) -> vehicles of buffer A land sorted in buffer B
//      (the per-lane order replaces the "traffic atlas" of Sec. 6.3.3);
//   2. stop-sign acquisition (one vehicle at a time, Sec. 6.3.2);
//   3. own-lane IDM acceleration (Eq. 7) with look-ahead over the link end and the
//      stop line, tentative ballistic move, admission candidates;
//   4. lane-change decisions (mandatory / discretionary + gap acceptance, Sec. 6.3.2);
//   5. conflict resolution, final move, edge transition, arrival -> buffer A;
//   6. departures from the per-link queues -> appended to buffer A.
//
// Every kernel reads the state at step t (buffer B and the per-step scratch written
// by earlier kernels of the same step) and writes the state at t+1, so the result
// does not depend on thread scheduling; ties are broken by vehicle id or by the
// rotating round-robin rank.
#include "gbt_rebuild.cuh"

namespace gbt {

// ------------------------------------------------------------------ occupancy
__global__ void k_count(Dev d) {
  griddep_wait();
  const int nA = d.ctl->nA;
  GRID_STRIDE(s, nA) {
    int e = d.A.link[s];
    if (e < 0) continue;
    int lane = d.A.lane[s];
    const LinkRec& L = d.links[e];
    if ((unsigned)lane >= L.lanes) { set_err(d, kErrLane, s); continue; }
    d.A.gid[s] = L.lane_base + lane;
    d.aidx[s] = atomicAdd(&d.cnt[L.lane_base + lane], 1);
  }
}

int scan_blocks(int n_lanes) { return (n_lanes + kScanChunk - 1) / kScanChunk; }

// Whether a lane of some link can hold more than kLongSeg vehicles (packed bumper to
// bumper with the shortest vehicle): only then does the step launch k_rank_long.
bool rank_long_needed(double max_len, float vlen_min) {
  return !(vlen_min > 0.0f) || max_len / (double)vlen_min > (double)kLongSeg;
}

__global__ void k_scan_sum(Dev d) {
  griddep_wait();
  if (step_timed_out(d)) return;
  ph_scan_sum(d);
}

__global__ void k_scan_fin(Dev d) {
  griddep_wait();
  if (step_timed_out(d)) return;
  ph_scan_fin(d);
}

__global__ void k_scatter(Dev d) {
  griddep_wait();
  if (step_timed_out(d)) return;
  ph_scatter(d);
}

// Rank of each vehicle inside its lane segment by (x, vid); the vehicle's state
// moves from its slot in A to position lane_start + rank in B.  The vehicle that
// lands first in its segment is the lane's rearmost: it writes the lane's rear record
// (the leader seen across the link end by vehicles entering or approaching the lane).
// The vehicle that lands last is the lane's front: if its link ends at a free stop-
// controlled node, it bids for the node here (Sec. 6.3.2 stop signs, one vehicle at
// a time): the bid with the smallest (round-robin rank of its link, lane) acquires it.
// Long lane segments (queues): one block per segment, keys (x, vid) staged in shared
// memory.  The scatter leaves a segment as a few ascending runs (each warp of the move
// kernel counts its vehicles of a lane in order; the warps' atomics interleave), so the
// rank of a key is its index in its own run plus, for every other run, the number of
// keys below it there (a binary search): an exact merge count.  Segments with more
// than kMaxRuns runs are sorted with a bitonic network (Batcher 1968) instead, and
// segments beyond the shared-memory capacity fall back to the per-vehicle count.
constexpr int kLongCap = 2048, kMaxRuns = 64;

__device__ __forceinline__ bool key_less(float xa, int va, float xb, int vb) {
  return xa < xb || (xa == xb && va < vb);
}

__global__ void __launch_bounds__(256) k_rank_long(Dev d) {
  griddep_wait();
  if (step_timed_out(d)) return;
  __shared__ float sx[kLongCap];
  __shared__ int32_t sv[kLongCap];
  __shared__ int16_t si[kLongCap];
  __shared__ int16_t run_start[kMaxRuns + 1];
  __shared__ int s_runs;
  const int nl = d.ctl->n_long;
  const int t = (int)d.ctl->t;
  const unsigned ep = d.ctl->occ_epoch;
  for (int j = blockIdx.x; j < nl; j += gridDim.x) {
    const int g = d.long_list[j];
    const int s0 = d.lane_start[g], s1 = d.lane_start[g + 1], k = s1 - s0;
    if (k > kLongCap) {
      for (int p = s0 + threadIdx.x; p < s1; p += blockDim.x) {
        const float xp = d.tx[p];
        const int vp = d.tvid[p];
        int rank = 0;
        for (int q = s0; q < s1; q++) {
          const float xq = d.tx[q];
          rank += (xq < xp || (xq == xp && d.tvid[q] < vp)) ? 1 : 0;
        }
        rank_emit(d, d.tsrc[p], xp, vp, g, s0 + rank, s1, rank == 0, t, ep);
      }
      continue;
    }
    if (threadIdx.x == 0) s_runs = 0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      sx[i] = d.tx[s0 + i];
      sv[i] = d.tvid[s0 + i];
    }
    __syncthreads();
    // run starts: positions whose key is below the previous one (and position 0)
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      if (i == 0 || key_less(sx[i], sv[i], sx[i - 1], sv[i - 1])) {
        const int r = atomicAdd(&s_runs, 1);
        if (r < kMaxRuns) run_start[r] = (int16_t)i;
      }
    }
    __syncthreads();
    const int R = s_runs;
    if (R <= kMaxRuns) {
      if (threadIdx.x == 0) {   // order the few run starts; the segment end closes the last
        for (int a = 1; a < R; a++) {
          const int16_t v = run_start[a];
          int b = a - 1;
          while (b >= 0 && run_start[b] > v) {
            run_start[b + 1] = run_start[b];
            b--;
          }
          run_start[b + 1] = v;
        }
        run_start[R] = (int16_t)k;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const float x = sx[i];
        const int v = sv[i];
        int rank = 0;
        for (int r = 0; r < R; r++) {
          const int a = run_start[r], b = run_start[r + 1];
          if (i >= a && i < b) {
            rank += i - a;
            continue;
          }
          int lo = a, hi = b;   // keys of run r below (x, v)
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (key_less(sx[mid], sv[mid], x, v)) lo = mid + 1;
            else hi = mid;
          }
          rank += lo - a;
        }
        rank_emit(d, d.tsrc[s0 + i], x, v, g, s0 + rank, s1, rank == 0, t, ep);
      }
      __syncthreads();
      continue;
    }
    int n = 1;
    while (n < k) n <<= 1;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (i >= k) {
        sx[i] = INFINITY;
        sv[i] = INT32_MAX;
      }
      si[i] = (int16_t)i;
    }
    __syncthreads();
    for (int size = 2; size <= n; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        // pair i compares lo and lo + stride, lo = i with a zero bit inserted at the
        // stride's position (stride is a power of two)
        for (int i = threadIdx.x; i < (n >> 1); i += blockDim.x) {
          const int lo = ((i & ~(stride - 1)) << 1) | (i & (stride - 1)), hi = lo + stride;
          const bool up = (lo & size) == 0;
          const float xa = sx[lo], xb = sx[hi];
          const int va = sv[lo], vb = sv[hi];
          const bool gt = xa > xb || (xa == xb && va > vb);
          if (gt == up) {
            sx[lo] = xb;
            sx[hi] = xa;
            sv[lo] = vb;
            sv[hi] = va;
            const int16_t ia = si[lo];
            si[lo] = si[hi];
            si[hi] = ia;
          }
        }
        __syncthreads();
      }
    }
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
      const int p = s0 + si[r];
      rank_emit(d, d.tsrc[p], sx[r], sv[r], g, s0 + r, s1, r == 0, t, ep);
    }
    __syncthreads();
  }
}

// SKIP_LONG: segments longer than kLongSeg are left to k_rank_long (launched after it);
// without, every segment is ranked here (networks whose lanes cannot hold that many).
template <bool SKIP_LONG>
__global__ void __launch_bounds__(256, 8) k_rank(Dev d) {
  griddep_wait();
  if (step_timed_out(d)) return;
  ph_rank<SKIP_LONG>(d);
}


// Own-lane step of the vehicle at sorted position p (front: the last of its lane):
// Eq. 7 behind the next vehicle of the lane, or for the front behind the rearmost
// vehicle of the next link's mapped lane and the stop line; tentative ballistic move;
// lane-change eligibility (returned); admission candidacy of a front whose move
// reaches the end.
template <bool TAPE, bool TYPES>
__device__ __forceinline__ bool own_core(const Dev& d, int p, bool front, int t, unsigned ep, int e, float x,
                                         float v, int vid, int lane, int nxt, float x1, float v1, int vid1) {
  const LinkRec L = d.links[e];
  // a front looks across the link end: its next link's record is loaded with its own
  LinkRec Lnx;
  if (front && nxt >= 0) Lnx = d.links[nxt];
  ClassPar P;
  float v0;
  veh_par<TYPES>(d, L, vid, P, v0);
  const bool hold = is_holder(d, L, t, vid, lane, front);
  float a;
  TapeForm f;
  bool closed = false, lead = false;
  int gt = 0;
  float room = 0.0f;
  if (!front) {
    const float sg = (x1 - x) - (TYPES ? veh_len<true>(d, vid1) : d.vlen);
    a = idm_acc(P, v0, d.s_min, sg, v, v1, true);
    if (TAPE) f = TapeForm{vid1, sg, v1, kFormLead, 0, 0, 0};
  } else {
    closed = nxt >= 0 && line_closed(d, L, t, hold);
    a = acc_front<TYPES>(d, ep, L, P, v0, vid, nxt, lane, x, v, closed, TAPE ? &f : nullptr, &gt, &lead, &room,
                         &Lnx);
  }
  if (TAPE) {
    TapeRec* rec = tape_slot(d, t, vid);
    rec->lead = f.lead;
    rec->kind = f.kind;
    rec->s = f.s;
    rec->vl = f.vl;
  }
  float xo, vo;
  ballistic(x, v, a, d.dt, d.hdt2, xo, vo);
  d.a_own[p] = a;
  d.xo[p] = xo;
  d.intent[p] = 0;
  // lane-change candidates: multi-lane link, away from both link ends
  const bool elig = L.lanes >= 2 && x >= d.zone && xo < L.len - d.zone;
  uint8_t fl = (front ? kFlagFront : 0) | (hold ? kFlagHolder : 0);
  // admission candidate: front, route continues, stop line open, move reaches the
  // end and lands behind the rearmost vehicle of the mapped lane
  if (front && nxt >= 0 && !closed && xo >= L.len) {
    const bool ok = !lead || (xo - L.len) <= room;
    if (ok) {
      fl |= kFlagCand;
      atomicMin(&d.best[gt], epoch_key(t, rr_rank(L, t), lane));
    }
  }
  d.flags[p] = fl;
  return elig;
}

template <bool TAPE, bool TYPES>
__device__ __forceinline__ bool own_one(const Dev& d, int p, bool front, int t, unsigned ep) {
  const float x1 = front ? 0.0f : d.B.x[p + 1], v1 = front ? 0.0f : d.B.v[p + 1];
  const int vid1 = front ? 0 : d.B.vid[p + 1];
  return own_core<TAPE, TYPES>(d, p, front, t, ep, d.B.link[p], d.B.x[p], d.B.v[p], d.B.vid[p], d.B.lane[p],
                               d.B.nxt[p], x1, v1, vid1);
}

// Append the positions of the block's threads where `pred` holds to the lane-change
// candidate list, in thread order, with one atomic on the list counter per block.
// Every thread of the block must call it (it holds two block barriers).
constexpr int kMaxWarps = 32;   // blocks of up to 1024 threads

__device__ __forceinline__ void block_append(const Dev& d, bool pred, int pos) {
  __shared__ int wn[kMaxWarps + 1];
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, pred);
  if (ln == 0) wn[w] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    const int nw = (int)(blockDim.x >> 5);
    for (int k = 0; k < nw; k++) {
      const int c = wn[k];
      wn[k] = tot;
      tot += c;
    }
    wn[kMaxWarps] = tot ? atomicAdd(&d.ctl->n_elig, tot) : 0;
  }
  __syncthreads();
  if (pred) d.elig[wn[kMaxWarps] + wn[w] + __popc(m & ((1u << ln) - 1u))] = pos;
}

// The block walks blockDim consecutive sorted positions at a time (block-uniform trip
// count, for the candidate list's block barriers).
template <bool TAPE, bool TYPES>
__device__ __forceinline__ void ph_own(const Dev& d) {
  const int nB = d.ctl->nB;
  const int t = (int)d.ctl->t;
  const unsigned ep = d.ctl->occ_epoch;
  for (int base = blockIdx.x * blockDim.x; base < nB; base += gridDim.x * blockDim.x) {
    const int p = base + threadIdx.x;
    bool el = false;
    if (p < nB) {
      // the lane of sorted position p is tg[p]; p is its lane's front when the next
      // position starts another lane
      const int g = d.tg[p];
      const bool front = p + 1 == nB || d.tg[p + 1] != g;
      el = own_one<TAPE, TYPES>(d, p, front, t, ep);
    }
    block_append(d, el, p);
  }
}

template <bool TAPE, bool TYPES>
__global__ void __launch_bounds__(256, 6) k_own(Dev d) {
  griddep_wait();
  if (step_timed_out(d)) return;
  ph_own<TAPE, TYPES>(d);
}

// First position q in [s0, s1) whose (x, vid) exceeds (x, vid) of the probe.
__device__ __forceinline__ int upper_pos(const Dev& d, int s0, int s1, float x, int vid) {
  int lo = s0, hi = s1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    float xm = d.B.x[mid];
    bool greater = xm > x || (xm == x && d.B.vid[mid] > vid);
    if (greater) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Lane-change decision from the state at t: MOBIL incentive (Kesting, Treiber &
// Helbing 2007) for discretionary changes, mandatory changes toward the lanes of
// the next movement once within the drawn switch distance, and gap acceptance =
// no overlap and both the changer's and the new follower's accelerations >= -b_safe.
template <bool TAPE, bool TYPES>
__device__ __forceinline__ void decide_one(const Dev& d, int p, int t, unsigned ep) {
  {
    const int e = d.B.link[p];
    const LinkRec L = d.links[e];
    const float x = d.B.x[p];
    const float v = d.B.v[p];
    const int vid = d.B.vid[p], lane = d.B.lane[p], nxt = d.B.nxt[p], cur = d.B.cur[p];
    ClassPar P;
    float v0;
    veh_par<TYPES>(d, L, vid, P, v0);
    const int M = lane_mask(d.B.mv[p], L.lanes);
    int dirs[2];
    int nd = 0;
    bool mand = false;
    if ((M >> lane) & 1) {
      if (lane + 1 < L.lanes && ((M >> (lane + 1)) & 1)) dirs[nd++] = 1;
      if (lane >= 1 && ((M >> (lane - 1)) & 1)) dirs[nd++] = -1;
    } else {
      int ms = __ffs(M) - 1;
      int dd = ms > lane ? 1 : -1;
      int ncross = ms > lane ? ms - lane : lane - ms;
      float thr = (d.lam * (float)ncross) * d.tau[mand_index(d.hseed[vid], cur)];
      float drem = L.len - x;
      mand = drem <= thr;
      dirs[nd++] = dd;
    }
    const int g = L.lane_base + lane;
    const uint8_t flp = d.flags[p];
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
      const int s0 = d.lane_start[g2], s1 = d.lane_start[g2 + 1];
      const int up = upper_pos(d, s0, s1, x, vid);
      const int Ln = up < s1 ? up : -1;
      const int Fn = up > s0 ? up - 1 : -1;
      float ac;
      TapeForm cf;
      if (Ln >= 0) {
        float sl = (d.B.x[Ln] - x) - (TYPES ? veh_len<true>(d, d.B.vid[Ln]) : d.vlen);
        if (!(sl > 0.0f)) continue;
        ac = idm_acc(P, v0, d.s_min, sl, v, d.B.v[Ln], true);
        if (TAPE) cf = TapeForm{d.B.vid[Ln], sl, d.B.v[Ln], kFormLead, 0, 0, 0};
      } else {
        ac = acc_front<TYPES>(d, ep, L, P, v0, vid, nxt, l2, x, v, closed_self, TAPE ? &cf : nullptr);
      }
      if (!(ac >= -d.mbsafe)) continue;
      float an = 0.0f;
      if (Fn >= 0) {
        float sg = (x - d.B.x[Fn]) - veh_len<TYPES>(d, vid);
        if (!(sg > 0.0f)) continue;
        ClassPar PF = P;
        float v0F = v0;
        if (TYPES) veh_par<true>(d, L, d.B.vid[Fn], PF, v0F);
        an = idm_acc(PF, v0F, d.s_min, sg, d.B.v[Fn], v, true);
        if (!(an >= -d.mbsafe)) continue;
      }
      if (mand) {
        chosen = dd;
        chosen_at = ac;
        if (TAPE) d.tform[vid] = cf;
        break;
      }
      float dc = ac - d.a_own[p];
      float dn = Fn >= 0 ? an - d.a_own[Fn] : 0.0f;
      if (!dno_known) {   // the old follower's gain does not depend on the direction
        dno_known = true;
        if (p > 0 && d.tg[p - 1] == g) {   // old follower F = p - 1
          const int F = p - 1;
          ClassPar PF = P;
          float v0F = v0;
          if (TYPES) veh_par<true>(d, L, d.B.vid[F], PF, v0F);
          float ao;
          if (!front) {
            const float sF = (d.B.x[p + 1] - d.B.x[F]) - (TYPES ? veh_len<true>(d, d.B.vid[p + 1]) : d.vlen);
            ao = idm_acc(PF, v0F, d.s_min, sF, d.B.v[F], d.B.v[p + 1], true);
          } else {
            const int vF = d.B.vid[F];
            const int nF = d.B.nxt[F];
            bool holdF = is_holder(d, L, t, vF, lane, false);
            bool closedF = nF >= 0 && line_closed(d, L, t, holdF);
            ao = acc_front<TYPES>(d, ep, L, PF, v0F, vF, nF, lane, d.B.x[F], d.B.v[F], closedF);
          }
          dno = ao - d.a_own[F];
        }
      }
      float inc = dc + d.mp * (dn + dno);
      if (dd < 0) inc = inc + d.mbias;
      if (!(inc > d.mathr)) continue;
      if (chosen == 0 || inc > chosen_inc) {
        chosen = dd;
        chosen_inc = inc;
        chosen_at = ac;
        if (TAPE) d.tform[vid] = cf;
      }
    }
    d.intent[p] = (int8_t)chosen;
    d.at[p] = chosen_at;
  }
}

// One thread per lane-change candidate of the list built by the own-lane kernel.
template <bool TAPE, bool TYPES>
__device__ __forceinline__ void ph_decide(const Dev& d) {
  const int ne = d.ctl->n_elig;
  const int t = (int)d.ctl->t;
  const unsigned ep = d.ctl->occ_epoch;
  GRID_STRIDE(i, ne) decide_one<TAPE, TYPES>(d, d.elig[i], t, ep);
}

template <bool TAPE, bool TYPES>
__global__ void __launch_bounds__(256, 6) k_decide(Dev d) {
  griddep_wait();
  if (step_timed_out(d)) return;
  ph_decide<TAPE, TYPES>(d);
}

// ------------------------------------------------------------------ measured outputs

__global__ void k_edge_sample(Dev d) {
  griddep_wait();
  if (step_timed_out(d)) return;
  ph_edge_sample(d);
}

// ------------------------------------------------------------------ move
// OUT: the measured outputs are on (a separate instantiation keeps the plain kernel's
// register count, and so its occupancy, as it is without them); TYPES: vehicle types.
template <bool TAPE, bool OUT, bool TYPES>
__device__ __forceinline__ void ph_move(const Dev& d) {
  const int nB = d.ctl->nB;
  const int t = (int)d.ctl->t;
  GRID_STRIDE(p, nB) {
    const int e = d.B.link[p];
    const LinkRec L = d.links[e];
    const ClassPar P = d.cls[L.cls];
    const float x = d.B.x[p], v = d.B.v[p];
    const int vid = d.B.vid[p], lane = d.B.lane[p], nxt = d.B.nxt[p], cur = d.B.cur[p];
    const uint8_t fl = d.flags[p];
    int change = d.intent[p];
    // both candidate accelerations, read before the change is settled (at[] holds an
    // older step's value where no change was decided, and is then not used)
    const float a_own = d.a_own[p], a_chg = d.at[p];
    if (change != 0) {
      // cancelled by a lower-id vehicle changing into the same lane less than
      // (vehicle length + s0) away, the longer of the two lengths with vehicle types;
      // such vehicles sit in lanes tgt-1 and tgt+1
      const int tgt = lane + change;
      const float len_self = TYPES ? veh_len<true>(d, vid) : d.vlen;
      const float thr = d.vlen + P.s0;
      bool cancel = false;
      for (int src = tgt - 1; src <= tgt + 1 && !cancel; src += 2) {
        if (src < 0 || src >= L.lanes) continue;
        const int gs = L.lane_base + src;
        const int q0 = d.lane_start[gs], q1 = d.lane_start[gs + 1];
        for (int q = q0; q < q1 && !cancel; q++) {
          int iq = d.intent[q];
          if (iq == 0 || src + iq != tgt || d.B.vid[q] >= vid) continue;
          const float thr_q = TYPES ? fmaxf(len_self, veh_len<true>(d, d.B.vid[q])) + P.s0 : thr;
          if (fabsf(d.B.x[q] - x) < thr_q) cancel = true;
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
    TapeRec* rec = nullptr;
    if (TAPE) {
      rec = tape_slot(d, t, vid);
      if (change) {
        const TapeForm cf = d.tform[vid];
        rec->lead = cf.lead;
        rec->kind = cf.kind;
        rec->s = cf.s;
        rec->vl = cf.vl;
      }
      rec->link = e;
      rec->v = v;
      rec->a = acc;
      rec->branch = (v + acc * d.dt >= 0.0f) ? kBrNormal : kBrStop;
      rec->crossed = 0;
      rec->valid = 1;
    }
    const bool hold = (fl & kFlagHolder) != 0;
    int nl = lane + change, nlink = e, ncur = cur, nnxt = nxt;
    int nmv = -1;   // movement class after a crossing (else unchanged)
    float nx = x1, nv = v1;
    bool crossed = false;
    if (x1 >= L.len) {
      if (nxt < 0) {
        d.A.link[p] = -1;
        if (rec) rec->branch = kBrArrive;
        if (OUT && d.tt_sum) note_exit(d, vid, e, t);
        d.status[vid] = kArrived;
        d.arr_step[vid] = (int32_t)t;
        atomicAdd(&d.ctl->n_arr, 1);
        continue;
      }
      const LinkRec Ln = d.links[nxt];
      const int m = lane < Ln.lanes - 1 ? lane : Ln.lanes - 1;
      const int gt = Ln.lane_base + m;
      const bool won = (fl & kFlagCand) && d.best[gt] == epoch_key(t, rr_rank(L, t), lane);
      if (won) {
        const int off = d.roff[vid], len = d.rlen[vid];
        ncur = d.loop ? (cur + 1) % len : cur + 1;
        int k2 = ncur + 1;
        nnxt = k2 < len ? d.routes[off + k2] : (d.loop ? d.routes[off + k2 % len] : -1);
        nlink = nxt;
        nl = m;
        nx = x1 - L.len;
        crossed = true;
        nmv = move_class(d, nxt, nnxt);
        if (rec) rec->crossed = 1;
        if (OUT && d.tt_sum) {
          note_exit(d, vid, e, t);
          d.enter[vid] = t;
        }
      } else {
        nx = L.len;
        nv = 0.0f;
        if (rec) rec->branch = kBrClamp;
      }
    }
    if (hold) d.holder[L.to] = crossed ? -1 : vid;
    // a lane outside the link can only come from a step whose own-lane pass was cut
    // short by a wait that ran out (stale decisions): the vehicle is dropped and the
    // step reports it
    if (!crossed && (unsigned)nl >= L.lanes) {
      set_err(d, kErrLane, vid);
      d.A.link[p] = -1;
      continue;
    }
    // lane count for the next occupancy rebuild
    const int gb = crossed ? d.links[nlink].lane_base : L.lane_base;
    const int gn = gb + nl;
    d.A.gid[p] = gn;
    d.aidx[p] = count_in_lane(d, gn);
    d.A.mv[p] = nmv >= 0 ? (uint8_t)nmv : d.B.mv[p];
    d.adec[p] = (int8_t)change;
    d.A.x[p] = nx;
    d.A.v[p] = nv;
    d.A.vid[p] = vid;
    d.A.link[p] = nlink;
    d.A.nxt[p] = nnxt;
    d.A.cur[p] = ncur;
    d.A.lane[p] = nl;
  }
}


// Move and departures touch disjoint slots of buffer A (departures append after the
// sorted vehicles) and read only state of step t, so they share one launch.
template <bool TAPE, bool OUT, bool TYPES>
__global__ void k_move_insert(Dev d) {
  griddep_wait();
  if (step_timed_out(d)) return;
  ph_move<TAPE, OUT, TYPES>(d);
  if (d.n_qlinks > 0) ph_insert<OUT, TYPES>(d);
}

__global__ void k_finish(Dev d) {
  griddep_wait();
  if (step_timed_out(d)) return;
  ph_finish(d);
}


// ------------------------------------------------------------------ launch sequence
// Launch with programmatic stream serialization (the kernel starts with griddep_wait),
// which hides part of the launch gap between the kernels of a step.
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), int grid, int block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

void launch_kernel(int k, const Dev& d, int grid, cudaStream_t s);
void launch_count(const Dev& d, int grid, cudaStream_t s);

// Occupancy of the current state without stepping: rebuild B from the lane counts,
// then count buffer A again so that the next step finds its counts.
void launch_occupancy(const Dev& d, int grid, cudaStream_t s) {
  for (int k = kKScanSum; k <= kKRank; k++) launch_kernel(k, d, grid, s);
  launch_count(d, grid, s);
}

// Kernels of one step, in launch order (names reported by the timed step).  The
// lane counts the scan starts from are made by the previous step's chunk kernel (or by
// k_count after a state is loaded).  With the adjoint's tape on, "front" and "chunk"
// are the plain-load own-lane, decision and move kernels that write the tape.
const char* const kKernelNames[kNumKernels] = {"scan_sum", "scan_fin", "scatter", "rank", "front", "chunk",
                                               "finish"};

void launch_front(const Dev& d, cudaStream_t s);
void launch_chunk(const Dev& d, cudaStream_t s);

bool kernel_enabled(int k, const Dev& d, bool has_stop) {
  (void)k;
  (void)d;
  (void)has_stop;
  return true;
}

void launch_kernel(int k, const Dev& d, int grid, cudaStream_t s) {
  const int nb = scan_blocks(d.n_lanes);
  switch (k) {
    case kKScanSum: k_scan_sum<<<nb, kScanThreads, 0, s>>>(d); break;
    case kKScanFin: launch_pdl(k_scan_fin, nb, kScanThreads, s, d); break;
    case kKScatter: launch_pdl(k_scatter, grid, 256, s, d); break;
    case kKRank:
      if (d.rank_long) {
        launch_pdl(k_rank<true>, grid, 256, s, d);
        launch_pdl(k_rank_long, grid, 256, s, d);
      } else {
        launch_pdl(k_rank<false>, grid, 256, s, d);
      }
      break;
    case kKFront:
      // the per-edge sample (when enabled) reads the sorted state of step t; its time
      // is counted with the fronts'
      if (d.acc_u) launch_pdl(k_edge_sample, grid, 256, s, d);
      if (d.tape) launch_pdl(k_own<true, false>, grid, 256, s, d);
      else launch_front(d, s);
      break;
    case kKChunk:
      if (d.tape) {
        launch_pdl(k_decide<true, false>, grid, 256, s, d);
        launch_pdl(k_move_insert<true, false, false>, grid, 256, s, d);
      } else {
        launch_chunk(d, s);
      }
      break;
    case kKFinish: launch_pdl(k_finish, 1, 1, s, d); break;
    default: break;
  }
}

// lane counts of buffer A (after a state is loaded, or to restore them)
void launch_count(const Dev& d, int grid, cudaStream_t s) { launch_pdl(k_count, grid, 256, s, d); }

void launch_step(const Dev& d, int grid, bool has_stop, cudaStream_t s) {
  for (int k = 0; k < kNumKernels; k++)
    if (kernel_enabled(k, d, has_stop)) launch_kernel(k, d, grid, s);
}

// The same step with an event after every kernel: per-kernel device time (ms)
// accumulated into kernel_ms over n steps.
cudaError_t launch_steps_timed(const Dev& d, int grid, bool has_stop, cudaStream_t s, int n, float* kernel_ms) {
  cudaEvent_t ev[kNumKernels + 1];
  for (int k = 0; k <= kNumKernels; k++) {
    cudaError_t e = cudaEventCreate(&ev[k]);
    if (e != cudaSuccess) return e;
  }
  for (int k = 0; k < kNumKernels; k++) kernel_ms[k] = 0.0f;
  cudaError_t err = cudaSuccess;
  for (int it = 0; it < n && err == cudaSuccess; it++) {
    cudaEventRecord(ev[0], s);
    for (int k = 0; k < kNumKernels; k++) {
      if (kernel_enabled(k, d, has_stop)) launch_kernel(k, d, grid, s);
      cudaEventRecord(ev[k + 1], s);
    }
    err = cudaEventSynchronize(ev[kNumKernels]);
    for (int k = 0; k < kNumKernels && err == cudaSuccess; k++) {
      float ms = 0.0f;
      err = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
      kernel_ms[k] += ms;
    }
  }
  for (int k = 0; k <= kNumKernels; k++) cudaEventDestroy(ev[k]);
  return err;
}

// ------------------------------------------------------------------ state I/O kernels
__global__ void k_state_out(Dev d, uint8_t* status, int32_t* link, int32_t* lane, int32_t* cursor, float* x,
                            float* v, int32_t* ins, int32_t* arr, int8_t* dec) {
  // decisions of trips on the road are written per slot by k_state_out_active
  GRID_STRIDE(i, d.n_trips) {
    if (status) status[i] = d.status[i];
    if (link) link[i] = -1;
    if (lane) lane[i] = 0;
    if (cursor) cursor[i] = 0;
    if (x) x[i] = 0.0f;
    if (v) v[i] = 0.0f;
    if (ins) ins[i] = d.ins_step[i];
    if (arr) arr[i] = d.arr_step[i];
    if (dec) dec[i] = 0;
  }
}

__global__ void k_state_out_active(Dev d, int32_t* link, int32_t* lane, int32_t* cursor, float* x, float* v,
                                   int8_t* dec) {
  const int nA = d.ctl->nA;
  GRID_STRIDE(s, nA) {
    int e = d.A.link[s];
    if (e < 0) continue;
    int i = d.A.vid[s];
    if (link) link[i] = e;
    if (lane) lane[i] = d.A.lane[s];
    if (cursor) cursor[i] = d.A.cur[s];
    if (x) x[i] = d.A.x[s];
    if (v) v[i] = d.A.v[s];
    if (dec) dec[i] = d.adec[s];
  }
}

void launch_state_out(const Dev& d, int grid, cudaStream_t s, uint8_t* status, int32_t* link, int32_t* lane,
                      int32_t* cursor, float* x, float* v, int32_t* ins, int32_t* arr, int8_t* dec) {
  k_state_out<<<grid, 256, 0, s>>>(d, status, link, lane, cursor, x, v, ins, arr, dec);
  k_state_out_active<<<grid, 256, 0, s>>>(d, link, lane, cursor, x, v, dec);
}

// Validate a state given by vid: every active trip sits on route[cursor], in a lane
// of that link, with 0 <= x <= length and v >= 0.  Counts the violations.
__global__ void k_state_check(Dev d, const uint8_t* status, const int32_t* link, const int32_t* lane,
                              const int32_t* cursor, const float* x, const float* v, int* bad) {
  GRID_STRIDE(i, d.n_trips) {
    if (status[i] > kArrived) { atomicAdd(bad, 1); continue; }
    if (status[i] != kActive) continue;
    const int k = cursor[i], e = link[i];
    bool ok = k >= 0 && k < d.rlen[i] && e >= 0 && e < d.n_links && d.routes[d.roff[i] + k] == e;
    ok = ok && lane[i] >= 0 && lane[i] < d.links[e].lanes && x[i] >= 0.0f && x[i] <= d.links[e].len &&
         v[i] >= 0.0f;
    if (!ok) atomicAdd(bad, 1);
  }
}

void launch_state_check(const Dev& d, int grid, cudaStream_t s, const uint8_t* status, const int32_t* link,
                        const int32_t* lane, const int32_t* cursor, const float* x, const float* v, int* bad) {
  k_state_check<<<grid, 256, 0, s>>>(d, status, link, lane, cursor, x, v, bad);
}

// Load a state (by vid) into buffer A: active trips are packed into slots by an
// atomic counter (slot order is irrelevant: the next occupancy rebuild sorts).
__global__ void k_state_in(Dev d, const uint8_t* status, const int32_t* link, const int32_t* lane,
                           const int32_t* cursor, const float* x, const float* v) {
  GRID_STRIDE(i, d.n_trips) {
    d.status[i] = status[i];
    d.ins_step[i] = status[i] == kActive ? 0 : -1;
    d.arr_step[i] = -1;
    if (status[i] != kActive) continue;
    int slot = atomicAdd(&d.ctl->nA, 1);
    int off = d.roff[i], len = d.rlen[i];
    int k = cursor[i];
    int k2 = k + 1;
    d.A.x[slot] = x[i] + 0.0f;
    d.A.v[slot] = v[i];
    d.A.vid[slot] = i;
    d.A.link[slot] = link[i];
    d.A.lane[slot] = lane[i];
    d.A.cur[slot] = k;
    const int nx = k2 < len ? d.routes[off + k2] : (d.loop ? d.routes[off + k2 % len] : -1);
    d.A.nxt[slot] = nx;
    d.A.mv[slot] = (uint8_t)move_class(d, link[i], nx);
    d.adec[slot] = 0;
  }
}

void launch_state_in(const Dev& d, int grid, cudaStream_t s, const uint8_t* status, const int32_t* link,
                     const int32_t* lane, const int32_t* cursor, const float* x, const float* v) {
  k_state_in<<<grid, 256, 0, s>>>(d, status, link, lane, cursor, x, v);
}

// Trips by status at the current step: active, waiting (pending and due: departure step
// < t) and pending (not yet due), reduced per warp, one atomic per warp and class.
__global__ void k_status_counts(Dev d, unsigned long long* counts) {
  const long long t = d.ctl->t;
  const int n = d.n_trips;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += gridDim.x * blockDim.x) {
    const int i = base + (threadIdx.x & 31);
    int cls = -1;
    if (i < n) {
      const uint8_t s = d.status[i];
      if (s == kActive) cls = 0;
      else if (s == kPending) cls = (long long)d.depart[i] < t ? 1 : 2;
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const unsigned m = __ballot_sync(0xffffffffu, cls == k);
      if ((threadIdx.x & 31) == 0 && m) atomicAdd(&counts[k], (unsigned long long)__popc(m));
    }
  }
}

void launch_status_counts(const Dev& d, int grid, cudaStream_t s, unsigned long long* counts) {
  k_status_counts<<<grid, 256, 0, s>>>(d, counts);
}

__global__ void k_occ_out(Dev d, int32_t* sorted_vid) {
  const int nB = d.ctl->nB;
  GRID_STRIDE(p, nB) sorted_vid[p] = d.B.vid[p];
}

void launch_occ_out(const Dev& d, int grid, cudaStream_t s, int32_t* sorted_vid) {
  k_occ_out<<<grid, 256, 0, s>>>(d, sorted_vid);
}

}  // namespace gbt
