// Internal device data layout and per-vehicle model functions of libgbtraffic.
//
// Model (Waddell et al., Sec. 6): Intelligent Driver Model car following (Eq. 7),
// ballistic position update over dt (Sec. 6.3.2 gives dt = 0.5 s), mandatory /
// discretionary lane changes with gap acceptance (Sec. 6.3.2), stop and signal
// control (Sec. 6.3.2), per-lane ordered occupancy replacing the "traffic atlas"
// (Sec. 6.3.3).  Every binary32 expression below is written in the one fixed
// operation order of the model specification; the library is compiled with
// -fmad=false so no multiply-add is ever fused, which keeps results bit-identical
// to any IEEE implementation of the same order.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gbt {

constexpr int kCtrlNone = 0, kCtrlStop = 1, kCtrlSignal = 2;
constexpr int kPending = 0, kActive = 1, kArrived = 2;
constexpr int kTurnThrough = 0, kTurnLeft = 1, kTurnRight = 2, kTurnEnd = 3;

// Default bound of a device-side wait (grid barrier, tile copy), in SM cycles: about a
// second at GB300 clocks.
constexpr long long kDefaultWaitCycles = 2000000000LL;

// error word bits (device -> host)
constexpr int kErrLane = 1, kErrLink = 2, kErrSlot = 4, kErrRoute = 8, kErrUnreach = 16,
              kErrRouteCap = 32, kErrQueue = 64, kErrTimeout = 128;

// Grid barrier of the persistent step kernel (one per handle, in device memory).
struct GridSync {
  alignas(128) unsigned count;   // arrivals (atomics)
  alignas(128) unsigned gen;     // generation (polled): a line of its own
};

// Per-link record, 32 bytes: everything a vehicle step needs about its link and
// the node at its end, in one aligned load.
struct __align__(16) LinkRec {
  float len;           // link length, m
  float v0;            // IDM desired speed on this link, m/s
  int32_t lane_base;   // global id of lane 0
  int32_t to;          // head node
  uint8_t lanes, cls, ctrl, ew;   // lanes; parameter class; control of head node; approach is east-west
  uint8_t in_index, n_in;         // rank among the head node's in-links (ascending id), in-degree
  uint16_t sig_cyc;               // signal cycle, ds
  int32_t sig_off;                // signal offset, ds
  uint16_t sig_grn;               // north-south green, ds
  uint16_t pad;
};
static_assert(sizeof(LinkRec) == 32, "LinkRec must be 32 bytes");

struct ClassPar {      // IDM parameters of one link class
  float a, sab2, T, s0;   // sab2 = 2 * sqrt(a * b)
};

// Structure-of-arrays vehicle state, one entry per slot.
struct VehBuf {
  float* x;
  float* v;
  int32_t* vid;
  int32_t* link;   // -1: slot empty (vehicle arrived)
  int32_t* nxt;    // next link of the route, -1 on the last link
  int32_t* cur;    // index of the current link in the route
  int32_t* lane;
  int32_t* gid;    // global lane id (lane_base of the link + lane)
  uint8_t* mv;     // movement class of link -> nxt (kTurn*, kTurnEnd on the last link)
};

// Rearmost vehicle of a lane, written by the occupancy rebuild for every occupied
// lane; `tag` is the rebuild's epoch, so a lane whose tag is stale is empty.
struct __align__(16) RearRec {
  float x, v;
  int32_t vid;
  uint32_t tag;
};

// Front (last sorted position) of a lane, written by the occupancy rebuild for every
// occupied lane: what the lane-front kernel needs of it.
struct __align__(16) FrontRec {
  float x, v;
  int32_t vid, nxt;
};

// State after crossing of a lane front that bids for admission (written by the lane-front
// kernel for bidding fronts only; used when the bid wins): position on the next link,
// speed, target lane id, route cursor, the link after, movement class, lane.
struct __align__(16) CrossRec {
  float nx, nv;
  int32_t gt, ncur, nnxt;
  uint8_t nmv, m, pad0, pad1;
  int32_t pad[2];
};

// A chunk of the fused step kernel: sorted positions [c0, c1) (whole links), the links
// of its first and last vehicle and the lane ids [g_lo, g_hi) of those links.
struct __align__(16) ChunkInfo {
  int32_t c0, c1, e_lo, e_hi, g_lo, g_hi, pad0, pad1;
};

struct Ctl {
  long long t;
  int nA;          // slots filled in the unsorted buffer A
  int nB;          // vehicles in the sorted buffer B (active at step start)
  unsigned occ_epoch;               // occupancy rebuilds so far (tag of the rear records)
  int err, err_info;
  int active_last;
  unsigned long long veh_steps, departed, arrived;
  unsigned long long lc_evals;      // lane-change decisions evaluated, summed over steps
  unsigned long long route_cursor;  // bump allocator of the route store
  long long tape_t0;                // first step of the segment being taped
  double loss;                      // calibration loss accumulator
  long long samp_k0;                // first edge-sample index since the outputs were cleared
  unsigned long long gap_num, gap_den;  // measured-cost gap accumulators
  // counters bumped by atomics during a step, in a cache line of their own so that the
  // step kernels' reads of t, nB and the epoch do not queue behind them
  alignas(128) int n_ins;
  int n_arr;
  int n_elig;      // lane-change candidates listed this step
  int chunk_next;  // next chunk of the fused step kernel to take
  int n_long;      // long lane segments listed by the lane-start scan
  int n_big;       // chunks beyond the chunk kernel's staging capacity (lane-front phase)
};

// Forms of Eq. 7 an acceleration can come from (adjoint tape).
constexpr uint8_t kFormNone = 0, kFormLead = 1, kFormFree = 2, kFormStop = 3, kFormNext = 4;
// How a move ended.
constexpr uint8_t kBrNormal = 0, kBrStop = 1, kBrClamp = 2, kBrArrive = 3;

// One taped vehicle-step (32 bytes): leader, link, the gap / speeds / acceleration
// that entered Eq. 7 and the ballistic update, and the discrete outcome.
struct __align__(16) TapeRec {
  int32_t lead;
  int32_t link;
  float s, v, vl, a;
  uint8_t kind, branch, crossed, valid;
  int32_t pad;
};
static_assert(sizeof(TapeRec) == 32, "TapeRec must be 32 bytes");

// The form chosen for a lane change (per trip, rewritten each step).
struct TapeForm {
  int32_t lead;
  float s, vl;
  uint8_t kind, pad0, pad1, pad2;
};

struct Dev {
  // network
  const LinkRec* links;
  const int32_t* lfrom;
  const int32_t* node_x;
  const int32_t* node_y;
  const ClassPar* cls;
  const float* cls_b;            // comfortable deceleration b per class (adjoint)
  const uint8_t* cls_v0_param;   // 1 when the class sets v0 (else v0 = link speed limit)
  const float* tau;      // mandatory-switch table [256]
  int n_links, n_nodes, n_lanes, n_trips, n_cls;
  // parameters
  float dt, hdt2, vlen, s_min, zone, mp, mathr, mbsafe, mbias, lam, stop_acq;
  int dt_ds, loop;
  // trips
  const int32_t* depart;
  const int32_t* roff;
  const int32_t* rlen;
  const int32_t* routes;
  const unsigned long long* hseed;
  uint8_t* status;
  int32_t* ins_step;
  int32_t* arr_step;
  int8_t* adec;    // lane-change decision of the last step, per slot of buffer A
  // vehicle state: A = unsorted next state, B = sorted current state
  VehBuf A, B;
  // per-slot / per-lane scratch
  int32_t* aidx;
  float* tx;
  int32_t* tvid;
  int32_t* tsrc;
  int32_t* tg;
  int32_t* cnt;
  int32_t* lane_start;
  int32_t* bsum;
  unsigned long long* best;   // per lane: epoch-tagged admission key
  float* a_own;
  float* xo;
  float* at;
  int8_t* intent;
  uint8_t* flags;
  RearRec* rear;              // per lane: rearmost vehicle (current epoch only)
  FrontRec* fr;               // per lane: front vehicle (occupied lanes of this step only)
  const int32_t* lane_link;   // per lane: its link
  CrossRec* cr;               // per lane: the bidding front's state after crossing
  ChunkInfo* chunks;          // chunks of the fused step kernel (this step's)
  int32_t* long_list;         // lanes with long segments (sorted by a block each)
  ChunkInfo* big_chunks;       // chunks beyond the chunk kernel's staging capacity
  int32_t* elig;              // sorted positions of this step's lane-change candidates
  TapeRec* tape;              // adjoint tape of the current segment (nullptr: not taping)
  TapeForm* tform;            // lane-change forms of the current step (taping only)
  // per node
  int32_t* holder;
  unsigned long long* acq;
  // measured outputs (nullptr when off): fuel and CO per trip (Eq. 8-9); link
  // traversal times (Sec. 6.3.1); per-edge samples every samp_every steps averaged
  // over windows of samp_per samples (Sec. 6.4)
  double2* emis;                   // per trip: (fuel mL, CO g), one 16-byte record
  int32_t* enter;                  // per trip: step it entered its current link, -1 unknown
  unsigned long long* tt_sum;      // per link: summed traversal steps
  int32_t* tt_n;                   // per link: traversals
  double* acc_u;                   // per link: window sums of utilisation and speed
  double* acc_s;
  double* out_u;                   // [samp_max][n_links] window means
  double* out_s;
  int32_t* out_n;                  // [samp_max] samples in each finished window
  int samp_every, samp_per, samp_max;
  // vehicle types (Sec. 6.3.5; vtype == nullptr: one vehicle class of length vlen):
  // per trip a type, per (class, type) the Eq. 7 parameters, per type length and
  // maximum speed
  const uint8_t* vtype;
  const ClassPar* cls_ty;          // [class * n_vty + type]
  const float* vty_len;
  const float* vty_vmax;
  float vlen_max;                  // longest vehicle length (vlen without types)
  int n_vty;
  // departure queues
  const int32_t* qlinks;
  int n_qlinks;
  const int32_t* q_end;
  int32_t* q_head;
  const int32_t* q_items;
  Ctl* ctl;
  int chunk_split;                 // oversized chunks go to the big-chunk launch
  int rank_long;                   // long lane segments go to k_rank_long
  int front_grid[2];               // blocks of the lane-front kernel (without / with types)
  int chunk_grid[8];               // blocks of the chunk kernel (plain, outputs, types, both), then of
                                   // the big-chunk kernel (same order)
  long long wait_limit;            // SM cycles a staging wait of the chunk kernel may take
};

// Trip-planning work description (one shortest-path tree per distinct origin).
struct RouteDev {
  int nn, nl;
  const int32_t* out_start;
  const int32_t* out_link;
  const int32_t* in_start;
  const int32_t* in_link;
  const int32_t* lfrom;
  const int32_t* lto;
  const int32_t* cost;
  const int32_t* origins;
  int n_origins;
  const int32_t* otrip_start;   // per node: trips with this origin
  const int32_t* otrip_list;
  const int32_t* dest;
  unsigned long long* dist;     // [n_cta][nn]
  int32_t* qflag;
  int32_t* fflag;
  int32_t* qa;
  int32_t* qb;
  int32_t* fa;
  int32_t* fb;
  unsigned* cta_epoch;
  int32_t* cta_round;
  int32_t* roff;
  int32_t* rlen;
  int32_t* routes;
  unsigned long long cap;
  unsigned* flow;               // all-or-nothing mode: trips per link instead of stored routes
  int* work;
  int delta;
  Ctl* ctl;
};

void launch_route(const RouteDev& R, int n_cta, cudaStream_t s);

// kernels of one step, in launch order
enum { kKScanSum, kKScanFin, kKScatter, kKRank, kKFront, kKChunk, kKFinish, kNumKernels };
extern const char* const kKernelNames[kNumKernels];

constexpr uint8_t kFlagFront = 1, kFlagHolder = 2, kFlagCand = 4;

// spare elements at the end of every per-slot array (tiled bulk copies may read up to
// one tile of 256 + 4 elements past the last vehicle)
constexpr int kSlotPad = 512;

// ---------------------------------------------------------------- model functions

// Eq. 7 (IDM): a [1 - (v/v0)^4 - (s*/s)^2], s* = s0 + max(0, vT + v dv / (2 sqrt(ab))),
// dv = v - v_lead, gap floored at s_min; without a leader the interaction term is 0.
__host__ __device__ __forceinline__ float idm_acc(const ClassPar& P, float v0, float s_min, float s,
                                                  float v, float vl, bool has_leader) {
  float r = v / v0;
  float r2 = r * r;
  float r4 = r2 * r2;
  float q2 = 0.0f;
  if (has_leader) {
    float dv = v - vl;
    float t1 = v * P.T;
    float t2 = (v * dv) / P.sab2;
    float dyn = t1 + t2;
    float ss = P.s0 + fmaxf(0.0f, dyn);
    float se = fmaxf(s, s_min);
    float q = ss / se;
    q2 = q * q;
  }
  return P.a * ((1.0f - r4) - q2);
}

// Ballistic update: v' = v + a dt; x' = x + (v dt + a dt^2/2) unless the vehicle stops
// within the step, then x' = x - v^2 / (2a), v' = 0.
__host__ __device__ __forceinline__ void ballistic(float x, float v, float acc, float dt, float hdt2,
                                                   float& xo, float& vo) {
  float vn = v + acc * dt;
  if (vn >= 0.0f) {
    float d1 = v * dt;
    float d2 = acc * hdt2;
    xo = x + (d1 + d2);
    vo = vn;
  } else {
    float den = 2.0f * acc;
    float dx = -((v * v) / den);
    xo = x + dx;
    vo = 0.0f;
  }
}

// SplitMix64 (Steele, Lea & Flood 2014): golden-ratio increment, then its finaliser.
__host__ __device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Index into the mandatory-switch table: top 8 bits of SplitMix64 of
// (seed ^ vid << 32) ^ hop.  hseed = seed ^ (vid << 32).
__host__ __device__ __forceinline__ unsigned mand_index(unsigned long long hseed, int hop) {
  return (unsigned)(splitmix64(hseed ^ (unsigned long long)(unsigned)hop) >> 56);
}

// Reroute subset of round r (Sec. 6.3.1): the trip is in it when the top 16 bits of
// SplitMix64 of hseed ^ (2^31 | r) fall below fraction_q16 (1/65536 units).  Bit 31
// separates these draws from the mandatory-switch ones (hop < 2^31).
__host__ __device__ __forceinline__ bool reroute_selected(unsigned long long hseed, unsigned round,
                                                          unsigned fraction_q16) {
  const unsigned long long lo = 0x80000000ULL | (unsigned long long)(round & 0x7FFFFFFFu);
  return (unsigned)(splitmix64(hseed ^ lo) >> 48) < fraction_q16;
}

// Eq. 9, fuel rate (mL/s) at speed v (m/s), acceleration a (m/s^2): idle rate plus
// 0.072 mL/kJ times the tractive power (drag, inertia, extra engine drag 0.79296 a^2 v
// when accelerating), the power taken as 0 when negative (the engine idles).  binary32,
// terms accumulated left to right.
__device__ __forceinline__ float fuel_rate(float v, float a) {
  const float v2 = v * v;
  float pw = 0.269f * v + 0.0171f * v2;
  pw = pw + 0.000672f * (v2 * v);
  pw = pw + (1.680f * a) * v;
  if (a > 0.0f) pw = pw + ((0.79296f * a) * a) * v;
  return 0.666f + 0.072f * (pw > 0.0f ? pw : 0.0f);
}

// Eq. 8, CO emission rate (g/s); the equation's speed is in miles per hour.
__device__ __forceinline__ float co_rate(float v) {
  const float mph = v / 0.44704f;
  const float dm = mph - 50.0f;
  return (-0.064f + 0.0056f * mph) + 0.00026f * (dm * dm);
}

// Movement class of a -> b -> c from integer node positions.
__host__ __device__ __forceinline__ int turn_class(long long ax, long long ay, long long bx, long long by,
                                                   long long cx, long long cy) {
  long long ux = bx - ax, uy = by - ay, wx = cx - bx, wy = cy - by;
  long long cr = ux * wy - uy * wx;
  long long dot = ux * wx + uy * wy;
  long long acr = cr < 0 ? -cr : cr;
  if (dot > acr) return kTurnThrough;
  return cr < 0 ? kTurnRight : kTurnLeft;
}

// Movement class of e -> e2 (kTurnEnd when the route ends on e).
__device__ __forceinline__ int move_class(const Dev& d, int e, int e2) {
  if (e2 < 0) return kTurnEnd;
  int a = d.lfrom[e], b = d.lfrom[e2];   // head of e == tail of e2
  int c = d.links[e2].to;
  return turn_class(d.node_x[a], d.node_y[a], d.node_x[b], d.node_y[b], d.node_x[c], d.node_y[c]);
}

// Lanes allowed for a movement of class mc on a link of `lanes` lanes: right turns from
// lane 0, left turns (and U-turns) from the leftmost lane, through from any; all lanes
// at the route's end.
__host__ __device__ __forceinline__ int lane_mask(int mc, int lanes) {
  if (mc == kTurnRight) return 1;
  if (mc == kTurnLeft) return 1 << (lanes - 1);
  return (1 << lanes) - 1;
}

__device__ __forceinline__ int move_mask(const Dev& d, int e, int lanes, int e2) {
  return lane_mask(move_class(d, e, e2), lanes);
}

// Step time is kept below 2^31 / dt_ds (checked by sim_step), so the phase and
// round-robin arithmetic is exact in 32 bits.
__device__ __forceinline__ int rr_rank(const LinkRec& L, int t) {
  const int n = L.n_in;
  return (L.in_index + n - t % n) % n;
}

__device__ __forceinline__ bool signal_green(const LinkRec& L, int tds) {
  int p = (tds - L.sig_off) % (int)L.sig_cyc;
  if (p < 0) p += L.sig_cyc;
  const bool ns = p < (int)L.sig_grn;
  return L.ew ? !ns : ns;
}

// Epoch-tagged 64-bit priority key: entries of step t compare below all entries of
// earlier steps, so per-step minima need no reset.  Lower 32 bits: (rank, lane).
__device__ __forceinline__ unsigned long long epoch_key(int t, int rr, int lane) {
  unsigned hi = 0xFFFFFFFEu - (unsigned)t;
  return ((unsigned long long)hi << 32) | (unsigned long long)((rr << 8) | lane);
}
__device__ __forceinline__ bool epoch_current(unsigned long long k, int t) {
  return (unsigned)(k >> 32) == 0xFFFFFFFEu - (unsigned)t;
}

__device__ __forceinline__ void set_err(const Dev& d, int bit, int info) {
  atomicOr(&d.ctl->err, bit);
  atomicExch(&d.ctl->err_info, info);
}

}  // namespace gbt
