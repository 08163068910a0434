/* CPU oracle of the traffic microsimulation hot path.
 *
 * TEST INFRASTRUCTURE ONLY: plain, slow, obviously-correct C used to check the
 * CUDA library.  It shares no code with the library.  The product path never
 * loads it.
 *
 * Source: Waddell et al., "Architecture for Modular Microsimulation of Real
 * Estate Markets and Transportation", Sec. 6 ("Traffic microsimulation model"):
 *   - trip planning by shortest paths under estimated link times (Sec. 6.3.1),
 *     one tree per origin shared by its trips (Sec. 6 "Simulation scale");
 *   - free-flow link time t0 = d / s (Eq. 4), here in integer deciseconds;
 *   - time step dt = 0.5 s (Sec. 6.3.2);
 *   - car following by the Intelligent Driver Model (Eq. 7);
 *   - mandatory / discretionary lane changes with an exponential switch toward
 *     mandatory near the exit, plus lead/lag gap acceptance (Sec. 6.3.2);
 *   - stop signs (one vehicle at a time) and fixed-time traffic lights (Sec. 6.3.2).
 * Where the paper is silent a reading is taken; each reading is stated at the
 * function that applies it.
 *
 * Floating point: every kinematic quantity is IEEE binary32 evaluated in the
 * written operation order; build with -ffp-contract=off (no fused multiply-add).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OK 0
#define EINV -1
#define ENOMEM_ -2
#define EUNREACH -4
#define ESTATE -6

#define CTRL_NONE 0
#define CTRL_STOP 1
#define CTRL_SIGNAL 2

#define ST_PENDING 0
#define ST_ACTIVE 1
#define ST_ARRIVED 2

#define TURN_THROUGH 0
#define TURN_LEFT 1
#define TURN_RIGHT 2

struct orc_sim {
  /* network */
  int nn, nl;
  int64_t *px, *py;
  uint8_t *ctrl;
  int32_t *off, *cyc, *grn;
  int32_t *lf, *lt;
  float *len, *spd;
  int *lanes, *cls;
  float *v0l;               /* car-following desired speed per link */
  int *lane_base, n_lanes;  /* global lane id = lane_base[link] + lane */
  int *in_start, *in_list;  /* in-links of each node, ascending link id */
  int *in_index, *n_in;
  /* parameters */
  float dt, hdt2, len_v, s_min;
  int dt_ds;
  int ncls;
  float *pv0, *pT, *pa, *pb, *ps0, *psab;
  float mp, mathr, mbsafe, mbias, lam, stop_acq;
  uint64_t seed;
  int cost_mode, loop;
  float tau[256];
  /* demand and routes */
  int nt;
  int32_t *orig, *dest, *dep;
  int32_t *roff, *rl;
  int routed;
  /* vehicle state, by trip id */
  uint8_t *st;
  int32_t *link, *lane, *cur;
  float *x, *v;
  int32_t *ins_step, *arr_step;
  int8_t *dec;
  int32_t *holder;          /* per node: trip holding a stop-controlled node, or -1 */
  /* departure queues: trips by first link, ordered (depart_step, trip id) */
  int32_t *q_start, *q_items, *q_head;
  int64_t t, departed, arrived, veh_steps, active_last;
  int64_t lc_evals;    /* lane-change decisions evaluated, summed over steps */
  /* adjoint tape: per step, one record per vehicle advanced (see orc_adjoint) */
  int recording;
  struct orc_rec* rec;
  int64_t rec_n, rec_cap;
  int64_t* rec_step;        /* [steps + 1] start of each step's records */
  int rec_steps, rec_step_cap;
  /* start state of the taped run (for the replay) */
  uint8_t* st0;
  int32_t* cur0;
  float *x0, *v0s;
  double* tgt;              /* targets of the taped run */
  int tgt_nobs, tgt_every;
  /* measured outputs, each enabled by orc_set_outputs: per-trip fuel and CO (Eq. 8-9),
   * per-link traversal times (Sec. 6.3.1), per-edge samples (Sec. 6.4) */
  uint32_t out_flags;
  double *fuel, *co;        /* [nt] */
  int32_t* enter;           /* [nt] step at which the trip entered its current link, -1 unknown */
  int64_t* tt_sum;          /* [nl] summed traversal steps */
  int32_t* tt_n;            /* [nl] traversals */
  int samp_every, samp_per, samp_max;
  int64_t samp_k0;          /* first sample index taken since the outputs were cleared */
  double *acc_u, *acc_s, *out_u, *out_s;
  int32_t* out_n;
  /* vehicle types (Sec. 6.3.5: trucks differ in size, acceleration and maximum speed);
   * ttype == NULL: every vehicle is of the single class of orc_params */
  int n_vty;
  float *vty_len, *vty_ascale, *vty_vmax;
  uint8_t* ttype;
};

/* One taped vehicle-step: the form of Eq. 7 used (kind/lead/s/vl, see acc_form
 * below), the speed and acceleration, the link, and how the move ended. */
#define BR_NORMAL 0
#define BR_STOP 1
#define BR_CLAMP 2
#define BR_ARRIVE 3
typedef struct orc_rec {
  int32_t vid, lead, link;
  float s, v, vl, a;
  uint8_t kind, branch, crossed;
} orc_rec;

/* ------------------------------------------------------------------ helpers */
static void* xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz ? sz : 1); }
static size_t zsz(int n) { return n > 0 ? (size_t)n : 1; }

/* Intelligent Driver Model, Eq. 7, as in Treiber et al. (2000) which Sec. 6 cites:
 *   dv/dt = a [ 1 - (v/v0)^4 - (s*(v,dv)/s)^2 ],  s* = s0 + max(0, v T + v dv / (2 sqrt(a b))).
 * Reading: the printed "v dv / 2 sqrt(ab)" is the quotient v dv / (2 sqrt(ab)); the
 * dynamic part of s* is floored at 0; dv = v - v_lead; the gap s is floored at s_min.
 * No leader: the interaction term is 0.  Fixed binary32 operation order. */
static float idm_acc(float a, float sab, float T, float s0, float v0, float s_min,
                     float s, float v, float vl, int has_leader) {
  float r = v / v0;
  float r2 = r * r;
  float r4 = r2 * r2;
  float q2 = 0.0f;
  if (has_leader) {
    float dv = v - vl;
    float t1 = v * T;
    float t2 = (v * dv) / (2.0f * sab);
    float dyn = t1 + t2;
    float ss = s0 + fmaxf(0.0f, dyn);
    float se = fmaxf(s, s_min);
    float q = ss / se;
    q2 = q * q;
  }
  return a * ((1.0f - r4) - q2);
}

float orc_idm(float a, float b, float T, float s0, float v0, float s_min,
              float s, float v, float v_lead, int has_leader) {
  float sab = sqrtf(a * b);
  return idm_acc(a, sab, T, s0, v0, s_min, s, v, v_lead, has_leader);
}

/* Position/speed update over one step (Sec. 6.3.2 gives dt only).  Reading: the
 * ballistic scheme of Treiber & Kanagaraj (2015): v' = v + a dt; if v' >= 0 then
 * x' = x + v dt + a dt^2/2, otherwise the vehicle stops inside the step:
 * x' = x - v^2 / (2 a), v' = 0. */
static void ballistic(float x, float v, float acc, float dt, float hdt2, float* xo, float* vo) {
  float vn = v + acc * dt;
  if (vn >= 0.0f) {
    float d1 = v * dt;
    float d2 = acc * hdt2;
    *xo = x + (d1 + d2);
    *vo = vn;
  } else {
    float den = 2.0f * acc;
    float dx = -((v * v) / den);
    *xo = x + dx;
    *vo = 0.0f;
  }
}

void orc_ballistic(float x, float v, float acc, float dt, float* x_out, float* v_out) {
  float hdt2 = (0.5f * dt) * dt;
  ballistic(x, v, acc, dt, hdt2, x_out, v_out);
}

/* Free-flow link time, Eq. 4 (t0 = d / s seconds), as integer deciseconds rounded
 * half up and at least 1.  Mode 1 uses the routing weight of Sec. 6.3.1,
 * sqrt(lanes) * length / speed, in the same units. */
int32_t orc_link_cost(float length_m, float speed_mps, int lanes, int mode) {
  double d = (double)length_m, s = (double)speed_mps;
  double t = (mode == 1) ? ((10.0 * sqrt((double)lanes)) * d) / s : (10.0 * d) / s;
  double c = floor(t + 0.5);
  if (c < 1.0) c = 1.0;
  if (c > 2.0e9) c = 2.0e9;
  return (int32_t)c;
}

/* SplitMix64 (Steele, Lea & Flood 2014): one increment and the finaliser. */
static uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* SplitMix64 of seed ^ (vid << 32 | hop); the top 8 bits index the
 * mandatory-switch table. */
uint32_t orc_mand_index(uint64_t seed, int32_t vid, int32_t hop) {
  uint64_t z = splitmix64(seed ^ ((((uint64_t)(uint32_t)vid) << 32) | (uint64_t)(uint32_t)hop));
  return (uint32_t)(z >> 56);
}

/* Sec. 6.3.1 decaying reroute: trip vid is in the subset of round r when the top 16
 * bits of SplitMix64 of seed ^ (vid << 32 | 2^31 | r) are below fraction_q16 (a
 * fraction in 1/65536 units; 65536 takes every trip).  Bit 31 keeps these draws
 * apart from the mandatory-switch draws, whose hop index stays below 2^31. */
int orc_reroute_selected(uint64_t seed, int32_t vid, uint32_t round, uint32_t fraction_q16) {
  uint64_t lo = 0x80000000ULL | (uint64_t)(round & 0x7FFFFFFFu);
  uint64_t z = splitmix64(seed ^ ((((uint64_t)(uint32_t)vid) << 32) | lo));
  return (uint32_t)(z >> 48) < fraction_q16;
}

/* Eq. 8: CO emission rate in g/s.  The equation takes the speed in miles per hour
 * (1 mph = 0.44704 m/s); terms added left to right in binary32. */
float orc_co_rate(float v) {
  float vm = v / 0.44704f;
  float d = vm - 50.0f;
  return (-0.064f + 0.0056f * vm) + 0.00026f * (d * d);
}

/* Eq. 9: fuel rate in mL/s at speed v (m/s) and acceleration a (m/s^2), with the
 * extra engine drag P_ea = 0.79296 a^2 v for a > 0.  The bracket is the tractive
 * power (kW) of Akcelik's power-based model, which falls back to the idle rate
 * (0.666 mL/s) when that power is not positive; terms added left to right. */
float orc_fuel_rate(float v, float a) {
  float p = 0.269f * v + 0.0171f * (v * v);
  p = p + 0.000672f * ((v * v) * v);
  p = p + (1.680f * a) * v;
  if (a > 0.0f) p = p + ((0.79296f * a) * a) * v;
  if (!(p > 0.0f)) p = 0.0f;
  return 0.666f + 0.072f * p;
}

/* Mandatory switch (Sec. 6.3.2): a vehicle on the wrong lane turns mandatory with
 * probability exp(-(d/lambda)^2) at remaining distance d.  With one uniform draw u
 * per (vehicle, link), it is mandatory once d <= lambda sqrt(-ln u).  u is quantised
 * to 256 levels (k + 0.5) / 256 so that the threshold is a table lookup. */
float orc_mand_tau(int k) {
  return (float)sqrt(-log(((double)k + 0.5) / 256.0));
}

/* Turn class of the movement a->b->c from integer node positions (exact int64):
 * through when the heading changes by less than 45 degrees, else left (counter-
 * clockwise, and U-turns) or right. */
int orc_turn(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy) {
  int64_t d1x = bx - ax, d1y = by - ay, d2x = cx - bx, d2y = cy - by;
  int64_t cr = d1x * d2y - d1y * d2x;
  int64_t dot = d1x * d2x + d1y * d2y;
  int64_t acr = cr < 0 ? -cr : cr;
  if (dot > acr) return TURN_THROUGH;
  if (cr < 0) return TURN_RIGHT;
  return TURN_LEFT;
}

/* Fixed-time two-phase signal (Sec. 6.3.2 "traffic lights"; the grid workload
 * fixes 30 s green / 30 s red): phase time p = (t dt - offset) mod cycle in
 * deciseconds; north-south approaches are green for p < green, east-west otherwise. */
int orc_signal_green(int64_t t, int32_t dt_ds, int32_t offset, int32_t cycle, int32_t green, int ew) {
  int64_t p = (t * (int64_t)dt_ds - (int64_t)offset) % (int64_t)cycle;
  if (p < 0) p += cycle;
  int ns_green = p < (int64_t)green;
  return ew ? !ns_green : ns_green;
}

/* Dijkstra with a binary heap (the plain definition of single-source shortest
 * paths; Sec. 6 "Simulation scale" builds one tree per source). */
typedef struct { int64_t d; int32_t v; } hent;
static void heap_push(hent* h, int64_t* n, hent e) {
  int64_t i = (*n)++;
  h[i] = e;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h[p].d <= h[i].d) break;
    hent tmp = h[p]; h[p] = h[i]; h[i] = tmp;
    i = p;
  }
}
static hent heap_pop(hent* h, int64_t* n) {
  hent top = h[0];
  h[0] = h[--(*n)];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < *n && h[l].d < h[m].d) m = l;
    if (r < *n && h[r].d < h[m].d) m = r;
    if (m == i) break;
    hent tmp = h[m]; h[m] = h[i]; h[i] = tmp;
    i = m;
  }
  return top;
}

static int dijkstra(int nn, const int* out_start, const int* out_list, const int32_t* lt,
                    const int32_t* cost, int origin, int64_t* dist, hent* heap) {
  for (int i = 0; i < nn; i++) dist[i] = INT64_MAX;
  int64_t hn = 0;
  dist[origin] = 0;
  heap_push(heap, &hn, (hent){0, origin});
  while (hn > 0) {
    hent e = heap_pop(heap, &hn);
    if (e.d != dist[e.v]) continue;
    for (int k = out_start[e.v]; k < out_start[e.v + 1]; k++) {
      int l = out_list[k];
      int64_t nd = e.d + cost[l];
      if (nd < dist[lt[l]]) {
        dist[lt[l]] = nd;
        heap_push(heap, &hn, (hent){nd, lt[l]});
      }
    }
  }
  return OK;
}

static void build_csr(int n, int m, const int32_t* key, int* start, int* list) {
  for (int i = 0; i <= n; i++) start[i] = 0;
  for (int e = 0; e < m; e++) start[key[e] + 1]++;
  for (int i = 0; i < n; i++) start[i + 1] += start[i];
  int* fill = (int*)xcalloc(zsz(n), sizeof(int));
  for (int e = 0; e < m; e++) list[start[key[e]] + fill[key[e]]++] = e; /* ascending link id */
  free(fill);
}

int orc_sssp(int32_t n_nodes, int32_t n_links, const int32_t* from, const int32_t* to,
             const int32_t* cost, int32_t origin, int64_t* dist) {
  if (n_nodes <= 0 || origin < 0 || origin >= n_nodes) return EINV;
  int* os = (int*)xcalloc((size_t)n_nodes + 1, sizeof(int));
  int* ol = (int*)xcalloc((size_t)n_links, sizeof(int));
  hent* heap = (hent*)xcalloc((size_t)n_links + 1, sizeof(hent));
  build_csr(n_nodes, n_links, from, os, ol);
  dijkstra(n_nodes, os, ol, to, cost, origin, dist, heap);
  free(os); free(ol); free(heap);
  return OK;
}

/* ------------------------------------------------------------------ create */
int orc_create(const orc_network* N, const orc_demand* D, const orc_params* P, orc_sim** out) {
  if (!N || !D || !P || !out) return EINV;
  if (N->n_nodes <= 0 || N->n_links <= 0 || D->n_trips < 0) return EINV;
  if (P->n_class <= 0 || !(P->dt > 0.0f)) return EINV;
  int dt_ds = (int)lrintf(P->dt * 10.0f);
  if (dt_ds <= 0 || fabsf((float)dt_ds - P->dt * 10.0f) > 1e-3f) return EINV;
  orc_sim* S = (orc_sim*)xcalloc(1, sizeof(orc_sim));
  int nn = N->n_nodes, nl = N->n_links;
  S->nn = nn; S->nl = nl;
  S->px = (int64_t*)xcalloc(nn, 8); S->py = (int64_t*)xcalloc(nn, 8);
  S->ctrl = (uint8_t*)xcalloc(nn, 1);
  S->off = (int32_t*)xcalloc(nn, 4); S->cyc = (int32_t*)xcalloc(nn, 4); S->grn = (int32_t*)xcalloc(nn, 4);
  for (int i = 0; i < nn; i++) {
    S->px[i] = N->node_x_dm[i]; S->py[i] = N->node_y_dm[i];
    S->ctrl[i] = N->node_control[i];
    S->off[i] = N->signal_offset_ds[i]; S->cyc[i] = N->signal_cycle_ds[i]; S->grn[i] = N->signal_green_ds[i];
    if (S->ctrl[i] > 2 || (S->ctrl[i] == CTRL_SIGNAL && S->cyc[i] <= 0)) { orc_destroy(S); return EINV; }
  }
  S->lf = (int32_t*)xcalloc(nl, 4); S->lt = (int32_t*)xcalloc(nl, 4);
  S->len = (float*)xcalloc(nl, 4); S->spd = (float*)xcalloc(nl, 4);
  S->lanes = (int*)xcalloc(nl, sizeof(int)); S->cls = (int*)xcalloc(nl, sizeof(int));
  S->v0l = (float*)xcalloc(nl, 4);
  S->lane_base = (int*)xcalloc(nl + 1, sizeof(int));
  S->ncls = P->n_class;
  S->pv0 = (float*)xcalloc(S->ncls, 4); S->pT = (float*)xcalloc(S->ncls, 4);
  S->pa = (float*)xcalloc(S->ncls, 4); S->pb = (float*)xcalloc(S->ncls, 4);
  S->ps0 = (float*)xcalloc(S->ncls, 4); S->psab = (float*)xcalloc(S->ncls, 4);
  for (int c = 0; c < S->ncls; c++) {
    S->pv0[c] = P->v0[c]; S->pT[c] = P->T[c]; S->pa[c] = P->a[c]; S->pb[c] = P->b[c]; S->ps0[c] = P->s0[c];
    if (!(S->pa[c] > 0.0f) || !(S->pb[c] > 0.0f) || !(S->pT[c] >= 0.0f) || !(S->ps0[c] >= 0.0f)) { orc_destroy(S); return EINV; }
    S->psab[c] = sqrtf(S->pa[c] * S->pb[c]);
  }
  int nlanes = 0;
  for (int e = 0; e < nl; e++) {
    S->lf[e] = N->link_from[e]; S->lt[e] = N->link_to[e];
    S->len[e] = N->link_length_m[e]; S->spd[e] = N->link_speed_mps[e];
    S->lanes[e] = N->link_lanes[e]; S->cls[e] = N->link_class[e];
    if (S->lf[e] < 0 || S->lf[e] >= nn || S->lt[e] < 0 || S->lt[e] >= nn || S->lanes[e] < 1 || S->lanes[e] > 8 ||
        !(S->len[e] > 0.0f) || !(S->spd[e] > 0.0f) || S->cls[e] >= S->ncls) { orc_destroy(S); return EINV; }
    S->v0l[e] = S->pv0[S->cls[e]] > 0.0f ? S->pv0[S->cls[e]] : S->spd[e];
    S->lane_base[e] = nlanes;
    nlanes += S->lanes[e];
  }
  S->lane_base[nl] = nlanes;
  S->n_lanes = nlanes;
  S->in_start = (int*)xcalloc(nn + 1, sizeof(int)); S->in_list = (int*)xcalloc(nl, sizeof(int));
  build_csr(nn, nl, S->lt, S->in_start, S->in_list);
  S->in_index = (int*)xcalloc(nl, sizeof(int)); S->n_in = (int*)xcalloc(nn, sizeof(int));
  for (int n = 0; n < nn; n++) {
    S->n_in[n] = S->in_start[n + 1] - S->in_start[n];
    for (int k = S->in_start[n]; k < S->in_start[n + 1]; k++) S->in_index[S->in_list[k]] = k - S->in_start[n];
  }
  S->dt = P->dt; S->hdt2 = (0.5f * P->dt) * P->dt; S->dt_ds = dt_ds;
  S->len_v = P->veh_len; S->s_min = P->s_min;
  S->mp = P->mobil_p; S->mathr = P->mobil_athr; S->mbsafe = P->mobil_bsafe; S->mbias = P->mobil_bias_right;
  S->lam = P->lambda_mand; S->stop_acq = P->stop_acquire_m;
  S->seed = P->seed; S->cost_mode = P->cost_mode; S->loop = P->loop_routes;
  for (int k = 0; k < 256; k++) S->tau[k] = orc_mand_tau(k);
  int nt = D->n_trips;
  S->nt = nt;
  S->orig = (int32_t*)xcalloc(nt, 4); S->dest = (int32_t*)xcalloc(nt, 4); S->dep = (int32_t*)xcalloc(nt, 4);
  for (int i = 0; i < nt; i++) {
    S->orig[i] = D->origin[i]; S->dest[i] = D->dest[i]; S->dep[i] = D->depart_step[i];
    if (S->orig[i] < 0 || S->orig[i] >= nn || S->dest[i] < 0 || S->dest[i] >= nn) { orc_destroy(S); return EINV; }
  }
  S->roff = (int32_t*)xcalloc(nt + 1, 4);
  S->st = (uint8_t*)xcalloc(nt, 1);
  S->link = (int32_t*)xcalloc(nt, 4); S->lane = (int32_t*)xcalloc(nt, 4); S->cur = (int32_t*)xcalloc(nt, 4);
  S->x = (float*)xcalloc(nt, 4); S->v = (float*)xcalloc(nt, 4);
  S->ins_step = (int32_t*)xcalloc(nt, 4); S->arr_step = (int32_t*)xcalloc(nt, 4);
  S->dec = (int8_t*)xcalloc(nt, 1);
  S->holder = (int32_t*)xcalloc(nn, 4);
  for (int i = 0; i < nn; i++) S->holder[i] = -1;
  for (int i = 0; i < nt; i++) { S->link[i] = -1; S->ins_step[i] = -1; S->arr_step[i] = -1; }
  S->q_start = (int32_t*)xcalloc(nl + 1, 4); S->q_items = (int32_t*)xcalloc(nt, 4); S->q_head = (int32_t*)xcalloc(nl, 4);
  *out = S;
  return OK;
}

void orc_destroy(orc_sim* S) {
  if (!S) return;
  void* ptrs[] = {S->px, S->py, S->ctrl, S->off, S->cyc, S->grn, S->lf, S->lt, S->len, S->spd, S->lanes, S->cls,
                  S->v0l, S->lane_base, S->in_start, S->in_list, S->in_index, S->n_in, S->pv0, S->pT, S->pa,
                  S->pb, S->ps0, S->psab, S->orig, S->dest, S->dep, S->roff, S->rl, S->st, S->link, S->lane,
                  S->cur, S->x, S->v, S->ins_step, S->arr_step, S->dec, S->holder, S->q_start, S->q_items,
                  S->q_head, S->rec, S->rec_step, S->st0, S->cur0, S->x0, S->v0s, S->tgt,
                  S->fuel, S->co, S->enter, S->tt_sum, S->tt_n, S->acc_u, S->acc_s, S->out_u,
                  S->out_s, S->out_n, S->vty_len, S->vty_ascale, S->vty_vmax, S->ttype};
  for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); i++) free(ptrs[i]);
  free(S);
}

/* ------------------------------------------------------------------ routes */
static int route_len(const orc_sim* S, int i) { return S->roff[i + 1] - S->roff[i]; }

/* Next link after hop k of trip i, or -1 at the end of a non-looping route. */
static int next_link(const orc_sim* S, int i, int k) {
  int n = route_len(S, i);
  if (k + 1 < n) return S->rl[S->roff[i] + k + 1];
  if (S->loop) return S->rl[S->roff[i] + (k + 1) % n];
  return -1;
}

/* Departure queues: per first link, trips not yet on the road ordered by
 * (depart_step, trip id). */
static const int32_t* g_dep;
static int cmp_trip(const void* A, const void* B) {
  int a = *(const int*)A, b = *(const int*)B;
  if (g_dep[a] != g_dep[b]) return g_dep[a] < g_dep[b] ? -1 : 1;
  return a < b ? -1 : (a > b);
}

static void rebuild_queues(orc_sim* S) {
  int nl = S->nl, nt = S->nt;
  for (int e = 0; e <= nl; e++) S->q_start[e] = 0;
  for (int i = 0; i < nt; i++)
    if (S->st[i] == ST_PENDING) S->q_start[S->rl[S->roff[i]] + 1]++;
  for (int e = 0; e < nl; e++) S->q_start[e + 1] += S->q_start[e];
  int* fill = (int*)xcalloc(nl, sizeof(int));
  for (int i = 0; i < nt; i++)
    if (S->st[i] == ST_PENDING) { int e = S->rl[S->roff[i]]; S->q_items[S->q_start[e] + fill[e]++] = i; }
  free(fill);
  g_dep = S->dep;
  for (int e = 0; e < nl; e++) {
    qsort(S->q_items + S->q_start[e], (size_t)(S->q_start[e + 1] - S->q_start[e]), sizeof(int32_t), cmp_trip);
    S->q_head[e] = S->q_start[e];
  }
}

/* Outputs restart with the run: totals at zero, no link entered yet, sampling
 * windows empty from the next sampling instant on. */
static void clear_outputs(orc_sim* S) {
  if (S->fuel)
    for (int i = 0; i < S->nt; i++) { S->fuel[i] = 0.0; S->co[i] = 0.0; }
  if (S->enter) {
    for (int i = 0; i < S->nt; i++) S->enter[i] = -1;
    for (int e = 0; e < S->nl; e++) { S->tt_sum[e] = 0; S->tt_n[e] = 0; }
  }
  if (S->acc_u) {
    for (int e = 0; e < S->nl; e++) { S->acc_u[e] = 0.0; S->acc_s[e] = 0.0; }
    for (int64_t q = 0; q < (int64_t)S->samp_max * S->nl; q++) { S->out_u[q] = 0.0; S->out_s[q] = 0.0; }
    for (int w = 0; w < S->samp_max; w++) S->out_n[w] = 0;
    S->samp_k0 = (S->t + S->samp_every - 1) / S->samp_every;
  }
}

static void reset_state(orc_sim* S) {
  for (int i = 0; i < S->nt; i++) {
    S->st[i] = ST_PENDING; S->link[i] = -1; S->lane[i] = 0; S->cur[i] = 0; S->x[i] = 0.0f; S->v[i] = 0.0f;
    S->ins_step[i] = -1; S->arr_step[i] = -1; S->dec[i] = 0;
  }
  for (int n = 0; n < S->nn; n++) S->holder[n] = -1;
  S->t = 0; S->departed = 0; S->arrived = 0; S->veh_steps = 0; S->active_last = 0; S->lc_evals = 0;
  clear_outputs(S);
}

/* Trip planning (Sec. 6.3.1): every trip follows a shortest path from its origin
 * node to its destination node; one shortest-path tree per distinct origin is
 * shared by all trips from it (Sec. 6 "Simulation scale").  Ties between equally
 * short paths: walking back from the destination, take the lowest-id in-link
 * (u -> v) with dist[u] + c = dist[v].  With sel, only the trips with sel[i] set get
 * a new path; the others keep theirs. */
static int route_core(orc_sim* S, const int32_t* cost_in, const uint8_t* sel) {
  int nn = S->nn, nl = S->nl, nt = S->nt;
  int32_t* cost = (int32_t*)xcalloc(nl, 4);
  for (int e = 0; e < nl; e++) {
    cost[e] = cost_in ? cost_in[e] : orc_link_cost(S->len[e], S->spd[e], S->lanes[e], S->cost_mode);
    if (cost[e] < 1) { free(cost); return EINV; }
  }
  for (int i = 0; i < nt; i++) if (S->orig[i] == S->dest[i]) { free(cost); return EINV; }
  int* os = (int*)xcalloc(nn + 1, sizeof(int));
  int* ol = (int*)xcalloc(nl, sizeof(int));
  build_csr(nn, nl, S->lf, os, ol);
  /* trips grouped by origin */
  int* ts = (int*)xcalloc(nn + 1, sizeof(int));
  int* tl = (int*)xcalloc(nt, sizeof(int));
  build_csr(nn, nt, S->orig, ts, tl);
  int64_t* dist = (int64_t*)xcalloc(nn, 8);
  hent* heap = (hent*)xcalloc(nl + 1, sizeof(hent));
  int32_t* rlen = (int32_t*)xcalloc(nt, 4);
  int32_t** paths = (int32_t**)xcalloc(nt, sizeof(int32_t*));
  int32_t* tmp = (int32_t*)xcalloc(nn + 1, 4);
  int rc = OK;
  for (int i = 0; i < nt; i++) {
    if (sel && !sel[i]) {   /* kept route */
      rlen[i] = route_len(S, i);
      paths[i] = (int32_t*)xcalloc(rlen[i], 4);
      memcpy(paths[i], S->rl + S->roff[i], (size_t)rlen[i] * 4);
    }
  }
  for (int o = 0; o < nn && rc == OK; o++) {
    int any = 0;
    for (int k = ts[o]; k < ts[o + 1]; k++) if (!sel || sel[tl[k]]) any = 1;
    if (!any) continue;
    dijkstra(nn, os, ol, S->lt, cost, o, dist, heap);
    for (int k = ts[o]; k < ts[o + 1]; k++) {
      int i = tl[k];
      if (sel && !sel[i]) continue;
      int d = S->dest[i];
      if (dist[d] == INT64_MAX) { rc = EUNREACH; break; }
      int n = 0, v = d;
      while (v != o) {
        int pick = -1;
        for (int q = S->in_start[v]; q < S->in_start[v + 1]; q++) {
          int e = S->in_list[q];
          int u = S->lf[e];
          if (dist[u] != INT64_MAX && dist[u] + cost[e] == dist[v]) { pick = e; break; }
        }
        if (pick < 0) { rc = ESTATE; break; }
        tmp[n++] = pick;
        v = S->lf[pick];
      }
      if (rc != OK) break;
      rlen[i] = n;
      paths[i] = (int32_t*)xcalloc(n, 4);
      for (int j = 0; j < n; j++) paths[i][j] = tmp[n - 1 - j];
    }
  }
  if (rc == OK) {
    S->roff[0] = 0;
    for (int i = 0; i < nt; i++) S->roff[i + 1] = S->roff[i] + rlen[i];
    free(S->rl);
    S->rl = (int32_t*)xcalloc((size_t)S->roff[nt], 4);
    for (int i = 0; i < nt; i++) memcpy(S->rl + S->roff[i], paths[i], (size_t)rlen[i] * 4);
    S->routed = 1;
    reset_state(S);
    rebuild_queues(S);
  }
  for (int i = 0; i < nt; i++) free(paths[i]);
  free(paths); free(tmp); free(rlen); free(heap); free(dist); free(ts); free(tl); free(os); free(ol); free(cost);
  return rc;
}

int orc_route(orc_sim* S, const int32_t* cost_in) { return route_core(S, cost_in, NULL); }

/* Sec. 6.3.1: new shortest paths under cost for the subset of round `round` (see
 * orc_reroute_selected); the other trips keep their routes.  Restarts the run. */
int orc_reroute(orc_sim* S, const int32_t* cost, uint32_t fraction_q16, uint32_t round) {
  if (!S->routed) return ESTATE;
  if (!cost || fraction_q16 > 65536u) return EINV;
  uint8_t* sel = (uint8_t*)xcalloc(S->nt, 1);
  for (int i = 0; i < S->nt; i++) sel[i] = (uint8_t)orc_reroute_selected(S->seed, i, round, fraction_q16);
  int rc = route_core(S, cost, sel);
  free(sel);
  return rc;
}

int orc_set_routes(orc_sim* S, const int32_t* offsets, const int32_t* links) {
  int nt = S->nt;
  if (offsets[0] != 0) return EINV;
  for (int i = 0; i < nt; i++) {
    if (offsets[i + 1] <= offsets[i]) return EINV;
    for (int k = offsets[i]; k < offsets[i + 1]; k++) {
      if (links[k] < 0 || links[k] >= S->nl) return EINV;
      if (k > offsets[i] && S->lf[links[k]] != S->lt[links[k - 1]]) return EINV;
    }
    if (S->loop && S->lt[links[offsets[i + 1] - 1]] != S->lf[links[offsets[i]]]) return EINV;
  }
  for (int i = 0; i <= nt; i++) S->roff[i] = offsets[i];
  free(S->rl);
  S->rl = (int32_t*)xcalloc((size_t)offsets[nt], 4);
  memcpy(S->rl, links, (size_t)offsets[nt] * 4);
  S->routed = 1;
  reset_state(S);
  rebuild_queues(S);
  return OK;
}

int orc_route_size(const orc_sim* S, int64_t* n) { *n = S->routed ? S->roff[S->nt] : 0; return S->routed ? OK : ESTATE; }

int orc_read_routes(const orc_sim* S, int32_t* offsets, int32_t* links) {
  if (!S->routed) return ESTATE;
  memcpy(offsets, S->roff, (size_t)(S->nt + 1) * 4);
  memcpy(links, S->rl, (size_t)S->roff[S->nt] * 4);
  return OK;
}

int orc_write_state(orc_sim* S, const uint8_t* status, const int32_t* link, const int32_t* lane,
                    const int32_t* cursor, const float* x, const float* v) {
  if (!S->routed) return ESTATE;
  for (int i = 0; i < S->nt; i++) {
    if (status[i] > ST_ARRIVED) return EINV;
    if (status[i] == ST_ACTIVE) {
      int k = cursor[i];
      if (k < 0 || k >= route_len(S, i) || S->rl[S->roff[i] + k] != link[i]) return EINV;
      if (lane[i] < 0 || lane[i] >= S->lanes[link[i]]) return EINV;
      if (!(x[i] >= 0.0f) || !(x[i] <= S->len[link[i]]) || !(v[i] >= 0.0f)) return EINV;
    }
  }
  reset_state(S);
  for (int i = 0; i < S->nt; i++) {
    S->st[i] = status[i];
    if (status[i] == ST_ACTIVE) {
      S->link[i] = link[i]; S->lane[i] = lane[i]; S->cur[i] = cursor[i];
      S->x[i] = x[i] + 0.0f; S->v[i] = v[i]; S->ins_step[i] = 0;
    }
  }
  rebuild_queues(S);
  return OK;
}

/* ------------------------------------------------------------------ one step */
/* Per-lane occupancy, ordered by (position, trip id): the function of the paper's
 * "traffic atlas" (Sec. 6.3.3): the leader of a vehicle is the next vehicle in
 * its lane. */
static const float* g_x;
static int cmp_pos(const void* A, const void* B) {
  int a = *(const int*)A, b = *(const int*)B;
  if (g_x[a] != g_x[b]) return g_x[a] < g_x[b] ? -1 : 1;
  return a < b ? -1 : (a > b);
}

typedef struct {
  int* start;   /* [n_lanes + 1] */
  int* vids;    /* sorted by (lane, x, vid) */
  int* pos;     /* position of each active trip in vids */
  int n;
} occ_t;

static void build_occ(const orc_sim* S, occ_t* O) {
  int nlan = S->n_lanes;
  O->start = (int*)xcalloc(nlan + 1, sizeof(int));
  O->pos = (int*)xcalloc(S->nt, sizeof(int));
  int n = 0;
  for (int i = 0; i < S->nt; i++)
    if (S->st[i] == ST_ACTIVE) { O->start[S->lane_base[S->link[i]] + S->lane[i] + 1]++; n++; }
  for (int g = 0; g < nlan; g++) O->start[g + 1] += O->start[g];
  O->vids = (int*)xcalloc(n, sizeof(int));
  int* fill = (int*)xcalloc(nlan, sizeof(int));
  for (int i = 0; i < S->nt; i++)
    if (S->st[i] == ST_ACTIVE) { int g = S->lane_base[S->link[i]] + S->lane[i]; O->vids[O->start[g] + fill[g]++] = i; }
  free(fill);
  g_x = S->x;
  for (int g = 0; g < nlan; g++) qsort(O->vids + O->start[g], (size_t)(O->start[g + 1] - O->start[g]), sizeof(int), cmp_pos);
  for (int p = 0; p < n; p++) O->pos[O->vids[p]] = p;
  O->n = n;
}

static void free_occ(occ_t* O) { free(O->start); free(O->vids); free(O->pos); }

static int lane_id(const orc_sim* S, int e, int l) { return S->lane_base[e] + l; }

/* Lane mask of a movement (bit l set when lane l may make it).  Reading of
 * Sec. 6.3.2's "necessary change to reach an exit or right/left turn": on a
 * multi-lane link right turns leave from lane 0 (rightmost), left turns and
 * U-turns from the leftmost lane, through movements from any lane. */
static int move_mask(const orc_sim* S, int e, int e2) {
  int nl = S->lanes[e];
  int all = (1 << nl) - 1;
  if (e2 < 0) return all;
  int a = S->lf[e], b = S->lt[e], c = S->lt[e2];
  int tc = orc_turn(S->px[a], S->py[a], S->px[b], S->py[b], S->px[c], S->py[c]);
  if (tc == TURN_RIGHT) return 1;
  if (tc == TURN_LEFT) return 1 << (nl - 1);
  return all;
}

/* Phase group of an approach: east-west when the link runs more along x than y. */
static int approach_ew(const orc_sim* S, int e) {
  int64_t dx = S->px[S->lt[e]] - S->px[S->lf[e]];
  int64_t dy = S->py[S->lt[e]] - S->py[S->lf[e]];
  if (dx < 0) dx = -dx;
  if (dy < 0) dy = -dy;
  return dx >= dy;
}

/* Round-robin rank of an incoming link at step t (Sec. 6.3.2: "round robin logic"):
 * the link whose in-index equals t mod n_in ranks first. */
static int rr_rank(const orc_sim* S, int e, int64_t t) {
  int n = S->n_in[S->lt[e]];
  return (int)((S->in_index[e] + n - (int)(t % n)) % n);
}

/* Whether the stop line of link e is closed to vehicle i at step t: red light for
 * its approach, or a stop-controlled node held by another vehicle / not yet
 * acquired by i. */
static int stopline_closed(const orc_sim* S, int i, int e) {
  int n = S->lt[e];
  if (S->ctrl[n] == CTRL_SIGNAL)
    return !orc_signal_green(S->t, S->dt_ds, S->off[n], S->cyc[n], S->grn[n], approach_ew(S, e));
  if (S->ctrl[n] == CTRL_STOP) return S->holder[n] != i;
  return 0;
}

/* Length of trip i's vehicle. */
static float len_of(const orc_sim* S, int i) { return S->ttype ? S->vty_len[S->ttype[i]] : S->len_v; }

/* Eq. 7 parameters of trip i on link e: its link class's, with the acceleration a
 * scaled by its vehicle type and the desired speed capped at the type's maximum. */
static void vpar(const orc_sim* S, int e, int i, float* a, float* sab, float* v0) {
  int c = S->cls[e];
  if (S->ttype) {
    int ty = S->ttype[i];
    *a = S->pa[c] * S->vty_ascale[ty];
    *sab = sqrtf(*a * S->pb[c]);
    *v0 = fminf(S->v0l[e], S->vty_vmax[ty]);
  } else {
    *a = S->pa[c]; *sab = S->psab[c]; *v0 = S->v0l[e];
  }
}

/* Eq. 7 for trip i on link e: free road, or behind a leader at gap s with speed vl. */
static float acc_free(const orc_sim* S, int e, int i, float v) {
  int c = S->cls[e];
  float a, sab, v0;
  vpar(S, e, i, &a, &sab, &v0);
  return idm_acc(a, sab, S->pT[c], S->ps0[c], v0, S->s_min, 0.0f, v, 0.0f, 0);
}

static float acc_gap(const orc_sim* S, int e, int i, float s, float v, float vl) {
  int c = S->cls[e];
  float a, sab, v0;
  vpar(S, e, i, &a, &sab, &v0);
  return idm_acc(a, sab, S->pT[c], S->ps0[c], v0, S->s_min, s, v, vl, 1);
}

/* Which form of Eq. 7 produced an acceleration (for the adjoint's tape): kind
 * 1 = leader on the same link, 4 = leader across the link end, 2 = free road,
 * 3 = closed stop line; lead = leader trip id, s and vl = the gap and leader speed
 * that entered Eq. 7. */
#define FORM_NONE 0
#define FORM_LEAD 1
#define FORM_FREE 2
#define FORM_STOP 3
#define FORM_NEXT 4
typedef struct { int kind, lead; float s, vl; } accform;

static void set_form(accform* f, int kind, int lead, float s, float vl) {
  if (f) { f->kind = kind; f->lead = lead; f->s = s; f->vl = vl; }
}

/* Acceleration of vehicle j at (x, v) on link e, lane l when nothing is ahead of it
 * on e: the leader is the rearmost vehicle of the mapped lane of j's next link
 * (gap counted across the link end), and a closed stop line acts as a standing
 * obstacle; the smaller acceleration applies.  On the last link of a route the
 * road ahead is free. */
static float acc_front(const orc_sim* S, const occ_t* O, int j, int e, int l, float x, float v, accform* f) {
  int nx = next_link(S, j, S->cur[j]);
  if (nx < 0) { set_form(f, FORM_FREE, -1, 0.0f, 0.0f); return acc_free(S, e, j, v); }
  int m = l < S->lanes[nx] - 1 ? l : S->lanes[nx] - 1;
  int g = lane_id(S, nx, m);
  float a1;
  accform f1;
  if (O->start[g] < O->start[g + 1] && O->vids[O->start[g]] != j) {
    int r = O->vids[O->start[g]];
    float s = ((S->len[e] - x) + S->x[r]) - len_of(S, r);
    a1 = acc_gap(S, e, j, s, v, S->v[r]);
    f1 = (accform){FORM_NEXT, r, s, S->v[r]};
  } else {
    a1 = acc_free(S, e, j, v);
    f1 = (accform){FORM_FREE, -1, 0.0f, 0.0f};
  }
  if (stopline_closed(S, j, e)) {
    float s2 = S->len[e] - x;
    float a2 = acc_gap(S, e, j, s2, v, 0.0f);
    if (a2 < a1) { set_form(f, FORM_STOP, -1, s2, 0.0f); return a2; }
  }
  if (f) *f = f1;
  return a1;
}

static int leader_of(const orc_sim* S, const occ_t* O, int i) {
  int p = O->pos[i];
  int g = lane_id(S, S->link[i], S->lane[i]);
  return (p + 1 < O->start[g + 1]) ? O->vids[p + 1] : -1;
}
static int follower_of(const orc_sim* S, const occ_t* O, int i) {
  int p = O->pos[i];
  int g = lane_id(S, S->link[i], S->lane[i]);
  return (p > O->start[g]) ? O->vids[p - 1] : -1;
}

static int key_less(const orc_sim* S, int a, int b) {   /* (x, vid) order */
  if (S->x[a] != S->x[b]) return S->x[a] < S->x[b];
  return a < b;
}

/* Own-lane acceleration (Eq. 7 with the own-lane leader, else acc_front). */
static float acc_own(const orc_sim* S, const occ_t* O, int i, accform* f) {
  int L = leader_of(S, O, i);
  int e = S->link[i];
  if (L >= 0) {
    float s = (S->x[L] - S->x[i]) - len_of(S, L);
    set_form(f, FORM_LEAD, L, s, S->v[L]);
    return acc_gap(S, e, i, s, S->v[i], S->v[L]);
  }
  return acc_front(S, O, i, e, S->lane[i], S->x[i], S->v[i], f);
}

static orc_rec* rec_push(orc_sim* S) {
  if (S->rec_n == S->rec_cap) {
    S->rec_cap = S->rec_cap ? 2 * S->rec_cap : 65536;
    S->rec = (orc_rec*)realloc(S->rec, (size_t)S->rec_cap * sizeof(orc_rec));
  }
  orc_rec* r = &S->rec[S->rec_n++];
  memset(r, 0, sizeof(*r));
  return r;
}

static void rec_begin_step(orc_sim* S) {
  if (S->rec_steps + 2 > S->rec_step_cap) {
    S->rec_step_cap = S->rec_step_cap ? 2 * S->rec_step_cap : 1024;
    S->rec_step = (int64_t*)realloc(S->rec_step, (size_t)S->rec_step_cap * sizeof(int64_t));
  }
  S->rec_step[S->rec_steps++] = S->rec_n;
  S->rec_step[S->rec_steps] = S->rec_n;
}

/* Sec. 6.4 per-edge sample at step t (taken from the state at t, when t is a multiple
 * of samp_every): utilisation = vehicles on the edge / (length * lanes / (vehicle
 * length + s0)), speed = mean speed of those vehicles, summed in occupancy order (lane,
 * then position), or the free-flow speed of an empty edge.  Window w averages the
 * samples w*samp_per .. w*samp_per + samp_per - 1 that were taken; it is written when
 * its last sample is. */
static void edge_sample(orc_sim* S, const occ_t* O, int64_t t) {
  int64_t k = t / S->samp_every;
  int64_t w = k / S->samp_per, j = k % S->samp_per;
  int64_t first = w * S->samp_per > S->samp_k0 ? w * S->samp_per : S->samp_k0;
  for (int e = 0; e < S->nl; e++) {
    int g0 = S->lane_base[e], g1 = g0 + S->lanes[e];
    int n = O->start[g1] - O->start[g0];
    double sum = 0.0;
    for (int p = O->start[g0]; p < O->start[g1]; p++) sum += (double)S->v[O->vids[p]];
    double cap = ((double)S->len[e] * (double)S->lanes[e]) / ((double)S->len_v + (double)S->ps0[S->cls[e]]);
    double util = (double)n / cap;
    double spd = n > 0 ? sum / (double)n : (double)S->v0l[e];
    S->acc_u[e] += util;
    S->acc_s[e] += spd;
    if (j == S->samp_per - 1) {
      double cnt = (double)(k - first + 1);
      S->out_u[w * S->nl + e] = S->acc_u[e] / cnt;
      S->out_s[w * S->nl + e] = S->acc_s[e] / cnt;
      S->acc_u[e] = 0.0;
      S->acc_s[e] = 0.0;
    }
  }
  if (j == S->samp_per - 1) S->out_n[w] = (int32_t)(k - first + 1);
}

/* Sec. 6.3.1 measurement: a trip leaving link e at step t (into its next link, or
 * arriving) traversed it in t - enter steps, if it was seen entering it. */
static void record_exit(orc_sim* S, int i, int e, int64_t t) {
  if (S->enter[i] >= 0) { S->tt_sum[e] += t - S->enter[i]; S->tt_n[e] += 1; }
}

int orc_step(orc_sim* S, int32_t n_steps) {
  if (!S->routed) return ESTATE;
  if (n_steps < 0) return EINV;
  if (S->acc_u && n_steps > 0 && (S->t + n_steps - 1) / S->samp_every / S->samp_per >= S->samp_max) return EINV;
  int nt = S->nt;
  float* a_own = (float*)xcalloc(nt, 4);
  float* xo = (float*)xcalloc(nt, 4);
  float* vo = (float*)xcalloc(nt, 4);
  float* at = (float*)xcalloc(nt, 4);
  int8_t* intent = (int8_t*)xcalloc(nt, 1);
  int8_t* change = (int8_t*)xcalloc(nt, 1);
  uint8_t* cand = (uint8_t*)xcalloc(nt, 1);
  int* best = (int*)xcalloc(S->n_lanes, sizeof(int));
  uint8_t* nst = (uint8_t*)xcalloc(nt, 1);
  int32_t *nlink = (int32_t*)xcalloc(nt, 4), *nlane = (int32_t*)xcalloc(nt, 4), *ncur = (int32_t*)xcalloc(nt, 4);
  float *nx_ = (float*)xcalloc(nt, 4), *nv = (float*)xcalloc(nt, 4);
  accform* own_f = (accform*)xcalloc(nt, sizeof(accform));
  accform* tgt_f = (accform*)xcalloc(nt, sizeof(accform));

  for (int step = 0; step < n_steps; step++) {
    int64_t t = S->t;
    if (S->recording) rec_begin_step(S);
    occ_t O;
    build_occ(S, &O);
    S->veh_steps += O.n;
    S->active_last = O.n;
    if (S->acc_u && t % S->samp_every == 0) edge_sample(S, &O, t);

    /* stop signs (Sec. 6.3.2): one vehicle at a time.  A free stop-controlled node is
     * acquired by the front vehicle, within stop_acquire_m of the stop line, of the
     * incoming lane ranked first by (round-robin rank of its link, lane). */
    for (int n = 0; n < S->nn; n++) {
      if (S->ctrl[n] != CTRL_STOP || S->holder[n] >= 0) continue;
      int bk = 1 << 30, bv = -1;
      for (int q = S->in_start[n]; q < S->in_start[n + 1]; q++) {
        int e = S->in_list[q];
        for (int l = 0; l < S->lanes[e]; l++) {
          int g = lane_id(S, e, l);
          if (O.start[g] == O.start[g + 1]) continue;
          int j = O.vids[O.start[g + 1] - 1];
          if (next_link(S, j, S->cur[j]) < 0) continue;
          if (!((S->len[e] - S->x[j]) <= S->stop_acq)) continue;
          int key = rr_rank(S, e, t) * 256 + l;
          if (key < bk) { bk = key; bv = j; }
        }
      }
      S->holder[n] = bv;
    }

    /* own-lane acceleration and tentative move of every vehicle */
    for (int i = 0; i < nt; i++) {
      if (S->st[i] != ST_ACTIVE) continue;
      a_own[i] = acc_own(S, &O, i, S->recording ? &own_f[i] : NULL);
      ballistic(S->x[i], S->v[i], a_own[i], S->dt, S->hdt2, &xo[i], &vo[i]);
    }

    /* admission into the next link (Sec. 6.3.2 intersection control): the front
     * vehicle of a lane whose stop line is open and whose move reaches the link end
     * is a candidate if it lands behind the rearmost vehicle of its target lane; at
     * most one candidate enters each target lane per step, the one ranked first by
     * (round-robin rank of its link, lane). */
    for (int g = 0; g < S->n_lanes; g++) best[g] = 1 << 30;
    for (int i = 0; i < nt; i++) {
      cand[i] = 0;
      if (S->st[i] != ST_ACTIVE) continue;
      int e = S->link[i];
      if (leader_of(S, &O, i) >= 0) continue;
      int nx = next_link(S, i, S->cur[i]);
      if (nx < 0 || stopline_closed(S, i, e)) continue;
      if (!(xo[i] >= S->len[e])) continue;
      int m = S->lane[i] < S->lanes[nx] - 1 ? S->lane[i] : S->lanes[nx] - 1;
      int g = lane_id(S, nx, m);
      if (O.start[g] < O.start[g + 1] && O.vids[O.start[g]] != i) {
        int r = O.vids[O.start[g]];
        float land = xo[i] - S->len[e];
        float room = S->x[r] - len_of(S, r);
        if (!(land <= room)) continue;
      }
      cand[i] = 1;
      int key = rr_rank(S, e, t) * 256 + S->lane[i];
      if (key < best[g]) best[g] = key;
    }

    /* lane-change decisions (Sec. 6.3.2), from the state at t only.  Reading:
     * MOBIL (Kesting, Treiber & Helbing 2007) for the discretionary incentive and
     * its safety criterion for gap acceptance; mandatory when the vehicle is off
     * the lanes of its next movement and within its drawn switch distance. */
    for (int i = 0; i < nt; i++) {
      intent[i] = 0;
      if (S->st[i] != ST_ACTIVE) continue;
      int e = S->link[i];
      int nlan = S->lanes[e];
      if (nlan < 2) continue;
      float zone = 2.0f * S->len_v;
      if (!(S->x[i] >= zone && xo[i] < S->len[e] - zone)) continue;
      S->lc_evals++;
      int l = S->lane[i];
      int nx = next_link(S, i, S->cur[i]);
      int M = move_mask(S, e, nx);
      int dirs[2], nd = 0, mand = 0;
      if ((M >> l) & 1) {
        if (l + 1 < nlan && ((M >> (l + 1)) & 1)) dirs[nd++] = +1;
        if (l - 1 >= 0 && ((M >> (l - 1)) & 1)) dirs[nd++] = -1;
      } else {
        int ms = 0;
        while (!((M >> ms) & 1)) ms++;
        int d = ms > l ? +1 : -1;
        int ncross = ms > l ? ms - l : l - ms;
        float thr = (S->lam * (float)ncross) * S->tau[orc_mand_index(S->seed, i, S->cur[i])];
        float drem = S->len[e] - S->x[i];
        mand = drem <= thr;
        dirs[nd++] = d;
      }
      int chosen = 0;
      float chosen_inc = 0.0f, chosen_at = 0.0f;
      for (int k = 0; k < nd; k++) {
        int d = dirs[k];
        int l2 = l + d;
        int g2 = lane_id(S, e, l2);
        int Ln = -1, Fn = -1;
        for (int p = O.start[g2]; p < O.start[g2 + 1]; p++) {
          int j = O.vids[p];
          if (key_less(S, j, i)) Fn = j;
          else if (Ln < 0) Ln = j;
        }
        float ac;
        accform cf;
        if (Ln >= 0) {
          float sl = (S->x[Ln] - S->x[i]) - len_of(S, Ln);
          if (!(sl > 0.0f)) continue;
          ac = acc_gap(S, e, i, sl, S->v[i], S->v[Ln]);
          cf = (accform){FORM_LEAD, Ln, sl, S->v[Ln]};
        } else {
          ac = acc_front(S, &O, i, e, l2, S->x[i], S->v[i], &cf);
        }
        if (!(ac >= -S->mbsafe)) continue;
        float an = 0.0f;
        if (Fn >= 0) {
          float sg = (S->x[i] - S->x[Fn]) - len_of(S, i);
          if (!(sg > 0.0f)) continue;
          an = acc_gap(S, e, Fn, sg, S->v[Fn], S->v[i]);
          if (!(an >= -S->mbsafe)) continue;
        }
        if (mand) { chosen = d; chosen_at = ac; tgt_f[i] = cf; break; }
        float dc = ac - a_own[i];
        float dn = Fn >= 0 ? an - a_own[Fn] : 0.0f;
        float dn_o = 0.0f;
        int F = follower_of(S, &O, i);
        if (F >= 0) {
          int L = leader_of(S, &O, i);
          float ao = (L >= 0) ? acc_gap(S, e, F, (S->x[L] - S->x[F]) - len_of(S, L), S->v[F], S->v[L])
                              : acc_front(S, &O, F, e, l, S->x[F], S->v[F], NULL);
          dn_o = ao - a_own[F];
        }
        float inc = dc + S->mp * (dn + dn_o);
        if (d < 0) inc = inc + S->mbias;
        if (!(inc > S->mathr)) continue;
        if (chosen == 0 || inc > chosen_inc) { chosen = d; chosen_inc = inc; chosen_at = ac; tgt_f[i] = cf; }
      }
      intent[i] = (int8_t)chosen;
      at[i] = chosen_at;
    }

    /* simultaneous changes into one lane (paper silent): a change is cancelled when
     * another vehicle with a lower trip id changes into the same lane of the same
     * link less than (vehicle length + s0) away; with vehicle types, the longer of
     * the two lengths. */
    for (int i = 0; i < nt; i++) {
      change[i] = 0;
      if (S->st[i] != ST_ACTIVE || intent[i] == 0) continue;
      int e = S->link[i];
      int tgt = S->lane[i] + intent[i];
      float len_i = len_of(S, i);
      int cancel = 0;
      /* changers into lane tgt come from lanes tgt - 1 and tgt + 1 of the same link */
      for (int src = tgt - 1; src <= tgt + 1 && !cancel; src += 2) {
        if (src < 0 || src >= S->lanes[e]) continue;
        int g = lane_id(S, e, src);
        for (int p = O.start[g]; p < O.start[g + 1] && !cancel; p++) {
          int j = O.vids[p];
          if (j >= i || intent[j] == 0 || S->lane[j] + intent[j] != tgt) continue;
          float thr = fmaxf(len_i, len_of(S, j)) + S->ps0[S->cls[e]];
          if (fabsf(S->x[j] - S->x[i]) < thr) cancel = 1;
        }
      }
      if (!cancel) change[i] = intent[i];
    }

    /* move every vehicle; transitions, arrivals, and vehicles held at the stop line */
    int64_t arrivals = 0;
    for (int i = 0; i < nt; i++) {
      nst[i] = S->st[i]; nlink[i] = S->link[i]; nlane[i] = S->lane[i]; ncur[i] = S->cur[i];
      nx_[i] = S->x[i]; nv[i] = S->v[i];
      S->dec[i] = 0;
      if (S->st[i] != ST_ACTIVE) continue;
      int e = S->link[i];
      float acc = change[i] ? at[i] : a_own[i];
      float x1, v1;
      ballistic(S->x[i], S->v[i], acc, S->dt, S->hdt2, &x1, &v1);
      if (S->fuel) {
        /* Eq. 8-9 rates at the speed and acceleration of this step, times dt */
        S->fuel[i] += (double)(orc_fuel_rate(S->v[i], acc) * S->dt);
        S->co[i] += (double)(orc_co_rate(S->v[i]) * S->dt);
      }
      orc_rec* rr = NULL;
      if (S->recording) {
        rr = rec_push(S);
        accform fu = change[i] ? tgt_f[i] : own_f[i];
        rr->vid = i; rr->lead = fu.lead; rr->link = e; rr->kind = (uint8_t)fu.kind;
        rr->s = fu.s; rr->v = S->v[i]; rr->vl = fu.vl; rr->a = acc;
        rr->branch = (S->v[i] + acc * S->dt >= 0.0f) ? BR_NORMAL : BR_STOP;
        rr->crossed = 0;
      }
      int l1 = S->lane[i] + change[i];
      S->dec[i] = change[i];
      int node = S->lt[e];
      int was_holder = S->ctrl[node] == CTRL_STOP && S->holder[node] == i;
      if (x1 >= S->len[e]) {
        int nx = next_link(S, i, S->cur[i]);
        if (nx < 0) {
          nst[i] = ST_ARRIVED; nlink[i] = -1; nx_[i] = 0.0f; nv[i] = 0.0f;
          if (rr) rr->branch = BR_ARRIVE;
          if (S->enter) record_exit(S, i, e, t);
          S->arr_step[i] = (int32_t)t;
          arrivals++;
          continue;
        }
        int m = S->lane[i] < S->lanes[nx] - 1 ? S->lane[i] : S->lanes[nx] - 1;
        int g = lane_id(S, nx, m);
        int won = cand[i] && best[g] == rr_rank(S, e, t) * 256 + S->lane[i];
        if (won) {
          nlink[i] = nx; nlane[i] = m;
          int rlen = route_len(S, i);
          ncur[i] = S->loop ? (S->cur[i] + 1) % rlen : S->cur[i] + 1;
          nx_[i] = x1 - S->len[e]; nv[i] = v1;
          if (was_holder) S->holder[node] = -1;
          if (rr) rr->crossed = 1;
          if (S->enter) { record_exit(S, i, e, t); S->enter[i] = (int32_t)t; }
        } else {
          nlane[i] = l1; nx_[i] = S->len[e]; nv[i] = 0.0f;
          if (rr) rr->branch = BR_CLAMP;
        }
      } else {
        nlane[i] = l1; nx_[i] = x1; nv[i] = v1;
      }
    }

    /* departures (Sec. 6.2.2 OD and departure time): the head of each link's queue
     * of due trips enters at x = 0, v = 0 in the permitted lane with the largest rear
     * space (ties to the lowest lane) that received no vehicle from upstream in this
     * step, when that space is at least s0 + vehicle length. */
    int64_t ins = 0;
    for (int e = 0; e < S->nl; e++) {
      if (S->q_head[e] >= S->q_start[e + 1]) continue;
      int h = S->q_items[S->q_head[e]];
      if (S->dep[h] > t) continue;
      int rlen = route_len(S, h);
      int e2 = rlen >= 2 ? S->rl[S->roff[h] + 1] : (S->loop ? S->rl[S->roff[h]] : -1);
      int M = move_mask(S, e, e2);
      int bl = -1;
      float brs = 0.0f;
      for (int l = 0; l < S->lanes[e]; l++) {
        if (!((M >> l) & 1)) continue;
        int g = lane_id(S, e, l);
        if (best[g] != (1 << 30)) continue;
        float rs = (O.start[g] < O.start[g + 1]) ? S->x[O.vids[O.start[g]]] - len_of(S, O.vids[O.start[g]]) : INFINITY;
        if (bl < 0 || rs > brs) { bl = l; brs = rs; }
      }
      if (bl < 0) continue;
      float need = S->ps0[S->cls[e]] + len_of(S, h);
      if (!(brs >= need)) continue;
      nst[h] = ST_ACTIVE; nlink[h] = e; nlane[h] = bl; ncur[h] = 0; nx_[h] = 0.0f; nv[h] = 0.0f;
      S->ins_step[h] = (int32_t)t;
      if (S->enter) S->enter[h] = (int32_t)t;
      S->q_head[e]++;
      ins++;
    }

    memcpy(S->st, nst, (size_t)nt);
    memcpy(S->link, nlink, (size_t)nt * 4); memcpy(S->lane, nlane, (size_t)nt * 4);
    memcpy(S->cur, ncur, (size_t)nt * 4);
    memcpy(S->x, nx_, (size_t)nt * 4); memcpy(S->v, nv, (size_t)nt * 4);
    S->departed += ins;
    S->arrived += arrivals;
    S->t = t + 1;
    free_occ(&O);
  }
  free(a_own); free(xo); free(vo); free(at); free(intent); free(change); free(cand); free(best);
  free(nst); free(nlink); free(nlane); free(ncur); free(nx_); free(nv); free(own_f); free(tgt_f);
  return OK;
}

/* ------------------------------------------------------------------ outputs */
int orc_read_state(const orc_sim* S, uint8_t* status, int32_t* link, int32_t* lane, int32_t* cursor,
                   float* x, float* v, int32_t* insert_step, int32_t* arrive_step, int8_t* lane_change) {
  for (int i = 0; i < S->nt; i++) {
    if (status) status[i] = S->st[i];
    int act = S->st[i] == ST_ACTIVE;
    if (link) link[i] = act ? S->link[i] : -1;
    if (lane) lane[i] = act ? S->lane[i] : 0;
    if (cursor) cursor[i] = act ? S->cur[i] : 0;
    if (x) x[i] = act ? S->x[i] : 0.0f;
    if (v) v[i] = act ? S->v[i] : 0.0f;
    if (insert_step) insert_step[i] = S->ins_step[i];
    if (arrive_step) arrive_step[i] = S->arr_step[i];
    if (lane_change) lane_change[i] = S->dec[i];
  }
  return OK;
}

int orc_occupancy(const orc_sim* S, int32_t* lane_start, int32_t* sorted_vid) {
  occ_t O;
  build_occ(S, &O);
  for (int g = 0; g <= S->n_lanes; g++) lane_start[g] = O.start[g];
  for (int p = 0; p < O.n; p++) sorted_vid[p] = O.vids[p];
  free_occ(&O);
  return OK;
}

int orc_n_lanes(const orc_sim* S) { return S->n_lanes; }

int orc_node_holder(const orc_sim* S, int32_t* holder) {
  memcpy(holder, S->holder, (size_t)S->nn * 4);
  return OK;
}

/* counters: t, departed, waiting (due, not on the road), active, arrived,
 * vehicle-steps, pending (not yet due), active at the last step start, lane-change
 * decisions evaluated */
int orc_counters(const orc_sim* S, int64_t out[9]) {
  int64_t waiting = 0, pending = 0, active = 0;
  for (int i = 0; i < S->nt; i++) {
    if (S->st[i] == ST_ACTIVE) active++;
    else if (S->st[i] == ST_PENDING) {
      if (S->dep[i] < S->t) waiting++;
      else pending++;
    }
  }
  out[0] = S->t; out[1] = S->departed; out[2] = waiting; out[3] = active;
  out[4] = S->arrived; out[5] = S->veh_steps; out[6] = pending; out[7] = S->active_last;
  out[8] = S->lc_evals;
  return OK;
}

/* ------------------------------------------------------------------ calibration adjoint
 * Not in the paper (a calibration workload of the simulator): loss
 *   L = sum over observations k and trips v of (p_v(t_k) - target_{k,v})^2,
 * t_k = k * obs_every steps after the start, p_v = route progress (length of the
 * completed links of the route plus x; 0 before departure; the whole route length
 * after arrival).  Its gradient with respect to the IDM parameters of every link
 * class (v0, T, a, b, s0) holds every discrete decision of the run fixed: leaders,
 * lane changes, admissions, the stop-within-the-step branch, the clamp at a closed
 * stop line, floors of Eq. 7, departures and arrivals (the "tape").
 */
static double route_prefix(const orc_sim* S, int i, int upto) {
  double p = 0.0;
  for (int k = 0; k < upto; k++) p += (double)S->len[S->rl[S->roff[i] + k]];
  return p;
}

static double progress_of(const orc_sim* S, int i) {
  if (S->st[i] == ST_ACTIVE) return route_prefix(S, i, S->cur[i]) + (double)S->x[i];
  if (S->st[i] == ST_ARRIVED) return route_prefix(S, i, route_len(S, i));
  return 0.0;
}

int orc_observe(orc_sim* S, int32_t n_steps, int32_t obs_every, double* progress) {
  if (!S->routed) return ESTATE;
  if (obs_every <= 0 || n_steps < 0) return EINV;
  int nobs = n_steps / obs_every;
  for (int k = 0; k < nobs; k++) {
    orc_step(S, obs_every);
    for (int i = 0; i < S->nt; i++) progress[(int64_t)k * S->nt + i] = progress_of(S, i);
  }
  return OK;
}

int orc_set_class_params(orc_sim* S, const float* v0, const float* T, const float* a, const float* b,
                         const float* s0) {
  for (int c = 0; c < S->ncls; c++)
    if (!(a[c] > 0.0f) || !(b[c] > 0.0f) || !(T[c] >= 0.0f) || !(s0[c] >= 0.0f)) return EINV;
  for (int c = 0; c < S->ncls; c++) {
    S->pv0[c] = v0[c]; S->pT[c] = T[c]; S->pa[c] = a[c]; S->pb[c] = b[c]; S->ps0[c] = s0[c];
    S->psab[c] = sqrtf(S->pa[c] * S->pb[c]);
  }
  for (int e = 0; e < S->nl; e++) S->v0l[e] = S->pv0[S->cls[e]] > 0.0f ? S->pv0[S->cls[e]] : S->spd[e];
  return OK;
}

/* Partial derivatives of Eq. 7 (binary64) at the taped point: acceleration a with
 * respect to the gap s, own speed v, leader speed vl and the class parameters
 * (A, B, T, s0, v0).  The floors (gap at s_min, dynamic term at 0) are decided as in
 * the binary32 forward pass and held fixed. */
typedef struct { double ds, dv, dvl, dA, dB, dT, ds0, dv0; } idm_grad;

static idm_grad idm_partials(const orc_sim* S, int c, double v0, int kind, float s32, float v32, float vl32) {
  idm_grad g;
  memset(&g, 0, sizeof g);
  double A = S->pa[c], Bb = S->pb[c], T = S->pT[c], s0 = S->ps0[c];
  double v = v32;
  double r = v / v0;
  double r3 = r * r * r, r4 = r3 * r;
  g.dA = 1.0 - r4;
  g.dv0 = 4.0 * A * r4 / v0;
  g.dv = -4.0 * A * r3 / v0;
  if (kind == FORM_FREE || kind == FORM_NONE) return g;
  /* decisions taken in binary32, exactly as the forward pass took them */
  float dv32 = v32 - vl32;
  float t1 = v32 * S->pT[c];
  float t2 = (v32 * dv32) / (2.0f * S->psab[c]);
  int dyn_on = (t1 + t2) > 0.0f;
  int floored = !(s32 >= S->s_min) || s32 == S->s_min;
  double vl = vl32, s = s32;
  double cc = 1.0 / (2.0 * sqrt(A * Bb));
  double dvv = v - vl;
  double ss = s0 + (dyn_on ? v * T + v * dvv * cc : 0.0);
  double se = floored ? (double)S->s_min : s;
  double q = ss / se;
  double k2 = -2.0 * A * q / se;      /* d a / d ss */
  g.dA += -q * q;
  g.ds0 = k2;
  if (dyn_on) {
    g.dT = k2 * v;
    g.dA += k2 * v * dvv * (-cc / (2.0 * A));
    g.dB = k2 * v * dvv * (-cc / (2.0 * Bb));
    g.dv += k2 * (T + (dvv + v) * cc);
    g.dvl = k2 * (-v * cc);
  }
  g.ds = floored ? 0.0 : 2.0 * A * q * q / se;
  return g;
}

int orc_adjoint(orc_sim* S, int32_t n_steps, int32_t obs_every, const double* target, double* grad, double* loss) {
  if (!S->routed) return ESTATE;
  if (S->ttype) return ESTATE;   /* the calibration covers the single vehicle class */
  if (obs_every <= 0 || n_steps <= 0 || n_steps % obs_every) return EINV;
  int nt = S->nt, nobs = n_steps / obs_every;
  /* start state, kept for the taped replay */
  free(S->st0); free(S->cur0); free(S->x0); free(S->v0s); free(S->tgt);
  S->st0 = (uint8_t*)xcalloc(nt, 1); S->cur0 = (int32_t*)xcalloc(nt, 4);
  S->x0 = (float*)xcalloc(nt, 4); S->v0s = (float*)xcalloc(nt, 4);
  memcpy(S->st0, S->st, (size_t)nt); memcpy(S->cur0, S->cur, (size_t)nt * 4);
  memcpy(S->x0, S->x, (size_t)nt * 4); memcpy(S->v0s, S->v, (size_t)nt * 4);
  S->tgt = (double*)xcalloc((size_t)nobs * nt, 8);
  memcpy(S->tgt, target, (size_t)nobs * nt * 8);
  S->tgt_nobs = nobs; S->tgt_every = obs_every;
  /* forward with the tape; residuals of the observations */
  double* res = (double*)xcalloc((size_t)nobs * nt, 8);
  double L = 0.0;
  S->rec_n = 0; S->rec_steps = 0; S->recording = 1;
  for (int k = 0; k < nobs; k++) {
    orc_step(S, obs_every);
    for (int i = 0; i < nt; i++) {
      double r = progress_of(S, i) - target[(int64_t)k * nt + i];
      L += r * r;
      res[(int64_t)k * nt + i] = S->st[i] == ST_ACTIVE ? r : 0.0;   /* only positions depend on the parameters */
    }
  }
  S->recording = 0;
  S->rec_step[S->rec_steps] = S->rec_n;
  /* reverse sweep in binary64 */
  double* lx = (double*)xcalloc(nt, 8); double* lv = (double*)xcalloc(nt, 8);
  double* nx = (double*)xcalloc(nt, 8); double* nv = (double*)xcalloc(nt, 8);
  for (int q = 0; q < S->ncls * 5; q++) grad[q] = 0.0;
  double dt = S->dt, h = 0.5 * dt * dt;
  for (int j = n_steps - 1; j >= 0; j--) {
    if ((j + 1) % obs_every == 0) {
      int k = (j + 1) / obs_every - 1;
      for (int i = 0; i < nt; i++) lx[i] += 2.0 * res[(int64_t)k * nt + i];
    }
    memset(nx, 0, (size_t)nt * 8); memset(nv, 0, (size_t)nt * 8);
    for (int64_t q = S->rec_step[j]; q < S->rec_step[j + 1]; q++) {
      const orc_rec* r = &S->rec[q];
      int i = r->vid;
      double mu = 0.0;
      if (r->branch == BR_NORMAL) {
        mu = lx[i] * h + lv[i] * dt;
        nx[i] += lx[i];
        nv[i] += lx[i] * dt + lv[i];
      } else if (r->branch == BR_STOP) {
        double a = r->a, v = r->v;
        mu = lx[i] * v * v / (2.0 * a * a);
        nx[i] += lx[i];
        nv[i] += lx[i] * (-v / a);
      }
      if (mu == 0.0 || r->kind == FORM_NONE) continue;
      int c = S->cls[r->link];
      double v0 = S->v0l[r->link];
      idm_grad g = idm_partials(S, c, v0, r->kind, r->s, r->v, r->vl);
      nv[i] += mu * g.dv;
      if (r->kind != FORM_FREE) nx[i] -= mu * g.ds;
      if (r->kind == FORM_LEAD || r->kind == FORM_NEXT) {
        nx[r->lead] += mu * g.ds;
        nv[r->lead] += mu * g.dvl;
      }
      if (S->pv0[c] > 0.0f) grad[c * 5 + 0] += mu * g.dv0;
      grad[c * 5 + 1] += mu * g.dT;
      grad[c * 5 + 2] += mu * g.dA;
      grad[c * 5 + 3] += mu * g.dB;
      grad[c * 5 + 4] += mu * g.ds0;
    }
    double* tx = lx; lx = nx; nx = tx;
    double* tv = lv; lv = nv; nv = tv;
  }
  *loss = L;
  free(lx); free(lv); free(nx); free(nv); free(res);
  return OK;
}

/* Test helper (not the method): run n_steps recording the tape of every vehicle-step,
 * without observations or the reverse sweep, so that runs at perturbed parameters can
 * be compared with the base run's tape by orc_tape_digest. */
int orc_record(orc_sim* S, int32_t n_steps) {
  if (!S->routed) return ESTATE;
  if (n_steps < 0) return EINV;
  S->rec_n = 0; S->rec_steps = 0; S->recording = 1;
  orc_step(S, n_steps);
  S->recording = 0;
  if (S->rec_step) S->rec_step[S->rec_steps] = S->rec_n;
  return OK;
}

/* Test helper (not the method): the discrete content of the last recorded run, the
 * decisions the adjoint holds fixed, folded into one 64-bit FNV-1a digest (Fowler,
 * Noll, Vo: offset basis 14695981039346656037, prime 1099511628211, one byte at a
 * time).  Per record, in order: step boundary, trip, link, form of Eq. 7, its leader,
 * how the move ended, whether it crossed, and the two floors of Eq. 7 as the taped
 * binary32 values decide them (dynamic term positive, gap at or below s_min).  Two
 * runs whose digests and record counts agree took the same discrete path.  With
 * step_digest ([rec_steps] or NULL), entry j is the digest of steps 0 .. j-1 alone, so
 * the first entry where two runs differ bounds their common discrete prefix. */
static uint64_t fnv_bytes(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; i++) { h ^= b[i]; h *= 1099511628211ULL; }
  return h;
}

int orc_tape_digest(const orc_sim* S, uint64_t* digest, int64_t* n_rec, uint64_t* step_digest) {
  if (!digest || !n_rec) return EINV;
  uint64_t h = 14695981039346656037ULL;
  for (int j = 0; j < S->rec_steps; j++) {
    int32_t mark = -1 - j;
    h = fnv_bytes(h, &mark, 4);
    if (step_digest) step_digest[j] = h;   /* digest of the steps before j */
    for (int64_t q = S->rec_step[j]; q < S->rec_step[j + 1]; q++) {
      const orc_rec* r = &S->rec[q];
      int c = S->cls[r->link];
      float dv32 = r->v - r->vl;
      float t1 = r->v * S->pT[c];
      float t2 = (r->v * dv32) / (2.0f * S->psab[c]);
      int32_t w[8] = {r->vid, r->link, r->kind, r->lead, r->branch, r->crossed,
                      (r->kind != FORM_FREE && r->kind != FORM_NONE) ? (t1 + t2) > 0.0f : 0,
                      (r->kind != FORM_FREE && r->kind != FORM_NONE) ? !(r->s > S->s_min) : 0};
      h = fnv_bytes(h, w, sizeof w);
    }
  }
  *digest = h;
  *n_rec = S->rec_steps > 0 ? S->rec_step[S->rec_steps] : 0;
  return OK;
}

/* Loss of the last taped run replayed in binary64 with other class parameters
 * (v0, T, a, b, s0 per class), every discrete decision taken from the tape. */
int orc_replay_loss(const orc_sim* S, const double* pv0, const double* pT, const double* pa, const double* pb,
                    const double* ps0, double* loss) {
  if (!S->st0 || S->rec_steps <= 0) return ESTATE;
  int nt = S->nt;
  double* x = (double*)xcalloc(nt, 8); double* v = (double*)xcalloc(nt, 8);
  double* off = (double*)xcalloc(nt, 8); double* acc = (double*)xcalloc(nt, 8);
  uint8_t* st = (uint8_t*)xcalloc(nt, 1);
  for (int i = 0; i < nt; i++) {
    st[i] = S->st0[i];
    if (st[i] == ST_ACTIVE) { x[i] = S->x0[i]; v[i] = S->v0s[i]; off[i] = route_prefix(S, i, S->cur0[i]); }
  }
  double dt = S->dt, h = 0.5 * dt * dt, L = 0.0;
  for (int j = 0; j < S->rec_steps; j++) {
    /* vehicles that entered at the end of the previous step */
    for (int64_t q = S->rec_step[j]; q < S->rec_step[j + 1]; q++) {
      int i = S->rec[q].vid;
      if (st[i] != ST_ACTIVE) { st[i] = ST_ACTIVE; x[i] = 0.0; v[i] = 0.0; off[i] = 0.0; }
    }
    for (int64_t q = S->rec_step[j]; q < S->rec_step[j + 1]; q++) {
      const orc_rec* r = &S->rec[q];
      int i = r->vid, c = S->cls[r->link];
      double A = pa[c], Bb = pb[c], T = pT[c], s0 = ps0[c];
      double v0 = S->pv0[c] > 0.0f ? pv0[c] : (double)S->spd[r->link];
      double rr = v[i] / v0, r4 = rr * rr * rr * rr;
      double a = A * (1.0 - r4);
      if (r->kind != FORM_FREE && r->kind != FORM_NONE) {
        double s, vl;
        double Lk = S->len[r->link];
        if (r->kind == FORM_LEAD) { s = (x[r->lead] - x[i]) - S->len_v; vl = v[r->lead]; }
        else if (r->kind == FORM_NEXT) { s = ((Lk - x[i]) + x[r->lead]) - S->len_v; vl = v[r->lead]; }
        else { s = Lk - x[i]; vl = 0.0; }
        float dv32 = r->v - r->vl;
        int c32 = c;
        float t1 = r->v * S->pT[c32];
        float t2 = (r->v * dv32) / (2.0f * S->psab[c32]);
        int dyn_on = (t1 + t2) > 0.0f;
        int floored = !(r->s >= S->s_min) || r->s == S->s_min;
        double ss = s0 + (dyn_on ? v[i] * T + v[i] * (v[i] - vl) / (2.0 * sqrt(A * Bb)) : 0.0);
        double se = floored ? (double)S->s_min : s;
        double qq = ss / se;
        a -= A * qq * qq;
      }
      acc[i] = a;
    }
    for (int64_t q = S->rec_step[j]; q < S->rec_step[j + 1]; q++) {
      const orc_rec* r = &S->rec[q];
      int i = r->vid;
      double Lk = S->len[r->link];
      if (r->branch == BR_ARRIVE) { st[i] = ST_ARRIVED; continue; }
      if (r->branch == BR_CLAMP) { x[i] = Lk; v[i] = 0.0; continue; }
      if (r->branch == BR_NORMAL) { x[i] = x[i] + (v[i] * dt + acc[i] * h); v[i] = v[i] + acc[i] * dt; }
      else { x[i] = x[i] - v[i] * v[i] / (2.0 * acc[i]); v[i] = 0.0; }
      if (r->crossed) { x[i] -= Lk; off[i] += Lk; }
    }
    if ((j + 1) % S->tgt_every == 0) {
      int k = (j + 1) / S->tgt_every - 1;
      for (int i = 0; i < nt; i++) {
        double p = st[i] == ST_ACTIVE ? off[i] + x[i] : (st[i] == ST_ARRIVED ? route_prefix(S, i, route_len(S, i)) : 0.0);
        double d = p - S->tgt[(int64_t)k * nt + i];
        L += d * d;
      }
    }
  }
  *loss = L;
  free(x); free(v); free(off); free(acc); free(st);
  return OK;
}

/* ------------------------------------------------------------------ measured outputs */
int orc_set_outputs(orc_sim* S, uint32_t flags, int32_t sample_every, int32_t per_window, int32_t max_windows) {
  if (flags & ~7u) return EINV;
  if ((flags & 4u) && (sample_every < 1 || per_window < 1 || max_windows < 1)) return EINV;
  free(S->fuel); free(S->co); free(S->enter); free(S->tt_sum); free(S->tt_n);
  free(S->acc_u); free(S->acc_s); free(S->out_u); free(S->out_s); free(S->out_n);
  S->fuel = S->co = NULL; S->enter = NULL; S->tt_sum = NULL; S->tt_n = NULL;
  S->acc_u = S->acc_s = S->out_u = S->out_s = NULL; S->out_n = NULL;
  S->out_flags = flags;
  if (flags & 1u) {
    S->fuel = (double*)xcalloc(zsz(S->nt), 8);
    S->co = (double*)xcalloc(zsz(S->nt), 8);
  }
  if (flags & 2u) {
    S->enter = (int32_t*)xcalloc(zsz(S->nt), 4);
    S->tt_sum = (int64_t*)xcalloc(zsz(S->nl), 8);
    S->tt_n = (int32_t*)xcalloc(zsz(S->nl), 4);
  }
  if (flags & 4u) {
    S->samp_every = sample_every; S->samp_per = per_window; S->samp_max = max_windows;
    S->acc_u = (double*)xcalloc(zsz(S->nl), 8);
    S->acc_s = (double*)xcalloc(zsz(S->nl), 8);
    S->out_u = (double*)xcalloc((size_t)max_windows * zsz(S->nl), 8);
    S->out_s = (double*)xcalloc((size_t)max_windows * zsz(S->nl), 8);
    S->out_n = (int32_t*)xcalloc((size_t)max_windows, 4);
  }
  clear_outputs(S);
  return OK;
}

/* Vehicle types (Sec. 6.3.5): n types with length, acceleration scale and maximum
 * speed; trip_type[i] < n for every trip.  n = 0 returns to the single class. */
int orc_set_vehicle_types(orc_sim* S, int32_t n, const float* length, const float* accel_scale,
                          const float* max_speed, const uint8_t* trip_type) {
  if (n < 0 || n > 8) return EINV;
  for (int k = 0; k < n; k++)
    if (!(length[k] > 0.0f) || !(accel_scale[k] > 0.0f) || !(max_speed[k] > 0.0f)) return EINV;
  for (int i = 0; n > 0 && i < S->nt; i++) if (trip_type[i] >= n) return EINV;
  free(S->vty_len); free(S->vty_ascale); free(S->vty_vmax); free(S->ttype);
  S->vty_len = S->vty_ascale = S->vty_vmax = NULL;
  S->ttype = NULL;
  S->n_vty = n;
  if (n == 0) return OK;
  S->vty_len = (float*)xcalloc(n, 4);
  S->vty_ascale = (float*)xcalloc(n, 4);
  S->vty_vmax = (float*)xcalloc(n, 4);
  S->ttype = (uint8_t*)xcalloc(zsz(S->nt), 1);
  memcpy(S->vty_len, length, (size_t)n * 4);
  memcpy(S->vty_ascale, accel_scale, (size_t)n * 4);
  memcpy(S->vty_vmax, max_speed, (size_t)n * 4);
  memcpy(S->ttype, trip_type, (size_t)S->nt);
  return OK;
}

/* clear the outputs in the middle of a run (windows restart at the next sampling instant) */
int orc_reset_outputs(orc_sim* S) {
  clear_outputs(S);
  return OK;
}

int orc_read_emissions(const orc_sim* S, double* fuel_ml, double* co_g) {
  if (!S->fuel) return ESTATE;
  memcpy(fuel_ml, S->fuel, (size_t)S->nt * 8);
  memcpy(co_g, S->co, (size_t)S->nt * 8);
  return OK;
}

int orc_read_link_times(const orc_sim* S, int64_t* sum_steps, int32_t* n_exits) {
  if (!S->enter) return ESTATE;
  memcpy(sum_steps, S->tt_sum, (size_t)S->nl * 8);
  memcpy(n_exits, S->tt_n, (size_t)S->nl * 4);
  return OK;
}

int orc_read_edge_samples(const orc_sim* S, double* util, double* speed, int32_t* n_samples) {
  if (!S->acc_u) return ESTATE;
  memcpy(util, S->out_u, (size_t)S->samp_max * S->nl * 8);
  memcpy(speed, S->out_s, (size_t)S->samp_max * S->nl * 8);
  memcpy(n_samples, S->out_n, (size_t)S->samp_max * 4);
  return OK;
}

/* Sec. 6.3.1: the measured travel time of a link is the mean of its traversal times
 * in deciseconds (traversal steps * dt_ds / traversals, rounded half up, kept within
 * 1 .. 1e6); a link no trip left keeps its previous cost.  gap (optional) compares
 * previous and measured costs, weighted by traversals:
 * sum n_e |prev_e - meas_e| / sum n_e prev_e. */
int orc_measured_costs(const orc_sim* S, const int32_t* prev, int32_t* out, double* gap) {
  if (!S->enter) return ESTATE;
  int64_t num = 0, den = 0;
  for (int e = 0; e < S->nl; e++) {
    int64_t n = S->tt_n[e];
    if (n == 0) { out[e] = prev[e]; continue; }
    int64_t c = (2 * S->tt_sum[e] * S->dt_ds + n) / (2 * n);
    if (c < 1) c = 1;
    if (c > 1000000) c = 1000000;
    out[e] = (int32_t)c;
    num += n * (c > prev[e] ? c - prev[e] : prev[e] - c);
    den += n * (int64_t)prev[e];
  }
  if (gap) *gap = den > 0 ? (double)num / (double)den : 0.0;
  return OK;
}

/* Sec. 6.3.1 iterative decaying equilibrium: iteration 0 routes every trip on the
 * initial costs (cost_mode) and runs n_steps; iteration k >= 1 reroutes the subset
 * fractions_q16[k] of round k on the costs measured in iteration k - 1 and runs again.
 * gap[k] is the measured-versus-routed gap of iteration k; cost_out the costs measured
 * in the last one.  Needs the link-time output. */
int orc_equilibrium(orc_sim* S, int32_t n_iter, const uint32_t* fractions_q16, int32_t n_steps, int32_t* cost_out,
                    double* gap) {
  if (!S->enter) return ESTATE;
  if (n_iter < 1 || n_steps < 1) return EINV;
  for (int k = 1; k < n_iter; k++) if (fractions_q16[k] > 65536u) return EINV;
  int32_t* cost = (int32_t*)xcalloc(zsz(S->nl), 4);
  int32_t* meas = (int32_t*)xcalloc(zsz(S->nl), 4);
  for (int e = 0; e < S->nl; e++) cost[e] = orc_link_cost(S->len[e], S->spd[e], S->lanes[e], S->cost_mode);
  int rc = OK;
  for (int k = 0; k < n_iter && rc == OK; k++) {
    rc = k == 0 ? orc_route(S, cost) : orc_reroute(S, cost, fractions_q16[k], (uint32_t)k);
    if (rc == OK) rc = orc_step(S, n_steps);
    if (rc == OK) rc = orc_measured_costs(S, cost, meas, &gap[k]);
    if (rc == OK) memcpy(cost, meas, (size_t)S->nl * 4);
  }
  if (rc == OK) memcpy(cost_out, cost, (size_t)S->nl * 4);
  free(cost); free(meas);
  return rc;
}

/* ------------------------------------------------------------------ static assignment */
/* Eq. 3 (BPR): t = t0 (1 + alpha (x / c)^beta), integer beta by repeated products,
 * t0 = length / speed (Eq. 4, seconds), binary64. */
static double bpr_time(double t0, double x, double c, double alpha, int beta) {
  double r = x / c, p = 1.0;
  for (int k = 0; k < beta; k++) p = p * r;
  return t0 * (1.0 + alpha * p);
}

/* Beckmann term of one link (Eq. 6 objective): integral of Eq. 3 from 0 to x. */
static double bpr_integral(double t0, double x, double c, double alpha, int beta) {
  double r = x / c, p = 1.0;
  for (int k = 0; k < beta; k++) p = p * r;
  return t0 * x * (1.0 + alpha * p / (double)(beta + 1));
}

/* Sums whose value steers the algorithm (the line search's derivative sign, the gap,
 * the objective) are taken exactly: every term is rounded to the grid 2^-S, with S the
 * largest shift for which n terms bounded by B stay below 2^62 in magnitude, and the
 * integers are added.  The result then depends on no summation order. */
static double fp_scale(double bound, int n) {
  int E = 0;
  frexp(bound * (double)(n > 0 ? n : 1), &E);
  int S = 62 - E;
  if (S > 100) S = 100;
  return ldexp(1.0, S);
}

/* All-or-nothing assignment (Sec. 5.2, step 2 of Frank-Wolfe): every trip on its
 * canonical shortest path under the integer costs q (the tie rule of orc_route);
 * flow[e] = number of trips using link e. */
static int aon_flows(const orc_sim* S, const int32_t* q, double* flow) {
  int nn = S->nn, nl = S->nl, nt = S->nt;
  int* os = (int*)xcalloc(nn + 1, sizeof(int));
  int* ol = (int*)xcalloc(zsz(nl), sizeof(int));
  build_csr(nn, nl, S->lf, os, ol);
  int* ts = (int*)xcalloc(nn + 1, sizeof(int));
  int* tl = (int*)xcalloc(zsz(nt), sizeof(int));
  build_csr(nn, nt, S->orig, ts, tl);
  int64_t* dist = (int64_t*)xcalloc(nn, 8);
  hent* heap = (hent*)xcalloc(nl + 1, sizeof(hent));
  int64_t* cnt = (int64_t*)xcalloc(zsz(nl), 8);
  int rc = OK;
  for (int o = 0; o < nn && rc == OK; o++) {
    if (ts[o] == ts[o + 1]) continue;
    dijkstra(nn, os, ol, S->lt, q, o, dist, heap);
    for (int k = ts[o]; k < ts[o + 1] && rc == OK; k++) {
      int d = S->dest[tl[k]];
      if (d == o) { rc = EINV; break; }
      if (dist[d] == INT64_MAX) { rc = EUNREACH; break; }
      int v = d;
      while (v != o) {
        int pick = -1;
        for (int j = S->in_start[v]; j < S->in_start[v + 1]; j++) {
          int e = S->in_list[j];
          int u = S->lf[e];
          if (dist[u] != INT64_MAX && dist[u] + q[e] == dist[v]) { pick = e; break; }
        }
        if (pick < 0) { rc = ESTATE; break; }
        cnt[pick]++;
        v = S->lf[pick];
      }
    }
  }
  for (int e = 0; e < nl; e++) flow[e] = (double)cnt[e];
  free(os); free(ol); free(ts); free(tl); free(dist); free(heap); free(cnt);
  return rc;
}

/* Integer routing costs of the travel times t: units of max(0.1 s, max t / qmax), rounded
 * half up, within 1 .. qmax, qmax = min(1e6, (2e9 - 1) / n_nodes) so that no path
 * length can pass 2^31 in the shortest-path search. */
static void quantize_costs(const orc_sim* S, const double* t, int32_t* q) {
  int64_t qmax = (2000000000LL - 1) / (S->nn > 0 ? S->nn : 1);
  if (qmax > 1000000) qmax = 1000000;
  double tmax = 0.0;
  for (int e = 0; e < S->nl; e++) if (t[e] > tmax) tmax = t[e];
  double unit = tmax / (double)qmax;
  if (unit < 0.1) unit = 0.1;
  for (int e = 0; e < S->nl; e++) {
    double c = floor(t[e] / unit + 0.5);
    if (c < 1.0) c = 1.0;
    if (c > (double)qmax) c = (double)qmax;
    q[e] = (int32_t)c;
  }
}

/* Static user equilibrium (Sec. 5.2, Eq. 6) by Frank-Wolfe with BPR link times (Eq. 3):
 *   x_0 = all-or-nothing on the free-flow times;
 *   iteration k: t = BPR(x_k); y_k = all-or-nothing on t; gap_k = (t.x - t.y) / t.x;
 *     step a_k in [0, 1] minimising the Beckmann objective along x_k + a (y_k - x_k):
 *     bisection (bisect_iter halvings) on the sign of its derivative
 *     sum_e t_e(x_e + a d_e) d_e, a_k = 1 when that is not positive at a = 1 and 0 when it
 *     is not negative at a = 0; x_{k+1} = x_k + a_k (y_k - x_k).
 * Demand: one vehicle per trip.  capacity[e] > 0 in vehicles over the same period.
 * Outputs: flow and BPR time at x_K, gap[k] and step[k] for k < K, objective[k] at
 * x_k for k <= K. */
int orc_assign_static(orc_sim* S, const double* capacity, double alpha, int32_t beta, int32_t max_iter,
                      int32_t bisect_iter, double* flow_out, double* time_out, double* gap, double* step,
                      double* objective) {
  int nl = S->nl;
  if (!capacity || beta < 1 || beta > 8 || !(alpha >= 0.0) || max_iter < 0 || bisect_iter < 0) return EINV;
  for (int e = 0; e < nl; e++) if (!(capacity[e] > 0.0)) return EINV;
  double* t0 = (double*)xcalloc(zsz(nl), 8);
  double* x = (double*)xcalloc(zsz(nl), 8);
  double* y = (double*)xcalloc(zsz(nl), 8);
  double* t = (double*)xcalloc(zsz(nl), 8);
  int32_t* q = (int32_t*)xcalloc(zsz(nl), 4);
  for (int e = 0; e < nl; e++) t0[e] = (double)S->len[e] / (double)S->spd[e];
  quantize_costs(S, t0, q);
  int rc = aon_flows(S, q, x);
  for (int k = 0; k <= max_iter && rc == OK; k++) {
    /* objective at x_k */
    double bo = 0.0;
    for (int e = 0; e < nl; e++) {
      double f = bpr_integral(t0[e], x[e], capacity[e], alpha, beta);
      if (f > bo) bo = f;
    }
    double so = fp_scale(bo, nl);
    long long io = 0;
    for (int e = 0; e < nl; e++) io += llrint(bpr_integral(t0[e], x[e], capacity[e], alpha, beta) * so);
    objective[k] = (double)io / so;
    if (k == max_iter) break;
    /* direction */
    for (int e = 0; e < nl; e++) t[e] = bpr_time(t0[e], x[e], capacity[e], alpha, beta);
    quantize_costs(S, t, q);
    rc = aon_flows(S, q, y);
    if (rc != OK) break;
    double bg = 0.0;
    for (int e = 0; e < nl; e++) {
      double m = (x[e] > y[e] ? x[e] : y[e]) * t[e];
      if (m > bg) bg = m;
    }
    double sg = fp_scale(bg, nl);
    long long tx = 0, ty = 0;
    for (int e = 0; e < nl; e++) { tx += llrint(t[e] * x[e] * sg); ty += llrint(t[e] * y[e] * sg); }
    gap[k] = tx > 0 ? (double)(tx - ty) / (double)tx : 0.0;
    /* line search */
    double bl = 0.0;
    for (int e = 0; e < nl; e++) {
      double d = y[e] - x[e];
      double m = bpr_time(t0[e], x[e] > y[e] ? x[e] : y[e], capacity[e], alpha, beta) * fabs(d);
      if (m > bl) bl = m;
    }
    double sl = fp_scale(bl, nl);
#define DERIV_SIGN(A, OUT) do { long long g_ = 0; \
      for (int e = 0; e < nl; e++) { double d_ = y[e] - x[e]; \
        g_ += llrint(bpr_time(t0[e], x[e] + (A) * d_, capacity[e], alpha, beta) * d_ * sl); } \
      (OUT) = g_; } while (0)
    long long g0, g1;
    DERIV_SIGN(0.0, g0);
    DERIV_SIGN(1.0, g1);
    double a;
    if (g0 >= 0) a = 0.0;
    else if (g1 <= 0) a = 1.0;
    else {
      double lo = 0.0, hi = 1.0;
      for (int it = 0; it < bisect_iter; it++) {
        double mid = 0.5 * (lo + hi);
        long long gm;
        DERIV_SIGN(mid, gm);
        if (gm > 0) hi = mid; else lo = mid;
      }
      a = 0.5 * (lo + hi);
    }
#undef DERIV_SIGN
    step[k] = a;
    for (int e = 0; e < nl; e++) x[e] = x[e] + a * (y[e] - x[e]);
  }
  if (rc == OK)
    for (int e = 0; e < nl; e++) {
      flow_out[e] = x[e];
      time_out[e] = bpr_time(t0[e], x[e], capacity[e], alpha, beta);
    }
  free(t0); free(x); free(y); free(t); free(q);
  return rc;
}

/* building block for the pins: all-or-nothing flows on integer costs */
int orc_aon(orc_sim* S, const int32_t* cost, double* flow) { return aon_flows(S, cost, flow); }
