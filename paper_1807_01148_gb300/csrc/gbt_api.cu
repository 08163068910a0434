// C-ABI of libgbtraffic (declared in include/gbtraffic.h): input validation, network
// preprocessing, device memory, the trip-planning driver and the CUDA-graph step loop.
// Waddell et al., Sec. 6 ("Traffic microsimulation model").
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gbt_internal.cuh"
#include "gbtraffic.h"

namespace gbt {
void launch_step(const Dev& d, int grid, bool has_stop, cudaStream_t s);
void launch_occupancy(const Dev& d, int grid, cudaStream_t s);
void launch_count(const Dev& d, int grid, cudaStream_t s);
int scan_blocks(int n_lanes);
void launch_state_out(const Dev& d, int grid, cudaStream_t s, uint8_t* status, int32_t* link, int32_t* lane,
                      int32_t* cursor, float* x, float* v, int32_t* ins, int32_t* arr, int8_t* dec);
void launch_state_in(const Dev& d, int grid, cudaStream_t s, const uint8_t* status, const int32_t* link,
                     const int32_t* lane, const int32_t* cursor, const float* x, const float* v);
void launch_occ_out(const Dev& d, int grid, cudaStream_t s, int32_t* sorted_vid);
void launch_status_counts(const Dev& d, int grid, cudaStream_t s, unsigned long long* counts);
void launch_state_check(const Dev& d, int grid, cudaStream_t s, const uint8_t* status, const int32_t* link,
                        const int32_t* lane, const int32_t* cursor, const float* x, const float* v, int* bad);
cudaError_t launch_steps_timed(const Dev& d, int grid, bool has_stop, cudaStream_t s, int n, float* kernel_ms);
void launch_observe(const Dev& d, int grid, cudaStream_t s, const double* target, double* res, double* p_out);
void launch_tape_begin(const Dev& d, cudaStream_t s);
void launch_adj_step(const Dev& d, int grid, cudaStream_t s, const TapeRec* slab, const double* lx,
                     const double* lv, const double* res, double* nx, double* nv, double* grad, int n_class);
void launch_first_links(const int32_t* roff, const int32_t* routes, int n, int32_t* out, cudaStream_t s);
void launch_measured_costs(const Dev& d, const int32_t* prev, int32_t* out, cudaStream_t s);
void launch_fw_t0(const float* len, const float* spd, double* t0, int n, cudaStream_t s);
void launch_fw_counts(const unsigned* cnt, double* x, int n, cudaStream_t s);
void launch_fw_time(const double* t0, const double* x, const double* cap, double alpha, int beta, double* t,
                    unsigned long long* tmax, int n, cudaStream_t s);
void launch_fw_quantize(const double* t, double unit, int qmax, int32_t* q, int n, cudaStream_t s);
void launch_fw_bounds(const double* t0, const double* x, const unsigned* y, const double* t, const double* cap,
                      double alpha, int beta, unsigned long long* out, int n, cudaStream_t s);
void launch_fw_gap_sums(const double* t, const double* x, const unsigned* y, double scale, unsigned long long* out,
                        int n, cudaStream_t s);
void launch_fw_deriv(const double* t0, const double* x, const unsigned* y, const double* cap, double alpha, int beta,
                     double a, double scale, unsigned long long* out, int n, cudaStream_t s);
void launch_fw_update(double* x, const unsigned* y, double a, int n, cudaStream_t s);
void launch_fw_objective(const double* t0, const double* x, const double* cap, double alpha, int beta, bool bound,
                         double scale, unsigned long long* out, int n, cudaStream_t s);
void launch_fw_final_time(const double* t0, const double* x, const double* cap, double alpha, int beta, double* t,
                          int n, cudaStream_t s);
void launch_compact_routes(const int32_t* roff, const int32_t* rlen, const int32_t* src, const int32_t* new_off,
                           int32_t* dst, int n, cudaStream_t s);
void chunk_setup(int blocks_per_sm[8]);
void front_setup(int blocks_per_sm[2]);
bool chunk_split_needed(const double* lane_m, int n_links, float vlen_min);
bool rank_long_needed(double max_len, float vlen_min);
size_t chunk_table_size(int n_trips);
int persistent_max_blocks_per_sm(int threads);
cudaError_t launch_persistent(const Dev& d, GridSync* gs, int blocks, int threads, int n_steps, long long limit,
                              cudaStream_t s);
}  // namespace gbt

using namespace gbt;

static std::string g_create_error;

// An NVTX range over one call of the C ABI (visible in Nsight timelines; header-only
// NVTX3, inactive unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct HostMirror {
  Ctl c;
  unsigned long long counts[3];   // active, waiting (due, not on the road), pending (not yet due)
};

struct sim_handle {
  std::string err;
  void* stage[9] = {};   // device staging of sim_read_state's host reads, per field
  bool state_lost = false;   // a bounded device wait ran out: the state must be reset
  // host copy of the device step counter, valid while only sim_step (and reads) ran
  // since it was taken: sim_step then checks the horizon without a device round trip
  long long t_host = 0;
  bool t_known = false;
  // pinned host copy of the control block and of the trip-status counts (read back by
  // every sim_step and sim_counters) and their device source for the counts
  HostMirror* mirror = nullptr;
  unsigned long long* d_counts = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int device = 0, sm_count = 0, grid = 0;
  // sizes
  int nn = 0, nl = 0, nt = 0, n_lanes = 0, ncls = 0;
  bool has_stop = false;
  std::vector<double> lane_m;   // lanes x length per link (chunk_split_needed)
  double max_len = 0.0;         // longest link (rank_long_needed)
  long long launches = 0;    // kernel launches made by sim_step (sim_launch_count)
  size_t graph_nodes = 0, graph_samp_nodes = 0;   // kernels per step of the step graphs
  // host copies
  std::vector<int32_t> lfrom, lto, depart, origin, dest;
  std::vector<float> len, spd;
  std::vector<uint8_t> lanes;
  std::vector<int32_t> lane_base;
  int cost_mode = 0, loop = 0;
  // device
  std::vector<void*> allocs;
  std::vector<size_t> alloc_sizes;   // bytes of each entry of allocs
  size_t bytes = 0, max_bytes = 0;   // device bytes held; cap (0: none)
  Dev d{};
  int32_t* routes = nullptr;
  unsigned long long route_cap = 0;
  int32_t* q_items = nullptr;
  int32_t* q_end = nullptr;
  int32_t* q_head = nullptr;
  int32_t* qlinks = nullptr;
  bool routed = false;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  bool graph_dirty = true;
  // the step graph with the per-edge sample kernel, launched at sampling instants only
  cudaGraphExec_t gexec_samp = nullptr;
  cudaGraph_t graph_samp = nullptr;
  // class parameters (host copies) and the adjoint's tape
  std::vector<float> v0c, Tc, ac, bc, s0c, spd_link;
  std::vector<uint8_t> cls_link;
  std::vector<LinkRec> recs;
  TapeRec* tape = nullptr;
  TapeForm* tform = nullptr;
  int tape_steps = 0;
  cudaGraphExec_t gexec_tape = nullptr;
  cudaGraph_t graph_tape = nullptr;
  bool tape_graph_dirty = true;
  // execution configuration of sim_step
  sim_exec exec{SIM_EXEC_GRAPH, 256, 0, 8, 0};
  GridSync* gs = nullptr;
  // the persistent launch captured as a graph (for one step count at a time)
  cudaGraphExec_t pexec = nullptr;
  cudaGraph_t pgraph = nullptr;
  int pgraph_n = -1;
  sim_exec pgraph_cfg{};
  bool pgraph_unsupported = false;
  // per-trip hash bases (mandatory-switch and reroute draws), measured outputs
  std::vector<unsigned long long> hseed;
  uint32_t out_flags = 0;
  // vehicle types: per type length, acceleration scale, maximum speed
  std::vector<float> vty_len, vty_ascale, vty_vmax;
};

namespace {

int fail(sim_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(sim_handle* h, cudaError_t e, const char* what) {
  return fail(h, e == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);         \
  } while (0)

template <class T>
int dalloc(sim_handle* h, T** p, size_t n) {
  const size_t nb = (n ? n : 1) * sizeof(T);
  if (h->max_bytes && h->bytes + nb > h->max_bytes)
    return fail(h, SIM_ENOMEM, "device memory cap (sim_params.max_device_bytes) reached");
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, nb);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc");
  h->allocs.push_back(q);
  h->alloc_sizes.push_back(nb);
  h->bytes += nb;
  *p = static_cast<T*>(q);
  return SIM_OK;
}

void dfree(sim_handle* h, void* p) {
  if (!p) return;
  auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
  if (it != h->allocs.end()) {
    const size_t k = (size_t)(it - h->allocs.begin());
    h->bytes -= h->alloc_sizes[k];
    h->alloc_sizes.erase(h->alloc_sizes.begin() + (long)k);
    h->allocs.erase(it);
  }
  cudaFree(p);
}

template <class T>
int upload(sim_handle* h, T** p, const T* src, size_t n) {
  int rc = dalloc(h, p, n);
  if (rc) return rc;
  if (n) CK(cudaMemcpy(*p, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return SIM_OK;
}

// ------------------------------------------------------------------ union of scenarios
struct Flat {
  int nn = 0, nl = 0, nt = 0, ncls = 0;
  std::vector<int32_t> nx, ny, off, cyc, grn, lf, lt, orig, dest, dep;
  std::vector<uint8_t> ctrl, lanes, cls;
  std::vector<float> len, spd, v0, T, a, b, s0;
  std::vector<unsigned long long> hseed;
  sim_params p{};
};

int flatten(int n, const sim_network* const* nets, const sim_demand* const* dems, const sim_params* const* pars,
            Flat& F) {
  if (n <= 0 || !nets || !dems || !pars) return fail(nullptr, SIM_EINVAL, "null or empty scenario list");
  for (int k = 0; k < n; k++) {
    const sim_network* N = nets[k];
    const sim_demand* D = dems[k];
    const sim_params* P = pars[k];
    if (!N || !D || !P) return fail(nullptr, SIM_EINVAL, "null scenario input");
    if (N->n_nodes <= 0 || N->n_links <= 0 || D->n_trips < 0)
      return fail(nullptr, SIM_EINVAL, "n_nodes and n_links must be > 0, n_trips >= 0");
    if (!N->node_x_dm || !N->node_y_dm || !N->node_control || !N->signal_offset_ds || !N->signal_cycle_ds ||
        !N->signal_green_ds || !N->link_from || !N->link_to || !N->link_length_m || !N->link_speed_mps ||
        !N->link_lanes || !N->link_class)
      return fail(nullptr, SIM_EINVAL, "null network array");
    if (D->n_trips > 0 && (!D->origin || !D->dest || !D->depart_step))
      return fail(nullptr, SIM_EINVAL, "null demand array");
    if (P->n_class <= 0 || P->n_class > SIM_MAX_CLASS || !P->v0 || !P->T || !P->a || !P->b || !P->s0)
      return fail(nullptr, SIM_EINVAL, "bad parameter classes");
    if (k == 0) {
      F.p = *P;
    } else {
      const sim_params& Q = F.p;
      if (P->dt != Q.dt || P->veh_len != Q.veh_len || P->s_min != Q.s_min || P->mobil_p != Q.mobil_p ||
          P->mobil_athr != Q.mobil_athr || P->mobil_bsafe != Q.mobil_bsafe ||
          P->mobil_bias_right != Q.mobil_bias_right || P->lambda_mand != Q.lambda_mand ||
          P->stop_acquire_m != Q.stop_acquire_m || P->cost_mode != Q.cost_mode || P->loop_routes != Q.loop_routes ||
          P->max_device_bytes != Q.max_device_bytes)
        return fail(nullptr, SIM_EINVAL, "batched scenarios must share dt and all scalar parameters");
    }
    const int nb = F.nn, lb = F.nl, cb = F.ncls;
    for (int i = 0; i < N->n_nodes; i++) {
      F.nx.push_back(N->node_x_dm[i]);
      F.ny.push_back(N->node_y_dm[i]);
      F.ctrl.push_back(N->node_control[i]);
      F.off.push_back(N->signal_offset_ds[i]);
      F.cyc.push_back(N->signal_cycle_ds[i]);
      F.grn.push_back(N->signal_green_ds[i]);
    }
    for (int e = 0; e < N->n_links; e++) {
      if (N->link_from[e] < 0 || N->link_from[e] >= N->n_nodes || N->link_to[e] < 0 || N->link_to[e] >= N->n_nodes)
        return fail(nullptr, SIM_EINVAL, "link end node out of range");
      if (N->link_class[e] >= P->n_class) return fail(nullptr, SIM_EINVAL, "link class out of range");
      F.lf.push_back(N->link_from[e] + nb);
      F.lt.push_back(N->link_to[e] + nb);
      F.len.push_back(N->link_length_m[e]);
      F.spd.push_back(N->link_speed_mps[e]);
      F.lanes.push_back(N->link_lanes[e]);
      F.cls.push_back((uint8_t)(N->link_class[e] + cb));
    }
    for (int c = 0; c < P->n_class; c++) {
      F.v0.push_back(P->v0[c]);
      F.T.push_back(P->T[c]);
      F.a.push_back(P->a[c]);
      F.b.push_back(P->b[c]);
      F.s0.push_back(P->s0[c]);
    }
    for (int i = 0; i < D->n_trips; i++) {
      if (D->origin[i] < 0 || D->origin[i] >= N->n_nodes || D->dest[i] < 0 || D->dest[i] >= N->n_nodes)
        return fail(nullptr, SIM_EINVAL, "trip origin/destination out of range");
      F.orig.push_back(D->origin[i] + nb);
      F.dest.push_back(D->dest[i] + nb);
      F.dep.push_back(D->depart_step[i]);
      // hash base of the mandatory-switch draw: scenario seed and scenario-local trip id
      F.hseed.push_back((unsigned long long)P->seed ^ ((unsigned long long)(uint32_t)i << 32));
    }
    F.nn += N->n_nodes;
    F.nl += N->n_links;
    F.nt += D->n_trips;
    F.ncls += P->n_class;
    if (F.ncls > SIM_MAX_CLASS) return fail(nullptr, SIM_EINVAL, "too many parameter classes in batch");
    (void)lb;
  }
  return SIM_OK;
}

int create_from_flat(Flat& F, sim_handle** out) {
  *out = nullptr;
  const sim_params& P = F.p;
  if (!(P.dt > 0.0f)) return fail(nullptr, SIM_EINVAL, "dt must be > 0");
  const int dt_ds = (int)lrintf(P.dt * 10.0f);
  if (dt_ds <= 0 || fabsf((float)dt_ds - P.dt * 10.0f) > 1e-3f)
    return fail(nullptr, SIM_EINVAL, "dt must be a whole number of deciseconds");
  if (!(P.veh_len > 0.0f) || !(P.s_min > 0.0f)) return fail(nullptr, SIM_EINVAL, "veh_len and s_min must be > 0");
  for (int c = 0; c < F.ncls; c++)
    if (!(F.a[c] > 0.0f) || !(F.b[c] > 0.0f) || !(F.T[c] >= 0.0f) || !(F.s0[c] >= 0.0f))
      return fail(nullptr, SIM_EINVAL, "IDM parameters must satisfy a > 0, b > 0, T >= 0, s0 >= 0");
  for (int i = 0; i < F.nn; i++) {
    if (F.ctrl[i] > 2) return fail(nullptr, SIM_EINVAL, "node_control must be 0, 1 or 2");
    if (F.ctrl[i] == SIM_CTRL_SIGNAL && (F.cyc[i] <= 0 || F.cyc[i] > 65535 || F.grn[i] < 0 || F.grn[i] > 65535))
      return fail(nullptr, SIM_EINVAL, "signal cycle must be 1..65535 ds and green 0..65535 ds");
  }
  for (int e = 0; e < F.nl; e++) {
    if (F.lanes[e] < 1 || F.lanes[e] > 8) return fail(nullptr, SIM_EINVAL, "lanes must be 1..8");
    if (!(F.len[e] > 0.0f) || !(F.spd[e] > 0.0f)) return fail(nullptr, SIM_EINVAL, "length and speed must be > 0");
    const float v0 = F.v0[F.cls[e]] > 0.0f ? F.v0[F.cls[e]] : F.spd[e];
    if (!(v0 > 0.0f)) return fail(nullptr, SIM_EINVAL, "desired speed must be > 0");
  }

  sim_handle* h = new sim_handle();
  h->max_bytes = (size_t)P.max_device_bytes;
  h->nn = F.nn;
  h->nl = F.nl;
  h->nt = F.nt;
  h->ncls = F.ncls;
  h->cost_mode = P.cost_mode;
  h->loop = P.loop_routes ? 1 : 0;
  h->lfrom = F.lf;
  h->lto = F.lt;
  h->len = F.len;
  h->spd = F.spd;
  h->lanes = F.lanes;
  h->depart = F.dep;
  h->origin = F.orig;
  h->dest = F.dest;
  h->hseed = F.hseed;
  cudaGetDevice(&h->device);
  cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  if (h->sm_count <= 0) h->sm_count = 1;
  h->grid = h->sm_count * 8;
  h->d.wait_limit = kDefaultWaitCycles;
  {
    // one resident wave of chunk-taking blocks per variant of the chunk kernel
    int bps[8];
    chunk_setup(bps);
    for (int v = 0; v < 8; v++) h->d.chunk_grid[v] = std::max(1, bps[v]) * h->sm_count;
    int fbs[2];
    front_setup(fbs);
    for (int v = 0; v < 2; v++) h->d.front_grid[v] = std::max(1, fbs[v]) * h->sm_count;
  }

  // in-links of every node in ascending link id -> round-robin index, in-degree
  std::vector<int> n_in(F.nn, 0), in_index(F.nl, 0);
  for (int e = 0; e < F.nl; e++) in_index[e] = n_in[F.lt[e]]++;
  for (int i = 0; i < F.nn; i++)
    if (n_in[i] > 255) {
      delete h;
      return fail(nullptr, SIM_EINVAL, "node in-degree above 255");
    }
  std::vector<LinkRec> recs(F.nl);
  h->lane_base.resize(F.nl + 1);
  h->lane_m.resize(F.nl);
  int nlan = 0;
  for (int e = 0; e < F.nl; e++) {
    LinkRec& r = recs[e];
    memset(&r, 0, sizeof(r));
    r.len = F.len[e];
    r.v0 = F.v0[F.cls[e]] > 0.0f ? F.v0[F.cls[e]] : F.spd[e];
    r.lane_base = nlan;
    h->lane_base[e] = nlan;
    nlan += F.lanes[e];
    const int n = F.lt[e];
    r.to = n;
    r.lanes = F.lanes[e];
    r.cls = F.cls[e];
    r.ctrl = F.ctrl[n];
    long long dx = (long long)F.nx[n] - F.nx[F.lf[e]], dy = (long long)F.ny[n] - F.ny[F.lf[e]];
    r.ew = (llabs(dx) >= llabs(dy)) ? 1 : 0;
    r.in_index = (uint8_t)in_index[e];
    r.n_in = (uint8_t)n_in[n];
    r.sig_cyc = (uint16_t)(F.ctrl[n] == SIM_CTRL_SIGNAL ? F.cyc[n] : 1);
    r.sig_off = F.off[n];
    r.sig_grn = (uint16_t)(F.ctrl[n] == SIM_CTRL_SIGNAL ? F.grn[n] : 0);
    if (F.ctrl[n] == SIM_CTRL_STOP) h->has_stop = true;
    h->lane_m[e] = (double)F.len[e] * (double)F.lanes[e];
    h->max_len = std::max(h->max_len, (double)F.len[e]);
  }
  h->lane_base[F.nl] = nlan;
  h->n_lanes = nlan;
  std::vector<ClassPar> cp(F.ncls);
  std::vector<uint8_t> v0p(F.ncls);
  for (int c = 0; c < F.ncls; c++) {
    float sab = sqrtf(F.a[c] * F.b[c]);
    cp[c] = ClassPar{F.a[c], 2.0f * sab, F.T[c], F.s0[c]};
    v0p[c] = F.v0[c] > 0.0f ? 1 : 0;
  }
  h->v0c = F.v0; h->Tc = F.T; h->ac = F.a; h->bc = F.b; h->s0c = F.s0;
  h->spd_link = F.spd;
  h->cls_link = F.cls;
  h->recs = recs;
  // mandatory-switch table: tau[k] = sqrt(-ln((k + 0.5) / 256)) in binary64, rounded once
  std::vector<float> tau(256);
  for (int k = 0; k < 256; k++) tau[k] = (float)std::sqrt(-std::log(((double)k + 0.5) / 256.0));

  Dev& d = h->d;
  int rc = SIM_OK;
#define TRY(x)            \
  do {                    \
    rc = (x);             \
    if (rc) goto fail_rc; \
  } while (0)
  {
    LinkRec* links;
    ClassPar* cls;
    float* taud;
    TRY(upload(h, &links, recs.data(), recs.size()));
    TRY(upload(h, &cls, cp.data(), cp.size()));
    TRY(upload(h, &taud, tau.data(), tau.size()));
    float* clsb;
    uint8_t* clsv0;
    TRY(upload(h, &clsb, F.b.data(), F.b.size()));
    TRY(upload(h, &clsv0, v0p.data(), v0p.size()));
    d.cls_b = clsb;
    d.cls_v0_param = clsv0;
    d.links = links;
    d.cls = cls;
    d.tau = taud;
    int32_t *lf, *nx, *ny, *dep;
    unsigned long long* hs;
    TRY(upload(h, &lf, F.lf.data(), F.lf.size()));
    TRY(upload(h, &nx, F.nx.data(), F.nx.size()));
    TRY(upload(h, &ny, F.ny.data(), F.ny.size()));
    TRY(upload(h, &dep, F.dep.data(), F.dep.size()));
    TRY(upload(h, &hs, F.hseed.data(), F.hseed.size()));
    d.lfrom = lf;
    d.node_x = nx;
    d.node_y = ny;
    d.depart = dep;
    d.hseed = hs;
    d.n_links = F.nl;
    d.n_nodes = F.nn;
    d.n_lanes = nlan;
    d.n_trips = F.nt;
    d.n_cls = F.ncls;
    d.dt = P.dt;
    d.hdt2 = (0.5f * P.dt) * P.dt;
    d.vlen = P.veh_len;
    d.vlen_max = P.veh_len;
    d.chunk_split = chunk_split_needed(h->lane_m.data(), F.nl, P.veh_len) ? 1 : 0;
    d.rank_long = rank_long_needed(h->max_len, P.veh_len) ? 1 : 0;
    d.s_min = P.s_min;
    d.zone = 2.0f * P.veh_len;
    d.mp = P.mobil_p;
    d.mathr = P.mobil_athr;
    d.mbsafe = P.mobil_bsafe;
    d.mbias = P.mobil_bias_right;
    d.lam = P.lambda_mand;
    d.stop_acq = P.stop_acquire_m;
    d.dt_ds = dt_ds;
    d.loop = h->loop;
    const size_t nt = (size_t)F.nt;
    TRY(dalloc(h, &d.status, nt));
    TRY(dalloc(h, &d.ins_step, nt));
    TRY(dalloc(h, &d.arr_step, nt));
    TRY(dalloc(h, &d.adec, nt));
    int32_t *roff, *rlen;
    TRY(dalloc(h, &roff, nt));
    TRY(dalloc(h, &rlen, nt));
    d.roff = roff;
    d.rlen = rlen;
    VehBuf* bufs[2] = {&d.A, &d.B};
    // per-slot arrays carry kSlotPad spare elements: tiled bulk copies of the sorted
    // state may read up to one tile past the last vehicle
    const size_t ntp = nt + kSlotPad;
    for (VehBuf* b : bufs) {
      TRY(dalloc(h, &b->x, ntp));
      TRY(dalloc(h, &b->v, ntp));
      TRY(dalloc(h, &b->vid, ntp));
      TRY(dalloc(h, &b->link, ntp));
      TRY(dalloc(h, &b->nxt, ntp));
      TRY(dalloc(h, &b->cur, ntp));
      TRY(dalloc(h, &b->lane, ntp));
      TRY(dalloc(h, &b->gid, ntp));
      TRY(dalloc(h, &b->mv, ntp));
    }
    TRY(dalloc(h, &d.aidx, nt));
    TRY(dalloc(h, &d.tx, nt));
    TRY(dalloc(h, &d.tvid, nt));
    TRY(dalloc(h, &d.tsrc, nt));
    TRY(dalloc(h, &d.tg, ntp));
    TRY(dalloc(h, &d.a_own, ntp));
    TRY(dalloc(h, &d.xo, nt));
    TRY(dalloc(h, &d.at, nt));
    TRY(dalloc(h, &d.intent, nt));
    TRY(dalloc(h, &d.flags, ntp));
    TRY(dalloc(h, &d.cnt, (size_t)nlan));
    // 8 spare entries: the chunk kernel stages lane starts in copies rounded up to 4
    TRY(dalloc(h, &d.lane_start, (size_t)nlan + 8));
    TRY(dalloc(h, &d.bsum, (size_t)scan_blocks(nlan) + 1));
    TRY(dalloc(h, &d.best, (size_t)nlan));
    TRY(dalloc(h, &d.rear, (size_t)nlan));
    TRY(dalloc(h, &d.fr, (size_t)nlan));
    TRY(dalloc(h, &d.cr, (size_t)nlan));
    TRY(dalloc(h, &d.chunks, chunk_table_size(F.nt)));
    TRY(dalloc(h, &d.long_list, (size_t)nlan));
    TRY(dalloc(h, &d.big_chunks, chunk_table_size(F.nt)));
    {
      std::vector<int32_t> ll((size_t)nlan);
      for (int e = 0; e < F.nl; e++)
        for (int l = 0; l < F.lanes[e]; l++) ll[(size_t)h->lane_base[e] + l] = e;
      int32_t* dll;
      TRY(upload(h, &dll, ll.data(), ll.size()));
      d.lane_link = dll;
    }
    TRY(dalloc(h, &d.elig, nt));
    TRY(dalloc(h, &d.holder, (size_t)F.nn));
    TRY(dalloc(h, &d.acq, (size_t)F.nn));
    TRY(dalloc(h, &d.ctl, 1));
    TRY(dalloc(h, &h->gs, 1));
    if (cudaMemset(d.cnt, 0, (size_t)nlan * 4) != cudaSuccess ||
        cudaMemset(d.best, 0xFF, (size_t)nlan * 8) != cudaSuccess ||
        cudaMemset(d.rear, 0, (size_t)nlan * sizeof(RearRec)) != cudaSuccess ||
        cudaMemset(d.at, 0, nt ? nt * 4 : 4) != cudaSuccess ||
        cudaMemset(d.a_own, 0, nt ? nt * 4 : 4) != cudaSuccess ||
        cudaMemset(d.xo, 0, nt ? nt * 4 : 4) != cudaSuccess ||
        cudaMemset(d.intent, 0, nt ? nt : 1) != cudaSuccess ||
        cudaMemset(d.flags, 0, nt ? nt : 1) != cudaSuccess ||
        cudaMemset(d.acq, 0xFF, (size_t)F.nn * 8) != cudaSuccess ||
        cudaMemset(d.holder, 0xFF, (size_t)F.nn * 4) != cudaSuccess ||
        cudaMemset(d.ctl, 0, sizeof(Ctl)) != cudaSuccess || cudaMemset(h->gs, 0, sizeof(GridSync)) != cudaSuccess ||
        cudaMemset(d.A.link, 0xFF, nt ? nt * 4 : 4) != cudaSuccess ||
        cudaMemset(d.status, 0, nt ? nt : 1) != cudaSuccess) {
      rc = fail(h, SIM_ECUDA, "initial cudaMemset failed");
      goto fail_rc;
    }
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      rc = fail(h, SIM_ECUDA, "cudaStreamCreate failed");
      goto fail_rc;
    }
    TRY(dalloc(h, &h->d_counts, 3));
    if (cudaMallocHost(&h->mirror, sizeof(HostMirror)) != cudaSuccess) {
      h->mirror = nullptr;
      rc = fail(h, SIM_ENOMEM, "cudaMallocHost of the control-block mirror failed");
      goto fail_rc;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
      rc = fail(h, SIM_ECUDA, "device synchronize after create failed");
      goto fail_rc;
    }
  }
  *out = h;
  return SIM_OK;
fail_rc:
  g_create_error = h->err;
  sim_destroy(h);
  return rc;
#undef TRY
}

// ------------------------------------------------------------------ queues
// Departure queues: per first link, the trips still pending in (depart_step, vid) order.
int build_queues(sim_handle* h, const std::vector<uint8_t>& status) {
  const int nt = h->nt, nl = h->nl;
  std::vector<int32_t> first(nt > 0 ? nt : 1);
  if (nt > 0) {
    int32_t* dfirst;
    int rc = dalloc(h, &dfirst, (size_t)nt);
    if (rc) return rc;
    launch_first_links(h->d.roff, h->routes, nt, dfirst, h->stream);
    cudaError_t e = cudaMemcpyAsync(first.data(), dfirst, (size_t)nt * 4, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dfree(h, dfirst);
    if (e != cudaSuccess) return cuda_fail(h, e, "first links");
  }
  // stable counting sort by depart_step (vid order kept), then stable by first link
  std::vector<int32_t> order;
  order.reserve(nt);
  for (int i = 0; i < nt; i++)
    if (status[i] == SIM_PENDING) order.push_back(i);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return h->depart[a] < h->depart[b]; });
  std::vector<int32_t> qstart(nl + 1, 0);
  for (int i : order) qstart[first[i] + 1]++;
  for (int e = 0; e < nl; e++) qstart[e + 1] += qstart[e];
  std::vector<int32_t> items(order.size() > 0 ? order.size() : 1), fill(qstart.begin(), qstart.end() - 1);
  for (int i : order) items[fill[first[i]]++] = i;
  std::vector<int32_t> qend(nl), qhead(nl), ql;
  for (int e = 0; e < nl; e++) {
    qhead[e] = qstart[e];
    qend[e] = qstart[e + 1];
    if (qend[e] > qhead[e]) ql.push_back(e);
  }
  dfree(h, h->q_items);
  dfree(h, h->q_end);
  dfree(h, h->q_head);
  dfree(h, h->qlinks);
  h->q_items = h->q_end = h->q_head = h->qlinks = nullptr;
  int rc;
  if ((rc = upload(h, &h->q_items, items.data(), items.size()))) return rc;
  if ((rc = upload(h, &h->q_end, qend.data(), qend.size()))) return rc;
  if ((rc = upload(h, &h->q_head, qhead.data(), qhead.size()))) return rc;
  if ((rc = upload(h, &h->qlinks, ql.data(), ql.size()))) return rc;
  h->d.q_items = h->q_items;
  h->d.q_end = h->q_end;
  h->d.q_head = h->q_head;
  h->d.qlinks = h->qlinks;
  h->d.n_qlinks = (int)ql.size();
  h->graph_dirty = true;
  h->pgraph_n = -1;
  h->tape_graph_dirty = true;
  return SIM_OK;
}

// Reset the dynamic state: all trips pending, no vehicles, t = 0.
// Measured outputs restart: totals at zero, no link entered yet, sampling windows
// empty from the first sampling instant at or after step t (t < 0: read it).
int clear_outputs(sim_handle* h, long long t) {
  Dev& d = h->d;
  const size_t nt = (size_t)std::max(1, h->nt), nl = (size_t)std::max(1, h->nl);
  if (d.emis) CK(cudaMemsetAsync(d.emis, 0, nt * 16, h->stream));
  if (d.enter) {
    CK(cudaMemsetAsync(d.enter, 0xFF, nt * 4, h->stream));
    CK(cudaMemsetAsync(d.tt_sum, 0, nl * 8, h->stream));
    CK(cudaMemsetAsync(d.tt_n, 0, nl * 4, h->stream));
  }
  if (d.acc_u) {
    CK(cudaMemsetAsync(d.acc_u, 0, nl * 8, h->stream));
    CK(cudaMemsetAsync(d.acc_s, 0, nl * 8, h->stream));
    CK(cudaMemsetAsync(d.out_u, 0, (size_t)d.samp_max * nl * 8, h->stream));
    CK(cudaMemsetAsync(d.out_s, 0, (size_t)d.samp_max * nl * 8, h->stream));
    CK(cudaMemsetAsync(d.out_n, 0, (size_t)d.samp_max * 4, h->stream));
    if (t < 0) {
      CK(cudaMemcpyAsync(&t, &d.ctl->t, sizeof(t), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
    }
    const long long k0 = (t + d.samp_every - 1) / d.samp_every;
    CK(cudaMemcpyAsync(&d.ctl->samp_k0, &k0, sizeof(k0), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return SIM_OK;
}

int reset_dynamic(sim_handle* h) {
  Dev& d = h->d;
  h->state_lost = false;
  h->t_known = false;
  const size_t nt = (size_t)h->nt;
  CK(cudaMemsetAsync(d.status, 0, nt ? nt : 1, h->stream));
  CK(cudaMemsetAsync(d.ins_step, 0xFF, (nt ? nt : 1) * 4, h->stream));
  CK(cudaMemsetAsync(d.arr_step, 0xFF, (nt ? nt : 1) * 4, h->stream));
  CK(cudaMemsetAsync(d.adec, 0, nt ? nt : 1, h->stream));
  CK(cudaMemsetAsync(d.rear, 0, (size_t)h->n_lanes * sizeof(RearRec), h->stream));
  CK(cudaMemsetAsync(d.holder, 0xFF, (size_t)h->nn * 4, h->stream));
  CK(cudaMemsetAsync(d.acq, 0xFF, (size_t)h->nn * 8, h->stream));
  CK(cudaMemsetAsync(d.best, 0xFF, (size_t)h->n_lanes * 8, h->stream));
  CK(cudaMemsetAsync(d.cnt, 0, (size_t)h->n_lanes * 4, h->stream));
  CK(cudaMemsetAsync(d.ctl, 0, sizeof(Ctl), h->stream));
  // a persistent launch that timed out left its barrier counts behind
  CK(cudaMemsetAsync(h->gs, 0, sizeof(GridSync), h->stream));
  return clear_outputs(h, 0);
}

// Step times stay below 2^31 / dt_ds so that the device's 32-bit phase arithmetic is exact.
int check_horizon(sim_handle* h, int n_steps, long long* t_now = nullptr) {
  if (!h->t_known) {
    CK(cudaMemcpyAsync(&h->mirror->c, h->d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->t_host = h->mirror->c.t;
    h->t_known = true;
  }
  const long long t = h->t_host;
  if (t_now) *t_now = t;
  const long long limit = 2147483647LL / (h->d.dt_ds + 1);
  if (t + (long long)n_steps > limit) return fail(h, SIM_EINVAL, "simulation horizon beyond 2^31 deciseconds");
  const Dev& d = h->d;
  if (d.acc_u && n_steps > 0 && (t + n_steps - 1) / d.samp_every / d.samp_per >= d.samp_max)
    return fail(h, SIM_EINVAL, "edge-sample windows would run past max_windows");
  return SIM_OK;
}

int check_device(sim_handle* h) {
  CK(cudaMemcpyAsync(&h->mirror->c, h->d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const Ctl c = h->mirror->c;
  h->t_host = c.t;
  h->t_known = true;
  if (c.err) {
    char buf[160];
    snprintf(buf, sizeof buf, "device error word 0x%x (info %d) at step %lld", c.err, c.err_info, c.t);
    const int code = (c.err & kErrTimeout) ? SIM_ETIMEOUT : SIM_EDEVICE;
    if (code == SIM_ETIMEOUT) h->state_lost = true;
    // clear the word so that the handle stays usable after the caller resets the state
    CK(cudaMemsetAsync(&h->d.ctl->err, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return fail(h, code, buf);
  }
  return SIM_OK;
}

// Eq. 7 parameters per (class, vehicle type): the class's with a scaled by the type.
int upload_type_params(sim_handle* h) {
  const int nty = (int)h->vty_len.size();
  if (!nty) return SIM_OK;
  std::vector<ClassPar> cp((size_t)h->ncls * nty);
  for (int c = 0; c < h->ncls; c++)
    for (int k = 0; k < nty; k++) {
      const float a = h->ac[c] * h->vty_ascale[k];
      const float sab = sqrtf(a * h->bc[c]);
      cp[(size_t)c * nty + k] = ClassPar{a, 2.0f * sab, h->Tc[c], h->s0c[c]};
    }
  CK(cudaMemcpyAsync(const_cast<ClassPar*>(h->d.cls_ty), cp.data(), cp.size() * sizeof(ClassPar),
                     cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

// Eq. 4: t0 = d / s, in deciseconds rounded half up, at least 1 (binary64); cost_mode 1
// scales it by sqrt(lanes), the initial routing weight of Sec. 6.3.1.
int32_t free_flow_cost(const sim_handle* h, int e) {
  const double dd = (double)h->len[e], ss = (double)h->spd[e];
  const double tt = h->cost_mode == 1 ? ((10.0 * std::sqrt((double)h->lanes[e])) * dd) / ss : (10.0 * dd) / ss;
  double c = std::floor(tt + 0.5);
  if (c < 1.0) c = 1.0;
  if (c > 1.0e6) c = 1.0e6;
  return (int32_t)c;
}

// Rewrite the route store with every trip's route back to back (in trip order).
int compact_routes(sim_handle* h) {
  const int nt = h->nt;
  std::vector<int32_t> len(nt > 0 ? nt : 1), off(nt > 0 ? nt : 1);
  if (nt) CK(cudaMemcpy(len.data(), h->d.rlen, (size_t)nt * 4, cudaMemcpyDeviceToHost));
  unsigned long long total = 0;
  for (int i = 0; i < nt; i++) {
    off[i] = (int32_t)total;
    total += (unsigned long long)len[i];
  }
  if (total >= 2147483647ULL) return fail(h, SIM_EINVAL, "route store above 2^31 links");
  int32_t *dst = nullptr, *doff = nullptr;
  int rc = dalloc(h, &dst, (size_t)std::max<unsigned long long>(1, total));
  if (rc) return rc;
  if ((rc = dalloc(h, &doff, (size_t)std::max(1, nt)))) {
    dfree(h, dst);
    return rc;
  }
  if (nt) {
    CK(cudaMemcpy(doff, off.data(), (size_t)nt * 4, cudaMemcpyHostToDevice));
    launch_compact_routes(h->d.roff, h->d.rlen, h->routes, doff, dst, nt, h->stream);
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy(const_cast<int32_t*>(h->d.roff), doff, (size_t)nt * 4, cudaMemcpyDeviceToDevice));
  }
  dfree(h, doff);
  dfree(h, h->routes);
  h->routes = dst;
  h->route_cap = total;
  return SIM_OK;
}

// Trip planning (Sec. 6.3.1) for every trip, or, with sel, only for the trips with
// sel[i] set: their new routes are appended to a copy of the route store, which is
// then compacted; the other trips keep theirs.  Restarts the run.
// With flow (device, [n_links]): all-or-nothing mode, flow[e] = trips whose path uses e;
// routes and vehicle state are left as they are.
int route_impl(sim_handle* h, const int32_t* link_cost_ds, const std::vector<uint8_t>* sel,
               unsigned* flow = nullptr) {
  const int nn = h->nn, nl = h->nl, nt = h->nt;
  std::vector<int32_t> cost(nl);
  long long cmax = 1;
  for (int e = 0; e < nl; e++) {
    cost[e] = link_cost_ds ? link_cost_ds[e] : free_flow_cost(h, e);
    if (cost[e] < 1 || cost[e] > 1000000) return fail(h, SIM_EINVAL, "link costs must be 1..1e6 ds");
    cmax = std::max<long long>(cmax, cost[e]);
  }
  if ((long long)nn * cmax >= 2000000000LL) return fail(h, SIM_EINVAL, "path costs could overflow int32");
  for (int i = 0; i < nt; i++)
    if (h->origin[i] == h->dest[i]) return fail(h, SIM_EINVAL, "trip with origin == destination");
  // CSR of out-links and in-links (ascending link id), trips by origin
  std::vector<int32_t> os(nn + 1, 0), ol(nl), is(nn + 1, 0), il(nl), ts(nn + 1, 0), tl(nt > 0 ? nt : 1);
  for (int e = 0; e < nl; e++) {
    os[h->lfrom[e] + 1]++;
    is[h->lto[e] + 1]++;
  }
  for (int i = 0; i < nt; i++)
    if (!sel || (*sel)[i]) ts[h->origin[i] + 1]++;
  for (int v = 0; v < nn; v++) {
    os[v + 1] += os[v];
    is[v + 1] += is[v];
    ts[v + 1] += ts[v];
  }
  {
    std::vector<int32_t> fo(os.begin(), os.end() - 1), fi(is.begin(), is.end() - 1), ft(ts.begin(), ts.end() - 1);
    for (int e = 0; e < nl; e++) {
      ol[fo[h->lfrom[e]]++] = e;
      il[fi[h->lto[e]]++] = e;
    }
    for (int i = 0; i < nt; i++)
      if (!sel || (*sel)[i]) tl[ft[h->origin[i]]++] = i;
  }
  std::vector<int32_t> origins;
  for (int v = 0; v < nn; v++)
    if (ts[v + 1] > ts[v]) origins.push_back(v);
  long long csum = 0;
  for (int e = 0; e < nl; e++) csum += cost[e];
  // bucket width of the near-far search: eight mean link costs (fewer far-pile splits
  // for a few more re-relaxations inside a bucket; measured fastest on the metro; the
  // distances, and so the routes, do not depend on it).  Below INT_MAX - 2e9 since a
  // link costs at most 1e6.
  const int delta = (int)std::max<long long>(1, 8 * csum / std::max(1, nl));

  // four trees in flight per SM (one per 256-thread block): a tree's rounds are short and
  // synchronous, so more trees hide more of their latency
  const int n_cta = std::max(1, std::min<int>((int)origins.size(), h->sm_count * 4));
  std::vector<void*> tmp;
  auto talloc = [&](auto** p, size_t n) -> int {
    int rc = dalloc(h, p, n);
    if (!rc) tmp.push_back(*p);
    return rc;
  };
  auto cleanup = [&]() {
    for (void* p : tmp) dfree(h, p);
    tmp.clear();
  };

  RouteDev R{};
  int rc = SIM_OK;
  int32_t *dos, *dol, *dis, *dil, *dlt, *dcost, *dorig, *dts, *dtl, *ddest;
  if ((rc = talloc(&dos, os.size())) || (rc = talloc(&dol, ol.size())) || (rc = talloc(&dis, is.size())) ||
      (rc = talloc(&dil, il.size())) || (rc = talloc(&dlt, (size_t)nl)) || (rc = talloc(&dcost, (size_t)nl)) ||
      (rc = talloc(&dorig, origins.size() + 1)) || (rc = talloc(&dts, ts.size())) ||
      (rc = talloc(&dtl, tl.size())) || (rc = talloc(&ddest, (size_t)std::max(1, nt)))) {
    cleanup();
    return rc;
  }
  cudaMemcpy(dos, os.data(), os.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(dol, ol.data(), ol.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(dis, is.data(), is.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(dil, il.data(), il.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(dlt, h->lto.data(), (size_t)nl * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(dcost, cost.data(), (size_t)nl * 4, cudaMemcpyHostToDevice);
  if (!origins.empty()) cudaMemcpy(dorig, origins.data(), origins.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(dts, ts.data(), ts.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(dtl, tl.data(), tl.size() * 4, cudaMemcpyHostToDevice);
  if (nt) cudaMemcpy(ddest, h->dest.data(), (size_t)nt * 4, cudaMemcpyHostToDevice);
  const size_t per = (size_t)n_cta * (size_t)nn;
  unsigned long long* ddist;
  int32_t *qf, *ff, *qa, *qb, *fa, *fb, *cround;
  unsigned* cep;
  int* work;
  if ((rc = talloc(&ddist, per)) || (rc = talloc(&qf, per)) || (rc = talloc(&ff, per)) || (rc = talloc(&qa, per)) ||
      (rc = talloc(&qb, per)) || (rc = talloc(&fa, per)) || (rc = talloc(&fb, per)) ||
      (rc = talloc(&cround, (size_t)n_cta)) || (rc = talloc(&cep, (size_t)n_cta)) || (rc = talloc(&work, 1))) {
    cleanup();
    return rc;
  }
  cudaMemset(ddist, 0xFF, per * 8);
  cudaMemset(qf, 0, per * 4);
  cudaMemset(ff, 0, per * 4);
  cudaMemset(cround, 0, (size_t)n_cta * 4);
  cudaMemset(cep, 0, (size_t)n_cta * 4);
  R.nn = nn;
  R.nl = nl;
  R.out_start = dos;
  R.out_link = dol;
  R.in_start = dis;
  R.in_link = dil;
  R.lfrom = h->d.lfrom;
  R.lto = dlt;
  R.cost = dcost;
  R.origins = dorig;
  R.n_origins = (int)origins.size();
  R.otrip_start = dts;
  R.otrip_list = dtl;
  R.dest = ddest;
  R.dist = ddist;
  R.qflag = qf;
  R.fflag = ff;
  R.qa = qa;
  R.qb = qb;
  R.fa = fa;
  R.fb = fb;
  R.cta_epoch = cep;
  R.cta_round = cround;
  R.roff = const_cast<int32_t*>(h->d.roff);
  R.rlen = const_cast<int32_t*>(h->d.rlen);
  R.work = work;
  R.delta = delta;
  R.ctl = h->d.ctl;
  if (flow) {
    // counts on a scratch control block, so that the simulation's counters stay intact
    Ctl* fctl;
    if ((rc = talloc(&fctl, 1))) {
      cleanup();
      return rc;
    }
    R.ctl = fctl;
    R.routes = nullptr;
    R.cap = 0;
    R.flow = flow;
    cudaMemset(work, 0, 4);
    cudaMemset(fctl, 0, sizeof(Ctl));
    cudaMemset(flow, 0, (size_t)std::max(1, nl) * 4);
    if (cudaDeviceSynchronize() != cudaSuccess) {
      cleanup();
      return fail(h, SIM_ECUDA, "all-or-nothing setup failed");
    }
    if (R.n_origins > 0) launch_route(R, n_cta, h->stream);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    Ctl c{};
    if (e == cudaSuccess) e = cudaMemcpy(&c, fctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(h, e, "all-or-nothing kernel");
    if (c.err & kErrUnreach) {
      char buf[96];
      snprintf(buf, sizeof buf, "trip %d: destination unreachable", c.err_info);
      return fail(h, SIM_EUNREACHABLE, buf);
    }
    if (c.err) return fail(h, SIM_EDEVICE, "all-or-nothing path extraction failed");
    return SIM_OK;
  }
  // the kept routes (subset mode) stay at the front of the store, new ones follow
  int32_t* old_routes = nullptr;
  unsigned long long kept = 0;
  if (sel) {
    old_routes = h->routes;
    kept = h->route_cap;
    h->routes = nullptr;
  }
  unsigned long long n_new = 0;
  for (int i = 0; i < nt; i++) n_new += (!sel || (*sel)[i]) ? 1 : 0;
  // initial reservation of the route store; a second pass with the exact size follows if it overflows
  unsigned long long cap = kept + std::max<unsigned long long>(1024, std::max<unsigned long long>(1, n_new) * 96ULL);
  for (int attempt = 0; attempt < 2; attempt++) {
    dfree(h, h->routes);
    h->routes = nullptr;
    if ((rc = dalloc(h, &h->routes, cap))) {
      dfree(h, old_routes);
      if (sel) h->routed = false;   // the kept routes are gone with the failed store
      cleanup();
      return rc;
    }
    if (kept) cudaMemcpy(h->routes, old_routes, kept * 4, cudaMemcpyDeviceToDevice);
    R.routes = h->routes;
    R.cap = cap;
    cudaMemset(work, 0, 4);
    cudaMemset(h->d.ctl, 0, sizeof(Ctl));
    if (kept) cudaMemcpy(&h->d.ctl->route_cursor, &kept, sizeof(kept), cudaMemcpyHostToDevice);
    if (cudaDeviceSynchronize() != cudaSuccess) {
      dfree(h, old_routes);
      if (sel) h->routed = false;   // the kept routes are gone with the failed store
      cleanup();
      return fail(h, SIM_ECUDA, "route setup failed");
    }
    if (R.n_origins > 0) launch_route(R, n_cta, h->stream);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      dfree(h, old_routes);
      if (sel) h->routed = false;   // the kept routes are gone with the failed store
      cleanup();
      return cuda_fail(h, e, "route kernel");
    }
    Ctl c;
    cudaMemcpy(&c, h->d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
    if (c.err & kErrUnreach) {
      dfree(h, old_routes);
      if (sel) h->routed = false;   // the kept routes are gone with the failed store
      cleanup();
      char buf[96];
      snprintf(buf, sizeof buf, "trip %d: destination unreachable", c.err_info);
      return fail(h, SIM_EUNREACHABLE, buf);
    }
    if (c.err) {
      dfree(h, old_routes);
      if (sel) h->routed = false;   // the kept routes are gone with the failed store
      cleanup();
      return fail(h, SIM_EDEVICE, "route extraction failed");
    }
    h->route_cap = c.route_cursor;
    if (c.route_cursor <= cap) break;
    cap = c.route_cursor;
  }
  cleanup();
  if (sel) {
    dfree(h, old_routes);
    if ((rc = compact_routes(h))) return rc;
  }
  h->d.routes = h->routes;
  if ((rc = reset_dynamic(h))) return rc;
  std::vector<uint8_t> st(nt, SIM_PENDING);
  if ((rc = build_queues(h, st))) return rc;
  CK(cudaStreamSynchronize(h->stream));
  h->routed = true;
  h->graph_dirty = true;
  h->pgraph_n = -1;
  return SIM_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

int sim_create(const sim_network* net, const sim_demand* dem, const sim_params* par, sim_handle** out) {
  NvtxRange nvtx_("sim_create");
  if (!out) return fail(nullptr, SIM_EINVAL, "out is NULL");
  *out = nullptr;
  Flat F;
  int rc = flatten(1, &net, &dem, &par, F);
  if (rc) return rc;
  return create_from_flat(F, out);
}

int sim_create_batch(int32_t n, const sim_network* const* nets, const sim_demand* const* dems,
                     const sim_params* const* pars, sim_handle** out) {
  NvtxRange nvtx_("sim_create_batch");
  if (!out) return fail(nullptr, SIM_EINVAL, "out is NULL");
  *out = nullptr;
  Flat F;
  int rc = flatten(n, nets, dems, pars, F);
  if (rc) return rc;
  return create_from_flat(F, out);
}

int sim_set_stream(sim_handle* h, void* stream) {
  if (!h) return SIM_EINVAL;
  h->t_known = false;
  h->stream = (cudaStream_t)stream;
  return SIM_OK;
}

int sim_route(sim_handle* h, const int32_t* link_cost_ds) {
  NvtxRange nvtx_("sim_route");
  if (!h) return SIM_EINVAL;
  h->t_known = false;
  return route_impl(h, link_cost_ds, nullptr);
}

int sim_reroute(sim_handle* h, const int32_t* link_cost_ds, uint32_t fraction_q16, uint32_t round) {
  NvtxRange nvtx_("sim_reroute");
  if (!h || !link_cost_ds) return SIM_EINVAL;
  h->t_known = false;
  if (!h->routed) return fail(h, SIM_ESTATE, "sim_reroute before routes exist");
  if (fraction_q16 > 65536u) return fail(h, SIM_EINVAL, "fraction_q16 must be 0..65536");
  std::vector<uint8_t> sel(h->nt);
  for (int i = 0; i < h->nt; i++) sel[i] = reroute_selected(h->hseed[i], round, fraction_q16) ? 1 : 0;
  return route_impl(h, link_cost_ds, &sel);
}

int sim_set_routes(sim_handle* h, const int32_t* offsets, const int32_t* links) {
  NvtxRange nvtx_("sim_set_routes");
  if (!h || !offsets || !links) return SIM_EINVAL;
  h->t_known = false;
  const int nt = h->nt;
  if (offsets[0] != 0) return fail(h, SIM_EINVAL, "offsets[0] must be 0");
  for (int i = 0; i < nt; i++) {
    if (offsets[i + 1] <= offsets[i]) return fail(h, SIM_EINVAL, "every route needs at least one link");
    for (int k = offsets[i]; k < offsets[i + 1]; k++) {
      if (links[k] < 0 || links[k] >= h->nl) return fail(h, SIM_EINVAL, "route link out of range");
      if (k > offsets[i] && h->lfrom[links[k]] != h->lto[links[k - 1]])
        return fail(h, SIM_EINVAL, "route links are not connected");
    }
    if (h->loop && h->lto[links[offsets[i + 1] - 1]] != h->lfrom[links[offsets[i]]])
      return fail(h, SIM_EINVAL, "loop route is not a cycle");
  }
  const long long total = nt ? offsets[nt] : 0;
  std::vector<int32_t> off(nt > 0 ? nt : 1), len(nt > 0 ? nt : 1);
  for (int i = 0; i < nt; i++) {
    off[i] = offsets[i];
    len[i] = offsets[i + 1] - offsets[i];
  }
  dfree(h, h->routes);
  h->routes = nullptr;
  int rc = dalloc(h, &h->routes, (size_t)std::max<long long>(1, total));
  if (rc) return rc;
  if (total) CK(cudaMemcpy(h->routes, links, (size_t)total * 4, cudaMemcpyHostToDevice));
  if (nt) {
    CK(cudaMemcpy(const_cast<int32_t*>(h->d.roff), off.data(), (size_t)nt * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(const_cast<int32_t*>(h->d.rlen), len.data(), (size_t)nt * 4, cudaMemcpyHostToDevice));
  }
  h->route_cap = (unsigned long long)total;
  h->d.routes = h->routes;
  if ((rc = reset_dynamic(h))) return rc;
  std::vector<uint8_t> st(nt, SIM_PENDING);
  if ((rc = build_queues(h, st))) return rc;
  CK(cudaStreamSynchronize(h->stream));
  h->routed = true;
  h->graph_dirty = true;
  h->pgraph_n = -1;
  return SIM_OK;
}

int sim_route_size(sim_handle* h, int64_t* n_hops) {
  if (!h || !n_hops) return SIM_EINVAL;
  if (!h->routed) return fail(h, SIM_ESTATE, "no routes");
  std::vector<int32_t> len(h->nt);
  if (h->nt) CK(cudaMemcpy(len.data(), h->d.rlen, (size_t)h->nt * 4, cudaMemcpyDeviceToHost));
  int64_t s = 0;
  for (int32_t l : len) s += l;
  *n_hops = s;
  return SIM_OK;
}

int sim_read_routes(sim_handle* h, int32_t* offsets, int32_t* links) {
  if (!h || !offsets || !links) return SIM_EINVAL;
  if (!h->routed) return fail(h, SIM_ESTATE, "no routes");
  const int nt = h->nt;
  std::vector<int32_t> off(nt), len(nt), all((size_t)std::max<unsigned long long>(1, h->route_cap));
  if (nt) {
    CK(cudaMemcpy(off.data(), h->d.roff, (size_t)nt * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(len.data(), h->d.rlen, (size_t)nt * 4, cudaMemcpyDeviceToHost));
  }
  if (h->route_cap) CK(cudaMemcpy(all.data(), h->routes, (size_t)h->route_cap * 4, cudaMemcpyDeviceToHost));
  offsets[0] = 0;
  for (int i = 0; i < nt; i++) {
    memcpy(links + offsets[i], all.data() + off[i], (size_t)len[i] * 4);
    offsets[i + 1] = offsets[i] + len[i];
  }
  return SIM_OK;
}

int sim_step(sim_handle* h, int32_t n_steps) {
  NvtxRange nvtx_("sim_step");
  if (!h || n_steps < 0) return SIM_EINVAL;
  if (h->state_lost) return fail(h, SIM_ESTATE, "the state is undefined after a timeout: sim_write_state or sim_route first");
  if (!h->routed) return fail(h, SIM_ESTATE, "sim_step before sim_route / sim_set_routes");
  if (n_steps == 0) return SIM_OK;
  long long t0 = 0;
  if (int rc = check_horizon(h, n_steps, &t0)) return rc;
  if (h->graph_dirty) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->gexec_samp) cudaGraphExecDestroy(h->gexec_samp);
    if (h->graph_samp) cudaGraphDestroy(h->graph_samp);
    h->gexec = h->gexec_samp = nullptr;
    h->graph = h->graph_samp = nullptr;
    Dev dn = h->d;
    dn.acc_u = nullptr;   // steps between sampling instants skip the sample kernel
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    launch_step(dn, h->grid, h->has_stop, h->cap_stream);
    CK(cudaStreamEndCapture(h->cap_stream, &h->graph));
    CK(cudaGraphInstantiate(&h->gexec, h->graph, 0));
    CK(cudaGraphGetNodes(h->graph, nullptr, &h->graph_nodes));
    if (h->d.acc_u) {
      CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      launch_step(h->d, h->grid, h->has_stop, h->cap_stream);
      CK(cudaStreamEndCapture(h->cap_stream, &h->graph_samp));
      CK(cudaGraphInstantiate(&h->gexec_samp, h->graph_samp, 0));
      CK(cudaGraphGetNodes(h->graph_samp, nullptr, &h->graph_samp_nodes));
    }
    h->graph_dirty = false;
  }
  if (h->exec.mode == SIM_EXEC_PERSISTENT) {
    const int blocks = h->exec.blocks_per_sm * h->sm_count;
    const long long limit = h->exec.barrier_timeout_cycles > 0 ? h->exec.barrier_timeout_cycles : kDefaultWaitCycles;
    const sim_exec& x = h->exec;
    const bool same = h->pexec && h->pgraph_n == n_steps && h->pgraph_cfg.threads == x.threads &&
                      h->pgraph_cfg.blocks_per_sm == x.blocks_per_sm &&
                      h->pgraph_cfg.barrier_timeout_cycles == x.barrier_timeout_cycles;
    if (!same && !h->pgraph_unsupported) {
      // capture the single persistent launch as a graph (rebuilt when the step count or
      // the configuration changes); direct launch where capture is not available
      if (h->pexec) cudaGraphExecDestroy(h->pexec);
      if (h->pgraph) cudaGraphDestroy(h->pgraph);
      h->pexec = nullptr;
      h->pgraph = nullptr;
      bool ok = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        cudaError_t le = launch_persistent(h->d, h->gs, blocks, x.threads, n_steps, limit, h->cap_stream);
        cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &h->pgraph);
        ok = le == cudaSuccess && ce == cudaSuccess && h->pgraph &&
             cudaGraphInstantiate(&h->pexec, h->pgraph, 0) == cudaSuccess;
      }
      if (!ok) {
        cudaGetLastError();
        if (h->pgraph) cudaGraphDestroy(h->pgraph);
        h->pgraph = nullptr;
        h->pexec = nullptr;
        h->pgraph_unsupported = true;
      } else {
        h->pgraph_n = n_steps;
        h->pgraph_cfg = x;
      }
    }
    if (h->pexec) CK(cudaGraphLaunch(h->pexec, h->stream));
    else CK(launch_persistent(h->d, h->gs, blocks, x.threads, n_steps, limit, h->stream));
    h->launches += 1;
  } else {
    const long long every = h->d.acc_u ? h->d.samp_every : 0;
    for (int s = 0; s < n_steps; s++) {
      const bool samp = every > 0 && (t0 + s) % every == 0;
      CK(cudaGraphLaunch(samp ? h->gexec_samp : h->gexec, h->stream));
      h->launches += (long long)(samp ? h->graph_samp_nodes : h->graph_nodes);
    }
  }
  return check_device(h);
}

int sim_set_exec(sim_handle* h, const sim_exec* e) {
  if (!h || !e) return SIM_EINVAL;
  h->t_known = false;
  sim_exec x = *e;
  if (x.mode == SIM_EXEC_GRAPH) {
    if (x.grid_per_sm < 1 || x.grid_per_sm > 64) return fail(h, SIM_EINVAL, "grid_per_sm must be 1..64");
    h->grid = x.grid_per_sm * h->sm_count;
    h->d.wait_limit = x.barrier_timeout_cycles > 0 ? x.barrier_timeout_cycles : kDefaultWaitCycles;
    h->graph_dirty = true;
  h->pgraph_n = -1;
    h->tape_graph_dirty = true;
  } else if (x.mode == SIM_EXEC_PERSISTENT) {
    // the lane-start scan gives each block 2048 lanes, 8 to each of 256 threads
    if (x.threads != 256 && x.threads != 512 && x.threads != 1024)
      return fail(h, SIM_EINVAL, "persistent threads must be 256, 512 or 1024");
    const int mx = persistent_max_blocks_per_sm(x.threads);
    if (mx < 1) return fail(h, SIM_EINVAL, "the persistent kernel does not fit this block size");
    if (x.blocks_per_sm < 1 || x.blocks_per_sm > mx)
      return fail(h, SIM_EINVAL, "blocks_per_sm exceeds the co-resident limit of the persistent kernel");
  } else {
    return fail(h, SIM_EINVAL, "unknown execution mode");
  }
  h->exec = x;
  return SIM_OK;
}

int sim_get_exec(sim_handle* h, sim_exec* e) {
  if (!h || !e) return SIM_EINVAL;
  *e = h->exec;
  return SIM_OK;
}

int sim_step_timed(sim_handle* h, int32_t n_steps, float* kernel_ms) {
  NvtxRange nvtx_("sim_step_timed");
  if (!h || n_steps < 0 || !kernel_ms) return SIM_EINVAL;
  h->t_known = false;
  if (h->state_lost) return fail(h, SIM_ESTATE, "the state is undefined after a timeout: sim_write_state or sim_route first");
  if (!h->routed) return fail(h, SIM_ESTATE, "sim_step_timed before sim_route / sim_set_routes");
  if (int rc = check_horizon(h, n_steps)) return rc;
  CK(launch_steps_timed(h->d, h->grid, h->has_stop, h->stream, n_steps, kernel_ms));
  return check_device(h);
}

int sim_launch_count(sim_handle* h, int64_t* launches) {
  if (!h || !launches) return SIM_EINVAL;
  *launches = h->launches;
  return SIM_OK;
}

const char* sim_kernel_name(int32_t k) { return (k >= 0 && k < kNumKernels) ? kKernelNames[k] : ""; }

int sim_read_state(sim_handle* h, const sim_state_view* out, uint32_t fields, int on_device) {
  NvtxRange nvtx_("sim_read_state");
  if (!h || !out || on_device < 0 || on_device > 2) return SIM_EINVAL;
  const size_t nt = (size_t)h->nt;
  void* ptr[9] = {out->status, out->link, out->lane, out->cursor, out->x, out->v,
                  out->insert_step, out->arrive_step, out->lane_change};
  const size_t esz[9] = {1, 4, 4, 4, 4, 4, 4, 4, 1};
  void* dptr[9] = {nullptr};
  for (int f = 0; f < 9; f++) {
    if (!(fields & (1u << f))) continue;
    if (!ptr[f]) return fail(h, SIM_EINVAL, "requested field has a NULL pointer");
    if (on_device) {
      dptr[f] = ptr[f];
    } else {
      // device staging buffer of the field, allocated at its first host read and kept
      // for the handle's lifetime
      if (!h->stage[f]) {
        uint8_t* q;
        if (int rc = dalloc(h, &q, nt ? nt * esz[f] : 1)) return rc;
        h->stage[f] = q;
      }
      dptr[f] = h->stage[f];
    }
  }
  if (nt)
    launch_state_out(h->d, h->grid, h->stream, (uint8_t*)dptr[0], (int32_t*)dptr[1], (int32_t*)dptr[2],
                     (int32_t*)dptr[3], (float*)dptr[4], (float*)dptr[5], (int32_t*)dptr[6], (int32_t*)dptr[7],
                     (int8_t*)dptr[8]);
  cudaError_t e = cudaSuccess;
  if (!on_device)
    for (int f = 0; f < 9 && e == cudaSuccess; f++)
      if (dptr[f] && nt) e = cudaMemcpyAsync(ptr[f], dptr[f], nt * esz[f], cudaMemcpyDeviceToHost, h->stream);
  if (on_device == 2) {   // enqueued only
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "read_state");
    return SIM_OK;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "read_state");
  return SIM_OK;
}

int sim_write_state(sim_handle* h, const uint8_t* status, const int32_t* link, const int32_t* lane,
                    const int32_t* cursor, const float* x, const float* v) {
  NvtxRange nvtx_("sim_write_state");
  if (!h || !status || !link || !lane || !cursor || !x || !v) return SIM_EINVAL;
  h->t_known = false;
  if (!h->routed) return fail(h, SIM_ESTATE, "sim_write_state before routes exist");
  const int nt = h->nt;
  uint8_t* ds;
  int32_t *dl, *dn, *dc, *dbad;
  float *dx, *dv;
  const size_t n = (size_t)std::max(1, nt);
  int rc;
  if ((rc = dalloc(h, &ds, n)) || (rc = dalloc(h, &dl, n)) || (rc = dalloc(h, &dn, n)) || (rc = dalloc(h, &dc, n)) ||
      (rc = dalloc(h, &dx, n)) || (rc = dalloc(h, &dv, n)) || (rc = dalloc(h, &dbad, 1)))
    return rc;
  void* tl[7] = {ds, dl, dn, dc, dx, dv, dbad};
  auto release = [&]() {
    for (void* p : tl) dfree(h, p);
  };
  int bad = 0;
  cudaError_t e = cudaMemsetAsync(dbad, 0, 4, h->stream);
  if (nt && e == cudaSuccess) {
    const cudaMemcpyKind k = cudaMemcpyHostToDevice;
    e = cudaMemcpyAsync(ds, status, (size_t)nt, k, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dl, link, (size_t)nt * 4, k, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dn, lane, (size_t)nt * 4, k, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dc, cursor, (size_t)nt * 4, k, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dx, x, (size_t)nt * 4, k, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dv, v, (size_t)nt * 4, k, h->stream);
    if (e == cudaSuccess) launch_state_check(h->d, h->grid, h->stream, ds, dl, dn, dc, dx, dv, dbad);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, dbad, 4, cudaMemcpyDeviceToHost, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(h, e, "write_state upload");
  }
  if (bad) {
    release();
    return fail(h, SIM_EINVAL, std::to_string(bad) +
                                   " trips: status not 0..2, or active trip not on route[cursor] with a valid lane, "
                                   "0 <= x <= length and v >= 0");
  }
  if ((rc = reset_dynamic(h))) {
    release();
    return rc;
  }
  if (nt) {
    launch_state_in(h->d, h->grid, h->stream, ds, dl, dn, dc, dx, dv);
    launch_count(h->d, h->grid, h->stream);
  }
  e = cudaStreamSynchronize(h->stream);
  release();
  if (e != cudaSuccess) return cuda_fail(h, e, "write_state");
  std::vector<uint8_t> st(status, status + nt);
  if ((rc = build_queues(h, st))) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

int sim_occupancy(sim_handle* h, int32_t* lane_start, int32_t* sorted_vid) {
  if (!h || !lane_start || !sorted_vid) return SIM_EINVAL;
  h->t_known = false;
  if (!h->routed) return fail(h, SIM_ESTATE, "no routes");
  launch_occupancy(h->d, h->grid, h->stream);
  int32_t* dv;
  int rc = dalloc(h, &dv, (size_t)std::max(1, h->nt));
  if (rc) return rc;
  launch_occ_out(h->d, h->grid, h->stream, dv);
  cudaError_t e = cudaMemcpyAsync(lane_start, h->d.lane_start, ((size_t)h->n_lanes + 1) * 4,
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess && lane_start[h->n_lanes] > 0)
    e = cudaMemcpy(sorted_vid, dv, (size_t)lane_start[h->n_lanes] * 4, cudaMemcpyDeviceToHost);
  dfree(h, dv);
  if (e != cudaSuccess) return cuda_fail(h, e, "occupancy");
  return check_device(h);
}

int sim_n_lanes(sim_handle* h, int64_t* n) {
  if (!h || !n) return SIM_EINVAL;
  *n = h->n_lanes;
  return SIM_OK;
}

int sim_counters(sim_handle* h, sim_counters_t* out) {
  NvtxRange nvtx_("sim_counters");
  if (!h || !out) return SIM_EINVAL;
  // trip statuses counted on the device against the step counter there
  CK(cudaMemsetAsync(h->d_counts, 0, 3 * sizeof(unsigned long long), h->stream));
  launch_status_counts(h->d, h->grid, h->stream, h->d_counts);
  CK(cudaMemcpyAsync(&h->mirror->c, h->d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->mirror->counts, h->d_counts, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const Ctl c = h->mirror->c;
  const int64_t active = (int64_t)h->mirror->counts[0], waiting = (int64_t)h->mirror->counts[1],
                pending = (int64_t)h->mirror->counts[2];
  out->t = c.t;
  out->departed = (int64_t)c.departed;
  out->waiting = waiting;
  out->active = active;
  out->arrived = (int64_t)c.arrived;
  out->veh_steps = (int64_t)c.veh_steps;
  out->pending = pending;
  out->active_last = c.active_last;
  out->lc_evals = (int64_t)c.lc_evals;
  return SIM_OK;
}

int sim_set_class_params(sim_handle* h, const float* v0, const float* T, const float* a, const float* b,
                         const float* s0) {
  if (!h || !v0 || !T || !a || !b || !s0) return SIM_EINVAL;
  h->t_known = false;
  for (int c = 0; c < h->ncls; c++)
    if (!(a[c] > 0.0f) || !(b[c] > 0.0f) || !(T[c] >= 0.0f) || !(s0[c] >= 0.0f) ||
        ((h->v0c[c] > 0.0f) != (v0[c] > 0.0f)))
      return fail(h, SIM_EINVAL, "class parameters need a > 0, b > 0, T >= 0, s0 >= 0, and v0 > 0 exactly for "
                                 "the classes created with v0 > 0");
  std::vector<ClassPar> cp(h->ncls);
  for (int c = 0; c < h->ncls; c++) {
    h->v0c[c] = v0[c]; h->Tc[c] = T[c]; h->ac[c] = a[c]; h->bc[c] = b[c]; h->s0c[c] = s0[c];
    float sab = sqrtf(a[c] * b[c]);
    cp[c] = ClassPar{a[c], 2.0f * sab, T[c], s0[c]};
  }
  for (int e = 0; e < h->nl; e++) {
    const int c = h->cls_link[e];
    h->recs[e].v0 = h->v0c[c] > 0.0f ? h->v0c[c] : h->spd_link[e];
  }
  CK(cudaMemcpyAsync(const_cast<ClassPar*>(h->d.cls), cp.data(), cp.size() * sizeof(ClassPar),
                     cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(const_cast<float*>(h->d.cls_b), h->bc.data(), h->bc.size() * 4, cudaMemcpyHostToDevice,
                     h->stream));
  CK(cudaMemcpyAsync(const_cast<LinkRec*>(h->d.links), h->recs.data(), h->recs.size() * sizeof(LinkRec),
                     cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return upload_type_params(h);
}

int sim_set_vehicle_types(sim_handle* h, int32_t n_types, const sim_vehicle_type* types, const uint8_t* trip_type) {
  if (!h || n_types < 0 || n_types > SIM_MAX_VEHICLE_TYPES) return SIM_EINVAL;
  h->t_known = false;
  if (n_types > 0 && (!types || (!trip_type && h->nt > 0))) return SIM_EINVAL;
  for (int k = 0; k < n_types; k++)
    if (!(types[k].length_m > 0.0f) || !(types[k].accel_scale > 0.0f) || !(types[k].max_speed_mps > 0.0f))
      return fail(h, SIM_EINVAL, "vehicle types need length, accel_scale and max_speed > 0");
  for (int i = 0; n_types > 0 && i < h->nt; i++)
    if (trip_type[i] >= n_types) return fail(h, SIM_EINVAL, "trip type out of range");
  Dev& d = h->d;
  void* olds[] = {const_cast<uint8_t*>(d.vtype), const_cast<ClassPar*>(d.cls_ty), const_cast<float*>(d.vty_len),
                  const_cast<float*>(d.vty_vmax)};
  for (void* q : olds) dfree(h, q);
  d.vtype = nullptr;
  d.cls_ty = nullptr;
  d.vty_len = d.vty_vmax = nullptr;
  d.n_vty = 0;
  d.vlen_max = d.vlen;
  d.chunk_split = chunk_split_needed(h->lane_m.data(), h->nl, d.vlen) ? 1 : 0;
  d.rank_long = rank_long_needed(h->max_len, d.vlen) ? 1 : 0;
  h->vty_len.clear();
  h->vty_ascale.clear();
  h->vty_vmax.clear();
  h->graph_dirty = true;
  h->pgraph_n = -1;
  h->tape_graph_dirty = true;
  if (n_types == 0) return SIM_OK;
  for (int k = 0; k < n_types; k++) {
    h->vty_len.push_back(types[k].length_m);
    h->vty_ascale.push_back(types[k].accel_scale);
    h->vty_vmax.push_back(types[k].max_speed_mps);
  }
  uint8_t* vt;
  ClassPar* ct;
  float *vl, *vm;
  int rc;
  if ((rc = upload(h, &vt, trip_type, (size_t)h->nt)) || (rc = dalloc(h, &ct, (size_t)h->ncls * n_types)) ||
      (rc = upload(h, &vl, h->vty_len.data(), (size_t)n_types)) ||
      (rc = upload(h, &vm, h->vty_vmax.data(), (size_t)n_types)))
    return rc;
  d.vtype = vt;
  d.cls_ty = ct;
  d.vty_len = vl;
  d.vty_vmax = vm;
  d.n_vty = n_types;
  d.vlen_max = *std::max_element(h->vty_len.begin(), h->vty_len.end());
  const float vmin = *std::min_element(h->vty_len.begin(), h->vty_len.end());
  d.chunk_split = chunk_split_needed(h->lane_m.data(), h->nl, vmin) ? 1 : 0;
  d.rank_long = rank_long_needed(h->max_len, vmin) ? 1 : 0;
  return upload_type_params(h);
}

int sim_observe(sim_handle* h, int32_t n_steps, int32_t obs_every, double* progress) {
  NvtxRange nvtx_("sim_observe");
  if (!h || !progress || obs_every <= 0 || n_steps < 0) return SIM_EINVAL;
  h->t_known = false;
  if (h->state_lost) return fail(h, SIM_ESTATE, "the state is undefined after a timeout: sim_write_state or sim_route first");
  if (!h->routed) return fail(h, SIM_ESTATE, "sim_observe before routes exist");
  const int nobs = n_steps / obs_every;
  const size_t nt = (size_t)h->nt;
  double* dp;
  int rc = dalloc(h, &dp, std::max<size_t>(1, nt));
  if (rc) return rc;
  for (int k = 0; k < nobs; k++) {
    if ((rc = sim_step(h, obs_every))) break;
    launch_observe(h->d, h->grid, h->stream, nullptr, nullptr, dp);
    cudaError_t e = cudaMemcpyAsync(progress + (size_t)k * nt, dp, nt * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      rc = cuda_fail(h, e, "observe");
      break;
    }
  }
  dfree(h, dp);
  return rc;
}

int sim_loss(sim_handle* h, const sim_loss_spec* spec, double* loss_out) {
  NvtxRange nvtx_("sim_loss");
  if (!h || !spec || !loss_out || !spec->target) return SIM_EINVAL;
  h->t_known = false;
  if (h->state_lost) return fail(h, SIM_ESTATE, "the state is undefined after a timeout: sim_write_state or sim_route first");
  if (!h->routed) return fail(h, SIM_ESTATE, "sim_loss before routes exist");
  const int n_steps = spec->n_steps, every = spec->obs_every;
  if (n_steps <= 0 || every <= 0 || n_steps % every) return fail(h, SIM_EINVAL, "n_steps must be a multiple of obs_every");
  if (int rc = check_horizon(h, n_steps)) return rc;
  h->t_known = false;
  const int nobs = n_steps / every;
  const size_t nt = (size_t)std::max(1, h->nt);
  double *tgt, *res;
  int rc = dalloc(h, &tgt, (size_t)nobs * nt);
  if (rc) return rc;
  if ((rc = dalloc(h, &res, nt))) {
    dfree(h, tgt);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(tgt, spec->target, (size_t)nobs * nt * 8, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(&h->d.ctl->loss, 0, 8, h->stream);
  if (e != cudaSuccess) rc = cuda_fail(h, e, "loss");
  for (int k = 0; k < nobs && rc == SIM_OK; k++) {
    if ((rc = sim_step(h, every))) break;
    launch_observe(h->d, h->grid, h->stream, tgt + (size_t)k * nt, res, nullptr);
  }
  if (rc == SIM_OK) {
    e = cudaMemcpyAsync(loss_out, &h->d.ctl->loss, 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(h, e, "loss");
  }
  dfree(h, tgt);
  dfree(h, res);
  if (rc) return rc;
  return check_device(h);
}

namespace {

// Everything a step changes, for the adjoint's checkpoints.
struct CkptLayout {
  size_t nt, nn, nl, nlan, bytes;
};

CkptLayout ckpt_layout(const sim_handle* h) {
  CkptLayout L;
  L.nt = (size_t)std::max(1, h->nt);
  L.nn = (size_t)h->nn;
  L.nl = (size_t)h->nl;
  L.nlan = (size_t)h->n_lanes;
  L.bytes = L.nt * (8 * 4 + 1 + 1 + 4 + 4 + 1 + 4) + L.nn * 4 + L.nl * 4 + L.nlan * 4 + sizeof(Ctl) + 64;
  return L;
}

cudaError_t ckpt_copy(sim_handle* h, unsigned char* buf, bool save) {
  const CkptLayout L = ckpt_layout(h);
  Dev& d = h->d;
  struct Item { void* p; size_t n; } items[] = {
      {d.A.x, L.nt * 4}, {d.A.v, L.nt * 4}, {d.A.vid, L.nt * 4}, {d.A.link, L.nt * 4}, {d.A.nxt, L.nt * 4},
      {d.A.cur, L.nt * 4}, {d.A.lane, L.nt * 4}, {d.A.gid, L.nt * 4}, {d.A.mv, L.nt}, {d.status, L.nt}, {d.ins_step, L.nt * 4}, {d.arr_step, L.nt * 4},
      {d.adec, L.nt}, {d.aidx, L.nt * 4}, {d.holder, L.nn * 4}, {h->q_head, L.nl * 4}, {d.cnt, L.nlan * 4},
      {d.ctl, sizeof(Ctl)}};
  size_t off = 0;
  for (const Item& it : items) {
    if (!it.p || !it.n) continue;
    cudaError_t e = save ? cudaMemcpyAsync(buf + off, it.p, it.n, cudaMemcpyDeviceToDevice, h->stream)
                         : cudaMemcpyAsync(it.p, buf + off, it.n, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return e;
    off += it.n;
  }
  if (!save) {
    h->t_known = false;   // the restored step counter
    // epoch-tagged keys written after the checkpoint would outrank the replayed steps' keys
    cudaError_t e = cudaMemsetAsync(d.best, 0xFF, L.nlan * 8, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.acq, 0xFF, L.nn * 8, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.rear, 0, L.nlan * sizeof(RearRec), h->stream);
    return e;
  }
  return cudaSuccess;
}

}  // namespace

int sim_adjoint(sim_handle* h, const sim_loss_spec* spec, double* grad_out, double* loss_out) {
  NvtxRange nvtx_("sim_adjoint");
  if (!h || !spec || !grad_out || !loss_out || !spec->target) return SIM_EINVAL;
  h->t_known = false;
  if (h->state_lost) return fail(h, SIM_ESTATE, "the state is undefined after a timeout: sim_write_state or sim_route first");
  if (!h->routed) return fail(h, SIM_ESTATE, "sim_adjoint before routes exist");
  if (h->out_flags) return fail(h, SIM_ESTATE, "sim_adjoint with measured outputs on (sim_set_outputs(h, 0, NULL))");
  if (h->d.vtype) return fail(h, SIM_ESTATE, "sim_adjoint covers the single vehicle class (sim_set_vehicle_types(h, 0, ...))");
  const int n_steps = spec->n_steps, every = spec->obs_every;
  const int seg = spec->checkpoint_every > 0 ? spec->checkpoint_every : 64;
  if (n_steps <= 0 || every <= 0 || n_steps % every) return fail(h, SIM_EINVAL, "n_steps must be a multiple of obs_every");
  if (int rc = check_horizon(h, n_steps)) return rc;
  h->t_known = false;   // the passes below advance and restore the step counter
  const int nobs = n_steps / every, nseg = (n_steps + seg - 1) / seg;
  const size_t nt = (size_t)std::max(1, h->nt);
  // sim_step's graph
  int rc = sim_step(h, 0);
  if (rc) return rc;
  if (h->graph_dirty) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    launch_step(h->d, h->grid, h->has_stop, h->cap_stream);
    CK(cudaStreamEndCapture(h->cap_stream, &h->graph));
    CK(cudaGraphInstantiate(&h->gexec, h->graph, 0));
    h->graph_dirty = false;
  }
  // tape of one segment and its graph
  if (h->tape_steps != seg || !h->tape) {
    dfree(h, h->tape);
    dfree(h, h->tform);
    h->tape = nullptr;
    h->tform = nullptr;
    if ((rc = dalloc(h, &h->tape, (size_t)seg * nt))) return rc;
    if ((rc = dalloc(h, &h->tform, nt))) return rc;
    h->tape_steps = seg;
    h->tape_graph_dirty = true;
  }
  if (h->tape_graph_dirty) {
    if (h->gexec_tape) cudaGraphExecDestroy(h->gexec_tape);
    if (h->graph_tape) cudaGraphDestroy(h->graph_tape);
    h->gexec_tape = nullptr;
    h->graph_tape = nullptr;
    Dev dt = h->d;
    dt.tape = h->tape;
    dt.tform = h->tform;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    launch_step(dt, h->grid, h->has_stop, h->cap_stream);
    CK(cudaStreamEndCapture(h->cap_stream, &h->graph_tape));
    CK(cudaGraphInstantiate(&h->gexec_tape, h->graph_tape, 0));
    h->tape_graph_dirty = false;
  }
  Dev dtape = h->d;
  dtape.tape = h->tape;
  dtape.tform = h->tform;
  // working memory of this call
  const CkptLayout CL = ckpt_layout(h);
  unsigned char* ck;
  double *tgt, *res, *lam, *grad;
  std::vector<void*> tmp;
  auto release = [&]() {
    for (void* p : tmp) dfree(h, p);
  };
  if ((rc = dalloc(h, &ck, CL.bytes * (size_t)(nseg + 1))) || (tmp.push_back(ck), false) ||
      (rc = dalloc(h, &tgt, (size_t)nobs * nt)) || (tmp.push_back(tgt), false) ||
      (rc = dalloc(h, &res, (size_t)nobs * nt)) || (tmp.push_back(res), false) ||
      (rc = dalloc(h, &lam, 4 * nt)) || (tmp.push_back(lam), false) ||
      (rc = dalloc(h, &grad, (size_t)h->ncls * 5)) || (tmp.push_back(grad), false)) {
    release();
    return rc;
  }
  const int ng = h->ncls * 5;
  cudaError_t e = cudaMemcpyAsync(tgt, spec->target, (size_t)nobs * nt * 8, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(grad, 0, (size_t)ng * 8, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(&h->d.ctl->loss, 0, 8, h->stream);
  // ---- forward: checkpoint every `seg` steps, observe every `every` steps
  for (int sg = 0; sg < nseg && e == cudaSuccess; sg++) {
    e = ckpt_copy(h, ck + (size_t)sg * CL.bytes, true);
    const int j1 = std::min(n_steps, (sg + 1) * seg);
    for (int j = sg * seg; j < j1 && e == cudaSuccess; j++) {
      e = cudaGraphLaunch(h->gexec, h->stream);
      if ((j + 1) % every == 0) {
        const int k = (j + 1) / every - 1;
        launch_observe(h->d, h->grid, h->stream, tgt + (size_t)k * nt, res + (size_t)k * nt, nullptr);
      }
    }
  }
  if (e == cudaSuccess) e = ckpt_copy(h, ck + (size_t)nseg * CL.bytes, true);   // end state
  // ---- reverse: per segment, replay it with the tape, then sweep it backwards
  double *lx = lam, *lv = lam + nt, *nx = lam + 2 * nt, *nv = lam + 3 * nt;
  if (e == cudaSuccess) e = cudaMemsetAsync(lam, 0, 2 * nt * 8, h->stream);
  for (int sg = nseg - 1; sg >= 0 && e == cudaSuccess; sg--) {
    const int j0 = sg * seg, j1 = std::min(n_steps, (sg + 1) * seg);
    e = ckpt_copy(h, ck + (size_t)sg * CL.bytes, false);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->tape, 0, (size_t)seg * nt * sizeof(TapeRec), h->stream);
    launch_tape_begin(h->d, h->stream);
    for (int j = j0; j < j1 && e == cudaSuccess; j++) e = cudaGraphLaunch(h->gexec_tape, h->stream);
    for (int j = j1 - 1; j >= j0 && e == cudaSuccess; j--) {
      e = cudaMemsetAsync(nx, 0, 2 * nt * 8, h->stream);
      const double* r = ((j + 1) % every == 0) ? res + (size_t)((j + 1) / every - 1) * nt : nullptr;
      launch_adj_step(dtape, h->grid, h->stream, h->tape + (size_t)(j - j0) * nt, lx, lv, r, nx, nv, grad, h->ncls);
      std::swap(lx, nx);
      std::swap(lv, nv);
    }
  }
  if (e == cudaSuccess) e = ckpt_copy(h, ck + (size_t)nseg * CL.bytes, false);
  if (e == cudaSuccess) e = cudaMemcpyAsync(grad_out, grad, (size_t)ng * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(loss_out, &h->d.ctl->loss, 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  release();
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint");
  return check_device(h);
}

// ---------------------------------------------------------------- autotuner
namespace {

std::string tune_key(const sim_handle* h) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, h->device);
  unsigned long long hsh = 1469598103934665603ULL;
  auto mix = [&](unsigned long long v) {
    hsh ^= v;
    hsh *= 1099511628211ULL;
  };
  mix((unsigned long long)h->nn);
  mix((unsigned long long)h->nl);
  mix((unsigned long long)h->nt);
  mix((unsigned long long)h->n_lanes);
  mix((unsigned long long)h->has_stop);
  char buf[sizeof(prop.name) + 48];
  snprintf(buf, sizeof buf, "%s|sm%d|%016llx", prop.name, h->sm_count, hsh);
  return buf;
}

bool tune_cache_lookup(const char* path, const std::string& key, sim_exec* out) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char k[300];
    sim_exec e{};
    long long lim = 0;
    if (sscanf(line, "{\"key\": \"%299[^\"]\", \"mode\": %d, \"threads\": %d, \"blocks_per_sm\": %d, "
                     "\"grid_per_sm\": %d, \"barrier_timeout_cycles\": %lld",
               k, &e.mode, &e.threads, &e.blocks_per_sm, &e.grid_per_sm, &lim) == 6 &&
        key == k) {
      e.barrier_timeout_cycles = lim;
      *out = e;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void tune_cache_store(const char* path, const std::string& key, const sim_exec& e, double us) {
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f,
          "{\"key\": \"%s\", \"mode\": %d, \"threads\": %d, \"blocks_per_sm\": %d, \"grid_per_sm\": %d, "
          "\"barrier_timeout_cycles\": %lld, \"us_per_step\": %.3f}\n",
          key.c_str(), e.mode, e.threads, e.blocks_per_sm, e.grid_per_sm, (long long)e.barrier_timeout_cycles, us);
  fclose(f);
}

}  // namespace

int sim_autotune(sim_handle* h, int32_t trial_steps, const char* cache_path, sim_exec* chosen) {
  NvtxRange nvtx_("sim_autotune");
  if (!h || trial_steps < 1) return SIM_EINVAL;
  h->t_known = false;
  if (h->state_lost) return fail(h, SIM_ESTATE, "the state is undefined after a timeout: sim_write_state or sim_route first");
  if (!h->routed) return fail(h, SIM_ESTATE, "sim_autotune before routes exist");
  if (h->out_flags) return fail(h, SIM_ESTATE, "sim_autotune with measured outputs on (its trial steps would count)");
  const std::string key = tune_key(h);
  sim_exec best{};
  if (tune_cache_lookup(cache_path, key, &best) && sim_set_exec(h, &best) == SIM_OK) {
    if (chosen) *chosen = h->exec;
    return SIM_OK;
  }
  if (int rc = check_horizon(h, trial_steps * 40)) return rc;
  // candidates; every one gives the same results, only the time differs
  std::vector<sim_exec> cand;
  for (int g : {2, 4, 8, 16}) cand.push_back(sim_exec{SIM_EXEC_GRAPH, 256, 0, g, 0});
  for (int t : {256, 512, 1024}) {
    const int mx = persistent_max_blocks_per_sm(t);
    for (int b = 1; b <= mx && b * t <= 1024; b++) cand.push_back(sim_exec{SIM_EXEC_PERSISTENT, t, b, 8, 0});
  }
  const CkptLayout CL = ckpt_layout(h);
  unsigned char* ck;
  int rc = dalloc(h, &ck, CL.bytes);
  if (rc) return rc;
  const sim_exec orig = h->exec;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t err = ckpt_copy(h, ck, true);
  double best_us = 1e30;
  for (const sim_exec& c : cand) {
    if (err != cudaSuccess) break;
    if (sim_set_exec(h, &c) != SIM_OK) continue;
    err = ckpt_copy(h, ck, false);
    if (err != cudaSuccess) break;
    if ((rc = sim_step(h, trial_steps))) break;   // warm-up (builds the graphs of this step count)
    err = ckpt_copy(h, ck, false);
    if (err != cudaSuccess) break;
    cudaEventRecord(e0, h->stream);
    if ((rc = sim_step(h, trial_steps))) break;
    cudaEventRecord(e1, h->stream);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double us = 1e3 * ms / trial_steps;
    if (us < best_us) {
      best_us = us;
      best = c;
    }
  }
  if (err == cudaSuccess && !rc) err = ckpt_copy(h, ck, false);
  if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dfree(h, ck);
  if (rc) {
    sim_set_exec(h, &orig);
    return rc;
  }
  if (err != cudaSuccess) return cuda_fail(h, err, "autotune");
  if (best_us >= 1e30) return fail(h, SIM_ECUDA, "no execution configuration ran");
  if ((rc = sim_set_exec(h, &best))) return rc;
  tune_cache_store(cache_path, key, best, best_us);
  if (chosen) *chosen = best;
  return SIM_OK;
}

// ------------------------------------------------------------------ measured outputs
int sim_set_outputs(sim_handle* h, uint32_t flags, const sim_sampling* sampling) {
  if (!h) return SIM_EINVAL;
  h->t_known = false;
  if (flags & ~(uint32_t)(SIM_OUT_EMISSIONS | SIM_OUT_LINK_TIMES | SIM_OUT_EDGE_SAMPLES))
    return fail(h, SIM_EINVAL, "unknown output flag");
  int every = 0, per = 0, maxw = 0;
  if (flags & SIM_OUT_EDGE_SAMPLES) {
    if (!sampling) return fail(h, SIM_EINVAL, "edge samples need a sim_sampling");
    every = sampling->every_steps;
    per = sampling->per_window;
    maxw = sampling->max_windows;
    if (every < 1 || per < 1 || maxw < 1) return fail(h, SIM_EINVAL, "sampling sizes must be >= 1");
    if ((double)maxw * (double)std::max(1, h->nl) * 16.0 > 64.0e9)
      return fail(h, SIM_EINVAL, "edge-sample store above 64 GB");
  }
  Dev& d = h->d;
  void* olds[] = {d.emis, d.enter, d.tt_sum, d.tt_n, d.acc_u, d.acc_s, d.out_u, d.out_s, d.out_n};
  for (void* q : olds) dfree(h, q);
  d.emis = nullptr;
  d.enter = nullptr;
  d.tt_sum = nullptr;
  d.tt_n = nullptr;
  d.acc_u = d.acc_s = d.out_u = d.out_s = nullptr;
  d.out_n = nullptr;
  d.samp_every = d.samp_per = d.samp_max = 0;
  h->out_flags = 0;
  h->graph_dirty = true;
  h->pgraph_n = -1;
  h->tape_graph_dirty = true;
  const size_t nt = (size_t)std::max(1, h->nt), nl = (size_t)std::max(1, h->nl);
  int rc = SIM_OK;
  if (flags & SIM_OUT_EMISSIONS) {
    if ((rc = dalloc(h, &d.emis, nt))) return rc;
  }
  if (flags & SIM_OUT_LINK_TIMES) {
    if ((rc = dalloc(h, &d.enter, nt)) || (rc = dalloc(h, &d.tt_sum, nl)) || (rc = dalloc(h, &d.tt_n, nl))) return rc;
  }
  if (flags & SIM_OUT_EDGE_SAMPLES) {
    if ((rc = dalloc(h, &d.acc_u, nl)) || (rc = dalloc(h, &d.acc_s, nl)) ||
        (rc = dalloc(h, &d.out_u, (size_t)maxw * nl)) || (rc = dalloc(h, &d.out_s, (size_t)maxw * nl)) ||
        (rc = dalloc(h, &d.out_n, (size_t)maxw)))
      return rc;
    d.samp_every = every;
    d.samp_per = per;
    d.samp_max = maxw;
  }
  h->out_flags = flags;
  return clear_outputs(h, -1);
}

int sim_reset_outputs(sim_handle* h) {
  if (!h) return SIM_EINVAL;
  h->t_known = false;
  return clear_outputs(h, -1);
}

int sim_read_emissions(sim_handle* h, double* fuel_ml, double* co_g) {
  if (!h || !fuel_ml || !co_g) return SIM_EINVAL;
  if (!h->d.emis) return fail(h, SIM_ESTATE, "emissions output is off");
  std::vector<double2> q((size_t)std::max(1, h->nt));
  if (h->nt) CK(cudaMemcpyAsync(q.data(), h->d.emis, (size_t)h->nt * 16, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int i = 0; i < h->nt; i++) {
    fuel_ml[i] = q[i].x;
    co_g[i] = q[i].y;
  }
  return SIM_OK;
}

int sim_read_link_times(sim_handle* h, int64_t* sum_steps, int32_t* n_exits) {
  if (!h || !sum_steps || !n_exits) return SIM_EINVAL;
  if (!h->d.tt_sum) return fail(h, SIM_ESTATE, "link-time output is off");
  if (h->nl) {
    CK(cudaMemcpyAsync(sum_steps, h->d.tt_sum, (size_t)h->nl * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(n_exits, h->d.tt_n, (size_t)h->nl * 4, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

int sim_read_edge_samples(sim_handle* h, double* util, double* speed, int32_t* n_samples) {
  if (!h || !util || !speed || !n_samples) return SIM_EINVAL;
  const Dev& d = h->d;
  if (!d.acc_u) return fail(h, SIM_ESTATE, "edge-sample output is off");
  const size_t n = (size_t)d.samp_max * (size_t)h->nl;
  if (n) {
    CK(cudaMemcpyAsync(util, d.out_u, n * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(speed, d.out_s, n * 8, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaMemcpyAsync(n_samples, d.out_n, (size_t)d.samp_max * 4, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

int sim_measured_costs(sim_handle* h, const int32_t* prev_cost_ds, int32_t* cost_ds, double* gap) {
  NvtxRange nvtx_("sim_measured_costs");
  if (!h || !prev_cost_ds || !cost_ds) return SIM_EINVAL;
  h->t_known = false;
  const Dev& d = h->d;
  if (!d.tt_sum) return fail(h, SIM_ESTATE, "link-time output is off");
  const int nl = h->nl;
  for (int e = 0; e < nl; e++)
    if (prev_cost_ds[e] < 1 || prev_cost_ds[e] > 1000000) return fail(h, SIM_EINVAL, "link costs must be 1..1e6 ds");
  int32_t *dp = nullptr, *dc = nullptr;
  int rc = dalloc(h, &dp, (size_t)std::max(1, nl));
  if (rc) return rc;
  if ((rc = dalloc(h, &dc, (size_t)std::max(1, nl)))) {
    dfree(h, dp);
    return rc;
  }
  cudaError_t e = cudaSuccess;
  unsigned long long nd[2] = {0, 0};
  if (nl) e = cudaMemcpyAsync(dp, prev_cost_ds, (size_t)nl * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(&d.ctl->gap_num, 0, 2 * sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess && nl) launch_measured_costs(d, dp, dc, h->stream);
  if (e == cudaSuccess && nl) e = cudaMemcpyAsync(cost_ds, dc, (size_t)nl * 4, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(nd, &d.ctl->gap_num, sizeof(nd), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dfree(h, dp);
  dfree(h, dc);
  if (e != cudaSuccess) return cuda_fail(h, e, "measured costs");
  if (gap) *gap = nd[1] ? (double)nd[0] / (double)nd[1] : 0.0;
  return SIM_OK;
}

int sim_equilibrium(sim_handle* h, int32_t n_iter, const uint32_t* fractions_q16, int32_t n_steps, int32_t* cost_out,
                    double* gap_out) {
  NvtxRange nvtx_("sim_equilibrium");
  if (!h || !fractions_q16 || !cost_out || !gap_out) return SIM_EINVAL;
  h->t_known = false;
  if (h->state_lost) return fail(h, SIM_ESTATE, "the state is undefined after a timeout: sim_write_state or sim_route first");
  if (!h->d.tt_sum) return fail(h, SIM_ESTATE, "sim_equilibrium needs the link-time output");
  if (n_iter < 1 || n_steps < 1) return fail(h, SIM_EINVAL, "n_iter and n_steps must be >= 1");
  for (int k = 1; k < n_iter; k++)
    if (fractions_q16[k] > 65536u) return fail(h, SIM_EINVAL, "fraction_q16 must be 0..65536");
  const int nl = h->nl;
  std::vector<int32_t> cost(std::max(1, nl)), meas(std::max(1, nl));
  for (int e = 0; e < nl; e++) cost[e] = free_flow_cost(h, e);
  for (int k = 0; k < n_iter; k++) {
    int rc = k == 0 ? sim_route(h, cost.data()) : sim_reroute(h, cost.data(), fractions_q16[k], (uint32_t)k);
    if (!rc) rc = sim_step(h, n_steps);
    if (!rc) rc = sim_measured_costs(h, cost.data(), meas.data(), &gap_out[k]);
    if (rc) return rc;
    cost.swap(meas);
  }
  if (nl) memcpy(cost_out, cost.data(), (size_t)nl * 4);
  return SIM_OK;
}

// ------------------------------------------------------------------ static assignment
namespace {
// 2^S with S the largest shift (<= 100) for which n terms of magnitude <= bound sum to
// less than 2^62
double fixed_scale(double bound, int n) {
  int E = 0;
  std::frexp(bound * (double)std::max(n, 1), &E);
  return std::ldexp(1.0, std::min(62 - E, 100));
}
}  // namespace

int sim_assign_static(sim_handle* h, const sim_assign_spec* spec, double* flow_out, double* time_out, double* gap_out,
                      double* step_out, double* objective_out) {
  NvtxRange nvtx_("sim_assign_static");
  if (!h || !spec || !spec->capacity || !flow_out || !time_out || !objective_out) return SIM_EINVAL;
  h->t_known = false;
  const int nl = h->nl, nn = h->nn, K = spec->max_iter, beta = spec->beta;
  const double alpha = spec->alpha;
  if (beta < 1 || beta > 8 || !(alpha >= 0.0) || K < 0 || spec->bisect_iter < 0 || spec->bisect_iter > 60)
    return fail(h, SIM_EINVAL, "need 1 <= beta <= 8, alpha >= 0, max_iter >= 0, 0 <= bisect_iter <= 60");
  if (K > 0 && (!gap_out || !step_out)) return SIM_EINVAL;
  for (int e = 0; e < nl; e++)
    if (!(spec->capacity[e] > 0.0) || !std::isfinite(spec->capacity[e]))
      return fail(h, SIM_EINVAL, "capacities must be finite and > 0");
  const size_t L = (size_t)std::max(1, nl);
  double *t0 = nullptr, *x = nullptr, *t = nullptr, *cap = nullptr;
  unsigned* y = nullptr;
  int32_t* q = nullptr;
  float *dlen = nullptr, *dspd = nullptr;
  unsigned long long* red = nullptr;
  std::vector<void*> mine;
  auto take = [&](auto** p, size_t n) -> int {
    int rc = dalloc(h, p, n);
    if (!rc) mine.push_back(*p);
    return rc;
  };
  auto release = [&]() {
    for (void* p : mine) dfree(h, p);
    mine.clear();
  };
  int rc = SIM_OK;
  if ((rc = take(&t0, L)) || (rc = take(&x, L)) || (rc = take(&t, L)) || (rc = take(&cap, L)) ||
      (rc = take(&y, L)) || (rc = take(&q, L)) || (rc = take(&dlen, L)) || (rc = take(&dspd, L)) ||
      (rc = take(&red, 4))) {
    release();
    return rc;
  }
  cudaStream_t s = h->stream;
  const long long qmax = std::min<long long>(1000000, (2000000000LL - 1) / std::max(1, nn));
  std::vector<int32_t> qh(L);
  unsigned long long hr[4];
  cudaError_t e = cudaSuccess;
  auto put = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  };
  auto get = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  };
  auto zero_red = [&]() {
    if (e == cudaSuccess) e = cudaMemsetAsync(red, 0, 4 * sizeof(unsigned long long), s);
  };
  // direction finding: integer costs of the times in t (largest time in red[0]), then
  // all-or-nothing counts into y
  auto aon = [&]() -> int {
    get(hr, red, sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(h, e, "assignment");
    double tmax;
    memcpy(&tmax, &hr[0], sizeof tmax);
    const double unit = std::max(0.1, tmax / (double)qmax);
    launch_fw_quantize(t, unit, (int)qmax, q, nl, s);
    get(qh.data(), q, (size_t)nl * 4);
    if (e != cudaSuccess) return cuda_fail(h, e, "assignment");
    return route_impl(h, qh.data(), nullptr, y);
  };
  put(dlen, h->len.data(), (size_t)nl * 4);
  put(dspd, h->spd.data(), (size_t)nl * 4);
  put(cap, spec->capacity, (size_t)nl * 8);
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, L * 8, s);
  launch_fw_t0(dlen, dspd, t0, nl, s);
  zero_red();
  launch_fw_time(t0, x, cap, alpha, beta, t, red, nl, s);   // x = 0: t = t0
  if ((rc = aon())) {
    release();
    return rc;
  }
  launch_fw_counts(y, x, nl, s);
  for (int k = 0; k <= K; k++) {
    // Beckmann objective at x_k
    zero_red();
    launch_fw_objective(t0, x, cap, alpha, beta, true, 0.0, red, nl, s);
    get(hr, red, 8);
    double bo;
    memcpy(&bo, &hr[0], 8);
    const double so = fixed_scale(bo, nl);
    zero_red();
    launch_fw_objective(t0, x, cap, alpha, beta, false, so, red, nl, s);
    get(hr, red, 8);
    objective_out[k] = (double)(long long)hr[0] / so;
    if (k == K) break;
    // direction
    zero_red();
    launch_fw_time(t0, x, cap, alpha, beta, t, red, nl, s);
    if ((rc = aon())) {
      release();
      return rc;
    }
    zero_red();
    launch_fw_bounds(t0, x, y, t, cap, alpha, beta, red, nl, s);
    get(hr, red, 16);
    double bg, bl;
    memcpy(&bg, &hr[0], 8);
    memcpy(&bl, &hr[1], 8);
    const double sg = fixed_scale(bg, nl), sl = fixed_scale(bl, nl);
    zero_red();
    launch_fw_gap_sums(t, x, y, sg, red, nl, s);
    get(hr, red, 16);
    const long long tx = (long long)hr[0], ty = (long long)hr[1];
    gap_out[k] = tx > 0 ? (double)(tx - ty) / (double)tx : 0.0;
    // step: exact line search by bisection on the sign of the derivative
    auto deriv = [&](double a) -> long long {
      zero_red();
      launch_fw_deriv(t0, x, y, cap, alpha, beta, a, sl, red, nl, s);
      get(hr, red, 8);
      return (long long)hr[0];
    };
    const long long g0 = deriv(0.0), g1 = deriv(1.0);
    double a;
    if (g0 >= 0) {
      a = 0.0;
    } else if (g1 <= 0) {
      a = 1.0;
    } else {
      double lo = 0.0, hi = 1.0;
      for (int it = 0; it < spec->bisect_iter; it++) {
        const double mid = 0.5 * (lo + hi);
        if (deriv(mid) > 0) hi = mid;
        else lo = mid;
      }
      a = 0.5 * (lo + hi);
    }
    step_out[k] = a;
    launch_fw_update(x, y, a, nl, s);
    if (e != cudaSuccess) break;
  }
  launch_fw_final_time(t0, x, cap, alpha, beta, t, nl, s);
  get(flow_out, x, (size_t)nl * 8);
  get(time_out, t, (size_t)nl * 8);
  release();
  if (e != cudaSuccess) return cuda_fail(h, e, "assignment");
  return SIM_OK;
}

const char* sim_last_error(const sim_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void sim_destroy(sim_handle* h) {
  if (!h) return;
  if (h->gexec_samp) cudaGraphExecDestroy(h->gexec_samp);
  if (h->graph_samp) cudaGraphDestroy(h->graph_samp);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->gexec_tape) cudaGraphExecDestroy(h->gexec_tape);
  if (h->graph_tape) cudaGraphDestroy(h->graph_tape);
  if (h->pexec) cudaGraphExecDestroy(h->pexec);
  if (h->pgraph) cudaGraphDestroy(h->pgraph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->mirror) cudaFreeHost(h->mirror);
  for (void* p : h->allocs) cudaFree(p);
  delete h;
}

}  // extern "C"
