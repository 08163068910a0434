/* gbtraffic — GB300 (sm_103a) traffic microsimulation hot path, C ABI.
 *
 * Implements the time-stepped microsimulation of Waddell et al., "Architecture
 * for Modular Microsimulation of Real Estate Markets and Transportation",
 * Sec. 6 ("Traffic microsimulation model"): vehicles follow precomputed
 * shortest-path routes on a lane-level network (Sec. 6.2.1, 6.3.1), accelerate
 * by the Intelligent Driver Model (Eq. 7), change lanes (mandatory /
 * discretionary with gap acceptance, Sec. 6.3.2) and are admitted through stop
 * signs and traffic lights (Sec. 6.3.2), with dt = 0.5 s (Sec. 6.3.2).
 *
 * Conventions
 *  - All pointers in the input structs are HOST pointers owned by the caller;
 *    sim_create copies everything it needs to the device, so the caller may free
 *    its arrays as soon as sim_create returns.
 *  - A trip id (vid) is the index of the trip in sim_demand; every per-trip
 *    output is indexed by vid.  Link and node ids are indices into sim_network.
 *  - Lanes are numbered 0 (rightmost) to lanes-1 (leftmost); at most 8 per link.
 *  - All device work is ordered on the stream given by sim_set_stream (default:
 *    the legacy default stream).  A handle is not thread-safe.
 *  - Every call returns SIM_OK or a negative SIM_E* code; the message of the
 *    last failure is available from sim_last_error.  No call aborts, throws or
 *    traps on the device.  Device-side index checks set an error word that the
 *    next synchronising call reports as SIM_EDEVICE.
 */
#ifndef GBTRAFFIC_H
#define GBTRAFFIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SIM_OK = 0,
  SIM_EINVAL = -1,        /* malformed input or argument */
  SIM_ENOMEM = -2,        /* device or host allocation failed */
  SIM_ECUDA = -3,         /* a CUDA runtime call failed */
  SIM_EUNREACHABLE = -4,  /* a trip's destination cannot be reached from its origin */
  SIM_ETIMEOUT = -5,      /* a bounded device wait expired */
  SIM_ESTATE = -6,        /* call out of order (e.g. sim_step before routes exist) */
  SIM_EDEVICE = -7        /* the device error word was set (index out of range, capacity) */
};

enum { SIM_CTRL_NONE = 0, SIM_CTRL_STOP = 1, SIM_CTRL_SIGNAL = 2 };
enum { SIM_PENDING = 0, SIM_ACTIVE = 1, SIM_ARRIVED = 2 };

/* Road network (Sec. 6.2.1: nodes = intersections, directed edges = roads with
 * speed and lanes; Sec. 4: directed multigraph, self-loops allowed). */
typedef struct {
  int32_t n_nodes, n_links;
  const int32_t* node_x_dm;          /* [n_nodes] position, integer decimetres (turns, signal phases) */
  const int32_t* node_y_dm;          /* [n_nodes] */
  const uint8_t* node_control;       /* [n_nodes] SIM_CTRL_* */
  const int32_t* signal_offset_ds;   /* [n_nodes] offset of the fixed-time plan, deciseconds */
  const int32_t* signal_cycle_ds;    /* [n_nodes] cycle length, deciseconds (1..65535) */
  const int32_t* signal_green_ds;    /* [n_nodes] north-south green per cycle, deciseconds */
  const int32_t* link_from;          /* [n_links] tail node */
  const int32_t* link_to;            /* [n_links] head node */
  const float* link_length_m;        /* [n_links] > 0 */
  const float* link_speed_mps;       /* [n_links] speed limit > 0 */
  const uint8_t* link_lanes;         /* [n_links] 1..8 */
  const uint8_t* link_class;         /* [n_links] < sim_params.n_class (selects IDM parameters) */
} sim_network;

/* Travel demand (Sec. 6.2.2: origin, destination and departure time per vehicle). */
typedef struct {
  int32_t n_trips;
  const int32_t* origin;             /* [n_trips] node id */
  const int32_t* dest;               /* [n_trips] node id, != origin for routed trips */
  const int32_t* depart_step;        /* [n_trips] earliest step at which the trip may enter */
} sim_demand;

#define SIM_MAX_CLASS 256

/* Model parameters.  IDM per link class (Eq. 7); v0 <= 0 uses the link speed
 * limit (Sec. 6.3.2: "v0 is the edge speed limit"). */
typedef struct {
  float dt;                          /* step, seconds; dt*10 must be an integer (0.5 in the paper) */
  float veh_len;                     /* vehicle length, m */
  float s_min;                       /* floor of the bumper gap in Eq. 7, m */
  int32_t n_class;                   /* 1..SIM_MAX_CLASS */
  const float *v0, *T, *a, *b, *s0;  /* [n_class] host arrays */
  float mobil_p, mobil_athr, mobil_bsafe, mobil_bias_right;  /* lane-change incentive / safety */
  float lambda_mand;                 /* mandatory-switch length scale per lane to cross, m */
  float stop_acquire_m;              /* distance to the stop line within which a stop is acquired, m */
  uint64_t seed;                     /* draws of the mandatory-switch distance */
  int32_t cost_mode;                 /* 0: free-flow length/speed; 1: sqrt(lanes)*length/speed */
  int32_t loop_routes;               /* 1: routes repeat forever (ring roads) */
  uint64_t max_device_bytes;         /* cap on the device memory the handle allocates, 0: none;
                                        a call that would pass it returns SIM_ENOMEM (all
                                        scenarios of a batch must give the same value) */
} sim_params;

typedef struct sim_handle sim_handle;

/* Counters after the last completed step. */
typedef struct {
  int64_t t;            /* steps simulated since the state was set */
  int64_t departed;     /* trips that entered the network */
  int64_t waiting;      /* due trips (depart_step < t) not yet on the network */
  int64_t active;       /* vehicles on the network now */
  int64_t arrived;      /* trips that reached their destination */
  int64_t veh_steps;    /* sum over steps of the vehicles advanced in that step */
  int64_t pending;      /* trips not yet due */
  int64_t active_last;  /* vehicles advanced in the last step */
  int64_t lc_evals;     /* sum over steps of the lane-change decisions evaluated (vehicles
                           on a multi-lane link away from both of its ends) */
} sim_counters_t;

/* Field bits for sim_read_state. */
enum {
  SIM_F_STATUS = 1 << 0, SIM_F_LINK = 1 << 1, SIM_F_LANE = 1 << 2, SIM_F_CURSOR = 1 << 3,
  SIM_F_X = 1 << 4, SIM_F_V = 1 << 5, SIM_F_INSERT = 1 << 6, SIM_F_ARRIVE = 1 << 7,
  SIM_F_LANECHANGE = 1 << 8
};

/* Per-trip state view.  Each pointer addresses n_trips elements (or is NULL when
 * its field is not requested).  Non-active trips read link -1, lane 0, cursor 0,
 * x 0, v 0. */
typedef struct {
  uint8_t* status;      /* SIM_PENDING / SIM_ACTIVE / SIM_ARRIVED */
  int32_t* link;        /* current link */
  int32_t* lane;        /* current lane */
  int32_t* cursor;      /* index of the current link in the trip's route */
  float* x;             /* distance from the start of the link, m, in [0, length] */
  float* v;             /* speed, m/s */
  int32_t* insert_step; /* step at which the trip entered (-1: not yet; 0 for written state) */
  int32_t* arrive_step; /* step at which the trip arrived (-1: not yet) */
  int8_t* lane_change;  /* lane change applied in the last step: -1 right, +1 left, 0 none */
} sim_state_view;

/* Create a simulation.  Validates and deep-copies the inputs to the device of the
 * current CUDA context.  Errors: SIM_EINVAL (bad ids, lengths, lanes, classes,
 * dt), SIM_ENOMEM, SIM_ECUDA.  *out is NULL on failure. */
int sim_create(const sim_network* net, const sim_demand* dem, const sim_params* par, sim_handle** out);

/* Create one simulation over the disjoint union of n scenarios (independent
 * networks and demands with their own parameters), advanced together by every
 * sim_step.  Trip t of scenario k has vid = (sum of n_trips of scenarios < k) + t;
 * node, link and class ids are offset the same way.  Each scenario evolves exactly
 * as it would in its own handle.  All scenarios must share dt and loop_routes. */
int sim_create_batch(int32_t n, const sim_network* const* nets, const sim_demand* const* dems,
                     const sim_params* const* pars, sim_handle** out);

/* Order all further device work of the handle on this cudaStream_t (NULL = legacy
 * default stream). */
int sim_set_stream(sim_handle* h, void* cuda_stream);

/* Trip planning (Sec. 6.3.1, Sec. 6 "Simulation scale"): one shortest-path tree per
 * distinct origin on the GPU (near-far delta-stepping on integer link costs), and
 * for every trip the path origin -> destination.  Among equally short paths, the
 * walk back from the destination takes the lowest-id in-link u->v with
 * dist[u] + cost = dist[v].  link_cost_ds: host array [n_links] of costs >= 1 in
 * deciseconds, or NULL for the free-flow cost of Eq. 4,
 * max(1, floor(10*length/speed + 0.5)) (cost_mode 1: times sqrt(lanes)).
 * Resets the vehicle state: all trips pending, t = 0.
 * Errors: SIM_EINVAL (cost < 1, origin == dest), SIM_EUNREACHABLE, SIM_ENOMEM. */
int sim_route(sim_handle* h, const int32_t* link_cost_ds);

/* Set explicit routes instead: host CSR offsets [n_trips+1] and link ids; each
 * route must be a connected link sequence (and a cycle when loop_routes).
 * Resets the vehicle state like sim_route. */
int sim_set_routes(sim_handle* h, const int32_t* offsets, const int32_t* links);

/* Total number of route hops (for sizing sim_read_routes). */
int sim_route_size(sim_handle* h, int64_t* n_hops);

/* Copy routes to host: offsets [n_trips+1], links [n_hops], in trip order. */
int sim_read_routes(sim_handle* h, int32_t* offsets, int32_t* links);

/* Advance the simulation by n_steps steps of dt.  All steps run on the device
 * without a host round trip.  Errors: SIM_ESTATE (no routes), SIM_EDEVICE,
 * SIM_EINVAL when the horizon would pass 2^31 deciseconds of simulated time. */
int sim_step(sim_handle* h, int32_t n_steps);

/* Size of sim_step_timed's kernel_ms array: at least the number of kernel groups of a
 * step that sim_kernel_name names (the rest of the array stays zero). */
#define SIM_N_KERNELS 8

/* Advance n_steps like sim_step, but launch every kernel directly with a CUDA event
 * after each one, and add each kernel's device time (ms, including its launch gap)
 * into kernel_ms[SIM_N_KERNELS] (host array, zeroed first).  Results are identical
 * to sim_step.  For profiling; slower than sim_step's graph launch. */
int sim_step_timed(sim_handle* h, int32_t n_steps, float* kernel_ms);

/* Name of kernel group k of a step (0 <= k < SIM_N_KERNELS), "" past the last group. */
const char* sim_kernel_name(int32_t k);

/* Kernel launches sim_step has made on this handle since its creation, into *launches:
 * in graph execution the kernels of the captured step graph, per step; in persistent
 * execution one cooperative launch per sim_step call.  (Launches of the other calls
 * are not counted.)  Errors: SIM_EINVAL on a NULL argument. */
int sim_launch_count(sim_handle* h, int64_t* launches);

/* How sim_step runs the steps.  SIM_EXEC_GRAPH: one CUDA graph of the step's kernels
 * per step, grid = grid_per_sm x SMs blocks of 256 threads for the kernels that do not
 * size their own grid (the chunk kernel runs one resident wave); the chunk kernel's
 * waits for its staged chunks (bulk copies into shared memory) are bounded by
 * barrier_timeout_cycles SM cycles (<= 0: 2e9), after which sim_step returns
 * SIM_ETIMEOUT (the state is then undefined until the next sim_write_state /
 * sim_route, and stepping calls return SIM_ESTATE until then).  SIM_EXEC_PERSISTENT: all
 * n steps in one cooperative launch of blocks_per_sm x SMs blocks of `threads`
 * threads (the same phases as the graph's kernels), the phases of a step separated by a
 * grid barrier whose wait, like the chunk staging wait, is bounded by
 * barrier_timeout_cycles SM cycles (<= 0: 2e9, about a second); a wait that runs out
 * makes sim_step return SIM_ETIMEOUT (the state is then undefined until the next
 * sim_write_state / sim_route).  Every configuration gives identical results. */
enum { SIM_EXEC_GRAPH = 0, SIM_EXEC_PERSISTENT = 1 };
typedef struct {
  int32_t mode;
  int32_t threads;                  /* persistent: 256, 512 or 1024 */
  int32_t blocks_per_sm;            /* persistent: 1 .. co-resident limit */
  int32_t grid_per_sm;              /* graph: 1 .. 64 */
  int64_t barrier_timeout_cycles;   /* persistent: bound of a barrier wait; graph: bound of a
                                       staging wait of the chunk kernel */
} sim_exec;

int sim_set_exec(sim_handle* h, const sim_exec* e);
int sim_get_exec(sim_handle* h, sim_exec* e);

/* Pick the fastest execution configuration for this handle: time trial_steps steps
 * from the current state under every candidate (graph with 2/4/8/16 blocks per SM;
 * persistent with 256/512/1024 threads and co-resident blocks per SM up to 1024
 * threads per SM), each after an untimed run of the same length from the same state
 * (which builds its launch graphs), restore the state, and keep the best.  The choice
 * holds for states like the current one: few vehicles favour the persistent launch,
 * many the graph.  cache_path (or NULL): a JSON-lines file keyed by
 * device name, SM count and a hash of the network and demand sizes; a hit skips the
 * trials, a new result is appended.  *chosen (or NULL) receives the choice. */
int sim_autotune(sim_handle* h, int32_t trial_steps, const char* cache_path, sim_exec* chosen);

/* Read the per-trip state (fields = OR of SIM_F_*).  on_device = 1: the view's
 * pointers are device pointers (e.g. from torch tensors) of n_trips elements each;
 * on_device = 0: host pointers (pinned host memory copies fastest); the first host read
 * of a field allocates a device staging buffer of n_trips elements that the handle keeps
 * until sim_destroy.  Both synchronise the stream before returning.  on_device = 2:
 * device pointers as for 1, but the gather is only enqueued on the handle's stream
 * (sim_set_stream) and the call returns at once: the buffers hold the state once that
 * stream reaches this point, and must not be reused before (order other streams after
 * an event recorded on it).  Other values: SIM_EINVAL. */
int sim_read_state(sim_handle* h, const sim_state_view* out, uint32_t fields, int on_device);

/* Replace the vehicle state (resume, tests).  Host arrays [n_trips]: status,
 * link, lane, cursor, x, v (only SIM_ACTIVE trips need link..v).  Active trips
 * must sit on route[cursor] with 0 <= x <= length; pending trips re-enter the
 * departure queues; t, counters and stop-sign holders are reset. */
int sim_write_state(sim_handle* h, const uint8_t* status, const int32_t* link, const int32_t* lane,
                    const int32_t* cursor, const float* x, const float* v);

/* Per-lane occupancy of the current state, the sorted order the next step uses:
 * lane_start [n_lanes+1] and sorted_vid [active] (lanes are numbered link by link,
 * lane 0 first; within a lane by position, then vid).  Host arrays. */
int sim_occupancy(sim_handle* h, int32_t* lane_start, int32_t* sorted_vid);
int sim_n_lanes(sim_handle* h, int64_t* n_lanes);

int sim_counters(sim_handle* h, sim_counters_t* out);

/* Replace the IDM parameters of every class (arrays [n_class], host): the next steps
 * use them.  Classes created with v0 <= 0 (desired speed = link speed limit) must
 * keep v0 <= 0 and the others v0 > 0.  Errors: SIM_EINVAL. */
int sim_set_class_params(sim_handle* h, const float* v0, const float* T, const float* a, const float* b,
                         const float* s0);

/* Advance n_steps and record the route progress of every trip after every obs_every
 * steps: progress[k * n_trips + v] (host, double, metres) = length of the completed
 * links of trip v's route plus its position, 0 before departure, the whole route
 * after arrival; k = 0 .. n_steps / obs_every - 1. */
int sim_observe(sim_handle* h, int32_t n_steps, int32_t obs_every, double* progress);

/* Calibration loss of a trajectory (not in the paper). */
typedef struct {
  int32_t n_steps;            /* horizon, a multiple of obs_every */
  int32_t obs_every;          /* observation period, steps */
  int32_t checkpoint_every;   /* steps between stored states (<= 0: 64) */
  const double* target;       /* host [n_steps / obs_every][n_trips] target progress, m */
} sim_loss_spec;

/* Loss L = sum_k sum_v (p_v(t_k) - target[k][v])^2 over the n_steps from the current
 * state (t_k = (k+1) * obs_every steps later; p as in sim_observe) and its gradient
 * with respect to the IDM parameters of every class, grad_out[5 * c + {0..4}] =
 * dL/d{v0, T, a, b, s0} of class c (host, double; the v0 entry is 0 for classes that
 * use the link speed limit).  The discrete decisions of the run (leaders, lane
 * changes, admissions, clamps at the stop line, stops within a step, departures,
 * arrivals) are held fixed.  The forward pass stores the state every
 * checkpoint_every steps; the reverse pass replays each segment with a tape of the
 * vehicle-steps and sweeps it backwards in binary64.  On return the state is the one
 * after the n_steps.  Errors: SIM_EINVAL, SIM_ESTATE, SIM_ENOMEM. */
int sim_adjoint(sim_handle* h, const sim_loss_spec* spec, double* grad_out, double* loss_out);

/* The same loss L without the gradient: steps n_steps from the current state (plain
 * step kernels, no tape, no checkpoints) and adds the squared residuals of every trip
 * at each observation on the device (binary64; the per-block partial sums are added
 * atomically, so the last bits may depend on the order of the blocks).  On return the
 * state is the one after the n_steps.  Errors: SIM_EINVAL, SIM_ESTATE, SIM_ENOMEM. */
int sim_loss(sim_handle* h, const sim_loss_spec* spec, double* loss_out);

/* ---------------------------------------------------------------- vehicle types
 * Sec. 6.3.5: a second vehicle type for trucks, differing in size, acceleration and
 * maximum speed.  With types set, every trip has a type; a vehicle's gap to its leader
 * is measured to the leader's rear (its own length), Eq. 7 uses the link class's
 * parameters with a multiplied by accel_scale (and 2 sqrt(ab) from that a) and v0 =
 * min(class or link v0, max_speed_mps); a departure needs s0 + the entering vehicle's
 * length of rear space; two changes into one lane closer than s0 + the longer of the
 * two lengths keep only the lower trip id's.  The lane-change zone (2 * veh_len) and the
 * edge-sample capacity keep sim_params.veh_len. */
#define SIM_MAX_VEHICLE_TYPES 8
typedef struct {
  float length_m;        /* > 0 */
  float accel_scale;     /* > 0, multiplies the class's a */
  float max_speed_mps;   /* > 0, caps v0 */
} sim_vehicle_type;

/* types [n_types] and trip_type [n_trips] (host; each < n_types).  n_types = 0 returns
 * to the single class of sim_params.  Takes effect from the next step; sim_set_class_params
 * keeps applying to every type.  sim_adjoint refuses to run with types set (SIM_ESTATE).
 * Errors: SIM_EINVAL (sizes, values, type ids), SIM_ENOMEM. */
int sim_set_vehicle_types(sim_handle* h, int32_t n_types, const sim_vehicle_type* types, const uint8_t* trip_type);

/* ---------------------------------------------------------------- measured outputs
 * Optional per-run measurements taken by the step kernels (sim_step in either
 * execution mode; sim_step_timed counts the edge-sample kernel under "own").  All
 * enabled outputs are cleared by sim_set_outputs, sim_reset_outputs, sim_route,
 * sim_reroute, sim_set_routes and sim_write_state (after which t = 0).
 *
 * SIM_OUT_EMISSIONS (Eq. 8-9, Sec. 6.3.4): per trip, the fuel burnt (mL) and the CO
 *   emitted (g).  Every step a vehicle on the road adds dt times the rates at its speed
 *   v and the acceleration a it applies in that step, computed in binary32:
 *   fuel = 0.666 + 0.072 * max(0, 0.269 v + 0.0171 v^2 + 0.000672 v^3 + 1.680 a v
 *   + [a > 0] 0.79296 a^2 v) mL/s (the bracket is tractive power in kW; the engine
 *   idles when it is not positive) and CO = -0.064 + 0.0056 m + 0.00026 (m - 50)^2
 *   g/s, m = v / 0.44704 the speed in mph.  Sums are binary64.
 * SIM_OUT_LINK_TIMES (Sec. 6.3.1): per link, the number of trips that left it (into
 *   their next link, or arriving at its end) and their summed traversal times in
 *   steps, from the step they entered it (departure or crossing) to the step they
 *   left.  Trips already on a link when the outputs were cleared are not counted on
 *   that link.
 * SIM_OUT_EDGE_SAMPLES (Sec. 6.4): every every_steps steps (at t = 0, every_steps,
 *   ...), per link, the utilisation n / (length * lanes / (veh_len + s0)) with n the
 *   vehicles on the link and s0 its class's minimum gap, and the mean speed of those
 *   vehicles (the desired speed v0 of the link when it is empty).  Window w averages
 *   the samples w*per_window .. w*per_window + per_window - 1 taken since the last
 *   clear and is written when its last sample is; the paper samples every minute and
 *   averages over 6 minutes (every_steps = 60 / dt, per_window = 6). */
#define SIM_OUT_EMISSIONS 1u
#define SIM_OUT_LINK_TIMES 2u
#define SIM_OUT_EDGE_SAMPLES 4u
typedef struct {
  int32_t every_steps;   /* >= 1 */
  int32_t per_window;    /* >= 1 */
  int32_t max_windows;   /* windows stored; sim_step refuses (SIM_EINVAL) to run past them */
} sim_sampling;

/* Turn the outputs in flags on (and the others off), allocating their device
 * arrays (emissions 16 B per trip; link times 4 B per trip + 12 B per link; edge
 * samples 16 B per link and 16 B per link per window).  sampling is read for
 * SIM_OUT_EDGE_SAMPLES only.  sim_adjoint and sim_autotune refuse to run (SIM_ESTATE)
 * while any output is on.
 * Errors: SIM_EINVAL (unknown flag, sizes < 1), SIM_ENOMEM. */
int sim_set_outputs(sim_handle* h, uint32_t flags, const sim_sampling* sampling);

/* Clear the enabled outputs without touching the vehicle state; sampling windows
 * restart at the next sampling instant. */
int sim_reset_outputs(sim_handle* h);

/* Per-trip totals (host arrays [n_trips], trip order).  SIM_ESTATE when off. */
int sim_read_emissions(sim_handle* h, double* fuel_ml, double* co_g);

/* Per-link traversal sums (host arrays [n_links]).  SIM_ESTATE when off. */
int sim_read_link_times(sim_handle* h, int64_t* sum_steps, int32_t* n_exits);

/* Window means, host arrays util[max_windows][n_links], speed[max_windows][n_links]
 * (m/s), and n_samples[max_windows], the samples behind each finished window (0: not
 * finished; its util and speed are 0).  SIM_ESTATE when off. */
int sim_read_edge_samples(sim_handle* h, double* util, double* speed, int32_t* n_samples);

/* Sec. 6.3.1 measured routing weights: cost_ds[e] = the mean traversal time of link
 * e in deciseconds (summed steps * dt_ds / traversals, rounded half up, within
 * 1..1e6), or prev_cost_ds[e] when no trip left e.  gap (may be NULL) =
 * sum_e n_e |cost_e - prev_e| / sum_e n_e prev_e, n_e the traversals (0 when none).
 * Host arrays [n_links].  Needs SIM_OUT_LINK_TIMES (SIM_ESTATE); SIM_EINVAL when a
 * previous cost is outside 1..1e6. */
int sim_measured_costs(sim_handle* h, const int32_t* prev_cost_ds, int32_t* cost_ds, double* gap);

/* Sec. 6.3.1 decaying reroute: new shortest paths (as sim_route, on link_cost_ds)
 * for the subset of trips of round `round`, the others keep their routes.  Trip
 * vid (scenario-local id in a batch) is in the subset when the top 16 bits of
 * SplitMix64(seed ^ (vid << 32) ^ (2^31 | round)) are below fraction_q16 (0..65536;
 * 65536 reroutes every trip, 32768 about half).  Resets the vehicle state like
 * sim_route.  Errors as sim_route, SIM_ESTATE before any routes; a failure after
 * the search started leaves the handle without routes. */
int sim_reroute(sim_handle* h, const int32_t* link_cost_ds, uint32_t fraction_q16, uint32_t round);

/* Sec. 6.3.1 iterative decaying equilibrium, n_iter runs of n_steps from t = 0:
 * iteration 0 routes every trip on the initial weights (Eq. 4; cost_mode 1 for the
 * paper's sqrt(lanes) * length / speed), iteration k >= 1 reroutes the subset
 * fractions_q16[k] of round k (fractions_q16[0] is not read) on the weights measured
 * in iteration k - 1.  gap_out[k] is sim_measured_costs's gap after iteration k and
 * cost_out [n_links] the weights measured in the last one.  The paper's schedule is
 * four iterations with 100%, 100%, 50% and 25% of the trips routed.  The handle is
 * left at the end of the last run.  Needs SIM_OUT_LINK_TIMES (SIM_ESTATE). */
int sim_equilibrium(sim_handle* h, int32_t n_iter, const uint32_t* fractions_q16, int32_t n_steps,
                    int32_t* cost_out, double* gap_out);

/* ---------------------------------------------------------------- static assignment
 * Static user equilibrium (Sec. 5.2, Eq. 6) of the handle's trips (one vehicle each) on
 * its network, by Frank-Wolfe with BPR link times (Eq. 3):
 *   t_e = t0_e (1 + alpha (x_e / capacity_e)^beta), t0_e = length / speed (Eq. 4, s);
 *   x_0 = all-or-nothing assignment on t0; iteration k: y_k = all-or-nothing on t(x_k),
 *   gap_k = (t.x_k - t.y_k) / t.x_k, step a_k in [0, 1] minimising the Beckmann objective
 *   sum_e int_0^{x_e} t_e along x_k + a (y_k - x_k) (bisection on the sign of its
 *   derivative; a_k = 0 when it is not negative at 0, 1 when it is not positive at 1),
 *   x_{k+1} = x_k + a_k (y_k - x_k).
 * All-or-nothing: every trip on the canonical shortest path of sim_route (GPU trees per
 * origin) under integer costs, the times on a grid of max(0.1 s, max t / qmax) with
 * qmax = min(1e6, (2e9 - 1) / n_nodes), rounded half up, within 1..qmax.  Sums that
 * decide anything are exact: terms rounded to a 2^-S grid (S from a bound of the terms)
 * and added as 64-bit integers, so results do not depend on the order of the GPU's
 * atomics.  The vehicle state and routes of the handle are not touched. */
typedef struct {
  const double* capacity;   /* host [n_links], vehicles over the same period as the demand, > 0 */
  double alpha;             /* 0.15 in the original BPR curve */
  int32_t beta;             /* 4 in the original BPR curve; 1..8 */
  int32_t max_iter;         /* Frank-Wolfe iterations after the initial assignment, >= 0 */
  int32_t bisect_iter;      /* halvings of the line search, 0..60 (30 gives 1e-9) */
} sim_assign_spec;

/* Outputs (host arrays): flow [n_links] = x_K, time [n_links] = t(x_K), gap [max_iter],
 * step [max_iter], objective [max_iter + 1] (at x_0 .. x_K; gap and step may be NULL when
 * max_iter = 0).  Errors: SIM_EINVAL (spec, capacities, origin == destination),
 * SIM_EUNREACHABLE, SIM_ENOMEM, SIM_ECUDA. */
int sim_assign_static(sim_handle* h, const sim_assign_spec* spec, double* flow, double* time, double* gap,
                      double* step, double* objective);

/* Largest graph sim_sssp_static accepts (nodes). */
#define SIM_SSSP_STATIC_MAX_NODES 262144

/* One shortest-path tree without any device allocation.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc, such as code
 * running while a framework owns the whole device memory pool, processes whose
 * device memory is capped by a supervisor, or plug-ins that must not change the
 * device's allocation state.
 *
 * It runs the same near-far search as sim_route's per-origin trees on a graph the
 * caller already holds in device memory, and writes dist_out[v] = length of the
 * shortest path origin -> v in the caller's integer costs (INT32_MAX when v is
 * unreachable).  All pointers are DEVICE pointers owned by the caller:
 *   out_start [n_nodes+1]  CSR offsets of the links leaving each node (out_start[0] = 0,
 *                          out_start[n_nodes] = n_links, non-decreasing)
 *   out_link  [n_links]    link ids grouped by tail node
 *   link_to   [n_links]    head node of each link
 *   link_cost [n_links]    cost of each link, 1..1e6
 *   dist_out  [n_nodes]    output
 * stream: cudaStream_t to run on (NULL = legacy default stream).  The call
 * synchronises that stream before returning.
 *
 * Working memory is one fixed device array inside the library (about 9 MB, enough
 * for SIM_SSSP_STATIC_MAX_NODES nodes) that every GPU loading the library keeps
 * until the process exits.  n_nodes above SIM_SSSP_STATIC_MAX_NODES, an origin
 * out of range, or a malformed graph (offsets, link ids, head nodes or costs out
 * of range; costs whose path sums could overflow) return SIM_EINVAL without
 * running the search.  The first call on each device looks up the array's device
 * address (with that device current) and fills its distance words once (a device
 * synchronisation); make that first call before any stream capture.  All calls share the array: calls that overlap on the GPU (different
 * streams or host threads at the same time) race and give wrong results, so
 * serialise them.  Only a small per-call control block is cleared on each call;
 * the distance and queue words are tagged with a per-call epoch and need no
 * clearing, except once every 2^30 calls or search rounds, when the call that
 * reaches that count refills them after its output is written.  Returns SIM_OK, SIM_EINVAL or SIM_ECUDA; sim_last_error is not set. */
int sim_sssp_static(int32_t n_nodes, int32_t n_links, const int32_t* out_start, const int32_t* out_link,
                    const int32_t* link_to, const int32_t* link_cost, int32_t origin, int32_t* dist_out,
                    void* stream);

/* Test hook of sim_sssp_static (no counterpart in the paper): sets the two counters the
 * fixed array keeps across calls, the search epoch that tags distance words and the
 * round number that tags queue flags.  After any call that leaves either at 2^30 or
 * more, sim_sssp_static puts the array back to its first-use state (distance words
 * all-ones, flags and counters zero) so that neither counter can wrap around in a
 * long-lived process; this hook lets a test reach that point without a billion calls.
 * The counters may only be moved forward (below their current values, stale tags in
 * the array would look current).  Same set-up and serialisation rules as
 * sim_sssp_static; allocates nothing.  Returns
 * SIM_OK or SIM_ECUDA. */
int sim_sssp_static_set_counters(uint32_t epoch, int32_t round, void* stream);

/* Message of the last failed call on this handle (or of the last failed
 * sim_create when h is NULL). */
const char* sim_last_error(const sim_handle* h);

void sim_destroy(sim_handle* h);

#ifdef __cplusplus
}
#endif
#endif
